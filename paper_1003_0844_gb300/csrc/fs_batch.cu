// Batched search over many segments (the coherent first stage of a
// hierarchical search, Sec. I) and the launch-configuration tuner.
//
// fs_search_batch orders the segments by transform cost, assigns them to two
// branches (longest first onto the less loaded branch), gives each branch its
// own workspace, and records every launch of every segment into one CUDA graph
// whose branches run concurrently: a branch's persistent kernel can start on
// the SMs that the other branch's kernel leaves idle in its tail, and the
// per-sky demodulation of one segment overlaps the transforms of another.
// The graph is replayed as long as the arguments match.
//
// Safety of two concurrent persistent kernels: every wait of a work item is on
// items that were taken from the same kernel's queue earlier, hence by CTAs
// that are already running; the kernels never wait on each other.
#include <float.h>
#include <math.h>
#include <algorithm>
#include <vector>
#include "fs_pass32.cuh"

// The templates one segment of a batch searches: a grid (alpha, delta [nsky] x f1
// [nspin], offset NULL) or lattice templates (f1 and offset [nsky][nspin]).
struct SegTemplates {
  const double *alpha = nullptr, *delta = nullptr, *f1 = nullptr, *offset = nullptr;
  int nsky = 0, nspin = 0;
  bool operator==(const SegTemplates &o) const {
    return alpha == o.alpha && delta == o.delta && f1 == o.f1 && offset == o.offset && nsky == o.nsky &&
           nspin == o.nspin;
  }
};

struct BatchPlan {
  std::vector<uint64_t> serials;
  std::vector<SegTemplates> tpl;
  float thr = 0.f;
  fs_candidate *cand = nullptr;
  int64_t cap = 0;
  int64_t *ncand = nullptr;
  uint64_t tune_version = 0;
  void *ws[fs_ctx::kWsSlots] = {};
  bool persistent = true;
  cudaGraphExec_t exec = nullptr;
  int64_t launches = 0;  // kernels per replay
};

namespace fs {

void batch_plan_release(fs_ctx *ctx) {
  if (!ctx->plan) return;
  if (ctx->plan->exec) cudaGraphExecDestroy(ctx->plan->exec);
  delete ctx->plan;
  ctx->plan = nullptr;
}

static double transform_cost(const fs_seg *s) {
  const double n = (double)s->g.nfft;
  return n * log2(n);
}

static fs_status ensure_side_streams(fs_ctx *ctx) {
  for (int i = 0; i < 2; i++) {
    if (!ctx->side[i] && cudaStreamCreateWithFlags(&ctx->side[i], cudaStreamNonBlocking) != cudaSuccess)
      return FS_ERR_CUDA;
    if (!ctx->join[i] && cudaEventCreateWithFlags(&ctx->join[i], cudaEventDisableTiming) != cudaSuccess)
      return FS_ERR_CUDA;
  }
  if (!ctx->fork && cudaEventCreateWithFlags(&ctx->fork, cudaEventDisableTiming) != cudaSuccess) return FS_ERR_CUDA;
  return FS_OK;
}

static bool plan_matches(const fs_ctx *ctx, const BatchPlan &p, fs_seg *const *segs, int nseg,
                         const SegTemplates *tpl, float thr, fs_candidate *cand, int64_t cap, int64_t *ncand) {
  if ((int)p.serials.size() != nseg) return false;
  for (int i = 0; i < nseg; i++)
    if (p.serials[i] != segs[i]->serial || !(p.tpl[i] == tpl[i])) return false;
  for (int i = 0; i < fs_ctx::kWsSlots; i++)
    if (p.ws[i] != ctx->ws[i]) return false;
  return p.thr == thr && p.cand == cand && p.cap == cap && p.ncand == ncand && p.tune_version == ctx->tune_version &&
         p.persistent == ctx->persistent;
}

// lattice templates run from the persistent queue's lattice items (lattice_supported)
bool lattice_supported(const Cfg32 &c);

static fs_status batch_run(fs_ctx *ctx, fs_seg *const *segs, int nseg, const SegTemplates *tpl, float thr,
                           fs_candidate *cand, int64_t cap, int64_t *ncand, cudaStream_t st) {
  if (ctx->plan && plan_matches(ctx, *ctx->plan, segs, nseg, tpl, thr, cand, cap, ncand)) {
    if (cudaGraphLaunch(ctx->plan->exec, st) != cudaSuccess) return FS_ERR_CUDA;
    ctx->launches += ctx->plan->launches;
    return FS_OK;
  }
  batch_plan_release(ctx);
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (st && cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) return FS_ERR_ARG;

  // the F row length of each segment: the band's bins, or the half-bin grid of an
  // interbinning segment (candidate bins are indices on that row)
  auto seg_nbins = [](const fs_seg *sg) {
    return (sg->d.options & FS_OPT_INTERBIN) ? sg->g.nfft : sg->g.nfft / 2;
  };
  std::vector<Cfg32> cfg(nseg);
  for (int i = 0; i < nseg; i++) {
    fs_status s = config32(ctx, segs[i], tpl[i].nsky, seg_nbins(segs[i]), &cfg[i]);
    if (s != FS_OK) return s;
    if (tpl[i].offset && !lattice_supported(cfg[i])) return FS_ERR_UNSUPPORTED;
  }
  // longest transforms first, each onto the branch with less work so far
  std::vector<int> order(nseg);
  for (int i = 0; i < nseg; i++) order[i] = i;
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return transform_cost(segs[a]) > transform_cost(segs[b]); });
  std::vector<int> branch(nseg);
  double load[2] = {0.0, 0.0};
  for (int i : order) {
    const int b = load[1] < load[0] ? 1 : 0;
    branch[i] = b;
    load[b] += transform_cost(segs[i]);
  }
  // size both branch workspaces before recording (no allocation inside the graph)
  for (int i : order) {
    Ws32 w;
    fs_status s = workspace32(ctx, 1 + branch[i], segs[i], cfg[i], tpl[i].nsky, tpl[i].nspin, true, st, &w);
    if (s != FS_OK) return s;
  }
  fs_status s = ensure_side_streams(ctx);
  if (s != FS_OK) return s;
  if (cudaStreamSynchronize(st) != cudaSuccess) return FS_ERR_CUDA;

  const bool prof = ctx->prof;
  const int64_t launches0 = ctx->launches;
  ctx->prof = false;  // no timing events inside a graph
  cudaStream_t s0 = ctx->side[0], s1 = ctx->side[1];
  cudaGraph_t graph = nullptr;
  fs_status r = FS_OK;
  if (cudaStreamBeginCapture(s0, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
    ctx->prof = prof;
    return FS_ERR_CUDA;
  }
  if (cudaEventRecord(ctx->fork, s0) != cudaSuccess || cudaStreamWaitEvent(s1, ctx->fork, 0) != cudaSuccess)
    r = FS_ERR_CUDA;
  for (int k = 0; k < nseg && r == FS_OK; k++) {
    const int i = order[k];
    cudaStream_t sb = branch[i] ? s1 : s0;
    Ws32 w;
    const SegTemplates &t = tpl[i];
    r = workspace32(ctx, 1 + branch[i], segs[i], cfg[i], t.nsky, t.nspin, false, sb, &w);
    if (r == FS_OK)
      r = search32_run(ctx, segs[i], cfg[i], w, t.alpha, t.delta, t.nsky, t.f1, t.nspin, thr, nullptr,
                       seg_nbins(segs[i]), cand ? cand + (int64_t)i * cap : nullptr, cap, ncand + i, sb, t.offset);
  }
  if (r == FS_OK && (cudaEventRecord(ctx->join[1], s1) != cudaSuccess || cudaStreamWaitEvent(s0, ctx->join[1], 0) != cudaSuccess))
    r = FS_ERR_CUDA;
  const cudaError_t ec = cudaStreamEndCapture(s0, &graph);
  ctx->prof = prof;
  const int64_t per_replay = ctx->launches - launches0;
  ctx->launches = launches0;
  if (r == FS_OK && (ec != cudaSuccess || !graph)) r = FS_ERR_CUDA;
  cudaGraphExec_t exec = nullptr;
  if (r == FS_OK && cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) r = FS_ERR_CUDA;
  if (graph) cudaGraphDestroy(graph);
  if (r != FS_OK) {
    cudaGetLastError();
    return r;
  }
  BatchPlan *p = new BatchPlan();
  for (int i = 0; i < nseg; i++) p->serials.push_back(segs[i]->serial);
  p->tpl.assign(tpl, tpl + nseg);
  p->thr = thr;
  p->cand = cand;
  p->cap = cap;
  p->ncand = ncand;
  p->tune_version = ctx->tune_version;
  for (int i = 0; i < fs_ctx::kWsSlots; i++) p->ws[i] = ctx->ws[i];
  p->persistent = ctx->persistent;
  p->exec = exec;
  p->launches = per_replay;
  ctx->plan = p;
  if (cudaGraphLaunch(exec, st) != cudaSuccess) return FS_ERR_CUDA;
  ctx->launches += per_replay;
  return FS_OK;
}

fs_status search32_batch(fs_ctx *ctx, fs_seg *const *segs, int nseg, const double *alpha, const double *delta,
                         int nsky, const double *f1, int nspin, float thr, fs_candidate *cand, int64_t cap,
                         int64_t *ncand, cudaStream_t st) {
  SegTemplates t;
  t.alpha = alpha;
  t.delta = delta;
  t.f1 = f1;
  t.nsky = nsky;
  t.nspin = nspin;
  std::vector<SegTemplates> tpl((size_t)nseg, t);
  return batch_run(ctx, segs, nseg, tpl.data(), thr, cand, cap, ncand, st);
}

fs_status search32_lattice_batch(fs_ctx *ctx, fs_seg *const *segs, int nseg, const double *const *alpha,
                                 const double *const *delta, const int32_t *nsky, const double *const *f1,
                                 const double *const *offset, const int32_t *nspin, float thr, fs_candidate *cand,
                                 int64_t cap, int64_t *ncand, cudaStream_t st) {
  std::vector<SegTemplates> tpl((size_t)nseg);
  for (int i = 0; i < nseg; i++) {
    tpl[i].alpha = alpha[i];
    tpl[i].delta = delta[i];
    tpl[i].f1 = f1[i];
    tpl[i].offset = offset[i];
    tpl[i].nsky = nsky[i];
    tpl[i].nspin = nspin[i];
  }
  return batch_run(ctx, segs, nseg, tpl.data(), thr, cand, cap, ncand, st);
}

// ------------------------------------------------------------------ tuner
static fs_status read_clear_flags(fs_ctx *ctx, uint32_t *f) {
  *f = 0;
  if (cudaMemcpy(f, ctx->d_flags, sizeof(uint32_t), cudaMemcpyDeviceToHost) != cudaSuccess) return FS_ERR_CUDA;
  if (*f && cudaMemset(ctx->d_flags, 0, sizeof(uint32_t)) != cudaSuccess) return FS_ERR_CUDA;
  return FS_OK;
}

fs_status autotune32(fs_ctx *ctx, fs_seg *seg, const double *alpha, const double *delta, int nsky,
                     const double *f1, int nspin, int reps, fs_tuning *out, cudaStream_t st) {
  int p = 0;
  while (((int64_t)1 << p) < seg->g.nfft) p++;
  const int vshift = p > 20 ? p - 20 : 0;
  const int64_t nsub = (int64_t)1 << (p - vshift);
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  std::vector<fs_tuning> cands;
  const int n1s[] = {64, 128, 256, 512, 1024};
  for (int n1 : n1s) {
    if (nsub % n1 != 0 || !split_instantiated(n1, (int)(nsub / n1))) continue;
    const int n2 = (int)(nsub / n1);
    int t1 = 0, t2 = 0;
    queue_tiles(n1, n2, kPersistThreads, &t1, &t2);
    const int ctas = passes_blocks_per_sm(n1, n2) * nsm;
    int last_kr = -1;
    for (double frac : {0.5, 0.85, 1.2}) {
      int kr = (int)(frac * ctas / t1 + 0.5);
      if (kr < 1) kr = 1;
      if (kr == last_kr) continue;
      last_kr = kr;
      for (int lag : {1, 2}) {
        fs_tuning t{};
        t.n1 = n1;
        t.queue_round = kr;
        t.queue_lag = lag;
        cands.push_back(t);
      }
    }
  }
  if (cands.empty()) return FS_ERR_SHAPE;

  const fs_tuning saved = ctx->tune[p];
  const bool saved_on = ctx->tuned[p];
  int64_t *dcount = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  fs_status r = FS_OK;
  if (cudaMalloc(&dcount, sizeof(int64_t)) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess)
    r = FS_ERR_CUDA;
  // the segment's own F row: the band's bins, or the half-bin grid with interbinning
  const int64_t nbins = (seg->d.options & FS_OPT_INTERBIN) ? seg->g.nfft : seg->g.nfft / 2;
  fs_tuning best{};
  float best_ms = FLT_MAX;
  for (size_t c = 0; c < cands.size() && r == FS_OK; c++) {
    ctx->tune[p] = cands[c];
    ctx->tuned[p] = true;
    // warm-up (sizes the workspace), then the timed searches
    r = search32(ctx, seg, alpha, delta, nsky, f1, nspin, FLT_MAX, nullptr, nbins, nullptr, 0, dcount, st);
    if (r != FS_OK) break;
    if (cudaStreamSynchronize(st) != cudaSuccess) { r = FS_ERR_CUDA; break; }
    uint32_t fl = 0;
    if ((r = read_clear_flags(ctx, &fl)) != FS_OK) break;
    if (fl & ERRF_CORRUPT) { r = FS_ERR_CORRUPT; break; }
    if (fl & ERRF_TIMEOUT) { r = FS_ERR_TIMEOUT; break; }
    if (fl & ERRF_NONFINITE) { r = FS_ERR_NONFINITE; break; }
    cudaEventRecord(e0, st);
    for (int k = 0; k < reps && r == FS_OK; k++)
      r = search32(ctx, seg, alpha, delta, nsky, f1, nspin, FLT_MAX, nullptr, nbins, nullptr, 0, dcount, st);
    cudaEventRecord(e1, st);
    if (r != FS_OK) break;
    if (cudaEventSynchronize(e1) != cudaSuccess) { r = FS_ERR_CUDA; break; }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if ((r = read_clear_flags(ctx, &fl)) != FS_OK) break;
    if (fl & ERRF_TIMEOUT) { r = FS_ERR_TIMEOUT; break; }
    const float per = ms / ((float)reps * (float)nsky * (float)nspin);
    if (per < best_ms) {
      best_ms = per;
      best = cands[c];
      best.ms_per_template = per;
    }
  }
  if (dcount) cudaFree(dcount);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (r != FS_OK) {
    ctx->tune[p] = saved;
    ctx->tuned[p] = saved_on;
    cudaGetLastError();
    return r;
  }
  ctx->tune[p] = best;
  ctx->tuned[p] = true;
  ctx->tune_version++;
  *out = best;
  return FS_OK;
}

}  // namespace fs
