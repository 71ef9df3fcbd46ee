// FP32 search path with compensated (double-float) phases: per-sky constants,
// the per-sky resampling/demodulation (A1) and the host orchestration of the
// transform passes (device code in fs_pass32.cuh).
//
// Per sky (A1, k_demod32): source times t_j of Eq. (eq:Bt) by one Newton
// step from a first delay estimate, the spline value x~_j (Sec. VI.A),
// a_j, b_j (Sec. II), the heterodyne factor exp(-2 pi i fl phi_m(t_j)) and
// the spindown phase argument Q_j = t_j^2/2 + t_j phi_m(t_j) (Eq. phas) kept
// as a double-float.  Output per sky: y^a_j, y^b_j (float2) and Q_j.
#include <stdio.h>
#include "fs_demod.cuh"
#include "fs_pass32.cuh"

namespace fs {

// Spindowns as double-floats, once per search (the FP64 conversion in every
// transform item would occupy the slow FP64 pipe).
__global__ void k_f1_df32(const double *f1, int64_t n, float2 *out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) {
    const df32 d = df_from_double(f1[i]);
    out[i] = make_float2(d.hi, d.lo);
  }
}

static cudaError_t f1_to_df32(const double *f1, int64_t n, float2 *out, cudaStream_t st) {
  k_f1_df32<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(f1, n, out);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ self-test of the bounded waits
__device__ unsigned g_never_incremented = 0;  // nothing writes it

__global__ void k_selftest_wait(uint32_t *flags) {
  if (threadIdx.x == 0) wait_at_least(&g_never_incremented, 1u, flags);
  __syncthreads();
}

cudaError_t selftest_wait(uint32_t *flags, cudaStream_t st) {
  k_selftest_wait<<<1, 32, 0, st>>>(flags);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ per-sky constants
__global__ void k_skyconst(const double *alpha, const double *delta, int nsky, SegGeom g, double eps,
                           double lat, double gamma, SkyConst32 *out32, SkyConst64 *out64) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nsky) return;
  SkyConst64 k;
  sky_constants(alpha[s], delta[s], eps, lat, gamma, g, &k);
  if (out64) out64[s] = k;
  if (out32) {
    SkyConst32 c;
    c.nx = df_from_double(k.nx);  // the tables carry the factor AU/c
    c.nyp = df_from_double(k.nyp);
    c.nz = df_from_double(k.nz);
    c.ca = (float)k.ca;
    c.sa = (float)k.sa;
    c.rcd = (float)k.rcd;
    c.zsd = (float)k.zsd;
    for (int i = 0; i < 5; i++) c.ea[i] = (float)k.ea[i];
    for (int i = 0; i < 4; i++) c.eb[i] = (float)k.eb[i];
    out32[s] = c;
  }
}

cudaError_t sky_constants32(const double *alpha, const double *delta, int nsky, const SegGeom &g,
                            const fs_detector &det, SkyConst32 *out, cudaStream_t st) {
  k_skyconst<<<(nsky + 127) / 128, 128, 0, st>>>(alpha, delta, nsky, g, det.eps, det.lat, det.gamma, out,
                                                  nullptr);
  return cudaGetLastError();
}
cudaError_t sky_constants64(const double *alpha, const double *delta, int nsky, const SegGeom &g,
                            const fs_detector &det, SkyConst64 *out, cudaStream_t st) {
  k_skyconst<<<(nsky + 127) / 128, 128, 0, st>>>(alpha, delta, nsky, g, det.eps, det.lat, det.gamma,
                                                  nullptr, out);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ A1: resample + demodulate one sky
// EPH: the delay from the caller's position table (eph0..2: r_m as double-floats
// and v_m on the grid) in place of the analytic orbit and rotation terms.
template <int INTERP, bool EPH>
__global__ void __launch_bounds__(256) k_demod32(DemodArgs A) {
  const int s = blockIdx.y;
  const SkyConst32 K = A.sky[s];
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  float a2 = 0.f, b2 = 0.f;
  if (j < A.npad) {
    float2 oa = make_float2(0.f, 0.f), ob = oa, oq = oa;
    if (j < A.g.n) {
      const ResampledSample r = resample_sample<INTERP, EPH>(A, K, j);
      a2 = r.av * r.av;
      b2 = r.bv * r.bv;
      // 7) heterodyne exp(-2 pi i fl phi_m(t_j))
      const float2 h = expm2pi(df_mul_frac(A.fl, r.phim));
      oa = make_float2(r.xr * r.av * h.x, r.xr * r.av * h.y);
      ob = make_float2(r.xr * r.bv * h.x, r.xr * r.bv * h.y);
      oq = make_float2(r.Q.hi, r.Q.lo);
      if (A.tsrc && s == 0) A.tsrc[j] = (double)r.m1 * A.g.dt + (double)r.tau;
    }
    A.ya[s * A.stride + j] = oa;
    A.yb[s * A.stride + j] = ob;
    A.qq[s * A.stride + j] = oq;
  }
  // deterministic block sums of a^2, b^2 by pairwise trees in FP32 (relative error
  // below 8 roundings of the 256 positive terms); the blocks are summed in FP64 by
  // k_demod_finalize.  (FP64 here would cost half the kernel: its pipe runs at 1/64
  // of the FP32 rate on this GPU.)
  for (int o = 16; o > 0; o >>= 1) {
    a2 += __shfl_down_sync(kFull, a2, o);
    b2 += __shfl_down_sync(kFull, b2, o);
  }
  __shared__ float wa[8], wb[8];
  if ((threadIdx.x & 31) == 0) { wa[threadIdx.x >> 5] = a2; wb[threadIdx.x >> 5] = b2; }
  __syncthreads();
  if (threadIdx.x == 0) {
    const float sa = ((wa[0] + wa[1]) + (wa[2] + wa[3])) + ((wa[4] + wa[5]) + (wa[6] + wa[7]));
    const float sb = ((wb[0] + wb[1]) + (wb[2] + wb[3])) + ((wb[4] + wb[5]) + (wb[6] + wb[7]));
    A.partial[(int64_t)s * gridDim.x + blockIdx.x] = make_float2(sa, sb);
  }
}

// <a^2>, <b^2> over the n output samples and the per-sky F normalisation
// (cF / <a^2>, cF / <b^2>) with cF = 2 dt^2 / (S0 To) = 2 dt / (S0 n).
__global__ void k_demod_finalize(const float2 *partial, int nb, int64_t n, double dt, double S0, float2 *norm,
                                 double2 *ab2) {
  const int s = blockIdx.x;
  double sa = 0.0, sb = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) {
    const float2 v = partial[(int64_t)s * nb + i];
    sa += v.x;
    sb += v.y;
  }
  __shared__ double ra[256], rb[256];
  ra[threadIdx.x] = sa;
  rb[threadIdx.x] = sb;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) { ra[threadIdx.x] += ra[threadIdx.x + o]; rb[threadIdx.x] += rb[threadIdx.x + o]; }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double ma = ra[0] / (double)n, mb = rb[0] / (double)n;
    double cF = 2.0 * dt / (S0 * (double)n);
    if (norm) norm[s] = make_float2((float)(cF / ma), (float)(cF / mb));
    if (ab2) ab2[s] = make_double2(ma, mb);
  }
}

// ------------------------------------------------------------------ host orchestration
static int log2_exact(int64_t v) {
  int p = 0;
  while (p < 62 && ((int64_t)1 << p) < v) p++;
  return ((int64_t)1 << p) == v ? p : -1;
}
// Default split of a sub-transform of length 2^p: N1 = 2^ceil(p/2), N2 = 2^floor(p/2).
static FftShape default_split(int p) { return FftShape{1 << ((p + 1) / 2), 1 << (p / 2)}; }

// Transform splits N1 x N2 the library instantiates for the persistent kernel.
static const int kSplits[][2] = {
    {64, 64},    {128, 64},  {128, 128},  {256, 64},   {256, 128}, {256, 256},  {512, 128},
    {128, 512},  {512, 256}, {256, 512},  {1024, 128}, {512, 512}, {1024, 256}, {256, 1024},
    {1024, 512}, {512, 1024}, {1024, 1024}};

bool split_instantiated(int N1, int N2) {
  for (const auto &s : kSplits)
    if (s[0] == N1 && s[1] == N2) return true;
  return false;
}

cudaError_t dispatch_passes(int N1, int N2, const Pass1Args &a1, const Pass2Args &a2, const QueueArgs &qa,
                            cudaStream_t st) {
  const int64_t nf = (int64_t)N1 * N2;
  if (nf <= (1 << 16)) return dispatch_passes_small(N1, N2, a1, a2, qa, st);
  if (nf <= (1 << 18)) return dispatch_passes_mid(N1, N2, a1, a2, qa, st);
  return dispatch_passes_large(N1, N2, a1, a2, qa, st);
}
int passes_blocks_per_sm(int N1, int N2) {
  const int64_t nf = (int64_t)N1 * N2;
  if (nf <= (1 << 16)) return passes_blocks_per_sm_small(N1, N2);
  if (nf <= (1 << 18)) return passes_blocks_per_sm_mid(N1, N2);
  return passes_blocks_per_sm_large(N1, N2);
}

// Sub-transform split: 2^vshift sub-transforms of at most 2^20 points.
static bool sub_transform(int64_t nfft, int *vshift, int *psub) {
  const int p = log2_exact(nfft);
  if (p < 12 || p > 21) return false;
  *vshift = p > 20 ? p - 20 : 0;
  *psub = p - *vshift;
  return true;
}

bool tuning_valid(int64_t nfft, const fs_tuning &t) {
  int vs = 0, ps = 0;
  if (!sub_transform(nfft, &vs, &ps)) return false;
  if (t.n1 < 0 || t.queue_round < 0 || t.queue_lag < 0 || t.group_skies < 0) return false;
  if (t.queue_lag > 64 || t.queue_round > 4096) return false;
  if (t.n1 == 0) return true;
  const int64_t ns = (int64_t)1 << ps;
  return ns % t.n1 == 0 && split_instantiated(t.n1, (int)(ns / t.n1));
}

static QueueShape queue_shape(const fs_ctx *ctx, const fs_tuning *t, const FftShape &sh) {
  QueueShape q{};
  queue_tiles(sh.N1, sh.N2, kPersistThreads, &q.tiles1, &q.tiles2);
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  int bps = passes_blocks_per_sm(sh.N1, sh.N2);
  if (bps < 1) bps = 1;
  const int ctas = bps * (nsm > 0 ? nsm : 1);
  const int qr = (t && t->queue_round > 0) ? t->queue_round : ctx->queue_round;
  q.kr = qr > 0 ? qr : (int)(0.85 * ctas / q.tiles1 + 0.5);
  if (q.kr < 1) q.kr = 1;
  const int lg = (t && t->queue_lag > 0) ? t->queue_lag : ctx->queue_lag;
  q.lag = lg > 0 ? lg : 1;
  const int need = (q.lag + 2) * q.kr;
  q.slots = ctx->z_slots > need ? ctx->z_slots : need;
  return q;
}

fs_status config32(const fs_ctx *ctx, const fs_seg *seg, int nsky, int64_t nbins, Cfg32 *c) {
  int ps = 0;
  if (!sub_transform(seg->g.nfft, &c->vshift, &ps)) return FS_ERR_SHAPE;
  c->nsub = (int64_t)1 << ps;
  if (seg->g.n > c->nsub) return FS_ERR_SHAPE;
  const int p = ps + c->vshift;
  const fs_tuning *t = ctx->tuned[p] ? &ctx->tune[p] : nullptr;
  c->sh = default_split(ps);
  // interbinning with an odd power: the split with the shorter first pass where its
  // items are built (2^17: 256 x 512 measured 15% faster than 512 x 256)
  if ((seg->d.options & FS_OPT_INTERBIN) && (ps & 1) && passes_ib_instantiated(c->sh.N1 / 2, c->sh.N2 * 2))
    c->sh = FftShape{c->sh.N1 / 2, c->sh.N2 * 2};
  if (t && t->n1 > 0) c->sh = FftShape{t->n1, (int)(c->nsub / t->n1)};
  c->n1max = (int)((seg->g.n + c->sh.N2 - 1) / c->sh.N2);
  c->npad = (int64_t)c->n1max * c->sh.N2;
  const int gsk = (t && t->group_skies > 0) ? t->group_skies : ctx->group_skies;
  c->G = gsk < nsky ? gsk : nsky;
  c->interbin = (seg->d.options & FS_OPT_INTERBIN) != 0;
  if (c->interbin && (c->vshift || nbins != seg->g.nfft)) return FS_ERR_SHAPE;
  c->full = (nbins == seg->g.nfft);
  // interbinning runs from the persistent queue for the splits built with its items
  c->persistent = ctx->persistent && (c->interbin ? passes_ib_instantiated(c->sh.N1, c->sh.N2) : !c->full);
  c->qs = queue_shape(ctx, t, c->sh);
  c->B = c->persistent ? c->qs.slots : ctx->batch_templates;
  return FS_OK;
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

fs_status workspace32(fs_ctx *ctx, int slot, const fs_seg *seg, const Cfg32 &c, int nsky, int nspin,
                      bool may_alloc, cudaStream_t st, Ws32 *w) {
  (void)seg;
  if (slot < 0 || slot >= fs_ctx::kWsSlots) return FS_ERR_ARG;
  const int G = c.G;
  const int64_t stride = (c.npad + 63) & ~(int64_t)63;
  const int nblk = (int)((c.npad + 255) / 256);
  const size_t vt = ((size_t)G * nspin) << c.vshift;  // virtual templates of a group
  size_t off = 0;
  size_t o_sky = off; off = align256(off + sizeof(SkyConst32) * (nsky > G ? nsky : G));
  size_t o_ya = off; off = align256(off + sizeof(float2) * stride * G);
  size_t o_yb = off; off = align256(off + sizeof(float2) * stride * G);
  size_t o_qq = off; off = align256(off + sizeof(float2) * stride * G);
  size_t o_nm = off; off = align256(off + sizeof(float2) * G);
  size_t o_ab = off; off = align256(off + sizeof(double2) * G);
  size_t o_pa = off; off = align256(off + sizeof(float2) * (size_t)nblk * G);
  size_t o_f1 = off; off = align256(off + sizeof(float2) * (size_t)nsky * nspin);
  const size_t gb = kDebug ? kGuardBytes : 0;  // debug builds: guard words around the ring
  size_t o_g0 = off; off = align256(off + gb);
  size_t o_z = off; off = align256(off + sizeof(float2) * 2 * (size_t)c.nsub * c.B);
  size_t o_g1 = off; off = align256(off + gb);
  const size_t xn = !c.interbin ? 0
                    : c.persistent ? vt * (size_t)ib_edge_stride(c.sh.N1, c.sh.N2, kPersistThreads)
                                   : 2 * (size_t)c.nsub * c.B;
  size_t o_x = off; off = align256(off + sizeof(float2) * xn);
  size_t o_ct = off; off = align256(off + sizeof(unsigned) * (1 + 2 * vt));
  size_t o_g2 = off; off = align256(off + gb);
  if (may_alloc) {
    fs_status s = ensure_buffer(&ctx->ws[slot], &ctx->ws_bytes[slot], off, st);
    if (s != FS_OK) return s;
  } else if (ctx->ws_bytes[slot] < off || !ctx->ws[slot]) {
    return FS_ERR_NOMEM;
  }
  char *base = (char *)ctx->ws[slot];
  w->skyc = (SkyConst32 *)(base + o_sky);
  w->ya = (float2 *)(base + o_ya);
  w->yb = (float2 *)(base + o_yb);
  w->qq = (float2 *)(base + o_qq);
  w->norm = (float2 *)(base + o_nm);
  w->ab2 = (double2 *)(base + o_ab);
  w->partial = (float2 *)(base + o_pa);
  w->f1df = (float2 *)(base + o_f1);
  w->Z = (float2 *)(base + o_z);
  w->X = c.interbin ? (float2 *)(base + o_x) : nullptr;
  w->counters = (unsigned *)(base + o_ct);
  w->stride = stride;
  w->nblk_a1 = nblk;
  w->guard[0] = kDebug ? (uint32_t *)(base + o_g0) : nullptr;
  w->guard[1] = kDebug ? (uint32_t *)(base + o_g1) : nullptr;
  w->guard[2] = kDebug ? (uint32_t *)(base + o_g2) : nullptr;
  return FS_OK;
}

// Debug builds: fill the guard words of a workspace before a search and check
// them after it (an overwritten word latches ERRF_CORRUPT).
__global__ void k_guard(uint32_t *g0, uint32_t *g1, uint32_t *g2, int check, uint32_t *flags) {
  constexpr int W = (int)(kGuardBytes / sizeof(uint32_t));
  uint32_t *g[3] = {g0, g1, g2};
  for (int i = threadIdx.x; i < 3 * W; i += blockDim.x) {
    uint32_t *p = g[i / W] + (i % W);
    if (!check) *p = kGuardWord;
    else if (*p != kGuardWord) atomicOr(flags, ERRF_CORRUPT);
  }
}

static cudaError_t guards(const Ws32 &w, bool check, uint32_t *flags, cudaStream_t st) {
  if (!w.guard[0]) return cudaSuccess;
  k_guard<<<1, 256, 0, st>>>(w.guard[0], w.guard[1], w.guard[2], check ? 1 : 0, flags);
  return cudaGetLastError();
}

static DemodArgs demod_args(const fs_seg *seg, const Ws32 &w, int64_t npad) {
  DemodArgs A{};
  A.g = seg->g;
  A.dt2 = df_from_double(seg->g.dt);
  A.dt = (float)seg->g.dt;
  A.inv_dt = (float)(1.0 / seg->g.dt);
  A.two_over_dt = (float)(2.0 / seg->g.dt);
  A.fl = df_from_double(seg->g.fl);
  A.sky = w.skyc;
  A.tab0 = seg->tab0;
  A.tab1 = seg->tab1;
  A.eph0 = seg->eph0;
  A.eph1 = seg->eph1;
  A.eph2 = seg->eph2;
  A.coef = (const float4 *)seg->coef;
  A.x32 = seg->x32;
  A.ya = w.ya;
  A.yb = w.yb;
  A.qq = w.qq;
  A.stride = w.stride;
  A.npad = npad;
  A.partial = w.partial;
  A.tsrc = nullptr;
  return A;
}

static cudaError_t launch_demod(const DemodArgs &A, int nsky, int nblk, int interp, cudaStream_t st) {
  dim3 grid(nblk, nsky);
  const bool eph = A.eph0 != nullptr;
  if (interp == FS_INTERP_NEAREST) {
    if (eph) k_demod32<FS_INTERP_NEAREST, true><<<grid, 256, 0, st>>>(A);
    else k_demod32<FS_INTERP_NEAREST, false><<<grid, 256, 0, st>>>(A);
  } else {
    if (eph) k_demod32<FS_INTERP_SPLINE2X, true><<<grid, 256, 0, st>>>(A);
    else k_demod32<FS_INTERP_SPLINE2X, false><<<grid, 256, 0, st>>>(A);
  }
  return cudaGetLastError();
}

static void pass_args(const fs_seg *seg, const Cfg32 &c, const Ws32 &w, int nspin, float thr,
                      fs_candidate *cand, int64_t cap, int64_t *ncand, uint32_t *flags, Pass1Args *p1,
                      Pass2Args *p2) {
  *p1 = Pass1Args{};
  p1->ya = w.ya;
  p1->yb = w.yb;
  p1->qq = w.qq;
  p1->sky_stride = w.stride;
  p1->f1df = w.f1df;  // filled by f1_to_df32 before the launches
  p1->nspin = nspin;
  p1->nspin_fd = make_fastdiv((uint32_t)nspin);
  p1->N2 = c.sh.N2;
  p1->n1max = c.n1max;
  p1->nfft = c.nsub;
  p1->vshift = c.vshift;
  p1->inv_nfft_total = (float)(1.0 / (double)seg->g.nfft);
  p1->Z = w.Z;
  p1->z_elems = 2 * c.nsub * (int64_t)c.B;
  p1->yq_elems = w.stride * (int64_t)c.G;
  p1->flags = flags;
  *p2 = Pass2Args{};
  p2->Z = w.Z;
  p2->N1 = c.sh.N1;
  p2->N2 = c.sh.N2;
  p2->nfft = c.nsub;
  p2->norm = w.norm;
  p2->nspin = nspin;
  p2->nspin_fd = make_fastdiv((uint32_t)nspin);
  p2->vshift = c.vshift;
  p2->thr = thr;
  p2->cand = cand;
  p2->cap = cap;
  p2->ncand = (unsigned long long *)ncand;
  p2->flags = flags;
  p2->z_elems = 2 * c.nsub * (int64_t)c.B;
}

fs_status search32_run(fs_ctx *ctx, fs_seg *seg, const Cfg32 &c, const Ws32 &w, const double *alpha,
                       const double *delta, int nsky, const double *f1, int nspin, float thr, float *F,
                       int64_t nbins, fs_candidate *cand, int64_t cap, int64_t *ncand, cudaStream_t st,
                       const double *lat_offset) {
  if (lat_offset && !c.persistent) return FS_ERR_UNSUPPORTED;
  const int64_t n = seg->g.n;
  if (cudaMemsetAsync(ncand, 0, sizeof(int64_t), st) != cudaSuccess) return FS_ERR_CUDA;
  if (guards(w, false, ctx->d_flags, st) != cudaSuccess) return FS_ERR_CUDA;
  DemodArgs DA = demod_args(seg, w, c.npad);
  {
    ProfScope ps(ctx, PROF_OTHER, st);
    if (sky_constants32(alpha, delta, nsky, seg->g, ctx->det, w.skyc, st) != cudaSuccess) return FS_ERR_CUDA;
    ctx->launches += 1;
  }
  Pass1Args p1;
  Pass2Args p2;
  pass_args(seg, c, w, nspin, thr, cand, cap, ncand, ctx->d_flags, &p1, &p2);
  p2.nbins = nbins;
  if (f1_to_df32(f1, lat_offset ? (int64_t)nsky * nspin : nspin, w.f1df, st) != cudaSuccess) return FS_ERR_CUDA;
  ctx->launches += 1;
  for (int g0 = 0; g0 < nsky; g0 += c.G) {
    const int gs = (nsky - g0) < c.G ? (nsky - g0) : c.G;
    DA.sky = w.skyc + g0;
    {
      NvtxRange nv("fs.demodulate");
      {
        ProfScope ps(ctx, PROF_DEMOD, st);
        if (launch_demod(DA, gs, w.nblk_a1, seg->d.interp, st) != cudaSuccess) return FS_ERR_CUDA;
      }
      ProfScope ps(ctx, PROF_OTHER, st);
      k_demod_finalize<<<gs, 256, 0, st>>>(w.partial, w.nblk_a1, n, seg->g.dt, seg->g.S0, w.norm, w.ab2);
    }
    ctx->launches += 2;
    const int ntm = (gs * nspin) << c.vshift;  // virtual templates of the group
    p2.sky_base = g0;
    if (lat_offset) {  // the group's rows of per-template spindowns and bin offsets
      p1.f1df = w.f1df + (int64_t)g0 * nspin;
      p1.bin_offset = lat_offset + (int64_t)g0 * nspin;
    }
    p2.F = F ? F + (int64_t)g0 * nspin * nbins : nullptr;
    p2.f_elems = (int64_t)(nsky - g0) * nspin * nbins;
    if (c.persistent) {
      QueueArgs qa{};
      qa.ntm = ntm;
      qa.tiles1 = c.qs.tiles1;
      qa.tiles2 = c.qs.tiles2;
      qa.kr = c.qs.kr;
      qa.lag = c.qs.lag;
      qa.slots = c.qs.slots;
      qa.ipr_fd = make_fastdiv((uint32_t)(qa.kr * (qa.tiles1 + qa.tiles2)));
      qa.slots_fd = make_fastdiv((uint32_t)qa.slots);
      qa.counter = w.counters;
      if (cudaMemsetAsync(w.counters, 0, sizeof(unsigned) * (1 + 2 * (size_t)ntm), st) != cudaSuccess)
        return FS_ERR_CUDA;
      {
        NvtxRange nv("fs.transform");
        ProfScope ps(ctx, PROF_PASS2, st);
        if (c.interbin) {
          p2.X = w.X;
          p2.eb_stride = ib_edge_stride(c.sh.N1, c.sh.N2, kPersistThreads);
          if (dispatch_passes_ib(c.sh.N1, c.sh.N2, p1, p2, qa, st) != cudaSuccess) return FS_ERR_CUDA;
          ctx->launches += 1;  // the edge bins
        } else if (lat_offset) {
          if (dispatch_passes_lat(c.sh.N1, c.sh.N2, p1, p2, qa, st) != cudaSuccess) return FS_ERR_CUDA;
        } else if (dispatch_passes(c.sh.N1, c.sh.N2, p1, p2, qa, st) != cudaSuccess) {
          return FS_ERR_CUDA;
        }
      }
      ctx->launches += 1;
      continue;
    }
    NvtxRange nv("fs.transform");
    for (int b0 = 0; b0 < ntm; b0 += c.B) {
      const int nb = (ntm - b0) < c.B ? (ntm - b0) : c.B;
      p1.tmpl0 = b0;
      p2.tmpl0 = b0;
      {
        ProfScope ps(ctx, PROF_PASS1, st);
        if (dispatch_pass1(c.sh.N1, p1, nb, st) != cudaSuccess) return FS_ERR_CUDA;
      }
      if (c.interbin) {
        ProfScope ps(ctx, PROF_PASS2, st);
        p2.X = w.X;
        if (dispatch_pass2x(c.sh.N2, p2, nb, st) != cudaSuccess) return FS_ERR_CUDA;
        if (launch_interbin(p2, nb, st) != cudaSuccess) return FS_ERR_CUDA;
        ctx->launches += 1;
      } else {
        ProfScope ps(ctx, PROF_PASS2, st);
        if (dispatch_pass2(c.sh.N2, c.full, p2, nb, st) != cudaSuccess) return FS_ERR_CUDA;
      }
      ctx->launches += 2;
    }
  }
  if (guards(w, true, ctx->d_flags, st) != cudaSuccess) return FS_ERR_CUDA;
  return FS_OK;
}

// Lattice templates run as lattice items of the persistent queue: the split's items
// must be built, and 2^21 takes its sub-transforms on the 1024 x 1024 split only.
bool lattice_supported(const Cfg32 &c) {
  if (c.interbin || c.full || !c.persistent || !passes_lat_instantiated(c.sh.N1, c.sh.N2)) return false;
  return !c.vshift || (c.vshift == 1 && c.sh.N1 == 1024 && c.sh.N2 == 1024);
}

fs_status search32_lattice(fs_ctx *ctx, fs_seg *seg, const double *alpha, const double *delta, int nsky,
                           const double *f1, const double *offset, int nspin, float thr, float *F, int64_t nbins,
                           fs_candidate *cand, int64_t cap, int64_t *ncand, cudaStream_t st) {
  Cfg32 c;
  fs_status s = config32(ctx, seg, nsky, nbins, &c);
  if (s != FS_OK) return s;
  if (!lattice_supported(c)) return FS_ERR_UNSUPPORTED;
  Ws32 w;
  s = workspace32(ctx, 0, seg, c, nsky, nspin, true, st, &w);
  if (s != FS_OK) return s;
  return search32_run(ctx, seg, c, w, alpha, delta, nsky, f1, nspin, thr, F, nbins, cand, cap, ncand, st, offset);
}

fs_status search32(fs_ctx *ctx, fs_seg *seg, const double *alpha, const double *delta, int nsky,
                   const double *f1, int nspin, float thr, float *F, int64_t nbins, fs_candidate *cand,
                   int64_t cap, int64_t *ncand, cudaStream_t st) {
  Cfg32 c;
  fs_status s = config32(ctx, seg, nsky, nbins, &c);
  if (s != FS_OK) return s;
  Ws32 w;
  s = workspace32(ctx, 0, seg, c, nsky, nspin, true, st, &w);
  if (s != FS_OK) return s;
  return search32_run(ctx, seg, c, w, alpha, delta, nsky, f1, nspin, thr, F, nbins, cand, cap, ncand, st);
}

// Stage access: A1 for one sky, widened to double.
__global__ void k_widen(const float2 *ya, const float2 *yb, double *oa, double *ob, int64_t n) {
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= n) return;
  oa[2 * j] = ya[j].x;
  oa[2 * j + 1] = ya[j].y;
  ob[2 * j] = yb[j].x;
  ob[2 * j + 1] = yb[j].y;
}

fs_status demod32_debug(fs_ctx *ctx, fs_seg *seg, double alpha, double delta, double *ya, double *yb,
                        double *tsrc, double *ab2, cudaStream_t st) {
  const int64_t n = seg->g.n;
  Cfg32 c{};
  c.G = 1;
  c.npad = n;
  c.nsub = 0;
  c.B = 0;
  Ws32 w;
  fs_status s = workspace32(ctx, 0, seg, c, 1, 1, true, st, &w);
  if (s != FS_OK) return s;
  // alpha/delta are host values: stage them through the partial buffer's tail is not
  // possible before allocation, so use a small device copy.
  double hd[2] = {alpha, delta};
  double *dd = (double *)w.ab2;  // 16 bytes, overwritten by finalize afterwards
  if (cudaMemcpyAsync(dd, hd, sizeof(hd), cudaMemcpyHostToDevice, st) != cudaSuccess) return FS_ERR_CUDA;
  if (sky_constants32(dd, dd + 1, 1, seg->g, ctx->det, w.skyc, st) != cudaSuccess) return FS_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return FS_ERR_CUDA;  // hd is on the stack
  DemodArgs A = demod_args(seg, w, n);
  A.tsrc = tsrc;
  if (launch_demod(A, 1, w.nblk_a1, seg->d.interp, st) != cudaSuccess) return FS_ERR_CUDA;
  k_demod_finalize<<<1, 256, 0, st>>>(w.partial, w.nblk_a1, n, seg->g.dt, seg->g.S0, nullptr, (double2 *)ab2);
  k_widen<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(w.ya, w.yb, ya, yb, n);
  return cuda_status(cudaGetLastError());
}

// ------------------------------------------------------------------ allocation-free search
// The working memory of fs_search_noalloc: one fixed array per device, alive
// until the process exits.  In host code the symbol is only a host-side stand-in
// for the array: fs_create looks up its device address once for each context,
// with the context's device current, and the searches pass that address on.
static __device__ __align__(256) unsigned char g_noalloc_scratch[FS_NOALLOC_SCRATCH_BYTES];

fs_status noalloc_address(unsigned char **addr) {
  void *p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || !p) {
    cudaGetLastError();
    *addr = nullptr;
    return FS_ERR_CUDA;
  }
  *addr = (unsigned char *)p;
  return FS_OK;
}

// offset non-NULL: lattice templates (f1 and offset [nsky][nspin]), one sky row per launch
fs_status search32_noalloc(fs_ctx *ctx, fs_seg *seg, const double *alpha, const double *delta, int nsky,
                           const double *f1, int nspin, float thr, float *F, int64_t nbins, fs_candidate *cand,
                           int64_t cap, int64_t *ncand, cudaStream_t st, const double *offset) {
  if (seg->d.precision != FS_PREC_F32 || nbins != seg->g.nfft / 2) return FS_ERR_UNSUPPORTED;
  int vshift = 0, ps = 0;
  if (!sub_transform(seg->g.nfft, &vshift, &ps) || seg->g.n > seg->g.nfft) return FS_ERR_SHAPE;
  if (vshift) return FS_ERR_SCRATCH;  // a 2^21 transform ring alone exceeds the array
  const FftShape sh = default_split(ps);
  if (offset && !passes_lat_instantiated(sh.N1, sh.N2)) return FS_ERR_UNSUPPORTED;
  const int64_t n = seg->g.n;
  const int n1max = (int)((n + sh.N2 - 1) / sh.N2);
  const int64_t npad = (int64_t)n1max * sh.N2;
  const int64_t stride = (npad + 63) & ~(int64_t)63;
  const int nblk = (int)((npad + 255) / 256);
  const int lag = 4, slots = 6;  // one sky per launch: a short ring suffices
  // layout inside the fixed array (one sky at a time)
  size_t off = 0;
  const size_t o_sky = off; off = align256(off + sizeof(SkyConst32));
  const size_t o_ya = off; off = align256(off + sizeof(float2) * stride);
  const size_t o_yb = off; off = align256(off + sizeof(float2) * stride);
  const size_t o_qq = off; off = align256(off + sizeof(float2) * stride);
  const size_t o_nm = off; off = align256(off + sizeof(float2));
  const size_t o_ab = off; off = align256(off + sizeof(double2));
  const size_t o_pa = off; off = align256(off + sizeof(float2) * (size_t)nblk);
  const size_t o_f1 = off; off = align256(off + sizeof(float2) * (size_t)nspin);
  const size_t o_z = off; off = align256(off + sizeof(float2) * 2 * (size_t)seg->g.nfft * slots);
  const size_t o_ct = off; off = align256(off + sizeof(unsigned) * (1 + 2 * (size_t)nspin));
  if (off > (size_t)FS_NOALLOC_SCRATCH_BYTES) return FS_ERR_SCRATCH;
  unsigned char *base = ctx->noalloc;
  if (!base) return FS_ERR_CUDA;
  Ws32 w{};
  w.skyc = (SkyConst32 *)(base + o_sky);
  w.ya = (float2 *)(base + o_ya);
  w.yb = (float2 *)(base + o_yb);
  w.qq = (float2 *)(base + o_qq);
  w.norm = (float2 *)(base + o_nm);
  w.ab2 = (double2 *)(base + o_ab);
  w.partial = (float2 *)(base + o_pa);
  w.f1df = (float2 *)(base + o_f1);
  w.Z = (float2 *)(base + o_z);
  w.counters = (unsigned *)(base + o_ct);
  w.stride = stride;
  w.nblk_a1 = nblk;
  if (cudaMemsetAsync(ncand, 0, sizeof(int64_t), st) != cudaSuccess) return FS_ERR_CUDA;
  if (!offset) {
    if (f1_to_df32(f1, nspin, w.f1df, st) != cudaSuccess) return FS_ERR_CUDA;
    ctx->launches += 1;
  }
  DemodArgs DA = demod_args(seg, w, npad);
  for (int g0 = 0; g0 < nsky; g0++) {
    if (offset) {  // this sky's row of spindowns
      if (f1_to_df32(f1 + (int64_t)g0 * nspin, nspin, w.f1df, st) != cudaSuccess) return FS_ERR_CUDA;
      ctx->launches += 1;
    }
    {
      ProfScope ps(ctx, PROF_OTHER, st);
      if (sky_constants32(alpha + g0, delta + g0, 1, seg->g, ctx->det, w.skyc, st) != cudaSuccess)
        return FS_ERR_CUDA;
    }
    {
      NvtxRange nv("fs.demodulate");
      ProfScope ps(ctx, PROF_DEMOD, st);
      if (launch_demod(DA, 1, nblk, seg->d.interp, st) != cudaSuccess) return FS_ERR_CUDA;
    }
    {
      ProfScope ps(ctx, PROF_OTHER, st);
      k_demod_finalize<<<1, 256, 0, st>>>(w.partial, nblk, n, seg->g.dt, seg->g.S0, w.norm, w.ab2);
    }
    Cfg32 c{};
    c.sh = sh;
    c.vshift = 0;
    c.nsub = seg->g.nfft;
    c.n1max = n1max;
    c.npad = npad;
    Pass1Args p1;
    Pass2Args p2;
    pass_args(seg, c, w, nspin, thr, cand, cap, ncand, ctx->d_flags, &p1, &p2);
    p2.sky_base = g0;
    p2.F = F ? F + (int64_t)g0 * nspin * nbins : nullptr;
    p2.nbins = nbins;
    p1.z_elems = p2.z_elems = 2 * seg->g.nfft * (int64_t)slots;
    p1.yq_elems = stride;
    p2.f_elems = (int64_t)(nsky - g0) * nspin * nbins;
    QueueArgs qa{};
    qa.ntm = nspin;
    queue_tiles(sh.N1, sh.N2, kPersistThreads, &qa.tiles1, &qa.tiles2);
    qa.kr = 1;
    qa.lag = lag;
    qa.slots = slots;
    qa.ipr_fd = make_fastdiv((uint32_t)(qa.kr * (qa.tiles1 + qa.tiles2)));
    qa.slots_fd = make_fastdiv((uint32_t)qa.slots);
    qa.counter = w.counters;
    // the array keeps the previous call's contents: the queue counters start at zero
    if (cudaMemsetAsync(w.counters, 0, sizeof(unsigned) * (1 + 2 * (size_t)nspin), st) != cudaSuccess)
      return FS_ERR_CUDA;
    {
      NvtxRange nv("fs.transform");
      ProfScope ps(ctx, PROF_PASS2, st);
      if (offset) {
        p1.bin_offset = offset + (int64_t)g0 * nspin;
        if (dispatch_passes_lat(sh.N1, sh.N2, p1, p2, qa, st) != cudaSuccess) return FS_ERR_CUDA;
      } else if (dispatch_passes(sh.N1, sh.N2, p1, p2, qa, st) != cudaSuccess) {
        return FS_ERR_CUDA;
      }
    }
    ctx->launches += 4;
  }
  return FS_OK;
}

}  // namespace fs
