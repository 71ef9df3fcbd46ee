// C ABI of the library (include/fstat.h): argument checks, ownership of
// segment buffers and workspaces, dispatch to the FP32 or FP64 path.
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <atomic>
#include <new>
#include "fs_internal.h"
#include "fs_model.cuh"

using namespace fs;

namespace fs {
fs_status ensure_buffer(void **buf, size_t *cur, size_t bytes, cudaStream_t st) {
  if (*cur >= bytes && *buf) return FS_OK;
  if (*buf) {
    if (cudaStreamSynchronize(st) != cudaSuccess) return FS_ERR_CUDA;
    cudaFree(*buf);
    *buf = nullptr;
    *cur = 0;
  }
  void *p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return FS_ERR_NOMEM;
  }
  *buf = p;
  *cur = bytes;
  return FS_OK;
}
}  // namespace fs

static inline cudaStream_t as_stream(void *s) { return (cudaStream_t)s; }

static bool is_pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }

static std::atomic<uint64_t> g_seg_serial{0};

// Orbital and sidereal angles at the epoch t0 of a segment's first sample (Sec. V).
static void set_epoch(const fs_detector &det, double t0, SegGeom *g) {
  g->theta0 = fmod(det.theta_g0 + det.lon + fmod(kOmegaR * t0, kTwoPi), kTwoPi);
  g->lambda0 = fmod(det.lambda_e0 + fmod(kOmegaO * t0, kTwoPi), kTwoPi);
}

extern "C" {

const char *fs_strerror(fs_status s) {
  switch (s) {
    case FS_OK: return "ok";
    case FS_ERR_ARG: return "invalid argument";
    case FS_ERR_SHAPE: return "unsupported shape (n, nfft, nbins)";
    case FS_ERR_CAPACITY: return "candidate buffer overflow";
    case FS_ERR_NONFINITE: return "non-finite value in the data";
    case FS_ERR_CUDA: return "CUDA runtime error";
    case FS_ERR_TIMEOUT: return "device-side wait timed out";
    case FS_ERR_UNSUPPORTED: return "unsupported request";
    case FS_ERR_NOMEM: return "device allocation failed";
    case FS_ERR_SCRATCH: return "request exceeds the fixed scratch array of fs_search_noalloc";
    case FS_ERR_CORRUPT: return "debug build: an index outside its buffer or an overwritten guard word";
  }
  return "unknown status";
}

fs_status fs_create(fs_ctx **ctx, const fs_detector *det, int32_t device) {
  if (!ctx || !det) return FS_ERR_ARG;
  *ctx = nullptr;
  if (cudaSetDevice(device) != cudaSuccess) { cudaGetLastError(); return FS_ERR_CUDA; }
  fs_ctx *c = new (std::nothrow) fs_ctx();
  if (!c) return FS_ERR_NOMEM;
  c->device = device;
  c->det = *det;
  if (cudaMalloc(&c->d_flags, sizeof(uint32_t)) != cudaSuccess) { delete c; cudaGetLastError(); return FS_ERR_NOMEM; }
  if (cudaMemset(c->d_flags, 0, sizeof(uint32_t)) != cudaSuccess) { cudaFree(c->d_flags); delete c; return FS_ERR_CUDA; }
  if (noalloc_address(&c->noalloc) != FS_OK) { cudaFree(c->d_flags); delete c; return FS_ERR_CUDA; }
  const char *bt = getenv("FSTAT_BATCH_TEMPLATES");
  if (bt && atoi(bt) > 0) c->batch_templates = atoi(bt);
  const char *gs = getenv("FSTAT_GROUP_SKIES");
  if (gs && atoi(gs) > 0) c->group_skies = atoi(gs);
  const char *pk = getenv("FSTAT_PERSISTENT");
  if (pk) c->persistent = atoi(pk) != 0;
  const char *lg = getenv("FSTAT_QUEUE_LAG");
  if (lg && atoi(lg) > 0) c->queue_lag = atoi(lg);
  const char *zs = getenv("FSTAT_Z_SLOTS");
  if (zs && atoi(zs) > 1) c->z_slots = atoi(zs);
  const char *qr = getenv("FSTAT_QUEUE_ROUND");
  if (qr && atoi(qr) > 0) c->queue_round = atoi(qr);

  *ctx = c;
  return FS_OK;
}

static void seg_release(fs_seg *s) {
  cudaFree(s->tab0);
  cudaFree(s->tab1);
  cudaFree(s->x64);
  cudaFree(s->x32);
  cudaFree(s->x2);
  cudaFree(s->coef);
  cudaFree(s->blu_bhat);
  cudaFree(s->blu_tw);
  cudaFree(s->blu_chirp);
  cudaFree(s->etab64);
  cudaFree(s->etab32);
  cudaFree(s->eph);
  cudaFree(s->eph0);
  cudaFree(s->eph1);
  cudaFree(s->eph2);
  delete s;
}

void fs_destroy(fs_ctx *ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  for (fs_seg *s : ctx->segs) seg_release(s);
  ctx->segs.clear();
  batch_plan_release(ctx);
  for (int i = 0; i < 2; i++) {
    if (ctx->side[i]) cudaStreamDestroy(ctx->side[i]);
    if (ctx->join[i]) cudaEventDestroy(ctx->join[i]);
  }
  if (ctx->fork) cudaEventDestroy(ctx->fork);
  cudaFree(ctx->d_flags);
  for (int i = 0; i < fs_ctx::kWsSlots; i++) cudaFree(ctx->ws[i]);
  cudaFree(ctx->ws64);
  cudaFree(ctx->rws);
  cudaFree(ctx->aws);
  cudaFree(ctx->scratch);
  for (cudaEvent_t e : ctx->evpool) cudaEventDestroy(e);
  delete ctx;
}

// Both preparation entry points: r, v NULL for the analytic Earth, else the
// caller's position table (copied before the first load builds the tables).
static fs_status prepare_segment(fs_ctx *ctx, fs_seg **seg, const fs_segment_desc *d, const void *x_dev,
                                 const double *r_eph, const double *v_eph, void *stream) {
  if (!ctx || !seg || !d || !x_dev) return FS_ERR_ARG;
  *seg = nullptr;
  if (d->n < 16 || !(d->dt > 0.0) || !(d->S0 > 0.0) || !isfinite(d->fl) || !isfinite(d->dt)) return FS_ERR_ARG;
  if (d->precision != FS_PREC_F32 && d->precision != FS_PREC_F64) return FS_ERR_ARG;
  if (d->interp != FS_INTERP_SPLINE2X && d->interp != FS_INTERP_NEAREST) return FS_ERR_ARG;
  if (d->x_dtype != FS_X_F32 && d->x_dtype != FS_X_F64) return FS_ERR_ARG;
  if ((d->options & ~FS_OPT_INTERBIN) != 0 || !isfinite(d->t0)) return FS_ERR_ARG;
  if ((d->options & FS_OPT_INTERBIN) && d->precision == FS_PREC_F32 && d->nfft > (int64_t(1) << 20))
    return FS_ERR_SHAPE;
  if (!is_pow2(d->nfft) || d->nfft < d->n || d->nfft < 4096 || d->nfft > (int64_t(1) << 21)) return FS_ERR_SHAPE;
  // the FP32 path splits a 2^21 transform into two 2^20 ones: the data must fit one
  if (d->precision == FS_PREC_F32 && d->nfft > (int64_t(1) << 20) && d->n > (int64_t(1) << 20)) return FS_ERR_SHAPE;
  if (d->n > (int64_t(1) << 28)) return FS_ERR_SHAPE;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return FS_ERR_CUDA;
  cudaStream_t st = as_stream(stream);

  fs_seg *s = new (std::nothrow) fs_seg();
  if (!s) return FS_ERR_NOMEM;
  s->ctx = ctx;
  s->serial = ++g_seg_serial;
  s->d = *d;
  SegGeom &g = s->g;
  g.n = d->n;
  g.nfft = d->nfft;
  g.dt = d->dt;
  g.fl = d->fl;
  g.S0 = d->S0;
  g.margin = (int64_t)ceil((r_eph ? kMaxDelayEph : kMaxDelay) / d->dt) + 4;
  g.ngrid = g.n + 2 * g.margin;
  set_epoch(ctx->det, d->t0, &g);
  double re, z;
  site_radius(ctx->det.lat, &re, &z);
  g.re_c = re / kC;
  g.z_c = z / kC;

  const int64_t n = g.n;
  bool ok = cudaMalloc(&s->x64, sizeof(double) * n) == cudaSuccess &&
            cudaMalloc(&s->x32, sizeof(float) * n) == cudaSuccess &&
            cudaMalloc(&s->x2, sizeof(double) * 2 * n) == cudaSuccess;
  if (ok && d->precision == FS_PREC_F32) {
    ok = cudaMalloc(&s->tab0, sizeof(float4) * g.ngrid) == cudaSuccess &&
         cudaMalloc(&s->tab1, sizeof(float4) * g.ngrid) == cudaSuccess &&
         cudaMalloc(&s->coef, sizeof(float4) * 2 * n) == cudaSuccess;
  } else if (ok) {
    ok = cudaMalloc(&s->coef, sizeof(dcoef4) * 2 * n) == cudaSuccess;
  }
  if (ok && r_eph) {
    ok = cudaMalloc(&s->eph, sizeof(dbl4) * 2 * n) == cudaSuccess;
    if (ok && d->precision == FS_PREC_F32)
      ok = cudaMalloc(&s->eph0, sizeof(float4) * g.ngrid) == cudaSuccess &&
           cudaMalloc(&s->eph1, sizeof(float4) * g.ngrid) == cudaSuccess &&
           cudaMalloc(&s->eph2, sizeof(float) * g.ngrid) == cudaSuccess;
  }
  if (!ok) {
    cudaGetLastError();
    seg_release(s);
    return FS_ERR_NOMEM;
  }
  ctx->segs.insert(s);
  fs_status r = r_eph ? import_eph(s, r_eph, v_eph, st) : FS_OK;
  if (r == FS_OK) r = fs_seg_load(s, x_dev, stream);
  if (r != FS_OK) {
    fs_seg_destroy(s);
    return r;
  }
  *seg = s;
  return FS_OK;
}

fs_status fs_prepare_segment(fs_ctx *ctx, fs_seg **seg, const fs_segment_desc *d, const void *x_dev,
                             void *stream) {
  return prepare_segment(ctx, seg, d, x_dev, nullptr, nullptr, stream);
}

fs_status fs_prepare_segment_eph(fs_ctx *ctx, fs_seg **seg, const fs_segment_desc *d, const void *x_dev,
                                 const double *r_dev, const double *v_dev, void *stream) {
  if (!r_dev || !v_dev) return FS_ERR_ARG;
  return prepare_segment(ctx, seg, d, x_dev, r_dev, v_dev, stream);
}

fs_status fs_seg_load(fs_seg *s, const void *x_dev, void *stream) {
  if (!s || !x_dev) return FS_ERR_ARG;
  if (cudaSetDevice(s->ctx->device) != cudaSuccess) return FS_ERR_CUDA;
  cudaStream_t st = as_stream(stream);
  NvtxRange nv("fs.prepare");
  ProfScope ps(s->ctx, PROF_PREP, st);
  fs_status r = FS_OK;
  if (s->d.precision == FS_PREC_F32) r = prepare_tables(s, st);
  if (r == FS_OK) r = prepare_upsample(s, x_dev, st);
  if (r == FS_OK) r = prepare_spline(s, st);
  return r;
}

void fs_seg_destroy(fs_seg *s) {
  if (!s) return;
  fs_ctx *ctx = s->ctx;
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  ctx->segs.erase(s);
  seg_release(s);
}

fs_status fs_search(fs_ctx *ctx, fs_seg *seg, const double *alpha_dev, const double *delta_dev, int32_t nsky,
                    const double *f1_dev, int32_t nspin, float F_thr, void *F_out_dev, int64_t nbins,
                    fs_candidate *cand_dev, int64_t cand_cap, int64_t *n_cand_dev, void *stream) {
  if (!ctx || !seg || !alpha_dev || !delta_dev || !f1_dev || !n_cand_dev) return FS_ERR_ARG;
  if (seg->ctx != ctx) return FS_ERR_ARG;
  if (nsky < 1 || nspin < 1 || cand_cap < 0 || (cand_cap > 0 && !cand_dev)) return FS_ERR_ARG;
  if (seg->d.options & FS_OPT_INTERBIN) {
    if (nbins != seg->g.nfft) return FS_ERR_SHAPE;
  } else if (!(nbins == seg->g.nfft / 2 || nbins == seg->g.nfft)) {
    return FS_ERR_SHAPE;
  }
  if ((int64_t)nsky * nspin > (int64_t)1 << 31) return FS_ERR_SHAPE;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return FS_ERR_CUDA;
  cudaStream_t st = as_stream(stream);
  NvtxRange nv("fs.search");
  if (seg->d.precision == FS_PREC_F32)
    return search32(ctx, seg, alpha_dev, delta_dev, nsky, f1_dev, nspin, F_thr, (float *)F_out_dev, nbins,
                    cand_dev, cand_cap, n_cand_dev, st);
  return search64(ctx, seg, alpha_dev, delta_dev, nsky, f1_dev, nspin, F_thr, (double *)F_out_dev, nbins,
                  cand_dev, cand_cap, n_cand_dev, st);
}

fs_status fs_selftest_wait(fs_ctx *ctx, void *stream) {
  if (!ctx) return FS_ERR_ARG;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return FS_ERR_CUDA;
  ctx->launches++;
  return cuda_status(selftest_wait(ctx->d_flags, as_stream(stream)));
}

fs_status fs_search_lattice(fs_ctx *ctx, fs_seg *seg, const double *alpha_dev, const double *delta_dev,
                            int32_t nsky, const double *f1_dev, const double *offset_dev, int32_t nspin, float F_thr,
                            void *F_out_dev, int64_t nbins, fs_candidate *cand_dev, int64_t cand_cap,
                            int64_t *n_cand_dev, void *stream) {
  if (!ctx || !seg || !alpha_dev || !delta_dev || !f1_dev || !offset_dev || !n_cand_dev) return FS_ERR_ARG;
  if (seg->ctx != ctx) return FS_ERR_ARG;
  if (nsky < 1 || nspin < 1 || cand_cap < 0 || (cand_cap > 0 && !cand_dev)) return FS_ERR_ARG;
  if ((int64_t)nsky * nspin > (int64_t)1 << 31) return FS_ERR_SHAPE;
  if ((seg->d.options & FS_OPT_INTERBIN) || nbins != seg->g.nfft / 2) return FS_ERR_UNSUPPORTED;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return FS_ERR_CUDA;
  if (seg->d.precision == FS_PREC_F64)
    return search64(ctx, seg, alpha_dev, delta_dev, nsky, f1_dev, nspin, F_thr, (double *)F_out_dev, nbins,
                    cand_dev, cand_cap, n_cand_dev, as_stream(stream), offset_dev);
  return search32_lattice(ctx, seg, alpha_dev, delta_dev, nsky, f1_dev, offset_dev, nspin, F_thr,
                          (float *)F_out_dev, nbins, cand_dev, cand_cap, n_cand_dev, as_stream(stream));
}

fs_status fs_search_noalloc(fs_ctx *ctx, fs_seg *seg, const double *alpha_dev, const double *delta_dev,
                            int32_t nsky, const double *f1_dev, int32_t nspin, float F_thr, float *F_out_dev,
                            int64_t nbins, fs_candidate *cand_dev, int64_t cand_cap, int64_t *n_cand_dev,
                            void *stream) {
  if (!ctx || !seg || !alpha_dev || !delta_dev || !f1_dev || !n_cand_dev) return FS_ERR_ARG;
  if (seg->ctx != ctx) return FS_ERR_ARG;
  if (nsky < 1 || nspin < 1 || cand_cap < 0 || (cand_cap > 0 && !cand_dev)) return FS_ERR_ARG;
  if ((int64_t)nsky * nspin > (int64_t)1 << 31) return FS_ERR_SHAPE;
  if (seg->d.options & FS_OPT_INTERBIN) return FS_ERR_UNSUPPORTED;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return FS_ERR_CUDA;
  NvtxRange nv("fs.search_noalloc");
  return search32_noalloc(ctx, seg, alpha_dev, delta_dev, nsky, f1_dev, nspin, F_thr, F_out_dev, nbins, cand_dev,
                          cand_cap, n_cand_dev, as_stream(stream));
}

fs_status fs_search_lattice_noalloc(fs_ctx *ctx, fs_seg *seg, const double *alpha_dev, const double *delta_dev,
                                    int32_t nsky, const double *f1_dev, const double *offset_dev, int32_t nspin,
                                    float F_thr, float *F_out_dev, int64_t nbins, fs_candidate *cand_dev,
                                    int64_t cand_cap, int64_t *n_cand_dev, void *stream) {
  if (!ctx || !seg || !alpha_dev || !delta_dev || !f1_dev || !offset_dev || !n_cand_dev) return FS_ERR_ARG;
  if (seg->ctx != ctx) return FS_ERR_ARG;
  if (nsky < 1 || nspin < 1 || cand_cap < 0 || (cand_cap > 0 && !cand_dev)) return FS_ERR_ARG;
  if ((int64_t)nsky * nspin > (int64_t)1 << 31) return FS_ERR_SHAPE;
  if (seg->d.options & FS_OPT_INTERBIN) return FS_ERR_UNSUPPORTED;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return FS_ERR_CUDA;
  NvtxRange nv("fs.search_lattice_noalloc");
  return search32_noalloc(ctx, seg, alpha_dev, delta_dev, nsky, f1_dev, nspin, F_thr, F_out_dev, nbins, cand_dev,
                          cand_cap, n_cand_dev, as_stream(stream), offset_dev);
}

fs_status fs_search_batch(fs_ctx *ctx, fs_seg *const *segs, int32_t nseg, const double *alpha_dev,
                          const double *delta_dev, int32_t nsky, const double *f1_dev, int32_t nspin, float F_thr,
                          fs_candidate *cand_dev, int64_t cand_cap, int64_t *n_cand_dev, void *stream) {
  if (!ctx || !segs || nseg < 1 || !alpha_dev || !delta_dev || !f1_dev || !n_cand_dev) return FS_ERR_ARG;
  if (nsky < 1 || nspin < 1 || cand_cap < 0 || (cand_cap > 0 && !cand_dev)) return FS_ERR_ARG;
  if ((int64_t)nsky * nspin > (int64_t)1 << 31) return FS_ERR_SHAPE;
  for (int i = 0; i < nseg; i++) {
    if (!segs[i] || segs[i]->ctx != ctx || segs[i]->d.precision != FS_PREC_F32) return FS_ERR_ARG;
  }
  if (cudaSetDevice(ctx->device) != cudaSuccess) return FS_ERR_CUDA;
  NvtxRange nv("fs.search_batch");
  return search32_batch(ctx, segs, nseg, alpha_dev, delta_dev, nsky, f1_dev, nspin, F_thr, cand_dev, cand_cap,
                        n_cand_dev, as_stream(stream));
}

fs_status fs_search_lattice_batch(fs_ctx *ctx, fs_seg *const *segs, int32_t nseg, const double *const *alpha_dev,
                                  const double *const *delta_dev, const int32_t *nsky, const double *const *f1_dev,
                                  const double *const *offset_dev, const int32_t *nspin, float F_thr,
                                  fs_candidate *cand_dev, int64_t cand_cap, int64_t *n_cand_dev, void *stream) {
  if (!ctx || !segs || nseg < 1 || !alpha_dev || !delta_dev || !nsky || !f1_dev || !offset_dev || !nspin ||
      !n_cand_dev)
    return FS_ERR_ARG;
  if (cand_cap < 0 || (cand_cap > 0 && !cand_dev)) return FS_ERR_ARG;
  for (int i = 0; i < nseg; i++) {
    if (!segs[i] || segs[i]->ctx != ctx || segs[i]->d.precision != FS_PREC_F32) return FS_ERR_ARG;
    if (!alpha_dev[i] || !delta_dev[i] || !f1_dev[i] || !offset_dev[i] || nsky[i] < 1 || nspin[i] < 1)
      return FS_ERR_ARG;
    if ((int64_t)nsky[i] * nspin[i] > (int64_t)1 << 31) return FS_ERR_SHAPE;
    if (segs[i]->d.options & FS_OPT_INTERBIN) return FS_ERR_UNSUPPORTED;
  }
  if (cudaSetDevice(ctx->device) != cudaSuccess) return FS_ERR_CUDA;
  return search32_lattice_batch(ctx, segs, nseg, alpha_dev, delta_dev, nsky, f1_dev, offset_dev, nspin, F_thr,
                                cand_dev, cand_cap, n_cand_dev, as_stream(stream));
}

static int tune_index(int64_t nfft) {
  if (!is_pow2(nfft) || nfft < 4096 || nfft > (int64_t(1) << 21)) return -1;
  int p = 0;
  while (((int64_t)1 << p) < nfft) p++;
  return p;
}

fs_status fs_set_tuning(fs_ctx *ctx, int64_t nfft, const fs_tuning *t) {
  if (!ctx) return FS_ERR_ARG;
  const int p = tune_index(nfft);
  if (p < 0) return FS_ERR_SHAPE;
  if (!t) {
    ctx->tuned[p] = false;
    ctx->tune[p] = fs_tuning{};
  } else {
    if (!tuning_valid(nfft, *t)) return FS_ERR_ARG;
    ctx->tune[p] = *t;
    ctx->tune[p].ms_per_template = 0.f;
    ctx->tuned[p] = true;
  }
  ctx->tune_version++;
  return FS_OK;
}

fs_status fs_get_tuning(fs_ctx *ctx, int64_t nfft, fs_tuning *out) {
  if (!ctx || !out) return FS_ERR_ARG;
  const int p = tune_index(nfft);
  if (p < 0) return FS_ERR_SHAPE;
  if (!ctx->tuned[p]) return FS_ERR_UNSUPPORTED;
  *out = ctx->tune[p];
  return FS_OK;
}

fs_status fs_autotune(fs_ctx *ctx, fs_seg *seg, const double *alpha_dev, const double *delta_dev, int32_t nsky,
                      const double *f1_dev, int32_t nspin, int32_t reps, fs_tuning *out, void *stream) {
  if (!ctx || !seg || !alpha_dev || !delta_dev || !f1_dev || !out) return FS_ERR_ARG;
  if (seg->ctx != ctx || seg->d.precision != FS_PREC_F32) return FS_ERR_ARG;
  if (nsky < 1 || nspin < 1 || reps < 1 || reps > 100) return FS_ERR_ARG;
  if ((int64_t)nsky * nspin > (int64_t)1 << 31) return FS_ERR_SHAPE;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return FS_ERR_CUDA;
  return autotune32(ctx, seg, alpha_dev, delta_dev, nsky, f1_dev, nspin, reps, out, as_stream(stream));
}

fs_status fs_fstat_points(fs_ctx *ctx, fs_seg *seg, const fs_point *pts_dev, int32_t npt, double *F_dev,
                          double *grad_dev, double *hess_dev, double *metric_dev, void *stream) {
  if (!ctx || !seg || !pts_dev || !F_dev || seg->ctx != ctx) return FS_ERR_ARG;
  if (npt < 1) return FS_ERR_ARG;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return FS_ERR_CUDA;
  NvtxRange nv("fs.fstat_points");
  return fstat_points(ctx, seg, pts_dev, npt, F_dev, grad_dev, hess_dev, metric_dev, as_stream(stream));
}

fs_status fs_fstat_resampled(fs_ctx *ctx, fs_seg *seg, const fs_point *pts_dev, int32_t npt, double *F_dev,
                             void *stream) {
  if (!ctx || !seg || !pts_dev || !F_dev || seg->ctx != ctx || npt < 1) return FS_ERR_ARG;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return FS_ERR_CUDA;
  NvtxRange nv("fs.fstat_resampled");
  return fstat_resampled(ctx, seg, pts_dev, npt, nullptr, F_dev, nullptr, as_stream(stream));
}

fs_status fs_fstat_resampled_grad(fs_ctx *ctx, fs_seg *seg, const fs_point *pts_dev, int32_t npt,
                                  const double *gF_dev, double *F_dev, double *grad_dev, void *stream) {
  if (!ctx || !seg || !pts_dev || !grad_dev || seg->ctx != ctx || npt < 1) return FS_ERR_ARG;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return FS_ERR_CUDA;
  NvtxRange nv("fs.fstat_resampled_grad");
  return fstat_resampled(ctx, seg, pts_dev, npt, gF_dev, F_dev, grad_dev, as_stream(stream));
}

fs_status fs_refine_resampled(fs_ctx *ctx, fs_seg *seg, fs_point *pts_dev, int32_t npt, int32_t nsteps,
                              double *F_dev, void *stream) {
  if (!ctx || !seg || !pts_dev || !F_dev || seg->ctx != ctx) return FS_ERR_ARG;
  if (npt < 1 || nsteps < 0 || nsteps > 10000) return FS_ERR_ARG;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return FS_ERR_CUDA;
  NvtxRange nv("fs.refine_resampled");
  return refine_resampled(ctx, seg, pts_dev, npt, nsteps, F_dev, as_stream(stream));
}

fs_status fs_refine(fs_ctx *ctx, fs_seg *seg, fs_point *pts_dev, int32_t npt, int32_t nsteps, double *F_dev,
                    void *stream) {
  if (!ctx || !seg || !pts_dev || !F_dev || seg->ctx != ctx) return FS_ERR_ARG;
  if (npt < 1 || nsteps < 0 || nsteps > 10000) return FS_ERR_ARG;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return FS_ERR_CUDA;
  NvtxRange nv("fs.refine");
  return refine_points(ctx, seg, pts_dev, npt, nsteps, F_dev, as_stream(stream));
}

fs_status fs_points_from_candidates(fs_ctx *ctx, fs_seg *seg, const fs_candidate *cand_dev, int32_t n,
                                    const double *alpha_dev, const double *delta_dev, const double *f1_dev,
                                    fs_point *pts_dev, void *stream) {
  if (!ctx || !seg || !cand_dev || !alpha_dev || !delta_dev || !f1_dev || !pts_dev || seg->ctx != ctx)
    return FS_ERR_ARG;
  if (n < 1) return FS_ERR_ARG;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return FS_ERR_CUDA;
  return points_from_candidates(ctx, seg, cand_dev, n, alpha_dev, delta_dev, f1_dev, pts_dev, as_stream(stream));
}

fs_status fs_amplitudes(fs_ctx *ctx, fs_seg *seg, const fs_point *pts_dev, int32_t npt, double *amp_dev,
                        void *stream) {
  if (!ctx || !seg || !pts_dev || !amp_dev || seg->ctx != ctx || npt < 1) return FS_ERR_ARG;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return FS_ERR_CUDA;
  return amplitudes(ctx, seg, pts_dev, npt, amp_dev, as_stream(stream));
}

fs_status fs_sync_status(fs_ctx *ctx, void *stream) {
  if (!ctx) return FS_ERR_ARG;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return FS_ERR_CUDA;
  if (cudaStreamSynchronize(as_stream(stream)) != cudaSuccess) { cudaGetLastError(); return FS_ERR_CUDA; }
  if (cudaGetLastError() != cudaSuccess) return FS_ERR_CUDA;
  uint32_t f = 0;
  if (cudaMemcpy(&f, ctx->d_flags, sizeof(f), cudaMemcpyDeviceToHost) != cudaSuccess) return FS_ERR_CUDA;
  if (f) cudaMemset(ctx->d_flags, 0, sizeof(uint32_t));
  if (f & ERRF_CORRUPT) return FS_ERR_CORRUPT;
  if (f & ERRF_TIMEOUT) return FS_ERR_TIMEOUT;
  if (f & ERRF_NONFINITE) return FS_ERR_NONFINITE;
  if (f & ERRF_CAPACITY) return FS_ERR_CAPACITY;
  return FS_OK;
}

fs_status fs_set_profiling(fs_ctx *ctx, int32_t on) {
  if (!ctx) return FS_ERR_ARG;
  ctx->prof = on != 0;
  return FS_OK;
}

fs_status fs_get_stats(fs_ctx *ctx, fs_stats *out, int32_t reset) {
  if (!ctx || !out) return FS_ERR_ARG;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return FS_ERR_CUDA;
  if (cudaDeviceSynchronize() != cudaSuccess) return FS_ERR_CUDA;
  memset(out, 0, sizeof(*out));
  out->launches = ctx->launches;
  int64_t wb = (int64_t)(ctx->ws64_bytes + ctx->scratch_bytes + ctx->rws_bytes + ctx->aws_bytes);
  for (int i = 0; i < fs_ctx::kWsSlots; i++) wb += (int64_t)ctx->ws_bytes[i];
  out->workspace_bytes = wb;
  for (const auto &r : ctx->recs) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) return FS_ERR_CUDA;
    out->ms[r.kind] += ms;
    out->count[r.kind] += 1;
  }
  if (reset) {
    ctx->launches = 0;
    ctx->recs.clear();
    ctx->ev_used = 0;
  }
  return FS_OK;
}

fs_status fs_seg_upsampled(const fs_seg *seg, double *x2_dev, void *stream) {
  if (!seg || !x2_dev) return FS_ERR_ARG;
  return cuda_status(cudaMemcpyAsync(x2_dev, seg->x2, sizeof(double) * 2 * seg->g.n, cudaMemcpyDeviceToDevice,
                                     as_stream(stream)));
}

fs_status fs_demodulate(fs_ctx *ctx, fs_seg *seg, double alpha, double delta, double *ya_dev, double *yb_dev,
                        double *tsrc_dev, double *ab2_dev, void *stream) {
  if (!ctx || !seg || !ya_dev || !yb_dev || !tsrc_dev || !ab2_dev) return FS_ERR_ARG;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return FS_ERR_CUDA;
  if (seg->d.precision == FS_PREC_F32)
    return demod32_debug(ctx, seg, alpha, delta, ya_dev, yb_dev, tsrc_dev, ab2_dev, as_stream(stream));
  return demod64_debug(ctx, seg, alpha, delta, ya_dev, yb_dev, tsrc_dev, ab2_dev, as_stream(stream));
}

fs_status fs_inject(fs_ctx *ctx, double *x_dev, int64_t n, double dt, double fl, double sigma, double t0,
                    const fs_injection *inj_host, int32_t n_inj, void *stream) {
  if (!ctx || !x_dev || n < 1 || !(dt > 0.0) || !(sigma > 0.0) || n_inj < 0 || (n_inj > 0 && !inj_host))
    return FS_ERR_ARG;
  if (!isfinite(t0)) return FS_ERR_ARG;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return FS_ERR_CUDA;
  SegGeom g{};
  set_epoch(ctx->det, t0, &g);
  return inject64(ctx, x_dev, n, dt, fl, sigma, g.theta0, g.lambda0, inj_host, n_inj, as_stream(stream));
}

}  // extern "C"
