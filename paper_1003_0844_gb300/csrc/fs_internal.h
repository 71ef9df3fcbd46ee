// Host-side internals shared by the translation units of the library.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <unordered_set>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "fs_common.cuh"

struct fs_ctx {
  int device = 0;
  fs_detector det{};
  uint32_t *d_flags = nullptr;       // latched device error bits
  // FP32 search workspaces (grown on demand): slot 0 serves fs_search and
  // fs_autotune, slots 1 and 2 the two concurrent branches of fs_search_batch
  static constexpr int kWsSlots = 3;
  void *ws[kWsSlots] = {};
  size_t ws_bytes[kWsSlots] = {};
  // FP64 search workspace
  size_t ws64_bytes = 0;
  void *ws64 = nullptr;
  // scratch for stage access / injection
  size_t scratch_bytes = 0;
  void *scratch = nullptr;
  // fine-search workspace
  size_t rws_bytes = 0;
  void *rws = nullptr;
  // workspace of the resampled F at continuous points (fs_adjoint.cu)
  size_t aws_bytes = 0;
  void *aws = nullptr;
  // device address of the fixed array of the allocation-free searches, looked up
  // for this context by fs_create (the address belongs to the device's context)
  unsigned char *noalloc = nullptr;
  // tuning knobs (templates per batch, skies per group)
  int batch_templates = 16;
  int group_skies = 256;
  bool persistent = true;  // both transform passes in one persistent launch per sky group
  // persistent-queue shape; 0 = automatic (a round's pass-1 items fill ~85% of the
  // resident CTAs, pass 2 one round behind, a ring of three rounds)
  int queue_lag = 0;       // rounds between a template's pass-1 and pass-2 items
  int z_slots = 0;         // Z ring slots (each 2 x Nfft complex floats)
  int queue_round = 0;     // templates per queue round
  // launch configuration per transform length 2^p (fs_set_tuning / fs_autotune)
  fs_tuning tune[32] = {};
  bool tuned[32] = {};
  uint64_t tune_version = 0;
  // fs_search_batch: the captured graph and what it was captured for
  struct BatchPlan *plan = nullptr;
  cudaStream_t side[2] = {nullptr, nullptr};
  cudaEvent_t fork = nullptr, join[2] = {nullptr, nullptr};
  // live segments of this context (fs_destroy releases those still alive)
  std::unordered_set<fs_seg *> segs;
  // launch accounting and optional event profiling
  int64_t launches = 0;
  bool prof = false;
  std::vector<cudaEvent_t> evpool;
  size_t ev_used = 0;
  struct Rec { int kind; cudaEvent_t a, b; };
  std::vector<Rec> recs;
};

struct fs_seg {
  fs_ctx *ctx = nullptr;
  uint64_t serial = 0;      // unique per segment in the process (keys captured graphs)
  fs_segment_desc d{};
  fs::SegGeom g{};
  // FP32 path tables on the grid t_m = m dt, m in [-margin, n + margin):
  //   tab0[m] = (C.hi, C.lo, S.hi, S.lo) with C, S = (AU/c) (cos, sin) lambda_E(t_m)
  //   tab1[m] = (cos theta_m, sin theta_m, t_m.hi, t_m.lo)
  float4 *tab0 = nullptr, *tab1 = nullptr;
  bool tables_ready = false;  // built by the first load (they do not depend on the data)
  double *x64 = nullptr;    // input as double [n]
  float *x32 = nullptr;     // input as float [n] (nearest-neighbour path)
  double *x2 = nullptr;     // Fourier x2 upsampled [2n]
  void *coef = nullptr;     // spline coefficients per interval: float4 or double[4] x [2n]
  // Upsampler plan (depends on n only), built by the first load: transform length
  // m >= 2n - 1, the FFT twiddles, the Bluestein chirp and half-sample shift [2n];
  // blu_bhat holds the chirp's spectrum while the plan runs one Bluestein DFT, then
  // the spectrum of the interpolation kernel.  Computed in FP64, held as
  // double-floats (float4 per complex value, the same 16 bytes).
  int64_t blu_m = 0;
  double2 *blu_bhat = nullptr, *blu_tw = nullptr;
  double2 *blu_chirp = nullptr;
  // FP64 (cos, sin) of the orbital and sidereal angles on t_k = k dt, built by
  // the first fine-search call
  void *etab64 = nullptr;
  // the same angles and the data as double-floats, with the 257-entry table of
  // exp(-2 pi i j / 256), for the fine search's double-float kernels (same call)
  void *etab32 = nullptr;
  // caller's position table (fs_prepare_segment_eph), else NULL:
  //   eph[2m] = (r_m, 0), eph[2m + 1] = (v_m, 0), m < n (light-seconds, SSB ecliptic frame)
  fs::dbl4 *eph = nullptr;
  // its FP32-path form on the grid t_m, m in [-margin, n + margin) (clamped linear extrapolation):
  //   eph0[m] = (r_x.hi, r_x.lo, r_y.hi, r_y.lo), eph1[m] = (r_z.hi, r_z.lo, v_x, v_y), eph2[m] = v_z
  float4 *eph0 = nullptr, *eph1 = nullptr;
  float *eph2 = nullptr;
};

// ---- launchers implemented in the .cu files (all asynchronous on `st`) ----
namespace fs {

inline fs_status cuda_status(cudaError_t e) { return e == cudaSuccess ? FS_OK : FS_ERR_CUDA; }

// FP64 radix-2 Stockham FFT of `batch` contiguous sequences of length n
// (power of two) in place in `buf` using `tmp` as ping-pong space.
// sign = -1 forward (exp(-2 pi i ...)), +1 inverse (unnormalised).
cudaError_t fft64(double2 *buf, double2 *tmp, const double2 *twiddle, int64_t n, int batch,
                  int sign, cudaStream_t st, int64_t *launches);
// twiddle[q] = exp(-2 pi i q / n), q < n/2
cudaError_t fft64_twiddles(double2 *tw, int64_t n, cudaStream_t st);
// The same transform in double-float arithmetic: complex values as float4
// (re.hi, re.lo, im.hi, im.lo), twiddle[q] = exp(-2 pi i q / n) likewise (to_df32 of
// the FP64 table).  to_df32 converts n double2 to float4 (in place when out == in).
cudaError_t fftdf(float4 *buf, float4 *tmp, const float4 *twiddle, int64_t n, int batch, int sign, cudaStream_t st,
                  int64_t *launches);
cudaError_t to_df32(const double2 *in, float4 *out, int64_t n, cudaStream_t st);

// Segment preparation (P0 tables, P1 upsampling, P2 spline).
fs_status prepare_tables(fs_seg *seg, cudaStream_t st);
// Copy a caller's position table (component-major r, v, 3 x n each) into seg->eph.
fs_status import_eph(fs_seg *seg, const double *r, const double *v, cudaStream_t st);
fs_status prepare_upsample(fs_seg *seg, const void *x_dev, cudaStream_t st);
fs_status prepare_spline(fs_seg *seg, cudaStream_t st);

// Per-sky constants from alpha/delta device arrays.
cudaError_t sky_constants32(const double *alpha, const double *delta, int nsky, const fs::SegGeom &g,
                            const fs_detector &det, SkyConst32 *out, cudaStream_t st);
cudaError_t sky_constants64(const double *alpha, const double *delta, int nsky, const fs::SegGeom &g,
                            const fs_detector &det, SkyConst64 *out, cudaStream_t st);

// Searches.
fs_status search32(fs_ctx *ctx, fs_seg *seg, const double *alpha, const double *delta, int nsky,
                   const double *f1, int nspin, float thr, float *F, int64_t nbins,
                   fs_candidate *cand, int64_t cap, int64_t *ncand, cudaStream_t st);
fs_status search64(fs_ctx *ctx, fs_seg *seg, const double *alpha, const double *delta, int nsky,
                   const double *f1, int nspin, float thr, double *F, int64_t nbins,
                   fs_candidate *cand, int64_t cap, int64_t *ncand, cudaStream_t st,
                   const double *offset = nullptr);
// One bounded wait on a counter nothing increments (fs_selftest_wait).
cudaError_t selftest_wait(uint32_t *flags, cudaStream_t st);
// Coarse search of lattice templates (fs_search_lattice): f1 and the bin offset per template.
fs_status search32_lattice(fs_ctx *ctx, fs_seg *seg, const double *alpha, const double *delta, int nsky,
                           const double *f1, const double *offset, int nspin, float thr, float *F, int64_t nbins,
                           fs_candidate *cand, int64_t cap, int64_t *ncand, cudaStream_t st);
// Device address of the fixed array of the allocation-free searches (no allocation;
// called by fs_create with the context's device current).
fs_status noalloc_address(unsigned char **addr);
fs_status search32_noalloc(fs_ctx *ctx, fs_seg *seg, const double *alpha, const double *delta, int nsky,
                           const double *f1, int nspin, float thr, float *F, int64_t nbins, fs_candidate *cand,
                           int64_t cap, int64_t *ncand, cudaStream_t st, const double *offset = nullptr);
fs_status demod32_debug(fs_ctx *ctx, fs_seg *seg, double alpha, double delta, double *ya, double *yb,
                        double *tsrc, double *ab2, cudaStream_t st);
fs_status demod64_debug(fs_ctx *ctx, fs_seg *seg, double alpha, double delta, double *ya, double *yb,
                        double *tsrc, double *ab2, cudaStream_t st);
fs_status inject64(fs_ctx *ctx, double *x, int64_t n, double dt, double fl, double sigma, double theta0,
                   double lambda0, const fs_injection *inj, int n_inj, cudaStream_t st);

// Event profiling of one launch (or group of launches) of a given kind.
enum { PROF_PREP = 0, PROF_DEMOD = 1, PROF_PASS1 = 2, PROF_PASS2 = 3, PROF_OTHER = 4 };
inline cudaEvent_t prof_event(fs_ctx *c) {
  if (c->ev_used == c->evpool.size()) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    c->evpool.push_back(e);
  }
  return c->evpool[c->ev_used++];
}
struct ProfScope {
  fs_ctx *c;
  int kind;
  cudaStream_t st;
  cudaEvent_t a = nullptr;
  ProfScope(fs_ctx *c_, int k, cudaStream_t s) : c(c_), kind(k), st(s) {
    if (c->prof) { a = prof_event(c); cudaEventRecord(a, st); }
  }
  ~ProfScope() {
    if (c->prof) {
      cudaEvent_t b = prof_event(c);
      cudaEventRecord(b, st);
      c->recs.push_back({kind, a, b});
    }
  }
};

// NVTX range over the host-side enqueue of one stage ("fs.prepare",
// "fs.demodulate", "fs.transform", ...): a profiler or tracer attached through
// NVTX sees the stages on the host timeline and can filter launches by them;
// without one the calls do nothing.
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

// Workspace helper: grow *buf to at least `bytes` (synchronising `st` first).
fs_status ensure_buffer(void **buf, size_t *cur, size_t bytes, cudaStream_t st);

// Batched search over several segments and the launch-configuration tuner.
fs_status search32_batch(fs_ctx *ctx, fs_seg *const *segs, int nseg, const double *alpha, const double *delta,
                         int nsky, const double *f1, int nspin, float thr, fs_candidate *cand, int64_t cap,
                         int64_t *ncand, cudaStream_t st);
// The same over lattice templates, one template set per segment (host arrays of nseg).
fs_status search32_lattice_batch(fs_ctx *ctx, fs_seg *const *segs, int nseg, const double *const *alpha,
                                 const double *const *delta, const int32_t *nsky, const double *const *f1,
                                 const double *const *offset, const int32_t *nspin, float thr, fs_candidate *cand,
                                 int64_t cap, int64_t *ncand, cudaStream_t st);
void batch_plan_release(fs_ctx *ctx);

// Fine search (fs_refine.cu).
fs_status fstat_points(fs_ctx *ctx, fs_seg *seg, const fs_point *pts, int npt, double *F, double *grad,
                       double *hess, double *metric, cudaStream_t st);
fs_status refine_points(fs_ctx *ctx, fs_seg *seg, fs_point *pts, int npt, int nsteps, double *F, cudaStream_t st);
fs_status amplitudes(fs_ctx *ctx, fs_seg *seg, const fs_point *pts, int npt, double *amp, cudaStream_t st);
// The coarse search's F at continuous points and (grad != NULL) gF dF/dtheta (fs_adjoint.cu).
fs_status fstat_resampled(fs_ctx *ctx, fs_seg *seg, const fs_point *pts, int npt, const double *gF, double *F,
                          double *grad, cudaStream_t st);
// Fisher-preconditioned gradient ascent of the resampled F from each point (fs_refine.cu).
fs_status refine_resampled(fs_ctx *ctx, fs_seg *seg, fs_point *pts, int npt, int nsteps, double *F, cudaStream_t st);
fs_status points_from_candidates(fs_ctx *ctx, fs_seg *seg, const fs_candidate *cand, int n, const double *alpha,
                                 const double *delta, const double *f1, fs_point *pts, cudaStream_t st);
fs_status autotune32(fs_ctx *ctx, fs_seg *seg, const double *alpha, const double *delta, int nsky,
                     const double *f1, int nspin, int reps, fs_tuning *out, cudaStream_t st);
bool tuning_valid(int64_t nfft, const fs_tuning &t);

}  // namespace fs
