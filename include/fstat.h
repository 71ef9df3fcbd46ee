/*
 * fstat.h -- C ABI of the GB300 coherent F-statistic template loop.
 *
 * The library evaluates, for every template (sky position alpha, delta and
 * spindown f1) of a search grid, the F-statistic of Eq. (OS)
 *
 *     F_k = 2 / (S0 To) * ( |Fa_k|^2 / <a^2> + |Fb_k|^2 / <b^2> )
 *
 * on the Fourier bins k of a zero-padded transform, where Fa, Fb are the
 * integrals of Eqs. (Fab) written as Fourier transforms in barycentric time
 * (Eq. ia, Sec. VI.A):
 *
 *     Fa_k = dt * sum_{j<N} x~_j a_j exp(-2 pi i Phi_j) exp(-2 pi i j k / Nfft)
 *
 * with x~_j the data resampled to the source time t_j that solves
 * t_j + phi_m(t_j) = j dt (Eq. eq:Bt, phi_m of Eq. pham), a_j, b_j the
 * amplitude modulation functions at t_j (Sec. II), and
 * Phi_j = fl phi_m(t_j) + f1 (t_j^2/2 + t_j phi_m(t_j)) the
 * frequency-independent phase (Eq. phas with one spindown, plus the
 * heterodyne term of a narrow band starting at fl).  Threshold crossings
 * F_k > F_thr are compacted into a candidate list (Sec. VII, coarse search).
 *
 * Conventions shared by every entry point:
 *  - Array arguments named *_dev are device pointers on the context's
 *    device, owned by the caller; the library only reads inputs and writes
 *    outputs through them.  Arguments named *_host are host pointers.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls are asynchronous on that stream unless stated.
 *  - Argument errors are returned immediately and nothing is launched.
 *    Errors found on the device (candidate overflow, non-finite input,
 *    exhausted wait) are latched in the context and returned by
 *    fs_sync_status().
 *  - A context is not thread-safe; use one context per host thread.
 *  - No C++ exception crosses this boundary.
 */
#ifndef FSTAT_H
#define FSTAT_H

#include <stdint.h>

#if defined(__GNUC__)
#define FS_API __attribute__((visibility("default")))
#else
#define FS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FS_OK = 0,
  FS_ERR_ARG = 1,         /* null pointer, bad enum value, bad sizes         */
  FS_ERR_SHAPE = 2,       /* unsupported n / nfft / nbins combination        */
  FS_ERR_CAPACITY = 3,    /* more candidates than cand_cap (count is exact)  */
  FS_ERR_NONFINITE = 4,   /* NaN or Inf in the data series                   */
  FS_ERR_CUDA = 5,        /* a CUDA runtime call failed                      */
  FS_ERR_TIMEOUT = 6,     /* a bounded device-side wait ran out              */
  FS_ERR_UNSUPPORTED = 7, /* valid request the library does not implement    */
  FS_ERR_NOMEM = 8,       /* device allocation failed                        */
  FS_ERR_SCRATCH = 9,     /* request needs more than FS_NOALLOC_SCRATCH_BYTES */
  FS_ERR_CORRUPT = 10     /* debug build (-DFS_DEBUG) only: a device index outside
                             its buffer, or a workspace guard word overwritten */
} fs_status;

/* Detector site and analytic-Earth parameters, radians.
 * lat, lon: geodetic latitude and east longitude of the site on the
 *   reference ellipsoid (a = 6378.140 km, flattening 0.00335281, Sec. V);
 * gamma: orientation of the arms' bisector, counter-clockwise from local
 *   East (the gamma of the amplitude modulation functions, Sec. II);
 * eps: obliquity of the ecliptic (Eq. pha4);
 * lambda_e0: ecliptic longitude of the Earth seen from the SSB at t = 0 on
 *   a circular orbit of 1 AU (R_ES of Eq. pha5);
 * theta_g0: Greenwich sidereal angle at t = 0; the local sidereal angle is
 *   theta(t) = theta_g0 + lon + Omega_r t, Omega_r = 7.2921151467e-5 rad/s.
 */
typedef struct {
  double lat, lon, gamma, eps, lambda_e0, theta_g0;
} fs_detector;

enum { FS_PREC_F32 = 0, /* FP32 samples, spline and FFT; compensated (double-float) phases */
       FS_PREC_F64 = 1  /* plain FP64 throughout                                           */ };
enum { FS_INTERP_SPLINE2X = 0, /* Fourier x2 + natural cubic spline (Sec. VI.A) */
       FS_INTERP_NEAREST = 1   /* nearest neighbour, "stroboscopic" (Sec. VI.A)  */ };
enum { FS_X_F32 = 0, FS_X_F64 = 1 };
/* Segment options.  FS_OPT_INTERBIN: the search returns F on the half-bin grid
 * f = j / (2 nfft dt), j < nfft, from the length-nfft transform: even j = 2k
 * from the bin X(k), odd j = 2k + 1 from X(k + 1/2) ~ (X(k+1) - X(k)) / sqrt(2)
 * (interbinning, Eq. intbin, Sec. VI.B) for both Fa and Fb -- the frequency grid
 * of a transform padded to 2 nfft at the cost of one of length nfft.  Searches
 * of such a segment take nbins = nfft (the F row length) and report candidate
 * bins j on that grid (also in fs_search_batch); FP32 segments need
 * nfft <= 2^20; the allocation-free searches do not take them (FS_ERR_UNSUPPORTED). */
enum { FS_OPT_INTERBIN = 1 };

/* One data segment: x_k = x(k dt), k < n, t = 0 at the first sample.
 * nfft: zero-padded transform length, a power of two with nfft >= n and
 *   4096 <= nfft <= 2^21 (with FS_PREC_F32 and nfft = 2^21, n <= 2^20);
 * fl: lower edge of the band [Hz] (heterodyne reference);
 * S0: one-sided noise spectral density (2 sigma^2 dt for white noise). */
typedef struct {
  int64_t n;
  int64_t nfft;
  double dt;
  double fl;
  double S0;
  int32_t precision; /* FS_PREC_* */
  int32_t interp;    /* FS_INTERP_* */
  int32_t x_dtype;   /* FS_X_F32 or FS_X_F64: element type of x_dev */
  int32_t options;   /* 0 or FS_OPT_INTERBIN */
  /* Epoch of the first sample [s] after the detector's t = 0: the Earth's
   * orbital and sidereal angles at the segment start are
   * lambda_e0 + Omega_o t0 and theta_g0 + lon + Omega_r t0 (Sec. V).  Phases,
   * spindown and the bins keep t = 0 at the segment's first sample. */
  double t0;
} fs_segment_desc;

/* A threshold crossing: template (sky index, spindown index), bin k, F_k. */
typedef struct {
  uint32_t sky, spin, bin;
  float F;
} fs_candidate;

typedef struct fs_ctx fs_ctx;
typedef struct fs_seg fs_seg;

/* Create a context on CUDA device `device` for detector `det`.
 * Allocates the context's small device state (error flag, counters).
 * Returns FS_ERR_ARG for null pointers, FS_ERR_CUDA if the device cannot be
 * used.  On success *ctx must be released with fs_destroy. */
FS_API fs_status fs_create(fs_ctx **ctx, const fs_detector *det, int32_t device);
/* Release the context and every segment of it still alive (their handles are
 * invalid afterwards: do not pass them to fs_seg_destroy). */
FS_API void fs_destroy(fs_ctx *ctx);

/* Prepare the template-independent part of the resampler for one segment
 * (Sec. VI.A): time/ephemeris tables on the grid t_m = m dt (analytic Earth,
 * Eqs. pha4-pha5, Sec. V), the Fourier x2 upsampled series and its natural
 * cubic spline.  x_dev holds n samples of type desc->x_dtype.  The segment
 * keeps its own device copies (about 40 bytes per sample) and may be reused
 * by any number of fs_search calls.  Non-finite samples latch
 * FS_ERR_NONFINITE.  Release with fs_seg_destroy. */
FS_API fs_status fs_prepare_segment(fs_ctx *ctx, fs_seg **seg, const fs_segment_desc *desc,
                             const void *x_dev, void *stream);
/* fs_prepare_segment with the detector position taken from the caller's table
 * instead of the analytic Earth (Sec. V reads it from ephemerides).
 * r_dev, v_dev: device arrays of 3 x n doubles, component-major (x[0..n),
 *   y[0..n), z[0..n)): r_d(t_m)/c in light-seconds and v_d(t_m)/c, t_m = m dt
 *   (m < n, t = 0 at the segment's first sample), components in the SSB frame
 *   of Eq. pha5 (ecliptic axes: the delay is n0 . r_d with n0 of Eq. pha4).
 * Off the grid the position is extrapolated linearly from the nearest grid
 * point m, clamped to [0, n): r_d(t)/c = r_m + (t - t_m) v_m.  The sidereal
 * angle of a(t), b(t) still comes from the detector and desc->t0.  The
 * segment copies the table (64 bytes per sample; fs_seg_load keeps it) and
 * every search, FP32 or FP64, and the fine search use it.  Entries that are
 * not finite, or farther than 600 light-seconds from the SSB, latch
 * FS_ERR_NONFINITE and are taken as zero.  Same arguments and errors as
 * fs_prepare_segment otherwise; FS_ERR_ARG for a null table pointer.
 * (fs_inject always uses the analytic Earth.) */
FS_API fs_status fs_prepare_segment_eph(fs_ctx *ctx, fs_seg **seg, const fs_segment_desc *desc,
                                        const void *x_dev, const double *r_dev, const double *v_dev,
                                        void *stream);
FS_API void fs_seg_destroy(fs_seg *seg);

/* Coarse search over nsky x nspin templates (Eq. OS on every bin).
 * alpha_dev, delta_dev: nsky doubles (radians); f1_dev: nspin doubles
 *   [Hz/s]; template (s, m) is (alpha[s], delta[s], f1[m]).
 * F_out_dev: NULL (candidates only) or [nsky*nspin][nbins] values, template
 *   index s*nspin + m, bins k = 0..nbins-1 (float for FS_PREC_F32, double
 *   for FS_PREC_F64); nbins is nfft/2 (bins up to Nyquist) or nfft.
 * cand_dev: capacity cand_cap; n_cand_dev: one device int64 that receives
 *   the number of crossings F_k > F_thr (it may exceed cand_cap; then only
 *   cand_cap are stored, in no particular order, and FS_ERR_CAPACITY is
 *   latched).  n_cand_dev is overwritten, not accumulated.
 * The call uses the context workspace, which it grows on first use for the
 * segment's shape; it allocates nothing on later calls of the same shape. */
FS_API fs_status fs_search(fs_ctx *ctx, fs_seg *seg,
                    const double *alpha_dev, const double *delta_dev, int32_t nsky,
                    const double *f1_dev, int32_t nspin, float F_thr,
                    void *F_out_dev, int64_t nbins,
                    fs_candidate *cand_dev, int64_t cand_cap, int64_t *n_cand_dev,
                    void *stream);

/* Re-run the segment preparation on new data of the same shape (n samples
 * of desc->x_dtype at x_dev), reusing the segment's buffers and its length-n
 * transform plan: no allocation.  Same results and errors as
 * fs_prepare_segment. */
FS_API fs_status fs_seg_load(fs_seg *seg, const void *x_dev, void *stream);

/* Allocation-free search.  The paper has no counterpart: this entry point
 * exists for callers that must not allocate device memory while searching,
 * for example an application whose framework already owns the GPU's memory
 * through its own caching pool (a cudaMalloc here could fail or fragment that
 * pool), or a latency-sensitive loop that cannot afford the device-wide
 * synchronisation that cudaFree implies.
 *
 * Same arguments and results as fs_search, restricted to segments prepared
 * with FS_PREC_F32 and nbins = nfft/2 (else FS_ERR_UNSUPPORTED).  It serves
 * callers that cannot allocate device memory while they search: an application
 * whose framework already owns the GPU's memory through its own caching pool, or
 * a latency-bound loop that cannot absorb the device-wide synchronisation of
 * cudaFree.  The paper has no counterpart: it is a property of this library's
 * interface.  Its working memory is one fixed array of
 * FS_NOALLOC_SCRATCH_BYTES that the library holds on every device where it is
 * loaded, until the process exits; a request whose per-sky arrays, transform
 * ring and counters do not fit returns FS_ERR_SCRATCH before launching
 * anything (roughly: nfft up to 2^17).  The call allocates nothing: no
 * cudaMalloc, no cudaFree, no library allocator; fs_create looks up the
 * array's device address for its context (a lookup, no allocation).  The first
 * launches of a process may still make the CUDA driver load the library's
 * kernels (lazy module loading), which is the driver's own memory, not this
 * call's.  Every call shares the one array and the array keeps the last call's
 * contents (the call clears what must start at zero itself): calls whose work
 * overlaps on the GPU, from any context or stream, race with each other and
 * must be serialised by the caller. */
#define FS_NOALLOC_SCRATCH_BYTES (16u << 20)
FS_API fs_status fs_search_noalloc(fs_ctx *ctx, fs_seg *seg,
                                   const double *alpha_dev, const double *delta_dev, int32_t nsky,
                                   const double *f1_dev, int32_t nspin, float F_thr,
                                   float *F_out_dev, int64_t nbins,
                                   fs_candidate *cand_dev, int64_t cand_cap, int64_t *n_cand_dev,
                                   void *stream);

/* First, coherent stage of a hierarchical search (Sec. I): the same template
 * grid searched in each of nseg segments, candidates only.  Every segment
 * must be prepared with FS_PREC_F32 on this context; lengths and transform
 * sizes may differ.  Bins are nfft/2 per segment (bins up to Nyquist), or the
 * nfft half-bin frequencies of an interbinning segment (FS_OPT_INTERBIN).
 * cand_dev: [nseg][cand_cap] candidates, segment s at cand_dev + s cand_cap;
 * n_cand_dev: [nseg] device int64 counts, overwritten (semantics of
 * fs_search per segment).  The segments run longest transform first on two
 * concurrent branches, each with its own workspace.  The first call for a
 * given set of arguments sizes the workspaces, records the launches of all
 * segments into a CUDA graph and launches it; a later call with the same
 * arguments (same segments, pointers, sizes, threshold and tuning) launches
 * the recorded graph only, so a caller that reloads the segments with
 * fs_seg_load and calls again repeats the whole batch in one graph launch.
 * The call must not itself be made inside a stream capture.  FS_ERR_ARG for a
 * segment of another context or precision. */
FS_API fs_status fs_search_batch(fs_ctx *ctx, fs_seg *const *segs_host, int32_t nseg,
                                 const double *alpha_dev, const double *delta_dev, int32_t nsky,
                                 const double *f1_dev, int32_t nspin, float F_thr,
                                 fs_candidate *cand_dev, int64_t cand_cap, int64_t *n_cand_dev,
                                 void *stream);
/* fs_search_batch over lattice templates (Sec. IV; see fs_search_lattice), each
 * segment with its own lattice: segment s searches nsky_host[s] sky nodes
 * (alpha_dev[s], delta_dev[s]) with the rows f1_dev[s], offset_dev[s] of
 * nsky_host[s] x nspin_host[s] doubles.  The five pointer arrays and the two
 * count arrays are host arrays of nseg entries naming device arrays; candidates,
 * counts, the CUDA graph and its replay as for fs_search_batch (the recorded
 * graph is replayed when every pointer and count is the same).  FP32 segments
 * without interbinning (else FS_ERR_UNSUPPORTED), nfft as fs_search_lattice. */
FS_API fs_status fs_search_lattice_batch(fs_ctx *ctx, fs_seg *const *segs_host, int32_t nseg,
                                         const double *const *alpha_dev, const double *const *delta_dev,
                                         const int32_t *nsky_host, const double *const *f1_dev,
                                         const double *const *offset_dev, const int32_t *nspin_host,
                                         float F_thr, fs_candidate *cand_dev, int64_t cand_cap,
                                         int64_t *n_cand_dev, void *stream);

/* Launch configuration of the FP32 search for one transform length nfft
 * (no counterpart in the paper: it changes the speed, not the result beyond
 * rounding).  Zero fields take the defaults.
 * n1: first-pass length N1 of the split Nsub = N1 x N2 of each
 *   sub-transform (Nsub = nfft, or 2^20 for nfft = 2^21); the splits built
 *   are N1/N2 in {1/4, 1/2, 1, 2, 4} with 64 <= N1, N2 <= 1024;
 * queue_round: templates per round of the persistent work queue;
 * queue_lag: rounds between a template's first and second pass;
 * group_skies: skies demodulated per group;
 * ms_per_template: filled by fs_autotune (ignored by fs_set_tuning). */
typedef struct {
  int32_t n1, queue_round, queue_lag, group_skies;
  float ms_per_template;
  int32_t reserved;
} fs_tuning;
/* Set (t non-NULL) or clear (t NULL) the configuration for nfft.
 * FS_ERR_ARG for a split the library does not provide. */
FS_API fs_status fs_set_tuning(fs_ctx *ctx, int64_t nfft, const fs_tuning *t_host);
/* Current configuration for nfft; FS_ERR_UNSUPPORTED when none is set. */
FS_API fs_status fs_get_tuning(fs_ctx *ctx, int64_t nfft, fs_tuning *out_host);
/* Time the candidate configurations for the segment's transform length on
 * the given grid (candidates only; `reps` timed searches after one warm-up
 * per configuration) and keep the fastest for that length; *out_host
 * receives it.  Synchronous.  The candidates are every split built for the
 * length times queue rounds of about 1/2, 3/4 and 1 of the resident CTAs'
 * first-pass items times lags 1 and 2. */
FS_API fs_status fs_autotune(fs_ctx *ctx, fs_seg *seg,
                             const double *alpha_dev, const double *delta_dev, int32_t nsky,
                             const double *f1_dev, int32_t nspin, int32_t reps,
                             fs_tuning *out_host, void *stream);

/* ---- Fine search (Sec. VI.C) ----
 * A point of the continuous template space: f0 [Hz] the frequency above the
 * band edge fl (the coarse search's bin k is f0 = k / (nfft dt)), f1 [Hz/s],
 * alpha, delta [rad]. */
typedef struct {
  double f0, f1, alpha, delta;
} fs_point;

/* The F-statistic at npt points, evaluated exactly by the direct sums of
 * Eqs. OS and Fab over the segment's original samples (no resampling; phase
 * f0 (t + phi_m) + fl phi_m + f1 (t^2/2 + t phi_m), as in the fine search of
 * Sec. VI.C as run in Sec. VII): sums as double-floats with the orbital
 * phase in FP64 (FP64 throughout with a caller's position table).  F_dev: npt doubles.  grad_dev: NULL or [npt][4]
 * doubles dF/d(f0, f1, alpha, delta).  hess_dev: NULL or [npt][10] doubles,
 * the upper triangle row by row of the Hessian of F.  metric_dev: NULL or [npt][10]
 * doubles, the upper triangle row by row of the reduced Fisher matrix
 * <m_i m_j> - <m_i><m_j> of the phase derivatives m_i = 2 pi dPhi/dtheta_i
 * (Eq. redFm-def, rad^2 per unit parameter^2).  The first call on a segment
 * builds an FP64 table of the orbital and sidereal angles (32 bytes per
 * sample, released with the segment). */
FS_API fs_status fs_fstat_points(fs_ctx *ctx, fs_seg *seg, const fs_point *pts_dev, int32_t npt,
                                 double *F_dev, double *grad_dev, double *hess_dev, double *metric_dev,
                                 void *stream);

/* The coarse search's F at npt continuous points (the adjoint's forward call):
 * the sums of Eqs. ia and Fab over the resampled series of Sec. VI.A (source
 * times of Eq. eq:Bt, spline values, a and b at those times) with the phase
 * Psi_j = fl phi_m(t_j) + f1 (t_j^2/2 + t_j phi_m(t_j)) + f0 j dt, and F of Eq. OS.  At
 * f0 = k / (nfft dt) it is fs_search's F at bin k (the zero-padded DFT of
 * Eq. eq:DFT), between Fourier frequencies the same sum off the grid.  FP32 with
 * double-float phases, as fs_search.  F_dev: npt doubles.  Segments of
 * precision FS_PREC_F32 with FS_INTERP_SPLINE2X and the analytic Earth only
 * (otherwise FS_ERR_UNSUPPORTED). */
FS_API fs_status fs_fstat_resampled(fs_ctx *ctx, fs_seg *seg, const fs_point *pts_dev, int32_t npt,
                                    double *F_dev, void *stream);

/* The backward (adjoint) call of fs_fstat_resampled: grad_dev[4 i + k] =
 * gF_dev[i] * dF_i/dtheta_k, theta = (f0, f1, alpha, delta), gF_dev NULL for
 * ones.  The resampled series is recomputed sample by sample, not stored; its
 * sky dependence enters through the source times (Eq. eq:Bt differentiated:
 * dt_j/dsky = -(d phi_m/dsky) / (1 + d phi_m/dt)), the spline's slope, a and b at
 * the moved times and the phase.  F_dev: NULL or npt doubles (F as the forward
 * call).  Same segments as fs_fstat_resampled. */
FS_API fs_status fs_fstat_resampled_grad(fs_ctx *ctx, fs_seg *seg, const fs_point *pts_dev, int32_t npt,
                                         const double *gF_dev, double *F_dev, double *grad_dev, void *stream);

/* Gradient ascent of the coarse search's F (fs_fstat_resampled) from each
 * point, the fine search driven by the adjoint's gradient: nsteps quasi-Newton
 * steps D = B^-1 grad F.  B starts as 2 F G, G the reduced Fisher matrix at
 * the starting point (Eq. redFm-def; near a maximum F(theta + tau) ~
 * F(theta) (1 - tau^T G tau), Eq. TaylorC2), and is updated by BFGS from the
 * gradient change of every accepted step.  Each step is limited to
 * D^T G D <= 1 and scaled by a factor that doubles (up to 1) when F grows and
 * quarters when it does not; a trial point replaces the current one only if its
 * F is larger.  One adjoint evaluation (F and gradient) per step.  pts_dev is updated in
 * place; F_dev (npt doubles) receives the final F.  Same segments as
 * fs_fstat_resampled. */
FS_API fs_status fs_refine_resampled(fs_ctx *ctx, fs_seg *seg, fs_point *pts_dev, int32_t npt, int32_t nsteps,
                                     double *F_dev, void *stream);

/* Hill climb of the exact F from each point (the fine search of Sec. VI.C,
 * here by Newton's method instead of the simplex search): nsteps steps, each
 * solving (-H + lambda diag(max(-H_ii, 2 F G_ii))) D = grad F with H the
 * Hessian of F and lambda raised from 0 until the matrix is positive definite,
 * limited to D^T G D <= 1 with G the reduced Fisher matrix at the starting
 * point (Eqs. redFm-def, hype: one full correlation length), and scaled by a
 * factor that doubles (up to 1) when F grows and quarters when it does not.
 * A trial point replaces the current one only if its F is larger, so F never
 * decreases.  One evaluation of F, its gradient and Hessian per step.  pts_dev is updated in place; F_dev (npt doubles) receives
 * the final F.  delta is kept in [-pi/2, pi/2] and alpha in [0, 2 pi). */
FS_API fs_status fs_refine(fs_ctx *ctx, fs_seg *seg, fs_point *pts_dev, int32_t npt, int32_t nsteps,
                           double *F_dev, void *stream);

/* Starting points of the fine search from n coarse candidates of fs_search
 * on this segment: f0 = bin / (nfft dt), f1 = f1_dev[spin],
 * (alpha, delta) = (alpha_dev[sky], delta_dev[sky]). */
FS_API fs_status fs_points_from_candidates(fs_ctx *ctx, fs_seg *seg, const fs_candidate *cand_dev, int32_t n,
                                           const double *alpha_dev, const double *delta_dev,
                                           const double *f1_dev, fs_point *pts_dev, void *stream);

/* ML estimators of the four amplitudes at each point (Eq. amle0):
 * A1 = 2 <x h1>/<a^2>, A2 = 2 <x h2>/<b^2>, A3 = 2 <x h3>/<a^2>,
 * A4 = 2 <x h4>/<b^2> with h1..h4 = a cos(phi), b cos(phi), a sin(phi),
 * b sin(phi) of Eq. sig and phi = 2 pi Phi the phase of fs_fstat_points,
 * averages over the segment's samples.  amp_dev: [npt][4] doubles. */
FS_API fs_status fs_amplitudes(fs_ctx *ctx, fs_seg *seg, const fs_point *pts_dev, int32_t npt,
                               double *amp_dev, void *stream);

/* ---- Detection threshold (Sec. III, host functions, no device work) ----
 * False-alarm probability of one cell for threshold F0, (1 + F0) exp(-F0)
 * (Eq. PF; 1 for F0 <= 0). */
FS_API double fs_false_alarm_cell(double F0);
/* Over n_cells independent cells: *alpha = 1 - (1 - P_F(F0))^n_cells
 * (Eq. FP) and, if n_false is not NULL, the expected number of false alarms
 * n_cells P_F(F0) (Eq. NF).  FS_ERR_ARG for n_cells <= 0 or non-finite input. */
FS_API fs_status fs_false_alarm(double F0, double n_cells, double *alpha, double *n_false);
/* The threshold F0 >= 0 whose false-alarm probability over n_cells cells is
 * alpha, 0 < alpha < 1 (Eq. FP inverted). */
FS_API fs_status fs_threshold(double alpha, double n_cells, double *F0);
/* Number of cells n_cells = v_total / V_cell with
 * V_cell = pi^(M/2) / (Gamma(M/2 + 1) sqrt(det G)) (Eqs. NT, vc); G_host is
 * the M x M reduced Fisher matrix (row-major, symmetric positive definite,
 * M <= 16), v_total the parameter-space volume in the same units. */
FS_API fs_status fs_cell_count(int32_t M, const double *G_host, double v_total, double *n_cells);

/* ---- Grid in the parameter space (Sec. IV, host functions, no device work) ----
 * Reduced Fisher matrix (Eq. redFm-def) of the linear phase model (Eq. philin)
 * with xi = (omega0, omega1, alpha1, alpha2) and m(t) = (t, t^2/2, mu1, mu2),
 * mu1 = (R_ES^y + R_E^y cos eps)/c, mu2 = (R_ES^x + R_E^x)/c, for n samples of
 * dt starting at epoch t0 (as fs_segment_desc.t0) in the detector's analytic
 * Earth model.  G_host: 4 x 4 doubles, row-major [s^2]. */
FS_API fs_status fs_linear_model_fisher(const fs_detector *det, int64_t n, double dt, double t0, double *G_host);
/* Lattice covering with constraints (Sec. IV.B): from A2* (dim 2, Eq. A2gen)
 * or A4* (dim 4, Eq. gen) of covering radius R = sqrt(1 - C0) in the
 * coordinates where tau^T G tau = 1 - C0 is a sphere, shrunk along a lattice
 * vector l by mu = |M^-1 a0|/|l| and expanded perpendicular to l by the nu
 * that restores the covering radius R (Eq. condition: minimal match exactly
 * C0), the l of largest mu nu^(dim-1) kept, l rotated onto M^-1 a0
 * (Eq. opt) and, with constraint2 (dim 4), a second lattice vector rotated
 * about it into the directions without sky components (Eq. opt2).
 * basis_host: dim x dim doubles, rows are basis vectors in the units of G;
 * row 0 = a0 = (dp0, 0, ...); with constraint2 row 1 has zero sky
 * (last two) components (Eq. constraint2).  *theta_host: covering thickness
 * theta_min / (mu nu^(dim-1)).  FS_ERR_ARG for G not positive definite or
 * C0 outside (0, 1). */
FS_API fs_status fs_lattice(int32_t dim, const double *G_host, double C0, double dp0, int32_t constraint2,
                            double *basis_host, double *theta_host);
/* Nodes of a 4-dimensional lattice (basis_host of fs_lattice with omega in
 * rad/s) in the band fl + [f0_min, f0_max] Hz and spindowns [f1_min, f1_max]
 * Hz/s over the whole sky, as template points (f0 above fl, f1 = omega1 /
 * 2 pi, and the sky position of (alpha1, alpha2) = omega0 (n0_y, n0_x) in
 * both ecliptic hemispheres, Eq. albe).  pts_host: capacity cap; *count: the
 * number of nodes (FS_ERR_CAPACITY if above cap, the first cap stored).
 * The basis must have the form fs_lattice gives with both constraints
 * (FS_ERR_ARG otherwise); nodes are visited sky node by sky node, then
 * spindown, then frequency. */
FS_API fs_status fs_lattice_nodes(const double *basis_host, const fs_detector *det, double fl, double f0_min,
                                  double f0_max, double f1_min, double f1_max, fs_point *pts_host, int64_t cap,
                                  int64_t *count);
/* Templates of the FFT search of that lattice (Sec. IV: a0 on the Fourier
 * spacing makes every line of nodes along a0 one zero-padded transform; Sec.
 * VII evaluates F over the whole band for each (omega1, alpha1, alpha2)).
 * basis_host: fs_lattice with both constraints and dp0 = 2 pi / (nfft dt).
 * Per sky node (alpha1, alpha2) and hemisphere one sky position (Eq. albe
 * read at the band's upper edge, omega0 = 2 pi (fl + 1/(2 dt))), inside the
 * ecliptic-component box box_host = (n_x lo, n_x hi, n_y lo, n_y hi) (NULL:
 * the whole sky); per sky a row of the spindown nodes in [f1_min, f1_max]
 * Hz/s and, for each, the fraction d in [0, 1) of a bin by which its line
 * falls off the Fourier grid: its nodes are f0 = (k + d) / (nfft dt) above fl.
 * Rows are padded to the longest, *nspin, by repeating their last node.
 * alpha_host, delta_host: sky_cap doubles; f1_host, offset_host: sky_cap x
 * spin_cap doubles, row-major with row length *nspin.  With sky_cap = spin_cap
 * = 0 the call only returns *nsky and *nspin; FS_ERR_CAPACITY (with both
 * counts) when they exceed the capacities; FS_ERR_ARG for a basis not of that
 * form.  Host only. */
FS_API fs_status fs_lattice_templates(const double *basis_host, const fs_detector *det, double fl, int64_t nfft,
                                      double dt, double f1_min, double f1_max, const double *box_host,
                                      double *alpha_host, double *delta_host, double *f1_host, double *offset_host,
                                      int64_t sky_cap, int32_t spin_cap, int64_t *nsky, int32_t *nspin);
/* Coarse search of lattice templates: as fs_search, but template (s, m) has its
 * own spindown f1_dev[s * nspin + m] and evaluates F at the frequencies
 * (k + offset_dev[s * nspin + m]) / (nfft dt) above fl (the data times
 * exp(-2 pi i d j / nfft) before the transform, Eq. eq:DFT at a shifted
 * frequency); a candidate's bin k means that frequency.  Device arrays of
 * nsky * nspin doubles, offsets in [0, 1); F_out_dev holds float for
 * FS_PREC_F32 segments, double for FS_PREC_F64.  Segments without interbinning,
 * nbins = nfft/2; FP32 segments take nfft <= 2^21 (2^21 as two 2^20
 * sub-transforms on the default 1024 x 1024 split); else FS_ERR_UNSUPPORTED. */
FS_API fs_status fs_search_lattice(fs_ctx *ctx, fs_seg *seg, const double *alpha_dev, const double *delta_dev,
                                   int32_t nsky, const double *f1_dev, const double *offset_dev, int32_t nspin,
                                   float F_thr, void *F_out_dev, int64_t nbins, fs_candidate *cand_dev,
                                   int64_t cand_cap, int64_t *n_cand_dev, void *stream);
/* fs_search_lattice from the fixed array of fs_search_noalloc, allocating
 * nothing: same arguments and results as fs_search_lattice for FP32 segments,
 * one sky row per launch; the limits and FS_ERR_SCRATCH of fs_search_noalloc
 * apply. */
FS_API fs_status fs_search_lattice_noalloc(fs_ctx *ctx, fs_seg *seg, const double *alpha_dev,
                                           const double *delta_dev, int32_t nsky, const double *f1_dev,
                                           const double *offset_dev, int32_t nspin, float F_thr,
                                           float *F_out_dev, int64_t nbins, fs_candidate *cand_dev,
                                           int64_t cand_cap, int64_t *n_cand_dev, void *stream);

/* Synchronise `stream` and return (and clear) the first device-side error
 * latched since the last call, or FS_OK. */
FS_API fs_status fs_sync_status(fs_ctx *ctx, void *stream);

/* Self-test of the bounded waits of the persistent transform queue (no
 * counterpart in the paper: it exercises the failure path without a GPU
 * fault).  Launches one block whose first thread waits, with the queue's own
 * wait routine and bound, for a device counter that nothing increments; the
 * wait runs out after its iteration limit (seconds), latches FS_ERR_TIMEOUT
 * for fs_sync_status and the block returns.  The context stays usable. */
FS_API fs_status fs_selftest_wait(fs_ctx *ctx, void *stream);

/* Launch accounting and optional per-kernel timing.
 * launches: kernels launched by this context since the last reset.
 * With profiling on, every launch of the kinds below is bracketed by CUDA
 * events on its stream; ms[k] / count[k] are their summed durations and
 * launch counts (read after the work completes; fs_get_stats synchronises
 * the device).  Kinds: 0 segment preparation (all of it), 1 per-sky
 * demodulation, 2 transform pass 1 (per-batch launches), 3 transform
 * pass 2 + F epilogue (per-batch launches) or both passes (the persistent
 * launch used for nbins = nfft/2), 4 other.
 * workspace_bytes: device bytes the context currently holds in the search and
 * fine-search workspaces it grows on demand (not reset; segments and the fixed
 * array of the allocation-free searches are not included). */
#define FS_PROF_KINDS 5
typedef struct {
  int64_t launches;
  double ms[FS_PROF_KINDS];
  int64_t count[FS_PROF_KINDS];
  int64_t workspace_bytes;
} fs_stats;
FS_API fs_status fs_set_profiling(fs_ctx *ctx, int32_t on);
FS_API fs_status fs_get_stats(fs_ctx *ctx, fs_stats *out, int32_t reset);

/* Human-readable name of a status code (static storage). */
FS_API const char *fs_strerror(fs_status s);

/* ---- stage access, for verification of each step against a reference ---- */

/* Copy the segment's Fourier x2 upsampled series (2n doubles, Sec. VI.A)
 * into x2_dev. */
FS_API fs_status fs_seg_upsampled(const fs_seg *seg, double *x2_dev, void *stream);

/* Resample and demodulate one sky position (the per-sky half of Sec. VI.A):
 * for j < n writes y^a_j = x~_j a_j exp(-2 pi i fl phi_m(t_j)) and y^b_j
 * (interleaved re, im: 2n doubles each), t_j (n doubles), and
 * ab2_dev[0..1] = <a^2>, <b^2> (means over the n output samples).
 * Values are computed by the segment's precision path and widened to double. */
FS_API fs_status fs_demodulate(fs_ctx *ctx, fs_seg *seg, double alpha, double delta,
                        double *ya_dev, double *yb_dev, double *tsrc_dev,
                        double *ab2_dev, void *stream);

/* Signal injection (software simulation of Eqs. resp-hphc, sig-eq:ampone):
 * adds to x_dev (n doubles, t_k = k dt) the response to each injection,
 * scaled so that its optimal SNR (Eq. snr-def with Eq. approx1,
 * S0 = 2 sigma^2 dt) is inj[i].snr.  t0: epoch of the first sample, as in
 * fs_segment_desc (the injection's phase, f0 and f1 refer to t = 0 at the
 * first sample).  Host array of n_inj records. FP64. */
typedef struct {
  double f0, f1, alpha, delta, psi, cos_iota, phi0, snr;
} fs_injection;
FS_API fs_status fs_inject(fs_ctx *ctx, double *x_dev, int64_t n, double dt, double fl, double sigma,
                           double t0, const fs_injection *inj_host, int32_t n_inj, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* FSTAT_H */
