// Segment preparation (template independent), Sec. VI.A and Sec. V.
//
//  P0  time/ephemeris tables on the grid t_m = m dt (analytic Earth, FP64
//      computed, stored as double-float for the FP32 path);
//  P1  Fourier x2 upsampling of the data (FP64).  With X = DFT_N(x), the
//      2N-point series of Sec. VI.A (DFT padded with N zeros, inverse DFT)
//      has x2[2m] = x[m] and x2[2m+1] = IDFT_N(Z)[m] with
//      Z_k = X_k exp(i pi k'/N), k' the signed frequency of bin k and the
//      Nyquist bin of even N set to zero (its split halves cancel on the odd
//      samples).  Both length-N transforms use Bluestein's chirp-z identity
//      on power-of-two FP64 FFTs, so any N is accepted;
//  P2  natural cubic spline through x2 at unit spacing: second derivatives
//      from the [1 4 1] tridiagonal system by the Thomas recurrences, exact at
//      the ends and as 21-tap filters (their pole (2 - sqrt 3)^21 ~ 1e-12)
//      one point per thread inside, then per-interval polynomial coefficients.
#include <stdio.h>
#include <algorithm>
#include "fs_internal.h"
#include "fs_dfc.cuh"
#include "fs_model.cuh"

namespace fs {

// ------------------------------------------------------------------ P0 tables
__global__ void k_tables32(SegGeom g, float4 *tab0, float4 *tab1) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= g.ngrid) return;
  double t = (double)(i - g.margin) * g.dt;
  double sl, cl, sth, cth;
  sincos(g.lambda0 + kOmegaO * t, &sl, &cl);
  sincos(g.theta0 + kOmegaR * t, &sth, &cth);
  df32 C = df_from_double(kAUls * cl), S = df_from_double(kAUls * sl), T = df_from_double(t);
  tab0[i] = make_float4(C.hi, C.lo, S.hi, S.lo);
  tab1[i] = make_float4((float)cth, (float)sth, T.hi, T.lo);
}

// A caller's position table (Sec. V: the ephemerides), component-major r and v,
// into (r, 0), (v, 0) pairs; entries that are not finite or beyond
// kMaxDelayEph light-seconds latch ERRF_NONFINITE and are taken as zero.
__global__ void k_eph_import(const double *r, const double *v, int64_t n, dbl4 *eph, uint32_t *flags) {
  const int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (m >= n) return;
  double rx = r[m], ry = r[n + m], rz = r[2 * n + m];
  double vx = v[m], vy = v[n + m], vz = v[2 * n + m];
  const double r2 = rx * rx + ry * ry + rz * rz;
  const bool ok = isfinite(rx) && isfinite(ry) && isfinite(rz) && isfinite(vx) && isfinite(vy) && isfinite(vz) &&
                  r2 <= kMaxDelayEph * kMaxDelayEph && vx * vx + vy * vy + vz * vz <= 1.0;
  if (!ok) {
    atomicOr(flags, ERRF_NONFINITE);
    rx = ry = rz = vx = vy = vz = 0.0;
  }
  eph[2 * m] = make_dbl4(rx, ry, rz, 0.0);
  eph[2 * m + 1] = make_dbl4(vx, vy, vz, 0.0);
}

// FP32-path form of the table on the grid with margins: position at t_m by
// linear extrapolation from the nearest table point (clamped), as double-floats.
__global__ void k_eph_tables32(SegGeom g, const dbl4 *eph, float4 *e0, float4 *e1, float *e2) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= g.ngrid) return;
  const int64_t m = i - g.margin;
  const int64_t mc = m < 0 ? 0 : (m >= g.n ? g.n - 1 : m);
  const double tau = (double)(m - mc) * g.dt;
  const dbl4 r = eph[2 * mc], v = eph[2 * mc + 1];
  const df32 X = df_from_double(r.x + tau * v.x), Y = df_from_double(r.y + tau * v.y),
             Z = df_from_double(r.z + tau * v.z);
  e0[i] = make_float4(X.hi, X.lo, Y.hi, Y.lo);
  e1[i] = make_float4(Z.hi, Z.lo, (float)v.x, (float)v.y);
  e2[i] = (float)v.z;
}

fs_status import_eph(fs_seg *seg, const double *r, const double *v, cudaStream_t st) {
  const int64_t n = seg->g.n;
  k_eph_import<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(r, v, n, seg->eph, seg->ctx->d_flags);
  seg->ctx->launches++;
  return cuda_status(cudaGetLastError());
}

fs_status prepare_tables(fs_seg *seg, cudaStream_t st) {
  if (seg->tables_ready) return FS_OK;  // they depend on the geometry only, not on the data
  const SegGeom &g = seg->g;
  k_tables32<<<(unsigned)((g.ngrid + 255) / 256), 256, 0, st>>>(g, seg->tab0, seg->tab1);
  seg->ctx->launches++;
  if (seg->eph) {
    k_eph_tables32<<<(unsigned)((g.ngrid + 255) / 256), 256, 0, st>>>(g, seg->eph, seg->eph0, seg->eph1,
                                                                      seg->eph2);
    seg->ctx->launches++;
  }
  const fs_status r = cuda_status(cudaGetLastError());
  seg->tables_ready = (r == FS_OK);
  return r;
}

// ------------------------------------------------------------------ P1 upsampling
template <typename T>
__global__ void k_load_x(const T *x, double *x64, float *x32, int64_t n, uint32_t *flags) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double v = (double)x[i];
  if (!isfinite(v)) { atomicOr(flags, ERRF_NONFINITE); v = 0.0; }
  x64[i] = v;
  x32[i] = (float)v;
}

// Bluestein chirp c_m = exp(sign * i pi m^2 / N) with m^2 reduced mod 2N exactly.
__device__ inline double2 bluestein_chirp(int64_t m, int64_t N, int sign) {
  unsigned long long q = ((unsigned long long)m * (unsigned long long)m) % (unsigned long long)(2 * N);
  double s, c;
  sincospi((double)q / (double)N, &s, &c);
  return make_double2(c, sign * s);
}

// b[m] = exp(+i pi m^2/N) for |m| < N placed circularly in a length-M buffer.
__global__ void k_bluestein_b(double2 *b, int64_t N, int64_t M) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= M) return;
  double2 v = make_double2(0.0, 0.0);
  if (i < N) v = bluestein_chirp(i, N, +1);
  else if (i > M - N) v = bluestein_chirp(M - i, N, +1);
  b[i] = v;
}

// Per-segment tables of the upsampler (they depend on N only): the chirp
// exp(-i pi m^2/N) and the half-sample shift exp(i pi k'/N) (k' the signed
// frequency of bin k; zero at the Nyquist bin of even N), m, k < N.
__global__ void k_bluestein_tables(double2 *chirp, double2 *shift, int64_t N) {
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= N) return;
  chirp[k] = bluestein_chirp(k, N, -1);
  if ((N % 2 == 0) && k == N / 2) {
    shift[k] = make_double2(0.0, 0.0);
  } else {
    const int64_t kp = (2 * k < N) ? k : k - N;  // signed frequency
    double sn, cs;
    sincospi((double)kp / (double)N, &sn, &cs);
    shift[k] = make_double2(cs, sn);
  }
}

// The per-load steps of the upsampler run in double-float arithmetic (FP32 pipe;
// ~1e-14 relative), on tables converted once per length from their FP64 form.
// a[n] = in[n] * exp(-i pi n^2/N) for n < N (in real or complex, optionally conjugated), 0 beyond.
__global__ void k_bluestein_a(float4 *a, const double *in_real, const float4 *in_cplx, int conj_in,
                              const float4 *chirp, int64_t N, int64_t M) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= M) return;
  dfc v{df32{0.f, 0.f}, df32{0.f, 0.f}};
  if (i < N) {
    dfc u = in_cplx ? dfc_ld(in_cplx[i]) : dfc{df_from_double(in_real[i]), df32{0.f, 0.f}};
    if (conj_in) u.im = df_neg(u.im);
    v = dfc_mul(u, dfc_ld(chirp[i]));
  }
  a[i] = dfc_st(v);
}

__global__ void k_pointwise_mul(float4 *a, const float4 *b, int64_t M) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < M) a[i] = dfc_st(dfc_mul(dfc_ld(a[i]), dfc_ld(b[i])));
}

// out[k] = exp(-i pi k^2/N) conv[k] / M   (k < N; M a power of two: exact scaling)
__global__ void k_bluestein_out(float4 *out, const float4 *conv, const float4 *chirp, int64_t N, int64_t M) {
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= N) return;
  const float inv = 1.0f / (float)M;
  dfc v = dfc_ld(conv[k]);
  v = dfc{df_scale(v.re, inv), df_scale(v.im, inv)};
  out[k] = dfc_st(dfc_mul(v, dfc_ld(chirp[k])));
}

// x2[2m] = x[m]; x2[2m+1] = Re(c[m]), c the circular convolution of x with the
// interpolation kernel (its spectrum carries the 1/M of the inverse transform)
__global__ void k_interleave(double *x2, const double *x, const float4 *c, int64_t N) {
  int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (m >= N) return;
  x2[2 * m] = x[m];
  const float4 v = c[m];
  x2[2 * m + 1] = (double)v.x + (double)v.y;
}

// a[i] = x[i] (i < N), 0 up to M, as double-float complex values
__global__ void k_pack_real(float4 *a, const double *x, int64_t N, int64_t M) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= M) return;
  const df32 v = i < N ? df_from_double(x[i]) : df32{0.f, 0.f};
  a[i] = make_float4(v.hi, v.lo, 0.f, 0.f);
}

// The interpolation kernel h = IDFT_N(shift) (real: shift is Hermitian) placed
// circularly in a length-M buffer, hM[d mod M] = h[d mod N] / M for |d| < N, zero
// elsewhere; X = DFT_N(conj(shift)), so h[j] = Re(X_j) / N.  M >= 2N - 1: the two
// ends do not overlap, and for outputs m < N and inputs j < N the circular
// convolution of length M reads h at m - j only, i.e. it equals the length-N one.
__global__ void k_place_kernel(float4 *hM, const float4 *X, int64_t N, int64_t M) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= M) return;
  const int64_t d = i < N ? i : i - M;  // signed offset
  float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
  if (d > -N) {
    const float4 x = X[d < 0 ? d + N : d];
    const df32 h = df_mul(df32{x.x, x.y}, df_from_double(1.0 / ((double)N * (double)M)));
    v = make_float4(h.hi, h.lo, 0.f, 0.f);
  }
  hM[i] = v;
}

static inline unsigned nblk(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

// DFT of length N of `in` (real, or complex double-floats optionally conjugated) into
// out (double-floats), by Bluestein.
static cudaError_t bluestein_dft(float4 *out, const double *in_real, const float4 *in_cplx, int conj_in,
                                 int64_t N, int64_t M, const float4 *Bhat, const float4 *chirp, float4 *a,
                                 float4 *tmp, const float4 *tw, cudaStream_t st, int64_t *launches) {
  k_bluestein_a<<<nblk(M), 256, 0, st>>>(a, in_real, in_cplx, conj_in, chirp, N, M);
  cudaError_t e = fftdf(a, tmp, tw, M, 1, -1, st, launches);
  if (e != cudaSuccess) return e;
  k_pointwise_mul<<<nblk(M), 256, 0, st>>>(a, Bhat, M);
  e = fftdf(a, tmp, tw, M, 1, +1, st, launches);
  if (e != cudaSuccess) return e;
  k_bluestein_out<<<nblk(N), 256, 0, st>>>(out, a, chirp, N, M);
  *launches += 3;
  return cudaGetLastError();
}

// Fourier x2 upsampling (Sec. VI.A, reading of the Nyquist split as the oracle):
// the odd samples are x2[2m+1] = sum_j x_j h[(m - j) mod N] with h = IDFT_N(s),
// s_k = exp(i pi k'/N) the half-sample shift (k' the signed frequency, zero at the
// Nyquist bin of even N), i.e. the inverse DFT of the DFT of x times s.  Per length N
// the plan computes h (one Bluestein DFT) and the spectrum of h placed in a
// power-of-two buffer of M >= 2N - 1 points; every load then takes one forward and
// one inverse transform of length M (double-float arithmetic on the FP32 pipe).
fs_status prepare_upsample(fs_seg *seg, const void *x_dev, cudaStream_t st) {
  int64_t N = seg->g.n;
  int64_t M = 1;
  while (M < 2 * N - 1) M <<= 1;
  int64_t *L = &seg->ctx->launches;
  if (seg->blu_m != M) {
    cudaFree(seg->blu_bhat);
    cudaFree(seg->blu_tw);
    cudaFree(seg->blu_chirp);
    seg->blu_bhat = seg->blu_tw = seg->blu_chirp = nullptr;
    seg->blu_m = 0;
    if (cudaMalloc(&seg->blu_bhat, sizeof(double2) * M) != cudaSuccess ||
        cudaMalloc(&seg->blu_tw, sizeof(double2) * (M / 2)) != cudaSuccess ||
        cudaMalloc(&seg->blu_chirp, sizeof(double2) * 2 * N) != cudaSuccess) {
      cudaGetLastError();
      return FS_ERR_NOMEM;
    }
  }
  // scratch: a, tmp, X (M each)
  size_t need = sizeof(float4) * 3 * (size_t)M;
  fs_status s = ensure_buffer(&seg->ctx->scratch, &seg->ctx->scratch_bytes, need, st);
  if (s != FS_OK) return s;
  float4 *a = (float4 *)seg->ctx->scratch;
  float4 *tmp = a + M, *X = tmp + M;
  float4 *Hhat = (float4 *)seg->blu_bhat;  // after the plan: the kernel's spectrum
  const float4 *tw = (const float4 *)seg->blu_tw;
  cudaError_t e;
  if (seg->blu_m != M) {
    // tables in FP64 (twiddles, Bluestein chirp and its spectrum, the half-sample
    // shift), then as double-floats in place (16 bytes per complex value either way)
    double2 *chirp64 = seg->blu_chirp, *shift64 = seg->blu_chirp + N;
    double2 *Bhat64 = seg->blu_bhat, *tw64 = seg->blu_tw;
    e = fft64_twiddles(tw64, M, st);
    if (e != cudaSuccess) return FS_ERR_CUDA;
    k_bluestein_b<<<nblk(M), 256, 0, st>>>(Bhat64, N, M);
    k_bluestein_tables<<<nblk(N), 256, 0, st>>>(chirp64, shift64, N);
    *L += 3;
    e = fft64(Bhat64, (double2 *)tmp, tw64, M, 1, -1, st, L);
    if (e != cudaSuccess) return FS_ERR_CUDA;
    if (to_df32(Bhat64, (float4 *)Bhat64, M, st) != cudaSuccess ||
        to_df32(tw64, (float4 *)tw64, M / 2, st) != cudaSuccess ||
        to_df32(chirp64, (float4 *)chirp64, 2 * N, st) != cudaSuccess)
      return FS_ERR_CUDA;
    *L += 3;
    const float4 *chirp = (const float4 *)chirp64, *shift = chirp + N;
    // X = DFT_N(conj(shift)): h = IDFT_N(shift) = Re(X) / N
    e = bluestein_dft(X, nullptr, shift, 1, N, M, (const float4 *)Bhat64, chirp, a, tmp, tw, st, L);
    if (e != cudaSuccess) return FS_ERR_CUDA;
    // the kernel placed circularly (scaled by 1/M), and its spectrum in place of Bhat
    k_place_kernel<<<nblk(M), 256, 0, st>>>(Hhat, X, N, M);
    *L += 1;
    e = fftdf(Hhat, tmp, tw, M, 1, -1, st, L);
    if (e != cudaSuccess) return FS_ERR_CUDA;
    seg->blu_m = M;
  }

  if (seg->d.x_dtype == FS_X_F32)
    k_load_x<float><<<nblk(N), 256, 0, st>>>((const float *)x_dev, seg->x64, seg->x32, N, seg->ctx->d_flags);
  else
    k_load_x<double><<<nblk(N), 256, 0, st>>>((const double *)x_dev, seg->x64, seg->x32, N, seg->ctx->d_flags);
  // odd samples: the circular convolution of x with the kernel
  k_pack_real<<<nblk(M), 256, 0, st>>>(a, seg->x64, N, M);
  *L += 2;
  e = fftdf(a, tmp, tw, M, 1, -1, st, L);
  if (e != cudaSuccess) return FS_ERR_CUDA;
  k_pointwise_mul<<<nblk(M), 256, 0, st>>>(a, Hhat, M);
  *L += 1;
  e = fftdf(a, tmp, tw, M, 1, +1, st, L);
  if (e != cudaSuccess) return FS_ERR_CUDA;
  k_interleave<<<nblk(N), 256, 0, st>>>(seg->x2, seg->x64, a, N);
  *L += 1;
  return cuda_status(cudaGetLastError());
}

// ------------------------------------------------------------------ P2 spline
// Thomas recurrences for M_{i-1} + 4 M_i + M_{i+1} = r_i (i = 1..n2-2), M_0 = M_{n2-1} = 0,
// r_i = 6 (y_{i+1} - 2 y_i + y_{i-1}):
//   c'_1 = 1/4, c'_i = 1/(4 - c'_{i-1});  d'_1 = r_1 c'_1, d'_i = (r_i - d'_{i-1}) c'_i
//   M_{n2-2} = d'_{n2-2},  M_i = d'_i - c'_i M_{i+1}
// c'_i reaches its limit c = 2 - sqrt(3) in double within ~20 steps.  Away
// from the ends both recurrences are first-order filters with pole -c, so
//   d'_i = c sum_{k=0}^{K} (-c)^k r_{i-k},   M_i = sum_{k=0}^{K} (-c)^k d'_{i+k}
// with K = 20; these run one point per thread.  The first and last kSplEnd
// points follow the exact recurrences serially.  The dropped tail weighs
// c^21 ~ 1e-12 of the data's scale: the result equals the sequential Thomas
// solution to that level, far below the FP32 coefficients' rounding and the
// FP64 path's 1e-8 tolerance on F.
constexpr int kSplK = 20;
constexpr int kSplEnd = 64;

__device__ inline double spline_climit() {
  double c = 0.25;
  for (int k = 2; k <= kSplEnd; k++) c = 1.0 / (4.0 - c);
  return c;
}

__global__ void k_spline_rhs(const double *y, double *r, int64_t n2) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= 1 && i <= n2 - 2) r[i] = 6.0 * (y[i + 1] - 2.0 * y[i] + y[i - 1]);
}

// d'_i for i in [1, n2-2]; thread 0 runs the exact head [1, kSplEnd) serially.
__global__ void k_spline_forward(const double *r, double *dp, int64_t n2) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t last = n2 - 2;
  if (i == 0) {
    double c = 0.25, d = 0.0;
    const int64_t h = last < kSplEnd - 1 ? last : kSplEnd - 1;
    for (int64_t k = 1; k <= h; k++) {
      if (k > 1) c = 1.0 / (4.0 - c);
      d = (r[k] - d) * c;
      dp[k] = d;
    }
    return;
  }
  if (i < kSplEnd || i > last) return;
  const double c = spline_climit();
  double acc = 0.0, w = c;
  for (int k = 0; k <= kSplK; k++) {
    acc = fma(w, r[i - k], acc);
    w *= -c;
  }
  dp[i] = acc;
}

// M_i for i in [1, n2-2]; thread 0 runs the exact tail from n2-2 down, thread 1
// the exact head from kSplEnd down to 1 (starting from the truncated-sum M_kSplEnd).
__global__ void k_spline_backward(const double *dp, double *Mout, int64_t n2) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t last = n2 - 2;
  const double c = spline_climit();
  if (i == 0) {
    double m = 0.0;
    const int64_t lo = last - kSplEnd + 1 > kSplEnd ? last - kSplEnd + 1 : kSplEnd;
    for (int64_t k = last; k >= lo; k--) {
      m = dp[k] - c * m;
      Mout[k] = m;
    }
    return;
  }
  if (i == 1) {
    double m = 0.0, w = 1.0;
    for (int k = 0; k <= kSplK; k++) {
      m = fma(w, dp[kSplEnd + k], m);
      w *= -c;
    }
    double cp[kSplEnd];
    cp[1] = 0.25;
    for (int k = 2; k < kSplEnd; k++) cp[k] = 1.0 / (4.0 - cp[k - 1]);
    for (int k = kSplEnd - 1; k >= 1; k--) {
      m = dp[k] - cp[k] * m;
      Mout[k] = m;
    }
    return;
  }
  if (i < kSplEnd || i > last - kSplEnd) return;
  double acc = 0.0, w = 1.0;
  for (int k = 0; k <= kSplK; k++) {
    acc = fma(w, dp[i + k], acc);
    w *= -c;
  }
  Mout[i] = acc;
}

// Short series: the sequential Thomas algorithm in one thread.
__global__ void k_spline_serial(const double *y, double *dp, double *Mout, int64_t n2) {
  const int64_t last = n2 - 2;
  double c = 0.25, d = 0.0;
  for (int64_t k = 1; k <= last; k++) {
    if (k > 1) c = 1.0 / (4.0 - c);
    d = (6.0 * (y[k + 1] - 2.0 * y[k] + y[k - 1]) - d) * c;
    dp[k] = d;
  }
  double m = 0.0;
  c = 0.25;
  // recompute c'_k on the way back (stored values would need another array)
  for (int64_t k = last; k >= 1; k--) {
    double ck = 0.25;
    for (int64_t q = 2; q <= (k < kSplEnd ? k : kSplEnd); q++) ck = 1.0 / (4.0 - ck);
    m = dp[k] - ck * m;
    Mout[k] = m;
  }
  (void)c;
}

// coef[i] for u = i + f, f in [0,1):
//   S = y_i + f (y_{i+1} - y_i - (2 M_i + M_{i+1})/6) + f^2 M_i/2 + f^3 (M_{i+1} - M_i)/6
template <typename C>
__global__ void k_spline_coef(const double *y, const double *Msd, C *coef, int64_t n2);

template <>
__global__ void k_spline_coef<float4>(const double *y, const double *Msd, float4 *coef, int64_t n2) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n2) return;
  if (i == n2 - 1) { coef[i] = make_float4(0.f, 0.f, 0.f, 0.f); return; }
  double Mi = (i == 0) ? 0.0 : Msd[i];
  double Mj = (i + 1 == n2 - 1) ? 0.0 : Msd[i + 1];
  double c1 = y[i + 1] - y[i] - (2.0 * Mi + Mj) / 6.0;
  coef[i] = make_float4((float)y[i], (float)c1, (float)(0.5 * Mi), (float)((Mj - Mi) / 6.0));
}

template <>
__global__ void k_spline_coef<dcoef4>(const double *y, const double *Msd, dcoef4 *coef, int64_t n2) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n2) return;
  if (i == n2 - 1) { coef[i] = dcoef4{0.0, 0.0, 0.0, 0.0}; return; }
  double Mi = (i == 0) ? 0.0 : Msd[i];
  double Mj = (i + 1 == n2 - 1) ? 0.0 : Msd[i + 1];
  double c1 = y[i + 1] - y[i] - (2.0 * Mi + Mj) / 6.0;
  coef[i] = dcoef4{y[i], c1, 0.5 * Mi, (Mj - Mi) / 6.0};
}

fs_status prepare_spline(fs_seg *seg, cudaStream_t st) {
  int64_t n2 = 2 * seg->g.n;
  size_t need = sizeof(double) * 3 * (size_t)n2;
  fs_status s = ensure_buffer(&seg->ctx->scratch, &seg->ctx->scratch_bytes, need, st);
  if (s != FS_OK) return s;
  double *r = (double *)seg->ctx->scratch;
  double *dp = r + n2;
  double *Msd = dp + n2;
  if (n2 - 2 < 4 * kSplEnd) {
    k_spline_serial<<<1, 1, 0, st>>>(seg->x2, dp, Msd, n2);
    seg->ctx->launches += 2;
  } else {
    k_spline_rhs<<<nblk(n2), 256, 0, st>>>(seg->x2, r, n2);
    k_spline_forward<<<nblk(n2), 256, 0, st>>>(r, dp, n2);
    k_spline_backward<<<nblk(n2), 256, 0, st>>>(dp, Msd, n2);
    seg->ctx->launches += 4;
  }
  if (seg->d.precision == FS_PREC_F32)
    k_spline_coef<float4><<<nblk(n2), 256, 0, st>>>(seg->x2, Msd, (float4 *)seg->coef, n2);
  else
    k_spline_coef<dcoef4><<<nblk(n2), 256, 0, st>>>(seg->x2, Msd, (dcoef4 *)seg->coef, n2);
  return cuda_status(cudaGetLastError());
}

// ------------------------------------------------------------------ injections (FP64)
struct InjConst {
  SkyConst64 K;
  double A[4];
  double f0, f1, fl;
};

// Unit-amplitude response of one injection at t_k = k dt (Eqs. sig, eq:ab), and
// per-block partial sums of h^2.
__global__ void k_inject_unit(InjConst c, SegGeom g, double *h, double *partial, int64_t n) {
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double v = 0.0;
  if (k < n) {
    double t = (double)k * g.dt;
    Geo64 q = geometry64(t, c.K, g);
    double a, b;
    ab_eval64(c.K, q.cx, q.sx, &a, &b);
    double cyc = c.f0 * (t + q.phi) + c.fl * q.phi + c.f1 * (0.5 * t * t + t * q.phi);
    cyc -= floor(cyc);
    double sp, cp;
    sincospi(2.0 * cyc, &sp, &cp);
    v = c.A[0] * a * cp + c.A[1] * b * cp + c.A[2] * a * sp + c.A[3] * b * sp;
    h[k] = v;
  }
  double sq = v * v;
  for (int o = 16; o > 0; o >>= 1) sq += __shfl_down_sync(0xffffffffu, sq, o);
  __shared__ double ws[32];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = sq;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) s += ws[w];
    partial[blockIdx.x] = s;
  }
}

// x += h * snr / rho_unit with rho_unit^2 = (2/S0) dt sum h^2 = sum h^2 / sigma^2.
__global__ void k_inject_add(double *x, const double *h, const double *partial, int nb, double snr,
                             double sigma, int64_t n) {
  __shared__ double scale;
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < nb; i++) s += partial[i];
    scale = (s > 0.0) ? snr * sigma / sqrt(s) : 0.0;
  }
  __syncthreads();
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k < n) x[k] += h[k] * scale;
}

fs_status inject64(fs_ctx *ctx, double *x, int64_t n, double dt, double fl, double sigma, double theta0,
                   double lambda0, const fs_injection *inj, int n_inj, cudaStream_t st) {
  int nb = (int)nblk(n);
  size_t need = sizeof(double) * ((size_t)n + (size_t)nb);
  fs_status s = ensure_buffer(&ctx->scratch, &ctx->scratch_bytes, need, st);
  if (s != FS_OK) return s;
  double *h = (double *)ctx->scratch;
  double *partial = h + n;
  SegGeom g{};
  g.n = n;
  g.dt = dt;
  g.fl = fl;
  g.theta0 = theta0;
  g.lambda0 = lambda0;
  double re, z;
  site_radius(ctx->det.lat, &re, &z);
  g.re_c = re / kC;
  g.z_c = z / kC;
  for (int i = 0; i < n_inj; i++) {
    InjConst c{};
    sky_constants(inj[i].alpha, inj[i].delta, ctx->det.eps, ctx->det.lat, ctx->det.gamma, g, &c.K);
    // A_i of Eq. eq:ampone with h0+ = (1 + cos^2 iota)/2, h0x = cos iota (Eq. h0iota, h0 = 1)
    double hp = 0.5 * (1.0 + inj[i].cos_iota * inj[i].cos_iota), hc = inj[i].cos_iota;
    double c2p = cos(2 * inj[i].psi), s2p = sin(2 * inj[i].psi);
    double cp = cos(inj[i].phi0), sp = sin(inj[i].phi0);
    c.A[0] = hp * c2p * cp - hc * s2p * sp;
    c.A[1] = hp * s2p * cp + hc * c2p * sp;
    c.A[2] = -hp * c2p * sp - hc * s2p * cp;
    c.A[3] = -hp * s2p * sp + hc * c2p * cp;
    c.f0 = inj[i].f0;
    c.f1 = inj[i].f1;
    c.fl = fl;
    k_inject_unit<<<nb, 256, 0, st>>>(c, g, h, partial, n);
    k_inject_add<<<nb, 256, 0, st>>>(x, h, partial, nb, inj[i].snr, sigma, n);
    ctx->launches += 2;
  }
  return cuda_status(cudaGetLastError());
}

}  // namespace fs
