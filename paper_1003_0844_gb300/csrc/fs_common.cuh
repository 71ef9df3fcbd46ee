// Shared definitions of the GB300 F-statistic kernels (device + host side).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <math.h>

#include "../../include/fstat.h"

namespace fs {

// Physical constants of the analytic Earth (Sec. II, Sec. V).
constexpr double kC = 299792458.0;                 // m/s
constexpr double kAU = 149597870700.0;             // m
constexpr double kOmegaR = 7.2921151467e-5;        // rad/s, Earth rotation (NOVAS value, Sec. V)
constexpr double kSiderealYear = 365.25636 * 86400.0;
constexpr double kTwoPi = 6.283185307179586476925286766559;
constexpr double kOmegaO = kTwoPi / kSiderealYear; // rad/s, circular orbit
constexpr double kEllA = 6378140.0;                // m, ellipsoid semi-major axis (Sec. V)
constexpr double kEllF = 0.00335281;               // flattening, NOVAS value (Sec. V)
constexpr double kAUls = kAU / kC;                 // 1 AU in light-seconds
constexpr double kMaxDelay = 500.0;                // bound on |phi_m| [s] (AU/c + Earth radius/c)
constexpr double kMaxDelayEph = 600.0;             // bound on |r_d/c| [s] accepted from a caller's table

// Device-side error bits latched in the context flag word.
enum : uint32_t { ERRF_CAPACITY = 1u, ERRF_NONFINITE = 2u, ERRF_TIMEOUT = 4u, ERRF_CORRUPT = 8u };

// Debug builds (-DFS_DEBUG): the transform kernels check every workspace and
// output index against the extent of its buffer; an index outside [0, limit)
// latches ERRF_CORRUPT and the access is skipped (no trap, the context stays
// usable).  Release builds compile the checks out.
#ifdef FS_DEBUG
constexpr bool kDebug = true;
#else
constexpr bool kDebug = false;
#endif
__device__ __forceinline__ bool dbg_in(int64_t i, int64_t limit, uint32_t *flags) {
  if constexpr (kDebug) {
    if (i < 0 || i >= limit) {
      atomicOr(flags, ERRF_CORRUPT);
      return false;
    }
  }
  return true;
}
// Guard words around debug-build workspace buffers.
constexpr uint32_t kGuardWord = 0xA5C3E10Fu;
constexpr size_t kGuardBytes = 256;

// ------------------------------------------------------------------ double-float (df32) arithmetic
// A value is represented as hi + lo with |lo| <= ulp(hi)/2.  The error-free
// transformations are Knuth's TwoSum and the FMA form of Dekker's TwoProd.
struct df32 { float hi, lo; };

__host__ __device__ inline df32 df_from_double(double x) {
  df32 r; r.hi = (float)x; r.lo = (float)(x - (double)r.hi); return r;
}
__host__ __device__ __forceinline__ df32 two_sum(float a, float b) {  // Knuth
  float s = a + b; float bb = s - a; float e = (a - (s - bb)) + (b - bb);
  df32 r; r.hi = s; r.lo = e; return r;
}
__host__ __device__ __forceinline__ df32 quick_two_sum(float a, float b) {  // requires |a| >= |b|
  float s = a + b; float e = b - (s - a); df32 r; r.hi = s; r.lo = e; return r;
}
__host__ __device__ __forceinline__ df32 two_prod(float a, float b) {  // Dekker with FMA
  float p = a * b; float e = fmaf(a, b, -p); df32 r; r.hi = p; r.lo = e; return r;
}
__host__ __device__ __forceinline__ df32 df_add(df32 a, df32 b) {
  df32 s = two_sum(a.hi, b.hi);
  float lo = s.lo + a.lo + b.lo;
  return quick_two_sum(s.hi, lo);
}
__host__ __device__ __forceinline__ df32 df_add_f(df32 a, float b) {
  df32 s = two_sum(a.hi, b);
  return quick_two_sum(s.hi, s.lo + a.lo);
}
__host__ __device__ __forceinline__ df32 df_mul(df32 a, df32 b) {
  df32 p = two_prod(a.hi, b.hi);
  float lo = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, p.lo));
  return quick_two_sum(p.hi, lo);
}
__host__ __device__ __forceinline__ df32 df_mul_f(df32 a, float b) {
  df32 p = two_prod(a.hi, b);
  return quick_two_sum(p.hi, fmaf(a.lo, b, p.lo));
}
__host__ __device__ inline df32 df_neg(df32 a) { return df32{-a.hi, -a.lo}; }
__host__ __device__ __forceinline__ df32 df_sub(df32 a, df32 b) { return df_add(a, df_neg(b)); }
// a * b for a df32 and an exactly representable power-of-two or small-integer factor
__host__ __device__ __forceinline__ df32 df_scale(df32 a, float b) { return df32{a.hi * b, a.lo * b}; }
// Fractional part of a df32 number of cycles, in [-0.5, 0.5].
__device__ __forceinline__ float df_frac_cycles(df32 c) {
  float r = c.hi - rintf(c.hi);  // exact: c.hi and its nearest integer are close
  float f = r + c.lo;
  return f - rintf(f);
}
// Fractional cycles of the product a*b of two df32 numbers.
__device__ __forceinline__ float df_mul_frac(df32 a, df32 b) {
  float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
  float r = p - rintf(p);
  float f = r + e;
  return f - rintf(f);
}

// ------------------------------------------------------------------ complex helpers
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
// exp(-2 pi i f) for f in cycles (|f| <= 1 for full accuracy)
__device__ __forceinline__ float2 expm2pi(float f) {
  float s, c; sincospif(2.0f * f, &s, &c); return make_float2(c, -s);
}

// Four doubles, 32-byte aligned (one vector load; CUDA 13 deprecates the
// unannotated double4).
struct alignas(32) dbl4 { double x, y, z, w; };
__host__ __device__ inline dbl4 make_dbl4(double x, double y, double z, double w) { return dbl4{x, y, z, w}; }

// Cubic spline coefficients of one interval in FP64 (c0, c1, c2, c3).
struct alignas(32) dcoef4 { double x, y, z, w; };

// ------------------------------------------------------------------ internal structures
// Per-sky constants of the FP32 demodulation kernel (computed in FP64 per sky).
struct SkyConst32 {
  df32 nx, nyp;      // n0 components multiplying R_ES^x and R_ES^y (Sec. II scalar product)
  df32 nz;           // n0 component along the ecliptic pole (a caller's position table)
  float ca, sa;      // cos(alpha), sin(alpha)
  float rcd, zsd;    // (r_e/c) cos(delta), (z/c) sin(delta)  [s]
  float ea[5];       // a = ea0 cos2x + ea1 sin2x + ea2 cos x + ea3 sin x + ea4, x = alpha - theta
  float eb[4];       // b = eb0 cos2x + eb1 sin2x + eb2 cos x + eb3 sin x
};
// FP64 counterpart.
struct SkyConst64 {
  double nx, nyp, nz, ca, sa, rcd, zsd;
  double ea[5];
  double eb[4];
};

// Segment-level geometry shared by the kernels.
struct SegGeom {
  int64_t n;        // samples
  int64_t nfft;
  int64_t margin;   // table points before 0 and after n-1
  int64_t ngrid;    // n + 2*margin
  double dt, fl, S0;
  double theta0;    // theta_g0 + lon
  double lambda0;   // lambda_e0
  double re_c, z_c; // site equatorial radius and polar height in light-seconds
};

}  // namespace fs
