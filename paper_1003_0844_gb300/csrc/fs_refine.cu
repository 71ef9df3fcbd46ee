// Fine search (Sec. VI.C): the F-statistic at continuous template points
// theta = (f0, f1, alpha, delta), evaluated exactly by the direct sums of
// Eqs. OS and Fab over the original samples (as the fine search of Sec. VII does), with its gradient and the reduced
// Fisher matrix of the phase (Eq. redFm-def) from the same pass, and a
// hill climb from the coarse-search candidates that uses them.
//
// Per sample k (t_k = k dt) and point:
//   phi_k = n0 . r_d(t_k) / c (Eq. pham) and its alpha, delta derivatives
//   (analytic Earth, or the caller's position table at t_k),
//   a_k, b_k and their derivatives (x = alpha - theta(t) and the delta
//   dependence of the coefficients),
//   Phi_k = f0 (t_k + phi_k) + fl phi_k + f1 (t_k^2/2 + t_k phi_k)   [cycles],
//   Sa += x_k a_k e_k, dSa_i += x_k (da_k,i - 2 pi i a_k dPhi_k,i) e_k with
//   e_k = exp(-2 pi i Phi_k), likewise for b, and the sums of a^2, a da_i,
//   dPhi_i, dPhi_i dPhi_j for <a^2>, its derivatives and the metric.
// F = 2 dt / (S0 N) (|Sa|^2/<a^2> + |Sb|^2/<b^2>) and dF follows by the
// quotient rule.  Everything is FP64: this runs on a few thousand points, not
// on the coarse grid.
//
// The hill climb is Newton's method on F with the analytic Hessian (second
// derivatives from the same pass), damped Levenberg-Marquardt style where F is
// not concave, each step limited to tau^T G tau <= 1 with G the reduced Fisher
// matrix at the start (one full correlation length, Eq. hype), scaled by eta,
// and kept only if F grew (eta doubles, up to 1), else eta quarters.
#include <math.h>
#include <algorithm>
#include "fs_internal.h"
#include "fs_model.cuh"
#include "fs_refine_df.cuh"

namespace fs {

constexpr int kPtThreads = 128;
// Samples per thread per block: 192 at most (a 2-day point in 4 blocks; measured
// fastest over 32..336 with 1024 points), fewer when the points alone leave the GPU
// short of blocks (about two waves of the kernels' 2 CTAs per SM), 8 at least.
constexpr int kPtSamplesMax = 192;
constexpr int kPtSamplesMin = 8;

// The samples [k0, k1) of this block: the n samples in gridDim.y blocks of equal size
// (a multiple of kPtThreads), so that no block is left with a sliver of the data.
__device__ __forceinline__ void block_range(int64_t n, int64_t *k0, int64_t *k1) {
  const int64_t per = ((n + gridDim.y - 1) / gridDim.y + kPtThreads - 1) / kPtThreads * kPtThreads;
  *k0 = (int64_t)blockIdx.y * per;
  *k1 = min(n, *k0 + per);
}

// Per-segment FP64 table on t_k = k dt: (cos, sin) of the orbital longitude
// lambda_E(t_k) and of the local sidereal angle theta(t_k).
__global__ void k_earth_table64(SegGeom g, dbl4 *tab) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= g.n) return;
  const double t = (double)k * g.dt;
  double sl, cl, sth, cth;
  sincos(g.lambda0 + kOmegaO * t, &sl, &cl);
  sincos(g.theta0 + kOmegaR * t, &sth, &cth);
  tab[k] = make_dbl4(cl, sl, cth, sth);
}

// The constants of each point, and their double-float form for the FP32-pipe kernels
// (computed once per point rather than by every block of those kernels).
__global__ void k_point_constants(const fs_point *pts, int npt, SegGeom g, fs_detector det, PointConst *out,
                                  FastConst *fast) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npt) return;
  const PointConst c = point_constants(pts[i], g, det);
  out[i] = c;
  fast[i] = fast_const(c, g);
}

// Accumulators per point:
//  [0, 4) Sa, Sb (re, im); [4, 20) dSa_i, dSb_i; [20, 26) sum a^2, b^2, a da_al, a da_de,
//  b db_al, b db_de;  MET: 14 more: sum dPhi_i, sum dPhi_i dPhi_j (i <= j) [cycles];
//  HESS: 46 more: d2Sa_ij, d2Sb_ij (i <= j), sum (a_i a_j + a a_ij), same for b (sky pairs).
template <bool HESS, bool MET>
struct PtLayout {
  static constexpr int kM = 26;
  static constexpr int kH = MET ? 40 : 26;
  static constexpr int kN = kH + (HESS ? 46 : 0);
};

// Grid: x = point, y = block of samples (block_range).
// EPH: phi and its sky derivatives from the caller's position table eph (r_k at
// t_k = k dt: n0 . r_k and the derivatives of n0 dotted with r_k) instead of the
// analytic orbit and rotation terms; the sidereal angle still comes from etab.
template <bool HESS, bool MET, bool EPH>
__global__ void __launch_bounds__(kPtThreads) k_points(SegGeom g, const dbl4 *__restrict__ etab,
                                                       const dbl4 *__restrict__ eph,
                                                       const double *__restrict__ x, const PointConst *pcs,
                                                       double *partial) {
  using Lt = PtLayout<HESS, MET>;
  constexpr int NA = Lt::kN;
  __shared__ PointConst c;
  __shared__ double red[kPtThreads / 32][NA];
  const int pt = blockIdx.x;
  if (threadIdx.x == 0) c = pcs[pt];
  __syncthreads();
  double acc[NA];
#pragma unroll
  for (int q = 0; q < NA; q++) acc[q] = 0.0;
  int64_t k0, k1;
  block_range(g.n, &k0, &k1);
  const double two_pi = 6.283185307179586476925286766559;
  const double four_pi2 = 39.478417604357434475337963999505;
  for (int64_t k = k0 + threadIdx.x; k < k1; k += kPtThreads) {
    const dbl4 e4 = etab[k];
    const double xk = x[k];
    const double t = (double)k * g.dt;
    const double cx = c.ca * e4.z + c.sa * e4.w;   // cos(alpha - theta)
    const double sx = c.sa * e4.z - c.ca * e4.w;   // sin(alpha - theta)
    dbl4 rk = make_dbl4(0.0, 0.0, 0.0, 0.0);
    if constexpr (EPH) rk = eph[2 * k];
    auto ndot = [&](int v) { return c.n3[v][0] * rk.x + c.n3[v][1] * rk.y + c.n3[v][2] * rk.z; };
    double phi, phi_a, phi_d;
    if constexpr (EPH) {
      phi = ndot(0);
      phi_a = ndot(1);
      phi_d = ndot(2);
    } else {
      phi = kAUls * (c.nx * e4.x + c.nyp * e4.y) + c.rcd * cx + c.zsd;
      phi_a = kAUls * (c.nx_a * e4.x + c.nyp_a * e4.y) - c.rcd * sx;
      phi_d = kAUls * (c.nx_d * e4.x + c.nyp_d * e4.y) + c.rcd_d * cx + c.zsd_d;
    }
    const double c2 = cx * cx - sx * sx, s2 = 2.0 * sx * cx;
    const double a = c.ea[0] * c2 + c.ea[1] * s2 + c.ea[2] * cx + c.ea[3] * sx + c.ea[4];
    const double b = c.eb[0] * c2 + c.eb[1] * s2 + c.eb[2] * cx + c.eb[3] * sx;
    const double a_a = -2.0 * c.ea[0] * s2 + 2.0 * c.ea[1] * c2 - c.ea[2] * sx + c.ea[3] * cx;
    const double b_a = -2.0 * c.eb[0] * s2 + 2.0 * c.eb[1] * c2 - c.eb[2] * sx + c.eb[3] * cx;
    const double a_d = c.ea_d[0] * c2 + c.ea_d[1] * s2 + c.ea_d[2] * cx + c.ea_d[3] * sx + c.ea_d[4];
    const double b_d = c.eb_d[0] * c2 + c.eb_d[1] * s2 + c.eb_d[2] * cx + c.eb_d[3] * sx;
    double ph = c.f0 * (t + phi) + g.fl * phi + c.f1 * t * (0.5 * t + phi);
    ph -= floor(ph);
    double sp, cp;
    sincospi(2.0 * ph, &sp, &cp);                   // e = cp - i sp
    const double w = c.f0 + g.fl + c.f1 * t;
    const double dP[4] = {t + phi, t * (0.5 * t + phi), w * phi_a, w * phi_d};
    const double da[4] = {0.0, 0.0, a_a, a_d}, db[4] = {0.0, 0.0, b_a, b_d};
    const double ua = xk * a, ub = xk * b;
    acc[0] += ua * cp;
    acc[1] -= ua * sp;
    acc[2] += ub * cp;
    acc[3] -= ub * sp;
#pragma unroll
    for (int i = 0; i < 4; i++) {
      // x (da_i - 2 pi i a dP_i) (cp - i sp)
      const double qa = xk * da[i], qb = xk * db[i];
      const double ra = -two_pi * ua * dP[i], rb = -two_pi * ub * dP[i];
      acc[4 + 2 * i] += qa * cp + ra * sp;
      acc[5 + 2 * i] += ra * cp - qa * sp;
      acc[12 + 2 * i] += qb * cp + rb * sp;
      acc[13 + 2 * i] += rb * cp - qb * sp;
    }
    acc[20] += a * a;
    acc[21] += b * b;
    acc[22] += a * a_a;
    acc[23] += a * a_d;
    acc[24] += b * b_a;
    acc[25] += b * b_d;
    if constexpr (MET) {
#pragma unroll
      for (int i = 0; i < 4; i++) acc[Lt::kM + i] += dP[i];
#pragma unroll
      for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = i; j < 4; j++) acc[Lt::kM + 4 + sym_idx(i, j)] += dP[i] * dP[j];
    }
    if constexpr (HESS) {
      double phi_aa, phi_ad, phi_dd;
      if constexpr (EPH) {
        phi_aa = ndot(3);
        phi_ad = ndot(4);
        phi_dd = ndot(5);
      } else {
        phi_aa = kAUls * (c.nx_aa * e4.x + c.nyp_aa * e4.y) - c.rcd * cx;
        phi_ad = kAUls * (c.nx_ad * e4.x + c.nyp_ad * e4.y) - c.rcd_d * sx;
        phi_dd = kAUls * (c.nx_dd * e4.x + c.nyp_dd * e4.y) + c.rcd_dd * cx + c.zsd_dd;
      }
      const double a_aa = -4.0 * c.ea[0] * c2 - 4.0 * c.ea[1] * s2 - c.ea[2] * cx - c.ea[3] * sx;
      const double b_aa = -4.0 * c.eb[0] * c2 - 4.0 * c.eb[1] * s2 - c.eb[2] * cx - c.eb[3] * sx;
      const double a_ad = -2.0 * c.ea_d[0] * s2 + 2.0 * c.ea_d[1] * c2 - c.ea_d[2] * sx + c.ea_d[3] * cx;
      const double b_ad = -2.0 * c.eb_d[0] * s2 + 2.0 * c.eb_d[1] * c2 - c.eb_d[2] * sx + c.eb_d[3] * cx;
      const double a_dd = c.ea_dd[0] * c2 + c.ea_dd[1] * s2 + c.ea_dd[2] * cx + c.ea_dd[3] * sx + c.ea_dd[4];
      const double b_dd = c.eb_dd[0] * c2 + c.eb_dd[1] * s2 + c.eb_dd[2] * cx + c.eb_dd[3] * sx;
#pragma unroll
      for (int i = 0; i < 4; i++) {
#pragma unroll
        for (int j = i; j < 4; j++) {
          // second derivative of Phi (cycles) and of a, b for the pair (i, j)
          double d2P = 0.0, d2a = 0.0, d2b = 0.0;
          if (i == 0 && j == 2) d2P = phi_a;
          if (i == 0 && j == 3) d2P = phi_d;
          if (i == 1 && j == 2) d2P = t * phi_a;
          if (i == 1 && j == 3) d2P = t * phi_d;
          if (i == 2 && j == 2) { d2P = w * phi_aa; d2a = a_aa; d2b = b_aa; }
          if (i == 2 && j == 3) { d2P = w * phi_ad; d2a = a_ad; d2b = b_ad; }
          if (i == 3 && j == 3) { d2P = w * phi_dd; d2a = a_dd; d2b = b_dd; }
          const int o = Lt::kH + 2 * sym_idx(i, j);
          const double Pa = xk * (d2a - four_pi2 * a * dP[i] * dP[j]);
          const double Qa = -two_pi * xk * (da[i] * dP[j] + da[j] * dP[i] + a * d2P);
          const double Pb = xk * (d2b - four_pi2 * b * dP[i] * dP[j]);
          const double Qb = -two_pi * xk * (db[i] * dP[j] + db[j] * dP[i] + b * d2P);
          acc[o] += Pa * cp + Qa * sp;
          acc[o + 1] += Qa * cp - Pa * sp;
          acc[o + 20] += Pb * cp + Qb * sp;
          acc[o + 21] += Qb * cp - Pb * sp;
        }
      }
      acc[Lt::kH + 40] += a_a * a_a + a * a_aa;
      acc[Lt::kH + 41] += a_a * a_d + a * a_ad;
      acc[Lt::kH + 42] += a_d * a_d + a * a_dd;
      acc[Lt::kH + 43] += b_a * b_a + b * b_aa;
      acc[Lt::kH + 44] += b_a * b_d + b * b_ad;
      acc[Lt::kH + 45] += b_d * b_d + b * b_dd;
    }
  }
  // block reduction in a fixed order: warps by shuffles, then over the warps
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NA; q++) {
    double v = acc[q];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) red[wp][q] = v;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < NA; q += kPtThreads) {
    double v = 0.0;
    for (int w2 = 0; w2 < kPtThreads / 32; w2++) v += red[w2][q];
    partial[((int64_t)pt * gridDim.y + blockIdx.y) * NA + q] = v;
  }
}

// ------------------------------------------------------------------ double-float form
// The same sums with the analytic Earth, arranged for the FP32 pipe (the FP64 pipe
// runs at 1/64 of its rate on this GPU).  Only the one term whose size needs more
// than the 48 bits of a double-float stays in FP64: the orbital part of the phase,
// (f0 + fl) (AU/c) n0 . (cos lambda, sin lambda) + f0 t, ~2.5e5 cycles, reduced to a
// fraction of a cycle (eight FP64 operations per sample).  The diurnal delay, the
// spindown term, exp(-2 pi i Phi) (a 257-entry table of exp(-2 pi i j/256) times a
// short series of the remainder), a, b and the F sums are double-floats; terms that
// enter a sum at ~1e-6 of its dominant part (the derivatives of a and b, the
// cross terms of the Hessian) are FP32.  Sums are kept as double-floats per thread
// and combined in FP64 in a fixed order, as in k_points.
//
// Layout of seg->etab32 (one allocation): L[n], T[n]: double-floats (cos hi, cos lo,
// sin hi, sin lo) of the orbital longitude and of the sidereal angle at t_k; X[n]:
// the data as double-floats; SC[257]: exp(-2 pi i j / 256) as (cos hi, cos lo, sin hi,
// sin lo), j = -128..128 (struct Etab32).
static size_t etab32_bytes(int64_t n) {
  return ((sizeof(float4) * 2 * n + sizeof(float2) * n + 255) & ~(size_t)255) + sizeof(float4) * 257;
}
static Etab32 etab32_view(const fs_seg *seg) {
  const int64_t n = seg->g.n;
  char *b = (char *)seg->etab32;
  Etab32 e;
  e.L = (float4 *)b;
  e.T = e.L + n;
  e.X = (float2 *)(e.T + n);
  e.SC = (float4 *)(b + ((sizeof(float4) * 2 * n + sizeof(float2) * n + 255) & ~(size_t)255));
  return e;
}

__global__ void k_earth_table32(int64_t n, const dbl4 *e64, Etab32 e) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k < n) {
    const dbl4 v = e64[k];
    const df32 cl = df_from_double(v.x), sl = df_from_double(v.y), ct = df_from_double(v.z),
               st = df_from_double(v.w);
    e.L[k] = make_float4(cl.hi, cl.lo, sl.hi, sl.lo);
    e.T[k] = make_float4(ct.hi, ct.lo, st.hi, st.lo);
  }
  if (k < 257) {
    double sj, cj;
    sincospi((double)(k - 128) / 128.0, &sj, &cj);  // angle 2 pi (k - 128) / 256
    const df32 c = df_from_double(cj), s = df_from_double(sj);
    e.SC[k] = make_float4(c.hi, c.lo, s.hi, s.lo);
  }
}

// The data as double-floats (rebuilt by every fine-search call: fs_seg_load may
// have replaced it).
__global__ void k_data32(int64_t n, const double *x64, float2 *X) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k < n) {
    const df32 v = df_from_double(x64[k]);
    X[k] = make_float2(v.hi, v.lo);
  }
}

// A point's FastConst into shared memory by the whole block (word by word).
__device__ __forceinline__ void load_fast_const(const FastConst *src, FastConst *dst) {
  static_assert(sizeof(FastConst) % 4 == 0, "copied as 32-bit words");
  const unsigned *s = (const unsigned *)src;
  unsigned *d = (unsigned *)dst;
  for (int i = threadIdx.x; i < (int)(sizeof(FastConst) / 4); i += blockDim.x) d[i] = s[i];
}

// Sums of the double-float kernels to FP64 block partials, in a fixed order.
template <int NQ>
__device__ __forceinline__ void fast_reduce(const df32 *acc, int q0, int NA, double *partial, int pt) {
  __shared__ double red[kPtThreads / 32][NQ];
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  // within a warp as double-floats (a DADD tree here cost the 1/64-rate FP64 pipe as
  // much as the orbital phase of 8 samples), across warps in FP64
#pragma unroll
  for (int q = 0; q < NQ; q++) {
    df32 v = acc[q];
    for (int o = 16; o > 0; o >>= 1)
      v = df_add(v, df32{__shfl_down_sync(0xffffffffu, v.hi, o), __shfl_down_sync(0xffffffffu, v.lo, o)});
    if (lane == 0) red[wp][q] = (double)v.hi + (double)v.lo;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < NQ; q += kPtThreads) {
    double v = 0.0;
    for (int w2 = 0; w2 < kPtThreads / 32; w2++) v += red[w2][q];
    partial[((int64_t)pt * gridDim.y + blockIdx.y) * NA + q0 + q] = v;
  }
}

// F and its gradient: accumulators [0, 26) of PtLayout (Sa, Sb, dSa_i, dSb_i, sums of
// a^2, b^2 and a da, b db).  NA: stride of a block's partials.
__global__ void __launch_bounds__(kPtThreads) k_points_fg(SegGeom g, const dbl4 *__restrict__ etab, Etab32 et,
                                                          const FastConst *fcs, double *partial, int NA) {
  __shared__ FastConst c;
  __shared__ float4 sc[257];
  const int pt = blockIdx.x;
  load_fast_const(fcs + pt, &c);
  for (int i = threadIdx.x; i < 257; i += blockDim.x) sc[i] = et.SC[i];
  __syncthreads();
  df32 acc[26];
#pragma unroll
  for (int q = 0; q < 26; q++) acc[q] = df32{0.f, 0.f};
  int64_t k0, k1;
  block_range(g.n, &k0, &k1);
  for (int64_t k = k0 + threadIdx.x; k < k1; k += kPtThreads) {
    const FastSample s = fast_sample(c, g, etab, et, sc, k);
    fg_sample(c, s, acc);
  }
  fast_reduce<26>(acc, 0, NA, partial, pt);
}

// The Hessian's accumulators [q0, q0 + 46) of PtLayout: d2Sa_ij, d2Sb_ij (i <= j) and
// the sums a_i a_j + a a_ij, b_i b_j + b b_ij over the sky pairs; SIG selects signal a
// or b (its 20 pair sums and 3 sums).
// One kernel per signal (SIG 0: a, 1: b), 23 sums each: 2% faster than one kernel with
// all 46 (255 registers and spills); forcing 3 CTAs per SM (168 registers) gained nothing.
template <int SIG>
__global__ void __launch_bounds__(kPtThreads) k_points_h(SegGeom g, const dbl4 *__restrict__ etab, Etab32 et,
                                                         const FastConst *fcs, double *partial, int NA, int q0) {
  __shared__ FastConst c;
  __shared__ float4 sc[257];
  const int pt = blockIdx.x;
  load_fast_const(fcs + pt, &c);
  for (int i = threadIdx.x; i < 257; i += blockDim.x) sc[i] = et.SC[i];
  __syncthreads();
  static_assert(SIG == 0 || SIG == 1, "one signal per kernel");
  constexpr int NQ = 23;
  df32 acc[NQ];
#pragma unroll
  for (int q = 0; q < NQ; q++) acc[q] = df32{0.f, 0.f};
  int64_t k0, k1;
  block_range(g.n, &k0, &k1);
  for (int64_t k = k0 + threadIdx.x; k < k1; k += kPtThreads) {
    const FastSample s = fast_sample(c, g, etab, et, sc, k);  // the same e as k_points_fg
    hess_sample<SIG>(c, s, acc);
  }
  // this signal's pairs, then its three sums of a_i a_j + a a_ij
  fast_reduce<20>(acc, q0 + 20 * SIG, NA, partial, pt);
  fast_reduce<3>(acc + 20, q0 + 40 + 3 * SIG, NA, partial, pt);
}

// The metric's accumulators [26, 40) in FP64 (first pass of a climb only): sums of
// dP_i and dP_i dP_j [cycles].
__global__ void __launch_bounds__(kPtThreads) k_points_met(SegGeom g, const dbl4 *__restrict__ etab,
                                                           const PointConst *pcs, double *partial, int NA) {
  __shared__ PointConst c;
  const int pt = blockIdx.x;
  if (threadIdx.x == 0) c = pcs[pt];
  __syncthreads();
  double acc[14];
#pragma unroll
  for (int q = 0; q < 14; q++) acc[q] = 0.0;
  int64_t k0, k1;
  block_range(g.n, &k0, &k1);
  for (int64_t k = k0 + threadIdx.x; k < k1; k += kPtThreads) {
    const dbl4 e4 = etab[k];
    const double t = (double)k * g.dt;
    const double cx = c.ca * e4.z + c.sa * e4.w;
    const double sx = c.sa * e4.z - c.ca * e4.w;
    const double phi = kAUls * (c.nx * e4.x + c.nyp * e4.y) + c.rcd * cx + c.zsd;
    const double phi_a = kAUls * (c.nx_a * e4.x + c.nyp_a * e4.y) - c.rcd * sx;
    const double phi_d = kAUls * (c.nx_d * e4.x + c.nyp_d * e4.y) + c.rcd_d * cx + c.zsd_d;
    const double w = c.f0 + g.fl + c.f1 * t;
    const double dP[4] = {t + phi, t * (0.5 * t + phi), w * phi_a, w * phi_d};
#pragma unroll
    for (int i = 0; i < 4; i++) acc[i] += dP[i];
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
      for (int j = i; j < 4; j++) acc[4 + sym_idx(i, j)] += dP[i] * dP[j];
  }
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  __shared__ double red[kPtThreads / 32][14];
#pragma unroll
  for (int q = 0; q < 14; q++) {
    double v = acc[q];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) red[wp][q] = v;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < 14; q += kPtThreads) {
    double v = 0.0;
    for (int w2 = 0; w2 < kPtThreads / 32; w2++) v += red[w2][q];
    partial[((int64_t)pt * gridDim.y + blockIdx.y) * NA + 26 + q] = v;
  }
}

// F, gradient, Hessian (upper triangle) and reduced Fisher matrix (rad^2, upper
// triangle) per point from the block partials, summed in block order.
template <bool HESS, bool MET>
__global__ void k_points_final(const double *partial, int nblk, int npt, SegGeom g, double *F, double *grad,
                               double *hess, double *metric, double *amp) {
  using Lt = PtLayout<HESS, MET>;
  constexpr int NA = Lt::kN;
  const int pt = blockIdx.x * blockDim.x + threadIdx.x;
  if (pt >= npt) return;
  double s[NA];
  for (int q = 0; q < NA; q++) s[q] = 0.0;
  for (int b = 0; b < nblk; b++)
    for (int q = 0; q < NA; q++) s[q] += partial[((int64_t)pt * nblk + b) * NA + q];
  const double n = (double)g.n;
  const double cF = 2.0 * g.dt / (g.S0 * n);
  double Fv = 0.0, gv[4] = {0, 0, 0, 0}, hv[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  for (int u = 0; u < 2; u++) {  // signal a, then b
    const double Sr = s[2 * u], Si = s[2 * u + 1];
    const double M = s[20 + u] / n;
    const double P = Sr * Sr + Si * Si;
    double dM[4] = {0.0, 0.0, 2.0 * s[22 + 2 * u] / n, 2.0 * s[23 + 2 * u] / n};
    double dSr[4], dSi[4], dPv[4];
    for (int i = 0; i < 4; i++) {
      dSr[i] = s[4 + 8 * u + 2 * i];
      dSi[i] = s[5 + 8 * u + 2 * i];
      dPv[i] = 2.0 * (Sr * dSr[i] + Si * dSi[i]);
    }
    Fv += P / M;
    for (int i = 0; i < 4; i++) gv[i] += dPv[i] / M - P * dM[i] / (M * M);
    if constexpr (HESS) {
      for (int i = 0; i < 4; i++) {
        for (int j = i; j < 4; j++) {
          const int p = sym_idx(i, j);
          const double d2r = s[Lt::kH + 20 * u + 2 * p], d2i = s[Lt::kH + 20 * u + 2 * p + 1];
          const double Pij = 2.0 * (dSr[i] * dSr[j] + dSi[i] * dSi[j] + Sr * d2r + Si * d2i);
          double Mij = 0.0;
          if (i >= 2 && j >= 2) Mij = 2.0 * s[Lt::kH + 40 + 3 * u + (i - 2) + (j - 2)] / n;
          hv[p] += Pij / M - (dPv[i] * dM[j] + dPv[j] * dM[i]) / (M * M) - P * Mij / (M * M) +
                   2.0 * P * dM[i] * dM[j] / (M * M * M);
        }
      }
    }
  }
  F[pt] = cF * Fv;
  if (amp) {  // Eq. amle0: 2 <x h_i> / <a^2> with <x a cos phi> = Re(Sa)/N, <x a sin phi> = -Im(Sa)/N
    amp[4 * pt + 0] = 2.0 * s[0] / s[20];
    amp[4 * pt + 1] = 2.0 * s[2] / s[21];
    amp[4 * pt + 2] = -2.0 * s[1] / s[20];
    amp[4 * pt + 3] = -2.0 * s[3] / s[21];
  }
  if (grad)
    for (int i = 0; i < 4; i++) grad[4 * pt + i] = cF * gv[i];
  if constexpr (HESS) {
    if (hess)
      for (int p = 0; p < 10; p++) hess[10 * pt + p] = cF * hv[p];
  }
  if constexpr (MET) {
    const double fp2 = 39.478417604357434475337963999505;  // (2 pi)^2
    for (int i = 0; i < 4; i++)
      for (int j = i; j < 4; j++)
        metric[10 * pt + sym_idx(i, j)] =
            fp2 * (s[Lt::kM + 4 + sym_idx(i, j)] / n - (s[Lt::kM + i] / n) * (s[Lt::kM + j] / n));
  }
}

__global__ void k_points_from_candidates(const fs_candidate *cand, int n, const double *alpha, const double *delta,
                                         const double *f1, double df, fs_point *pts) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const fs_candidate c = cand[i];
  pts[i] = fs_point{(double)c.bin * df, f1[c.spin], alpha[c.sky], delta[c.sky]};
}

// ------------------------------------------------------------------ hill climb
// State per point: F, gradient and Hessian of F at the current point, the
// reduced Fisher matrix at the starting point (it measures the step: one unit
// of tau^T G tau is a full loss of correlation, Eq. hype), and the step factor.
struct ClimbState {
  double F, g[4], H[10], G[10], eta;
};

// Newton step: solve (-H + lambda diag(max(-H_ii, 2 F G_ii))) D = g, raising
// lambda from 0 until the matrix is positive definite (Levenberg-Marquardt);
// then limit D to D^T G D <= 1.
__device__ inline bool climb_step(const ClimbState &s, double D[4]) {
  double dg[4];
  for (int i = 0; i < 4; i++) {
    dg[i] = fmax(-s.H[sym_idx(i, i)], 2.0 * s.F * s.G[sym_idx(i, i)]);
    if (!(dg[i] > 0.0)) return false;
  }
  double sc[4], r[4];
  for (int i = 0; i < 4; i++) {
    sc[i] = rsqrt(dg[i]);
    r[i] = sc[i] * s.g[i];
  }
  for (double lambda = 0.0; lambda <= 1e3; lambda = lambda == 0.0 ? 1e-6 : 10.0 * lambda) {
    double L[4][4] = {};
    bool ok = true;
    for (int i = 0; i < 4 && ok; i++) {
      for (int j = 0; j <= i; j++) {
        double v = -sc[i] * sc[j] * s.H[sym_idx(i, j)] + (i == j ? lambda : 0.0);
        for (int k = 0; k < j; k++) v -= L[i][k] * L[j][k];
        if (i == j) {
          if (!(v > 0.0)) { ok = false; break; }
          L[i][i] = sqrt(v);
        } else {
          L[i][j] = v / L[j][j];
        }
      }
    }
    if (!ok) continue;
    double y[4], u[4];
    for (int i = 0; i < 4; i++) {
      double v = r[i];
      for (int k = 0; k < i; k++) v -= L[i][k] * y[k];
      y[i] = v / L[i][i];
    }
    for (int i = 3; i >= 0; i--) {
      double v = y[i];
      for (int k = i + 1; k < 4; k++) v -= L[k][i] * u[k];
      u[i] = v / L[i][i];
    }
    for (int i = 0; i < 4; i++) D[i] = u[i] * sc[i];
    double m = 0.0;
    for (int i = 0; i < 4; i++)
      for (int j = 0; j < 4; j++) m += D[i] * s.G[sym_idx(i, j)] * D[j];
    if (m > 1.0) {
      const double f = rsqrt(m);
      for (int i = 0; i < 4; i++) D[i] *= f;
    }
    return true;
  }
  return false;
}

__global__ void k_climb_init(int npt, const double *F, const double *grad, const double *hess, const double *metric,
                             ClimbState *st) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npt) return;
  ClimbState s;
  s.F = F[i];
  for (int q = 0; q < 4; q++) s.g[q] = grad[4 * i + q];
  for (int q = 0; q < 10; q++) {
    s.H[q] = hess[10 * i + q];
    s.G[q] = metric[10 * i + q];
  }
  s.eta = 1.0;
  st[i] = s;
}

__global__ void k_climb_propose(int npt, const fs_point *pts, const ClimbState *st, fs_point *trial) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npt) return;
  const ClimbState s = st[i];
  fs_point p = pts[i];
  double D[4] = {0.0, 0.0, 0.0, 0.0};
  if (!(s.F > 0.0) || !climb_step(s, D)) D[0] = D[1] = D[2] = D[3] = 0.0;
  p.f0 += s.eta * D[0];
  p.f1 += s.eta * D[1];
  p.alpha += s.eta * D[2];
  p.delta += s.eta * D[3];
  const double half_pi = 1.5707963267948966192313216916398;
  if (p.delta > half_pi) { p.delta = 2 * half_pi - p.delta; p.alpha += 2 * half_pi; }
  if (p.delta < -half_pi) { p.delta = -2 * half_pi - p.delta; p.alpha += 2 * half_pi; }
  p.alpha -= 4 * half_pi * floor(p.alpha / (4 * half_pi));
  trial[i] = p;
}

__global__ void k_climb_accept(int npt, fs_point *pts, ClimbState *st, const fs_point *trial, const double *Ft,
                               const double *gt, const double *Ht) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npt) return;
  ClimbState s = st[i];
  if (Ft[i] > s.F) {
    pts[i] = trial[i];
    s.F = Ft[i];
    for (int q = 0; q < 4; q++) s.g[q] = gt[4 * i + q];
    for (int q = 0; q < 10; q++) s.H[q] = Ht[10 * i + q];
    s.eta = fmin(1.0, 2.0 * s.eta);
  } else {
    s.eta *= 0.25;
  }
  st[i] = s;
}

__global__ void k_climb_out(int npt, const ClimbState *st, double *F) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < npt) F[i] = st[i].F;
}

// ------------------------------------------------------------------ host
// The fine search's tables: built by the first call on a segment; the double-float
// copy of the data is refreshed by every call (fs_seg_load may have replaced it).
static fs_status earth_table(fs_seg *seg, cudaStream_t st) {
  const unsigned nb = (unsigned)((seg->g.n + 255) / 256);
  if (!seg->etab64) {
    if (cudaMalloc(&seg->etab64, sizeof(dbl4) * seg->g.n) != cudaSuccess) {
      cudaGetLastError();
      seg->etab64 = nullptr;
      return FS_ERR_NOMEM;
    }
    k_earth_table64<<<nb, 256, 0, st>>>(seg->g, (dbl4 *)seg->etab64);
    seg->ctx->launches += 1;
  }
  if (!seg->eph) {
    if (!seg->etab32) {
      if (cudaMalloc(&seg->etab32, etab32_bytes(seg->g.n)) != cudaSuccess) {
        cudaGetLastError();
        seg->etab32 = nullptr;
        return FS_ERR_NOMEM;
      }
      const unsigned nt = nb > 2 ? nb : 2;  // at least the 257 table entries
      k_earth_table32<<<nt, 256, 0, st>>>(seg->g.n, (const dbl4 *)seg->etab64, etab32_view(seg));
      seg->ctx->launches += 1;
    }
    k_data32<<<nb, 256, 0, st>>>(seg->g.n, seg->x64, etab32_view(seg).X);
    seg->ctx->launches += 1;
  }
  return cuda_status(cudaGetLastError());
}

static size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

// Fine-search workspace: point constants, block partials, and for the climb its
// state, trial points and their F, gradients, Hessians and metrics.
struct RefWs {
  PointConst *pc;
  FastConst *fc;
  double *partial;
  ClimbState *state;
  fs_point *trial;
  double *Ft, *gt, *Ht, *Gt;
  int nblk;
};

static fs_status refine_ws(fs_ctx *ctx, const fs_seg *seg, int npt, bool climb, cudaStream_t st, RefWs *w) {
  int nsm = 0;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device) != cudaSuccess) return FS_ERR_CUDA;
  const int64_t n = seg->g.n;
  const int64_t lo = (n + (int64_t)kPtThreads * kPtSamplesMax - 1) / ((int64_t)kPtThreads * kPtSamplesMax);
  const int64_t hi = (n + (int64_t)kPtThreads * kPtSamplesMin - 1) / ((int64_t)kPtThreads * kPtSamplesMin);
  const int64_t want = (4 * (int64_t)nsm + npt - 1) / npt;  // blocks per point for ~2 waves
  w->nblk = (int)std::min(hi, std::max(lo, want));  // <= 65535 for n <= 2^26
  constexpr int kMaxAcc = PtLayout<true, true>::kN;
  size_t off = 0;
  const size_t o_pc = off; off = al256(off + sizeof(PointConst) * npt);
  const size_t o_fc = off; off = al256(off + sizeof(FastConst) * npt);
  const size_t o_pa = off; off = al256(off + sizeof(double) * kMaxAcc * (size_t)w->nblk * npt);
  size_t o_st = 0, o_tr = 0, o_ft = 0, o_gt = 0, o_Ht = 0, o_Gt = 0;
  if (climb) {
    o_st = off; off = al256(off + sizeof(ClimbState) * npt);
    o_tr = off; off = al256(off + sizeof(fs_point) * npt);
    o_ft = off; off = al256(off + sizeof(double) * npt);
    o_gt = off; off = al256(off + sizeof(double) * 4 * npt);
    o_Ht = off; off = al256(off + sizeof(double) * 10 * npt);
    o_Gt = off; off = al256(off + sizeof(double) * 10 * npt);
  }
  fs_status s = ensure_buffer(&ctx->rws, &ctx->rws_bytes, off, st);
  if (s != FS_OK) return s;
  char *b = (char *)ctx->rws;
  w->pc = (PointConst *)(b + o_pc);
  w->fc = (FastConst *)(b + o_fc);
  w->partial = (double *)(b + o_pa);
  w->state = climb ? (ClimbState *)(b + o_st) : nullptr;
  w->trial = climb ? (fs_point *)(b + o_tr) : nullptr;
  w->Ft = climb ? (double *)(b + o_ft) : nullptr;
  w->gt = climb ? (double *)(b + o_gt) : nullptr;
  w->Ht = climb ? (double *)(b + o_Ht) : nullptr;
  w->Gt = climb ? (double *)(b + o_Gt) : nullptr;
  return FS_OK;
}

// With the analytic Earth the sums run in the double-float kernels (F and gradient;
// the Hessian; the metric in FP64); with a caller's position table in k_points.
template <bool HESS, bool MET>
static int launch_points(fs_seg *seg, const RefWs &w, int npt, double *F, double *grad, double *hess,
                         double *metric, double *amp, cudaStream_t st) {
  using Lt = PtLayout<HESS, MET>;
  const dim3 grid(npt, w.nblk);
  const dbl4 *et = (const dbl4 *)seg->etab64;
  int launches = 2;
  if (seg->eph) {
    k_points<HESS, MET, true><<<grid, kPtThreads, 0, st>>>(seg->g, et, seg->eph, seg->x64, w.pc, w.partial);
  } else {
    const Etab32 e32 = etab32_view(seg);
    k_points_fg<<<grid, kPtThreads, 0, st>>>(seg->g, et, e32, w.fc, w.partial, Lt::kN);
    if constexpr (HESS) {
      k_points_h<0><<<grid, kPtThreads, 0, st>>>(seg->g, et, e32, w.fc, w.partial, Lt::kN, Lt::kH);
      k_points_h<1><<<grid, kPtThreads, 0, st>>>(seg->g, et, e32, w.fc, w.partial, Lt::kN, Lt::kH);
      launches += 2;
    }
    if constexpr (MET) {
      k_points_met<<<grid, kPtThreads, 0, st>>>(seg->g, et, w.pc, w.partial, Lt::kN);
      launches++;
    }
  }
  k_points_final<HESS, MET><<<(unsigned)((npt + 127) / 128), 128, 0, st>>>(w.partial, w.nblk, npt, seg->g, F, grad,
                                                                            hess, metric, amp);
  return launches;
}

static fs_status points_pass(fs_ctx *ctx, fs_seg *seg, const RefWs &w, const fs_point *pts, int npt, double *F,
                             double *grad, double *hess, double *metric, cudaStream_t st, double *amp = nullptr) {
  k_point_constants<<<(unsigned)((npt + 127) / 128), 128, 0, st>>>(pts, npt, seg->g, ctx->det, w.pc, w.fc);
  int nl = 0;
  if (hess && metric) nl = launch_points<true, true>(seg, w, npt, F, grad, hess, metric, amp, st);
  else if (hess) nl = launch_points<true, false>(seg, w, npt, F, grad, hess, metric, amp, st);
  else if (metric) nl = launch_points<false, true>(seg, w, npt, F, grad, hess, metric, amp, st);
  else nl = launch_points<false, false>(seg, w, npt, F, grad, hess, metric, amp, st);
  ctx->launches += 1 + nl;
  return cuda_status(cudaGetLastError());
}

fs_status fstat_points(fs_ctx *ctx, fs_seg *seg, const fs_point *pts, int npt, double *F, double *grad,
                       double *hess, double *metric, cudaStream_t st) {
  ProfScope ps(ctx, PROF_OTHER, st);
  fs_status s = earth_table(seg, st);
  if (s != FS_OK) return s;
  RefWs w;
  s = refine_ws(ctx, seg, npt, false, st, &w);
  if (s != FS_OK) return s;
  return points_pass(ctx, seg, w, pts, npt, F, grad, hess, metric, st);
}

fs_status amplitudes(fs_ctx *ctx, fs_seg *seg, const fs_point *pts, int npt, double *amp, cudaStream_t st) {
  ProfScope ps(ctx, PROF_OTHER, st);
  fs_status s = earth_table(seg, st);
  if (s != FS_OK) return s;
  RefWs w;
  s = refine_ws(ctx, seg, npt, true, st, &w);  // the climb's F buffer receives the (unused) F
  if (s != FS_OK) return s;
  return points_pass(ctx, seg, w, pts, npt, w.Ft, nullptr, nullptr, nullptr, st, amp);
}

fs_status refine_points(fs_ctx *ctx, fs_seg *seg, fs_point *pts, int npt, int nsteps, double *F, cudaStream_t st) {
  ProfScope ps(ctx, PROF_OTHER, st);
  fs_status s = earth_table(seg, st);
  if (s != FS_OK) return s;
  RefWs w;
  s = refine_ws(ctx, seg, npt, true, st, &w);
  if (s != FS_OK) return s;
  const unsigned nb = (unsigned)((npt + 127) / 128);
  // state at the starting points: F, gradient, Hessian and the reduced Fisher matrix
  s = points_pass(ctx, seg, w, pts, npt, w.Ft, w.gt, w.Ht, w.Gt, st);
  if (s != FS_OK) return s;
  k_climb_init<<<nb, 128, 0, st>>>(npt, w.Ft, w.gt, w.Ht, w.Gt, w.state);
  ctx->launches += 1;
  for (int it = 0; it < nsteps; it++) {
    k_climb_propose<<<nb, 128, 0, st>>>(npt, pts, w.state, w.trial);
    s = points_pass(ctx, seg, w, w.trial, npt, w.Ft, w.gt, w.Ht, nullptr, st);
    if (s != FS_OK) return s;
    k_climb_accept<<<nb, 128, 0, st>>>(npt, pts, w.state, w.trial, w.Ft, w.gt, w.Ht);
    ctx->launches += 2;
  }
  k_climb_out<<<nb, 128, 0, st>>>(npt, w.state, F);
  ctx->launches += 1;
  return cuda_status(cudaGetLastError());
}

// The starting curvature of the resampled-F ascent: the Gauss-Newton Hessian of F
// near a maximum, H = -2 F G (F(theta + tau) ~ F(theta) (1 - tau^T G tau), Eq.
// TaylorC2), with which the first step is G^-1 grad F / (2 F).
__global__ void k_gauss_hessian(int npt, const double *F, const double *G, double *H) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npt) return;
  for (int q = 0; q < 10; q++) H[10 * i + q] = -2.0 * F[i] * G[10 * i + q];
}

// Accept the trial point if F grew; then update the curvature B = -H by BFGS from
// the step s and the gradient change y = g_old - g_new (the quasi-Newton secant
// condition B s = y for the minimisation of -F), skipped unless s^T y > 0 so that
// B stays positive definite.  Over a long, flat ridge of F (the f0-sky correlation)
// this learns the ridge's curvature, where the fixed -2 F G is far off.
__global__ void k_bfgs_accept(int npt, fs_point *pts, ClimbState *st, const fs_point *trial, const double *Ft,
                              const double *gt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npt) return;
  ClimbState c = st[i];
  if (Ft[i] > c.F) {
    const fs_point a = pts[i], b = trial[i];
    const double two_pi = 6.283185307179586476925286766559;
    const double sv[4] = {b.f0 - a.f0, b.f1 - a.f1, remainder(b.alpha - a.alpha, two_pi), b.delta - a.delta};
    double y[4], Bs[4], sBs = 0.0, sy = 0.0;
    for (int q = 0; q < 4; q++) y[q] = c.g[q] - gt[4 * i + q];
    for (int r = 0; r < 4; r++) {
      Bs[r] = 0.0;
      for (int q = 0; q < 4; q++) Bs[r] -= c.H[sym_idx(r, q)] * sv[q];
      sBs += sv[r] * Bs[r];
      sy += sv[r] * y[r];
    }
    if (sy > 0.0 && sBs > 0.0)
      for (int r = 0; r < 4; r++)
        for (int q = r; q < 4; q++) c.H[sym_idx(r, q)] += Bs[r] * Bs[q] / sBs - y[r] * y[q] / sy;
    pts[i] = b;
    c.F = Ft[i];
    for (int q = 0; q < 4; q++) c.g[q] = gt[4 * i + q];
    c.eta = fmin(1.0, 2.0 * c.eta);
  } else {
    c.eta *= 0.25;
  }
  st[i] = c;
}

fs_status refine_resampled(fs_ctx *ctx, fs_seg *seg, fs_point *pts, int npt, int nsteps, double *F, cudaStream_t st) {
  if (seg->d.precision != FS_PREC_F32 || seg->d.interp != FS_INTERP_SPLINE2X || seg->eph) return FS_ERR_UNSUPPORTED;
  ProfScope ps(ctx, PROF_OTHER, st);
  fs_status s = earth_table(seg, st);
  if (s != FS_OK) return s;
  RefWs w;
  s = refine_ws(ctx, seg, npt, true, st, &w);
  if (s != FS_OK) return s;
  const unsigned nb = (unsigned)((npt + 127) / 128);
  // the reduced Fisher matrix at the starting points (w.Ft receives the exact F, unused)
  s = points_pass(ctx, seg, w, pts, npt, w.Ft, nullptr, nullptr, w.Gt, st);
  if (s != FS_OK) return s;
  // F and its gradient from the adjoint kernels at the starting points
  s = fstat_resampled(ctx, seg, pts, npt, nullptr, w.Ft, w.gt, st);
  if (s != FS_OK) return s;
  k_gauss_hessian<<<nb, 128, 0, st>>>(npt, w.Ft, w.Gt, w.Ht);
  k_climb_init<<<nb, 128, 0, st>>>(npt, w.Ft, w.gt, w.Ht, w.Gt, w.state);
  ctx->launches += 2;
  for (int it = 0; it < nsteps; it++) {
    k_climb_propose<<<nb, 128, 0, st>>>(npt, pts, w.state, w.trial);
    s = fstat_resampled(ctx, seg, w.trial, npt, nullptr, w.Ft, w.gt, st);
    if (s != FS_OK) return s;
    k_bfgs_accept<<<nb, 128, 0, st>>>(npt, pts, w.state, w.trial, w.Ft, w.gt);
    ctx->launches += 2;
  }
  k_climb_out<<<nb, 128, 0, st>>>(npt, w.state, F);
  ctx->launches += 1;
  return cuda_status(cudaGetLastError());
}

fs_status points_from_candidates(fs_ctx *ctx, fs_seg *seg, const fs_candidate *cand, int n, const double *alpha,
                                 const double *delta, const double *f1, fs_point *pts, cudaStream_t st) {
  const double df = 1.0 / ((double)seg->g.nfft * seg->g.dt);
  k_points_from_candidates<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(cand, n, alpha, delta, f1, df, pts);
  ctx->launches += 1;
  return cuda_status(cudaGetLastError());
}

}  // namespace fs
