// One output sample of the FP32 resampling of Sec. VI.A (A1): the source time of
// Eq. (eq:Bt), the data there, a and b, the delay and the spindown phase argument,
// shared by the coarse search's demodulation (k_demod32) and the kernels of the
// resampled F at continuous points (fs_adjoint.cu).
#pragma once
#include "fs_common.cuh"

namespace fs {

struct DemodArgs {
  SegGeom g;
  df32 dt2;            // dt as double-float
  float dt, inv_dt, two_over_dt;
  df32 fl;
  const SkyConst32 *sky;
  const float4 *tab0, *tab1;  // indexed by m + margin
  const float4 *eph0, *eph1;  // caller's position table (EPH), indexed by m + margin
  const float *eph2;
  const float4 *coef;         // spline intervals [2n]
  const float *x32;           // data, nearest-neighbour path
  float2 *ya, *yb, *qq;       // [nsky][stride]
  int64_t stride, npad;
  float2 *partial;            // [nsky][gridDim.x]: block sums of a^2, b^2
  double *tsrc;               // optional [n] (first sky only)
};

// Steps 1-6 and 8 of one output sample j < n (t_b = j dt):
//  t_j = m1 dt + tau (one Newton step on t + phi_m(t) = t_b from a first delay
//  estimate), phi_m(t_j) and its time derivative, x~(t_j), a(t_j), b(t_j) and
//  Q_j = t_j (t_j/2 + phi_m(t_j)) as a double-float.  spl_c, spl_f: the spline interval
//  and the position in it (spl_c zero outside the data); U0: the orbit table at m1
//  (analytic Earth).
struct ResampledSample {
  float xr, av, bv, cx, sx, phidot, tau;
  int64_t m1;
  df32 phim, Q;
  float4 spl_c, U0;
  float spl_f;
};

template <int INTERP, bool EPH>
__device__ __forceinline__ ResampledSample resample_sample(const DemodArgs &A, const SkyConst32 &K, int64_t j) {
  ResampledSample r;
  r.spl_c = make_float4(0.f, 0.f, 0.f, 0.f);
  r.U0 = r.spl_c;
  r.spl_f = 0.f;
  const int64_t M = A.g.margin;
  // 1) delay at the output time t_b = j dt, plain FP32 (only seeds the solve)
  float phi0;
  if constexpr (EPH) {
    const float4 E0 = A.eph0[j + M], E1 = A.eph1[j + M];
    phi0 = fmaf(K.nx.hi, E0.x, fmaf(K.nyp.hi, E0.z, K.nz.hi * E1.x));
  } else {
    const float4 T0 = A.tab0[j + M], T1 = A.tab1[j + M];
    phi0 = fmaf(K.nx.hi, T0.x, K.nyp.hi * T0.z) + fmaf(K.rcd, K.ca * T1.x + K.sa * T1.y, K.zsd);
  }
  // 2) first source time t1 = m1 dt + tau1 with t1 - t_b = -phi0 (up to rounding)
  const float kf = rintf(-phi0 * A.inv_dt);
  const int k1 = (int)kf;
  const df32 kd = two_prod(kf, A.dt2.hi);  // k1 dt as an exact pair (plus kf * dt.lo)
  const float kdlo = fmaf(kf, A.dt2.lo, kd.lo);
  const float tau1 = (-phi0 - kd.hi) - kdlo;
  // |phi0| <= 600 s keeps m1 inside the margins; the clamp guards the table reads
  const int64_t m1 = j + k1;
  const int64_t mi = min(max(m1 + M, (int64_t)0), A.g.ngrid - 1);
  const float4 U1 = A.tab1[mi];
  df32 P;
  float orb, rot, phidot;
  const float er = (float)kOmegaR * tau1;
  const float ce = 1.f - 0.5f * er * er, se = er - er * er * er * (1.f / 6.f);
  const float cth = fmaf(U1.x, ce, -U1.y * se), sth = fmaf(U1.y, ce, U1.x * se);
  float cx = fmaf(K.ca, cth, K.sa * sth);   // cos(alpha - theta(t1))
  float sx = fmaf(K.sa, cth, -K.ca * sth);  // sin(alpha - theta(t1))
  if constexpr (EPH) {
    // 3) delay at t1: n0 . r_m1 as double-float plus tau1 n0 . v_m1
    const float4 V0 = A.eph0[mi], V1 = A.eph1[mi];
    const float vz = A.eph2[mi];
    P = df_add(df_add(df_mul(K.nx, df32{V0.x, V0.y}), df_mul(K.nyp, df32{V0.z, V0.w})),
               df_mul(K.nz, df32{V1.x, V1.y}));
    phidot = fmaf(K.nx.hi, V1.z, fmaf(K.nyp.hi, V1.w, K.nz.hi * vz));
    orb = tau1 * phidot;
    rot = 0.f;
  } else {
    // 3) delay at t1: orbit term as double-float at the grid point, rotated by Omega_o tau1
    const float4 U0 = A.tab0[mi];
    r.U0 = U0;
    P = df_add(df_mul(K.nx, df32{U0.x, U0.y}), df_mul(K.nyp, df32{U0.z, U0.w}));
    const float eo = (float)kOmegaO * tau1;
    const float Qo = fmaf(-K.nx.hi, U0.z, K.nyp.hi * U0.x);  // d(orbit)/d(lambda)
    orb = fmaf(eo, Qo, -0.5f * eo * eo * P.hi);
    rot = fmaf(K.rcd, cx, K.zsd);
    phidot = fmaf((float)kOmegaO, Qo, K.rcd * (float)kOmegaR * sx);
  }
  // 4) Newton step on g(t) = t + phi_m(t) - t_b at t1
  const df32 Ah = two_sum(kd.hi, P.hi);
  const float gres = ((Ah.hi + tau1) + (Ah.lo + kdlo)) + ((P.lo + orb) + rot);
  const float delta = -gres / (1.f + phidot);
  const float tau = tau1 + delta;  // t_j = m1 dt + tau
  const float small = ((P.lo + orb) + rot) + phidot * delta;
  const df32 phim = quick_two_sum(P.hi, small);  // phi_m(t_j)
  const float eta = (float)kOmegaR * delta;
  const float cxj = fmaf(sx, eta, cx), sxj = fmaf(-cx, eta, sx);
  cx = cxj;
  sx = sxj;
  // 5) data at the source time
  float xr = 0.f;
  if (INTERP == FS_INTERP_SPLINE2X) {
    const float v = tau * A.two_over_dt;
    const float fv = floorf(v);
    const int64_t i = 2 * m1 + (int64_t)fv;
    const float f = v - fv;
    const int64_t ilast = 2 * A.g.n - 2;
    if ((i >= 0 && i < ilast) || (i == ilast && f == 0.f)) {
      const float4 c = A.coef[i];
      xr = fmaf(f, fmaf(f, fmaf(f, c.w, c.z), c.y), c.x);
      r.spl_c = c;
      r.spl_f = f;
    }
  } else {
    const int64_t kk = m1 + (int64_t)rintf(tau * A.inv_dt);
    if (kk >= 0 && kk < A.g.n) xr = A.x32[kk];
  }
  // 6) amplitude modulation at t_j
  const float c2 = fmaf(cx, cx, -sx * sx), s2 = 2.f * sx * cx;
  const float av = fmaf(K.ea[0], c2, fmaf(K.ea[1], s2, fmaf(K.ea[2], cx, fmaf(K.ea[3], sx, K.ea[4]))));
  const float bv = fmaf(K.eb[0], c2, fmaf(K.eb[1], s2, fmaf(K.eb[2], cx, K.eb[3] * sx)));
  // 8) Q_j = t_j (t_j/2 + phi_m(t_j)) as double-float
  const df32 tj = df_add_f(df32{U1.z, U1.w}, tau);
  const df32 U = df_add(df32{0.5f * tj.hi, 0.5f * tj.lo}, phim);
  r.Q = df_mul(tj, U);
  r.xr = xr;
  r.av = av;
  r.bv = bv;
  r.cx = cx;
  r.sx = sx;
  r.phidot = phidot;
  r.tau = tau;
  r.m1 = m1;
  r.phim = phim;
  return r;
}

}  // namespace fs
