// The fine search's per-point constants and the per-sample arithmetic of its
// double-float kernels (fs_refine.cu), as host-and-device functions so that a
// host-compiled check can run them against an FP64 evaluation of the same sums.
#pragma once
#include "fs_common.cuh"
#include "fs_model.cuh"

namespace fs {

// Per-point constants: the ecliptic-frame components of n0 (Eq. pha4) and of
// its alpha/delta derivatives (first and second), the site terms
// (r_e/c) cos(delta), (z/c) sin(delta) and derivatives, and the Fourier
// coefficients of a, b with their first and second delta derivatives.
struct PointConst {
  double f0, f1, ca, sa;
  double nx, nyp, nx_a, nyp_a, nx_d, nyp_d, nx_aa, nyp_aa, nx_ad, nyp_ad, nx_dd, nyp_dd;
  double rcd, rcd_d, rcd_dd, zsd, zsd_d, zsd_dd;
  double ea[5], eb[4], ea_d[5], eb_d[4], ea_dd[5], eb_dd[4];
  // n0 and its derivatives as full ecliptic-frame vectors (a caller's position table):
  // [0] n0, [1] d/dalpha, [2] d/ddelta, [3] d2/dalpha2, [4] d2/dalpha ddelta, [5] d2/ddelta2
  double n3[6][3];
};

// The constants of one point (k_point_constants, and the host checks of the fine
// search's arithmetic).
__host__ __device__ inline PointConst point_constants(const fs_point &p, const SegGeom &g, const fs_detector &det) {
  PointConst c;
  c.f0 = p.f0;
  c.f1 = p.f1;
  double sa, ca, sd, cd;
  sincos(p.alpha, &sa, &ca);
  sincos(p.delta, &sd, &cd);
  const double ce = cos(det.eps), se = sin(det.eps);
  c.ca = ca;
  c.sa = sa;
  c.nx = ca * cd;
  c.nyp = sa * cd * ce + sd * se;
  c.nx_a = -sa * cd;
  c.nyp_a = ca * cd * ce;
  c.nx_d = -ca * sd;
  c.nyp_d = -sa * sd * ce + cd * se;
  c.nx_aa = -ca * cd;
  c.nyp_aa = -sa * cd * ce;
  c.nx_ad = sa * sd;
  c.nyp_ad = -ca * sd * ce;
  c.nx_dd = -ca * cd;
  c.nyp_dd = -sa * cd * ce - sd * se;
  c.rcd = g.re_c * cd;
  c.rcd_d = -g.re_c * sd;
  c.rcd_dd = -g.re_c * cd;
  c.zsd = g.z_c * sd;
  c.zsd_d = g.z_c * cd;
  c.zsd_dd = -g.z_c * sd;
  {
    // equatorial components of n and its derivatives, rotated to the ecliptic frame (Eq. pha4)
    const double q[6][3] = {{ca * cd, sa * cd, sd},        {-sa * cd, ca * cd, 0.0}, {-ca * sd, -sa * sd, cd},
                            {-ca * cd, -sa * cd, 0.0},     {sa * sd, -ca * sd, 0.0}, {-ca * cd, -sa * cd, -sd}};
    for (int v = 0; v < 6; v++) {
      c.n3[v][0] = q[v][0];
      c.n3[v][1] = ce * q[v][1] + se * q[v][2];
      c.n3[v][2] = -se * q[v][1] + ce * q[v][2];
    }
  }
  ab_coefficients(p.delta, det.lat, det.gamma, c.ea, c.eb);
  const double s2g = sin(2 * det.gamma), c2g = cos(2 * det.gamma);
  const double sl = sin(det.lat), cl = cos(det.lat), s2l = sin(2 * det.lat), c2l = cos(2 * det.lat);
  const double s2d = sin(2 * p.delta), c2d = cos(2 * p.delta);
  c.ea_d[0] = s2g * (3 - c2l) * 2 * s2d / 16.0;
  c.ea_d[1] = -c2g * sl * 2 * s2d / 4.0;
  c.ea_d[2] = s2g * s2l * 2 * c2d / 4.0;
  c.ea_d[3] = -c2g * cl * c2d;
  c.ea_d[4] = -0.75 * s2g * cl * cl * s2d;
  c.eb_d[0] = c2g * sl * cd;
  c.eb_d[1] = s2g * (3 - c2l) * cd / 4.0;
  c.eb_d[2] = -c2g * cl * sd;
  c.eb_d[3] = -s2g * s2l * sd / 2.0;
  c.ea_dd[0] = s2g * (3 - c2l) * 4 * c2d / 16.0;
  c.ea_dd[1] = -c2g * sl * c2d;
  c.ea_dd[2] = -s2g * s2l * s2d;
  c.ea_dd[3] = 2 * c2g * cl * s2d;
  c.ea_dd[4] = -1.5 * s2g * cl * cl * c2d;
  c.eb_dd[0] = -c2g * sl * sd;
  c.eb_dd[1] = -s2g * (3 - c2l) * sd / 4.0;
  c.eb_dd[2] = -c2g * cl * cd;
  c.eb_dd[3] = -s2g * s2l * cd / 2.0;
  return c;
}

__host__ __device__ constexpr int sym_idx(int i, int j) {  // upper-triangle index of (i, j), row by row
  return i <= j ? i * 4 - i * (i - 1) / 2 + (j - i) : j * 4 - j * (j - 1) / 2 + (i - j);
}

// The double-float tables of a segment (layout in fs_refine.cu).
struct Etab32 {
  float4 *L, *T;
  float2 *X;
  float4 *SC;
};

// Per-point constants of the double-float kernels (from PointConst).
struct FastConst {
  double F0L, f0, nxA, nyA;                       // FP64 phase: f0 + fl, f0, (AU/c) nx, (AU/c) nyp
  df32 F0L2, f1, dt, ca, sa, nxA2, nyA2, rcd, zsd;
  df32 nxAa, nyAa, nxAd, nyAd, rcd_d, zsd_d;      // the alpha / delta derivatives of the delay
  df32 ea[5], eb[4];
  df32 nxAaa, nyAaa, nxAad, nyAad, nxAdd, nyAdd, rcd_dd, zsd_dd;  // second derivatives
  float eaf[5], ebf[4], ea_d[5], eb_d[4], ea_dd[5], eb_dd[4];
};

__host__ __device__ inline FastConst fast_const(const PointConst &p, const SegGeom &g) {
  FastConst c;
  c.F0L = p.f0 + g.fl;
  c.f0 = p.f0;
  c.nxA = kAUls * p.nx;
  c.nyA = kAUls * p.nyp;
  c.F0L2 = df_from_double(c.F0L);
  c.f1 = df_from_double(p.f1);
  c.dt = df_from_double(g.dt);
  c.ca = df_from_double(p.ca);
  c.sa = df_from_double(p.sa);
  c.nxA2 = df_from_double(c.nxA);
  c.nyA2 = df_from_double(c.nyA);
  c.rcd = df_from_double(p.rcd);
  c.zsd = df_from_double(p.zsd);
  c.nxAa = df_from_double(kAUls * p.nx_a);
  c.nyAa = df_from_double(kAUls * p.nyp_a);
  c.nxAd = df_from_double(kAUls * p.nx_d);
  c.nyAd = df_from_double(kAUls * p.nyp_d);
  c.rcd_d = df_from_double(p.rcd_d);
  c.zsd_d = df_from_double(p.zsd_d);
  c.nxAaa = df_from_double(kAUls * p.nx_aa);
  c.nyAaa = df_from_double(kAUls * p.nyp_aa);
  c.nxAad = df_from_double(kAUls * p.nx_ad);
  c.nyAad = df_from_double(kAUls * p.nyp_ad);
  c.nxAdd = df_from_double(kAUls * p.nx_dd);
  c.nyAdd = df_from_double(kAUls * p.nyp_dd);
  c.rcd_dd = df_from_double(p.rcd_dd);
  c.zsd_dd = df_from_double(p.zsd_dd);
  for (int i = 0; i < 5; i++) {
    c.ea[i] = df_from_double(p.ea[i]);
    c.eaf[i] = (float)p.ea[i];
    c.ea_d[i] = (float)p.ea_d[i];
    c.ea_dd[i] = (float)p.ea_dd[i];
  }
  for (int i = 0; i < 4; i++) {
    c.eb[i] = df_from_double(p.eb[i]);
    c.ebf[i] = (float)p.eb[i];
    c.eb_d[i] = (float)p.eb_d[i];
    c.eb_dd[i] = (float)p.eb_dd[i];
  }
  return c;
}

// 2 pi and -4 pi^2 as double-floats
__host__ __device__ __forceinline__ df32 df_two_pi() { return df32{6.2831854820251465f, -1.7484555314695172e-07f}; }
__host__ __device__ __forceinline__ df32 df_m4pi2() { return df32{-39.478416442871094f, -1.1614863524300745e-06f}; }

// exp(-2 pi i f) = cp - i sp for a double-float f (cycles): the nearest table angle
// j / 256 and the remainder x = 2 pi (f - j/256), |x| <= pi/256, by cos x - 1 =
// -x^2/2 + x^4/24 and sin x - x = -x^3/6 + x^5/120 (dropped terms < 5e-15).
__host__ __device__ __forceinline__ void df_expm(df32 f, const float4 *sc, df32 *cp, df32 *sp) {
  // two reductions: for |f| ~ 1e5 the low word can carry the first remainder past 1/2
  f = df_add_f(f, -rintf(f.hi));
  f = df_add_f(f, -rintf(f.hi));
  // the table index stays inside [-128, 128] whatever f is (the remainder is then
  // at most slightly beyond 1/512, where the series is still accurate)
  const float jf = fminf(fmaxf(rintf(f.hi * 256.f), -128.f), 128.f);
  const df32 r = df_add_f(f, -jf * (1.f / 256.f));
  const df32 x = df_mul(df_two_pi(), r);
  const float x2 = x.hi * x.hi;
  const float cm1 = x2 * fmaf(x2, 1.f / 24.f, -0.5f);
  const float sm = x.hi * x2 * fmaf(x2, 1.f / 120.f, -1.f / 6.f);
  const df32 sn = df_add_f(x, sm);
  const float4 q = sc[(int)jf + 128];
  const df32 C{q.x, q.y}, S{q.z, q.w};
  *cp = df_sub(df_add_f(C, C.hi * cm1), df_mul(S, sn));  // cos(2 pi f) = C cos x - S sin x
  *sp = df_add(df_add_f(S, S.hi * cm1), df_mul(C, sn));  // sin(2 pi f) = S cos x + C sin x
}

// Per-sample quantities shared by the double-float kernels.
struct FastSample {
  df32 x, t, cx, sx, c2, s2, cl, sl, phid, phi, tu, a, b, cp, sp;
};

// The orbital part of the phase, (f0 + fl) (AU/c) n0 . (cos lambda, sin lambda) + f0 t,
// reaches ~2.5e5 cycles: it is formed in FP64 and reduced to a fraction of a cycle
// before the rest of the phase is added in double-float (the Hessian's terms cancel to
// ~1e-4 near a maximum, so both kernels need the same accuracy).
__host__ __device__ __forceinline__ FastSample fast_sample(const FastConst &c, const SegGeom &g, const dbl4 *__restrict__ etab,
                                                  const Etab32 &et, const float4 *sc, int64_t k) {
  FastSample s;
  const dbl4 e4 = etab[k];
  double P = fma(c.F0L, fma(c.nxA, e4.x, c.nyA * e4.y), c.f0 * ((double)k * g.dt));
  P -= rint(P);
  const float4 Lq = et.L[k], Tq = et.T[k];
  const float2 Xq = et.X[k];
  s.cl = df32{Lq.x, Lq.y};
  s.sl = df32{Lq.z, Lq.w};
  const df32 ct{Tq.x, Tq.y}, st{Tq.z, Tq.w};
  s.x = df32{Xq.x, Xq.y};
  s.t = df_mul_f(c.dt, (float)k);  // k < 2^24 is exact as a float
  s.cx = df_add(df_mul(c.ca, ct), df_mul(c.sa, st));  // cos(alpha - theta)
  s.sx = df_sub(df_mul(c.sa, ct), df_mul(c.ca, st));  // sin(alpha - theta)
  s.phid = df_add(df_mul(c.rcd, s.cx), c.zsd);        // diurnal delay
  const df32 phio = df_add(df_mul(c.nxA2, s.cl), df_mul(c.nyA2, s.sl));
  s.phi = df_add(phio, s.phid);
  s.tu = df_mul(s.t, df_add(df_scale(s.t, 0.5f), s.phi));  // t (t/2 + phi)
  const float Ph = (float)P;
  const df32 f = df_add(df32{Ph, (float)(P - (double)Ph)}, df_add(df_mul(c.F0L2, s.phid), df_mul(c.f1, s.tu)));
  df_expm(f, sc, &s.cp, &s.sp);
  s.c2 = df_sub(df_mul(s.cx, s.cx), df_mul(s.sx, s.sx));
  s.s2 = df_scale(df_mul(s.sx, s.cx), 2.f);
  s.a = df_add(df_add(df_add(df_mul(c.ea[0], s.c2), df_mul(c.ea[1], s.s2)),
                      df_add(df_mul(c.ea[2], s.cx), df_mul(c.ea[3], s.sx))), c.ea[4]);
  s.b = df_add(df_add(df_mul(c.eb[0], s.c2), df_mul(c.eb[1], s.s2)),
               df_add(df_mul(c.eb[2], s.cx), df_mul(c.eb[3], s.sx)));
  return s;
}

// One sample's terms of F's and the gradient's accumulators (k_points_fg).
__host__ __device__ __forceinline__ void fg_sample(const FastConst &c, const FastSample &s, df32 *acc) {
  const df32 ua = df_mul(s.x, s.a), ub = df_mul(s.x, s.b);
  acc[0] = df_add(acc[0], df_mul(ua, s.cp));
  acc[1] = df_sub(acc[1], df_mul(ua, s.sp));
  acc[2] = df_add(acc[2], df_mul(ub, s.cp));
  acc[3] = df_sub(acc[3], df_mul(ub, s.sp));
  // derivatives of a, b (FP32: their terms are ~1e-6 of the phase-derivative terms)
  const float cx = s.cx.hi, sx = s.sx.hi, c2 = s.c2.hi, s2 = s.s2.hi, xf = s.x.hi;
  const float a_a = -2.f * c.eaf[0] * s2 + 2.f * c.eaf[1] * c2 - c.eaf[2] * sx + c.eaf[3] * cx;
  const float b_a = -2.f * c.ebf[0] * s2 + 2.f * c.ebf[1] * c2 - c.ebf[2] * sx + c.ebf[3] * cx;
  const float a_d = c.ea_d[0] * c2 + c.ea_d[1] * s2 + c.ea_d[2] * cx + c.ea_d[3] * sx + c.ea_d[4];
  const float b_d = c.eb_d[0] * c2 + c.eb_d[1] * s2 + c.eb_d[2] * cx + c.eb_d[3] * sx;
  // phase derivatives [cycles per unit]: t + phi, t (t/2 + phi), w phi_alpha, w phi_delta
  const df32 w = df_add(c.F0L2, df_mul(c.f1, s.t));
  const df32 phia = df_sub(df_add(df_mul(c.nxAa, s.cl), df_mul(c.nyAa, s.sl)), df_mul(c.rcd, s.sx));
  const df32 phide = df_add(df_add(df_add(df_mul(c.nxAd, s.cl), df_mul(c.nyAd, s.sl)), df_mul(c.rcd_d, s.cx)),
                            c.zsd_d);
  const df32 dP[4] = {df_add(s.t, s.phi), s.tu, df_mul(w, phia), df_mul(w, phide)};
  const float da[4] = {0.f, 0.f, a_a, a_d}, db[4] = {0.f, 0.f, b_a, b_d};
  const float cpf = s.cp.hi, spf = s.sp.hi;
#pragma unroll
  for (int i = 0; i < 4; i++) {
    // x (da_i - 2 pi i a dP_i) (cp - i sp)
    const df32 ra = df_mul(df_neg(df_two_pi()), df_mul(ua, dP[i]));
    const df32 rb = df_mul(df_neg(df_two_pi()), df_mul(ub, dP[i]));
    acc[4 + 2 * i] = df_add(acc[4 + 2 * i], df_mul(ra, s.sp));
    acc[5 + 2 * i] = df_add(acc[5 + 2 * i], df_mul(ra, s.cp));
    acc[12 + 2 * i] = df_add(acc[12 + 2 * i], df_mul(rb, s.sp));
    acc[13 + 2 * i] = df_add(acc[13 + 2 * i], df_mul(rb, s.cp));
    if (i >= 2) {
      const float qa = xf * da[i], qb = xf * db[i];
      acc[4 + 2 * i] = df_add_f(acc[4 + 2 * i], qa * cpf);
      acc[5 + 2 * i] = df_add_f(acc[5 + 2 * i], -qa * spf);
      acc[12 + 2 * i] = df_add_f(acc[12 + 2 * i], qb * cpf);
      acc[13 + 2 * i] = df_add_f(acc[13 + 2 * i], -qb * spf);
    }
  }
  acc[20] = df_add(acc[20], df_mul(s.a, s.a));
  acc[21] = df_add(acc[21], df_mul(s.b, s.b));
  const float af = s.a.hi, bf = s.b.hi;
  acc[22] = df_add_f(acc[22], af * a_a);
  acc[23] = df_add_f(acc[23], af * a_d);
  acc[24] = df_add_f(acc[24], bf * b_a);
  acc[25] = df_add_f(acc[25], bf * b_d);
}

// One sample's terms of the Hessian's accumulators (k_points_h).  Near a maximum the
// two parts of d2|S|^2 (|dS|^2 and Re(S* d2S)) cancel to ~1e-4 for the sky pairs,
// so every term of d2S is a double-float; only x d2a (~1e-12 of the dP_i dP_j term)
// and the sums a_i a_j + a a_ij (they enter F's curvature at ~1e-9 of its scale) are FP32.
// SIG: 0 signal a only (acc[0, 20) pairs, acc[20, 23) the a sums), 1 signal b only (same
// layout), 2 both (the 46 sums in PtLayout's order).
template <int SIG>
__host__ __device__ __forceinline__ void hess_sample(const FastConst &c, const FastSample &s, df32 *acc) {
  constexpr bool DA = SIG != 1, DB = SIG != 0;
  constexpr int OB = SIG == 2 ? 20 : 0;  // offset of signal b's pairs
  const float cx = s.cx.hi, sx = s.sx.hi, c2 = s.c2.hi, s2 = s.s2.hi, xf = s.x.hi, af = s.a.hi, bf = s.b.hi;
  // first derivatives of a, b (double-float)
  const df32 a_a = df_add(df_sub(df_scale(df_sub(df_mul(c.ea[1], s.c2), df_mul(c.ea[0], s.s2)), 2.f),
                                 df_mul(c.ea[2], s.sx)), df_mul(c.ea[3], s.cx));
  const df32 b_a = df_add(df_sub(df_scale(df_sub(df_mul(c.eb[1], s.c2), df_mul(c.eb[0], s.s2)), 2.f),
                                 df_mul(c.eb[2], s.sx)), df_mul(c.eb[3], s.cx));
  const df32 a_d = df_add(df_add(df_add(df_mul_f(s.c2, c.ea_d[0]), df_mul_f(s.s2, c.ea_d[1])),
                                 df_add(df_mul_f(s.cx, c.ea_d[2]), df_mul_f(s.sx, c.ea_d[3]))),
                          df32{c.ea_d[4], 0.f});
  const df32 b_d = df_add(df_add(df_mul_f(s.c2, c.eb_d[0]), df_mul_f(s.s2, c.eb_d[1])),
                          df_add(df_mul_f(s.cx, c.eb_d[2]), df_mul_f(s.sx, c.eb_d[3])));
  // second derivatives of a, b (FP32)
  const float a_aa = -4.f * c.eaf[0] * c2 - 4.f * c.eaf[1] * s2 - c.eaf[2] * cx - c.eaf[3] * sx;
  const float b_aa = -4.f * c.ebf[0] * c2 - 4.f * c.ebf[1] * s2 - c.ebf[2] * cx - c.ebf[3] * sx;
  const float a_ad = -2.f * c.ea_d[0] * s2 + 2.f * c.ea_d[1] * c2 - c.ea_d[2] * sx + c.ea_d[3] * cx;
  const float b_ad = -2.f * c.eb_d[0] * s2 + 2.f * c.eb_d[1] * c2 - c.eb_d[2] * sx + c.eb_d[3] * cx;
  const float a_dd = c.ea_dd[0] * c2 + c.ea_dd[1] * s2 + c.ea_dd[2] * cx + c.ea_dd[3] * sx + c.ea_dd[4];
  const float b_dd = c.eb_dd[0] * c2 + c.eb_dd[1] * s2 + c.eb_dd[2] * cx + c.eb_dd[3] * sx;
  // phase derivatives and the sky second derivatives of the delay (double-float)
  const df32 w = df_add(c.F0L2, df_mul(c.f1, s.t));
  const df32 phia = df_sub(df_add(df_mul(c.nxAa, s.cl), df_mul(c.nyAa, s.sl)), df_mul(c.rcd, s.sx));
  const df32 phide = df_add(df_add(df_add(df_mul(c.nxAd, s.cl), df_mul(c.nyAd, s.sl)), df_mul(c.rcd_d, s.cx)),
                            c.zsd_d);
  const df32 phi_aa = df_sub(df_add(df_mul(c.nxAaa, s.cl), df_mul(c.nyAaa, s.sl)), df_mul(c.rcd, s.cx));
  const df32 phi_ad = df_sub(df_add(df_mul(c.nxAad, s.cl), df_mul(c.nyAad, s.sl)), df_mul(c.rcd_d, s.sx));
  const df32 phi_dd = df_add(df_add(df_add(df_mul(c.nxAdd, s.cl), df_mul(c.nyAdd, s.sl)), df_mul(c.rcd_dd, s.cx)),
                             c.zsd_dd);
  const df32 dP[4] = {df_add(s.t, s.phi), s.tu, df_mul(w, phia), df_mul(w, phide)};
  const df32 ua = df_mul(s.x, s.a), ub = df_mul(s.x, s.b);
  const df32 uam = df_mul(df_m4pi2(), ua), ubm = df_mul(df_m4pi2(), ub);
  const df32 mtp = df_neg(df_two_pi());
  // x da_i, x db_i (i = alpha, delta)
  const df32 xa[2] = {df_mul(s.x, a_a), df_mul(s.x, a_d)}, xb[2] = {df_mul(s.x, b_a), df_mul(s.x, b_d)};
#pragma unroll
  for (int i = 0; i < 4; i++) {
#pragma unroll
    for (int j = i; j < 4; j++) {
      const int o = 2 * sym_idx(i, j);
      const df32 m = df_mul(dP[i], dP[j]);
      float d2a = 0.f, d2b = 0.f;
      if (i == 2 && j == 2) { d2a = a_aa; d2b = b_aa; }
      if (i == 2 && j == 3) { d2a = a_ad; d2b = b_ad; }
      if (i == 3 && j == 3) { d2a = a_dd; d2b = b_dd; }
      // P = x (d2a - 4 pi^2 a dP_i dP_j)
      if constexpr (DA) {
        const df32 Pa = df_add_f(df_mul(uam, m), xf * d2a);
        acc[o] = df_add(acc[o], df_mul(Pa, s.cp));
        acc[o + 1] = df_sub(acc[o + 1], df_mul(Pa, s.sp));
      }
      if constexpr (DB) {
        const df32 Pb = df_add_f(df_mul(ubm, m), xf * d2b);
        acc[o + OB] = df_add(acc[o + OB], df_mul(Pb, s.cp));
        acc[o + OB + 1] = df_sub(acc[o + OB + 1], df_mul(Pb, s.sp));
      }
      if (j >= 2) {
        // Q = -2 pi x (da_i dP_j + da_j dP_i + a d2P), d2P the mixed phase derivative
        df32 d2P;
        if (i == 0) d2P = j == 2 ? phia : phide;
        else if (i == 1) d2P = df_mul(s.t, j == 2 ? phia : phide);
        else if (j == 2) d2P = df_mul(w, phi_aa);
        else d2P = df_mul(w, i == 2 ? phi_ad : phi_dd);
        if constexpr (DA) {
          df32 qa = df_add(df_mul(ua, d2P), df_mul(xa[j - 2], dP[i]));
          if (i >= 2) qa = df_add(qa, df_mul(xa[i - 2], dP[j]));
          const df32 Qa = df_mul(mtp, qa);
          acc[o] = df_add(acc[o], df_mul(Qa, s.sp));
          acc[o + 1] = df_add(acc[o + 1], df_mul(Qa, s.cp));
        }
        if constexpr (DB) {
          df32 qb = df_add(df_mul(ub, d2P), df_mul(xb[j - 2], dP[i]));
          if (i >= 2) qb = df_add(qb, df_mul(xb[i - 2], dP[j]));
          const df32 Qb = df_mul(mtp, qb);
          acc[o + OB] = df_add(acc[o + OB], df_mul(Qb, s.sp));
          acc[o + OB + 1] = df_add(acc[o + OB + 1], df_mul(Qb, s.cp));
        }
      }
    }
  }
  const float aa = a_a.hi, ad = a_d.hi, ba = b_a.hi, bd = b_d.hi;
  constexpr int MA = SIG == 2 ? 40 : 20, MB = SIG == 2 ? 43 : 20;
  if constexpr (DA) {
    acc[MA] = df_add_f(acc[MA], aa * aa + af * a_aa);
    acc[MA + 1] = df_add_f(acc[MA + 1], aa * ad + af * a_ad);
    acc[MA + 2] = df_add_f(acc[MA + 2], ad * ad + af * a_dd);
  }
  if constexpr (DB) {
    acc[MB] = df_add_f(acc[MB], ba * ba + bf * b_aa);
    acc[MB + 1] = df_add_f(acc[MB + 1], ba * bd + bf * b_ad);
    acc[MB + 2] = df_add_f(acc[MB + 2], bd * bd + bf * b_dd);
  }
}

}  // namespace fs
