// Analytic detector model on the device, FP64 (Sec. II and Sec. V).
#pragma once
#include "fs_common.cuh"

namespace fs {

// Site on the reference ellipsoid at zero height (Sec. V): reduced latitude
// Psi = atan(b tan(phi) / a), equatorial radius a cos(Psi), height b sin(Psi).
__host__ __device__ inline void site_radius(double lat, double *re_m, double *z_m) {
  double b = kEllA * (1.0 - kEllF);
  double psi = atan(b * tan(lat) / kEllA);
  *re_m = kEllA * cos(psi);
  *z_m = b * sin(psi);
}

// Fourier coefficients of the amplitude modulation functions in
// x = alpha - theta(t) (the interferometer response of the series' first
// paper, Eqs. 12-13 there, cited in Sec. II):
//   a = ea0 cos2x + ea1 sin2x + ea2 cos x + ea3 sin x + ea4
//   b = eb0 cos2x + eb1 sin2x + eb2 cos x + eb3 sin x
__host__ __device__ inline void ab_coefficients(double delta, double lat, double gamma, double ea[5],
                                                double eb[4]) {
  double s2g = sin(2 * gamma), c2g = cos(2 * gamma);
  double sl = sin(lat), cl = cos(lat), s2l = sin(2 * lat), c2l = cos(2 * lat);
  double sd = sin(delta), cd = cos(delta), s2d = sin(2 * delta), c2d = cos(2 * delta);
  ea[0] = s2g * (3 - c2l) * (3 - c2d) / 16.0;
  ea[1] = -c2g * sl * (3 - c2d) / 4.0;
  ea[2] = s2g * s2l * s2d / 4.0;
  ea[3] = -c2g * cl * s2d / 2.0;
  ea[4] = 0.75 * s2g * cl * cl * cd * cd;
  eb[0] = c2g * sl * sd;
  eb[1] = s2g * (3 - c2l) * sd / 4.0;
  eb[2] = c2g * cl * cd;
  eb[3] = s2g * s2l * cd / 2.0;
}

// Per-sky constants of the delay n0 . r_d / c written as in Sec. II:
//   cos(a)cos(d) (R_ES^x + R_E^x) + (sin(a)cos(d)cos(eps) + sin(d)sin(eps)) R_ES^y
//   + sin(a)cos(d) R_E^y + sin(d) R_E^z
// with R_ES = AU (cos lambda_E, sin lambda_E, 0) and R_E = (r_e cos th, r_e sin th, z):
//   phi_m = AU/c (nx cos lambda_E + nyp sin lambda_E) + (r_e/c) cos(d) cos(a - th) + (z/c) sin(d)
__host__ __device__ inline void sky_constants(double alpha, double delta, double eps, double lat,
                                              double gamma, const SegGeom &g, SkyConst64 *k) {
  double ca = cos(alpha), sa = sin(alpha), cd = cos(delta), sd = sin(delta);
  k->nx = ca * cd;
  k->nyp = sa * cd * cos(eps) + sd * sin(eps);
  k->nz = -sa * cd * sin(eps) + sd * cos(eps);
  k->ca = ca;
  k->sa = sa;
  k->rcd = g.re_c * cd;
  k->zsd = g.z_c * sd;
  ab_coefficients(delta, lat, gamma, k->ea, k->eb);
}

struct Geo64 {  // delay and its time derivative, plus cos/sin of x = alpha - theta
  double phi, phidot, cx, sx;
};

__device__ inline Geo64 geometry64(double t, const SkyConst64 &K, const SegGeom &g) {
  double sl, cl, sth, cth;
  sincos(g.lambda0 + kOmegaO * t, &sl, &cl);
  sincos(g.theta0 + kOmegaR * t, &sth, &cth);
  double cx = K.ca * cth + K.sa * sth;
  double sx = K.sa * cth - K.ca * sth;
  Geo64 r;
  r.phi = kAUls * (K.nx * cl + K.nyp * sl) + K.rcd * cx + K.zsd;
  r.phidot = kAUls * kOmegaO * (-K.nx * sl + K.nyp * cl) + K.rcd * kOmegaR * sx;
  r.cx = cx;
  r.sx = sx;
  return r;
}

__device__ inline void ab_eval64(const SkyConst64 &K, double cx, double sx, double *a, double *b) {
  double c2 = cx * cx - sx * sx, s2 = 2.0 * sx * cx;
  *a = K.ea[0] * c2 + K.ea[1] * s2 + K.ea[2] * cx + K.ea[3] * sx + K.ea[4];
  *b = K.eb[0] * c2 + K.eb[1] * s2 + K.eb[2] * cx + K.eb[3] * sx;
}

// The same from a caller's position table eph[2m] = (r_m, 0), eph[2m + 1] =
// (v_m, 0) on t_m = m dt: r(t) = r_m + (t - t_m) v_m from the nearest grid
// point m clamped to [0, n); phi = n0 . r(t), phidot = n0 . v_m.  The sidereal
// angle (for a, b) is the analytic one.
__device__ inline Geo64 geometry64_eph(double t, const SkyConst64 &K, const SegGeom &g, const dbl4 *eph) {
  double mf = rint(t / g.dt);
  mf = fmin(fmax(mf, 0.0), (double)(g.n - 1));
  const int64_t m = (int64_t)mf;
  const double tau = t - mf * g.dt;
  const dbl4 r = eph[2 * m], v = eph[2 * m + 1];
  double sth, cth;
  sincos(g.theta0 + kOmegaR * t, &sth, &cth);
  Geo64 q;
  q.phidot = K.nx * v.x + K.nyp * v.y + K.nz * v.z;
  q.phi = K.nx * r.x + K.nyp * r.y + K.nz * r.z + tau * q.phidot;
  q.cx = K.ca * cth + K.sa * sth;
  q.sx = K.sa * cth - K.ca * sth;
  return q;
}

// Source time t with t + phi_m(t) = tb (Eq. eq:Bt) by Newton's method in FP64;
// eph: NULL for the analytic Earth, else the caller's table.
__device__ inline double source_time64(double tb, const SkyConst64 &K, const SegGeom &g, Geo64 *geo,
                                       const dbl4 *eph = nullptr) {
  auto geom = [&](double tt) { return eph ? geometry64_eph(tt, K, g, eph) : geometry64(tt, K, g); };
  double t = tb;
  Geo64 q = geom(t);
  t = tb - q.phi;
#pragma unroll 1
  for (int it = 0; it < 3; it++) {
    q = geom(t);
    double gres = t + q.phi - tb;
    t -= gres / (1.0 + q.phidot);
  }
  *geo = geom(t);
  return t;
}

}  // namespace fs
