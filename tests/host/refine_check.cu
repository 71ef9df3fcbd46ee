// Host-side check of the fine search's double-float arithmetic (fs_refine_df.cuh,
// compiled as host code) on the 2-day, 2 s series of the fine-search workload:
//  1. exp(-2 pi i f) from the 257-entry table and the remainder series, for phases up
//     to 2e5 cycles and for the double-floats whose low word carries the first
//     remainder past 1/2, against the FP64 sine and cosine of the reduced phase;
//  2. the per-point constants against central differences of the quantities they are
//     derivatives of (n0 in the ecliptic frame, Eq. pha4; the site terms; the Fourier
//     coefficients of a and b);
//  3. the per-sample sums of F, its gradient and its Hessian (Eqs. OS and Fab with
//     their alpha, delta, f0, f1 derivatives), accumulated in double-float over all
//     samples, against the same sums in FP64 with sin/cos of the FP64 phase; and that
//     the one-signal Hessian kernels' sums equal the two-signal layout's.
// Prints one "name value" line per measured error and "OK" at the end when every error
// is under its bound; exits non-zero otherwise.
#include <cmath>
#include <cstdio>
#include <random>
#include <vector>

#include "../../paper_1003_0844_gb300/csrc/fs_refine_df.cuh"

using namespace fs;

static int failures = 0;

static void check(const char *name, double err, double bound) {
  const bool ok = std::isfinite(err) && err <= bound;
  printf("%s %.3e (bound %.1e)%s\n", name, err, bound, ok ? "" : "  FAIL");
  if (!ok) failures++;
}

static double dval(const df32 &v) { return (double)v.hi + (double)v.lo; }

// 1. exp(-2 pi i f) = cp - i sp
static void check_expm(const std::vector<float4> &SC) {
  double worst = 0;
  auto one = [&](df32 f) {
    df32 cp, sp;
    df_expm(f, SC.data(), &cp, &sp);
    const double fv = dval(f), fr = fv - std::rint(fv);
    const double e = std::fabs(dval(cp) - std::cos(2 * M_PI * fr)) + std::fabs(dval(sp) - std::sin(2 * M_PI * fr));
    if (!(e <= worst)) worst = e;  // NaN propagates into worst
  };
  std::mt19937 rng(11);
  std::uniform_real_distribution<double> ud(-2e5, 2e5);
  for (int i = 0; i < 1000000; i++) one(df_from_double(ud(rng)));
  // a high word on a half cycle and a low word beyond it: one reduction leaves |f| > 1/2
  std::uniform_real_distribution<float> ul(-0.0078f, 0.0078f);
  for (int i = 0; i < 100000; i++) {
    const float hi = (float)(int)(ud(rng) / 2) + 0.5f;  // exact: |hi| < 2^17
    one(df32{hi, ul(rng)});
  }
  // remainders at the edges of the table intervals, j / 256 +- 1 / 512
  for (int j = -128; j <= 128; j++)
    for (int s = -1; s <= 1; s += 2) one(df_from_double(12345.0 + j / 256.0 + s / 512.0));
  check("expm_abs", worst, 1e-8);
}

// 2. per-point constants against central differences
static void check_point_constants(const SegGeom &g, const fs_detector &det, const fs_point &p) {
  const double h = 1e-5;
  auto at = [&](double da, double dd) {
    fs_point q = p;
    q.alpha += da;
    q.delta += dd;
    return point_constants(q, g, det);
  };
  const PointConst c = point_constants(p, g, det);
  const PointConst ap = at(h, 0), am = at(-h, 0), dp = at(0, h), dm = at(0, -h);
  auto rel = [](double fd, double an, double scale) { return std::fabs(fd - an) / scale; };
  double worst = 0;
  for (int v = 0; v < 3; v++) {
    // n0 and its derivatives: [1] = dn/dalpha, [2] = dn/ddelta, [3..5] the second ones
    worst = fmax(worst, rel((ap.n3[0][v] - am.n3[0][v]) / (2 * h), c.n3[1][v], 1.0));
    worst = fmax(worst, rel((dp.n3[0][v] - dm.n3[0][v]) / (2 * h), c.n3[2][v], 1.0));
    worst = fmax(worst, rel((ap.n3[1][v] - am.n3[1][v]) / (2 * h), c.n3[3][v], 1.0));
    worst = fmax(worst, rel((dp.n3[1][v] - dm.n3[1][v]) / (2 * h), c.n3[4][v], 1.0));
    worst = fmax(worst, rel((dp.n3[2][v] - dm.n3[2][v]) / (2 * h), c.n3[5][v], 1.0));
  }
  // the (x, y') components the kernels use are n0's ecliptic x and y
  worst = fmax(worst, rel(c.nx, c.n3[0][0], 1.0) + rel(c.nyp, c.n3[0][1], 1.0));
  worst = fmax(worst, rel((ap.nx - am.nx) / (2 * h), c.nx_a, 1.0) + rel((ap.nyp - am.nyp) / (2 * h), c.nyp_a, 1.0));
  worst = fmax(worst, rel((dp.nx - dm.nx) / (2 * h), c.nx_d, 1.0) + rel((dp.nyp - dm.nyp) / (2 * h), c.nyp_d, 1.0));
  worst = fmax(worst, rel((ap.nx_a - am.nx_a) / (2 * h), c.nx_aa, 1.0) + rel((ap.nyp_a - am.nyp_a) / (2 * h), c.nyp_aa, 1.0));
  worst = fmax(worst, rel((dp.nx_a - dm.nx_a) / (2 * h), c.nx_ad, 1.0) + rel((dp.nyp_a - dm.nyp_a) / (2 * h), c.nyp_ad, 1.0));
  worst = fmax(worst, rel((dp.nx_d - dm.nx_d) / (2 * h), c.nx_dd, 1.0) + rel((dp.nyp_d - dm.nyp_d) / (2 * h), c.nyp_dd, 1.0));
  const double rs = g.re_c, zs = g.z_c;
  worst = fmax(worst, rel((dp.rcd - dm.rcd) / (2 * h), c.rcd_d, rs) + rel((dp.rcd_d - dm.rcd_d) / (2 * h), c.rcd_dd, rs));
  worst = fmax(worst, rel((dp.zsd - dm.zsd) / (2 * h), c.zsd_d, zs) + rel((dp.zsd_d - dm.zsd_d) / (2 * h), c.zsd_dd, zs));
  for (int i = 0; i < 5; i++) {
    worst = fmax(worst, rel((dp.ea[i] - dm.ea[i]) / (2 * h), c.ea_d[i], 1.0));
    worst = fmax(worst, rel((dp.ea_d[i] - dm.ea_d[i]) / (2 * h), c.ea_dd[i], 1.0));
  }
  for (int i = 0; i < 4; i++) {
    worst = fmax(worst, rel((dp.eb[i] - dm.eb[i]) / (2 * h), c.eb_d[i], 1.0));
    worst = fmax(worst, rel((dp.eb_d[i] - dm.eb_d[i]) / (2 * h), c.eb_dd[i], 1.0));
  }
  check("point_constants_fd", worst, 1e-8);
}

// 3. the sums: FP64 reference, accumulators in the kernels' layout (26 of F and its
// gradient; 46 of the Hessian)
struct Ref {
  double fg[26] = {}, h[46] = {};
};

static void ref_sample(const PointConst &c, const SegGeom &g, const dbl4 &e, double x, int64_t k, Ref &r) {
  const double t = (double)k * g.dt;
  const double cx = c.ca * e.z + c.sa * e.w, sx = c.sa * e.z - c.ca * e.w;  // cos, sin (alpha - theta)
  const double c2 = cx * cx - sx * sx, s2 = 2 * sx * cx;
  // delay phi = n0 . r / c and its sky derivatives [s]
  const double phi = kAUls * (c.nx * e.x + c.nyp * e.y) + c.rcd * cx + c.zsd;
  const double ph_a = kAUls * (c.nx_a * e.x + c.nyp_a * e.y) - c.rcd * sx;
  const double ph_d = kAUls * (c.nx_d * e.x + c.nyp_d * e.y) + c.rcd_d * cx + c.zsd_d;
  const double ph_aa = kAUls * (c.nx_aa * e.x + c.nyp_aa * e.y) - c.rcd * cx;
  const double ph_ad = kAUls * (c.nx_ad * e.x + c.nyp_ad * e.y) - c.rcd_d * sx;
  const double ph_dd = kAUls * (c.nx_dd * e.x + c.nyp_dd * e.y) + c.rcd_dd * cx + c.zsd_dd;
  // a, b and their alpha (through x), delta (through the coefficients) derivatives
  double A[6], B[6];  // value, _a, _d, _aa, _ad, _dd
  A[0] = c.ea[0] * c2 + c.ea[1] * s2 + c.ea[2] * cx + c.ea[3] * sx + c.ea[4];
  A[1] = -2 * c.ea[0] * s2 + 2 * c.ea[1] * c2 - c.ea[2] * sx + c.ea[3] * cx;
  A[2] = c.ea_d[0] * c2 + c.ea_d[1] * s2 + c.ea_d[2] * cx + c.ea_d[3] * sx + c.ea_d[4];
  A[3] = -4 * c.ea[0] * c2 - 4 * c.ea[1] * s2 - c.ea[2] * cx - c.ea[3] * sx;
  A[4] = -2 * c.ea_d[0] * s2 + 2 * c.ea_d[1] * c2 - c.ea_d[2] * sx + c.ea_d[3] * cx;
  A[5] = c.ea_dd[0] * c2 + c.ea_dd[1] * s2 + c.ea_dd[2] * cx + c.ea_dd[3] * sx + c.ea_dd[4];
  B[0] = c.eb[0] * c2 + c.eb[1] * s2 + c.eb[2] * cx + c.eb[3] * sx;
  B[1] = -2 * c.eb[0] * s2 + 2 * c.eb[1] * c2 - c.eb[2] * sx + c.eb[3] * cx;
  B[2] = c.eb_d[0] * c2 + c.eb_d[1] * s2 + c.eb_d[2] * cx + c.eb_d[3] * sx;
  B[3] = -4 * c.eb[0] * c2 - 4 * c.eb[1] * s2 - c.eb[2] * cx - c.eb[3] * sx;
  B[4] = -2 * c.eb_d[0] * s2 + 2 * c.eb_d[1] * c2 - c.eb_d[2] * sx + c.eb_d[3] * cx;
  B[5] = c.eb_dd[0] * c2 + c.eb_dd[1] * s2 + c.eb_dd[2] * cx + c.eb_dd[3] * sx;
  // phase [cycles] Phi = f0 (t + phi) + fl phi + f1 t (t/2 + phi), reduced before sin/cos
  double P = c.f0 * (t + phi) + g.fl * phi + c.f1 * t * (0.5 * t + phi);
  P -= std::floor(P);
  const double cp = std::cos(2 * M_PI * P), sp = std::sin(2 * M_PI * P);
  // dPhi / d(f0, f1, alpha, delta) and the non-zero second derivatives
  const double w = c.f0 + g.fl + c.f1 * t;
  const double dP[4] = {t + phi, t * (0.5 * t + phi), w * ph_a, w * ph_d};
  double d2P[4][4] = {};
  d2P[0][2] = ph_a;
  d2P[0][3] = ph_d;
  d2P[1][2] = t * ph_a;
  d2P[1][3] = t * ph_d;
  d2P[2][2] = w * ph_aa;
  d2P[2][3] = w * ph_ad;
  d2P[3][3] = w * ph_dd;
  // d(signal)/d(theta_i) for the two signals: index 0 f0, 1 f1, 2 alpha, 3 delta
  const double *S[2] = {A, B};
  for (int s = 0; s < 2; s++) {
    const double *Q = S[s];
    const double d1[4] = {0, 0, Q[1], Q[2]};
    double d2[4][4] = {};
    d2[2][2] = Q[3];
    d2[2][3] = Q[4];
    d2[3][3] = Q[5];
    // S = sum x q e^{-2 pi i Phi}
    r.fg[2 * s] += x * Q[0] * cp;
    r.fg[2 * s + 1] -= x * Q[0] * sp;
    for (int i = 0; i < 4; i++) {
      // dS_i = sum x (q_i - 2 pi i q dPhi_i) e^{-2 pi i Phi}
      const double re = x * d1[i], im = -2 * M_PI * x * Q[0] * dP[i];
      r.fg[4 + 8 * s + 2 * i] += re * cp + im * sp;
      r.fg[5 + 8 * s + 2 * i] += im * cp - re * sp;
    }
    for (int i = 0; i < 4; i++)
      for (int j = i; j < 4; j++) {
        // d2S_ij = sum x (q_ij - 4 pi^2 q dPhi_i dPhi_j
        //                 - 2 pi i (q_i dPhi_j + q_j dPhi_i + q d2Phi_ij)) e^{-2 pi i Phi}
        const double re = x * (d2[i][j] - 4 * M_PI * M_PI * Q[0] * dP[i] * dP[j]);
        const double im = -2 * M_PI * x * (d1[i] * dP[j] + d1[j] * dP[i] + Q[0] * d2P[i][j]);
        const int o = 20 * s + 2 * sym_idx(i, j);
        r.h[o] += re * cp + im * sp;
        r.h[o + 1] += im * cp - re * sp;
      }
    // sums of q^2, q q_alpha, q q_delta and of q_i q_j + q q_ij over the sky pairs
    r.fg[20 + s] += Q[0] * Q[0];
    r.fg[22 + 2 * s] += Q[0] * Q[1];
    r.fg[23 + 2 * s] += Q[0] * Q[2];
    r.h[40 + 3 * s] += Q[1] * Q[1] + Q[0] * Q[3];
    r.h[41 + 3 * s] += Q[1] * Q[2] + Q[0] * Q[4];
    r.h[42 + 3 * s] += Q[2] * Q[2] + Q[0] * Q[5];
  }
}

// worst error of acc[lo, hi) relative to the root sum of squares of ref[lo, hi)
static double group_err(const df32 *acc, const double *ref, int lo, int hi) {
  double sc = 0, worst = 0;
  for (int q = lo; q < hi; q++) sc += ref[q] * ref[q];
  sc = std::sqrt(sc);
  for (int q = lo; q < hi; q++) {
    const double e = std::fabs(dval(acc[q]) - ref[q]) / sc;
    if (!(e <= worst)) worst = e;
  }
  return worst;
}

int main() {
  // the detector of the workloads (Virgo-like site), the 2-day series at 2 s in the
  // band starting at 435.1875 Hz
  const fs_detector det{0.761493, 0.183260, 0.338594, 0.409105, 2.2, 1.1};
  SegGeom g{};
  g.n = 86400;
  g.dt = 2.0;
  g.fl = 435.1875;
  g.S0 = 1.0;
  g.theta0 = det.theta_g0 + det.lon;
  g.lambda0 = det.lambda_e0;
  double re, z;
  site_radius(det.lat, &re, &z);
  g.re_c = re / kC;
  g.z_c = z / kC;

  const int64_t n = g.n;
  std::vector<dbl4> e64(n);
  std::vector<float4> L(n), T(n), SC(257);
  std::vector<float2> X(n);
  std::vector<double> x(n);
  std::mt19937 rng(5);
  std::normal_distribution<double> nd;
  for (int64_t k = 0; k < n; k++) {
    const double t = (double)k * g.dt;
    e64[k] = make_dbl4(std::cos(g.lambda0 + kOmegaO * t), std::sin(g.lambda0 + kOmegaO * t),
                       std::cos(g.theta0 + kOmegaR * t), std::sin(g.theta0 + kOmegaR * t));
    const df32 cl = df_from_double(e64[k].x), sl = df_from_double(e64[k].y);
    const df32 ct = df_from_double(e64[k].z), st = df_from_double(e64[k].w);
    L[k] = make_float4(cl.hi, cl.lo, sl.hi, sl.lo);
    T[k] = make_float4(ct.hi, ct.lo, st.hi, st.lo);
    x[k] = nd(rng);
    const df32 xv = df_from_double(x[k]);
    X[k] = make_float2(xv.hi, xv.lo);
  }
  for (int j = 0; j < 257; j++) {
    const df32 c = df_from_double(std::cos(M_PI * (j - 128) / 128.0));
    const df32 s = df_from_double(std::sin(M_PI * (j - 128) / 128.0));
    SC[j] = make_float4(c.hi, c.lo, s.hi, s.lo);
  }
  const Etab32 et{L.data(), T.data(), X.data(), SC.data()};

  check_expm(SC);

  // points: mid-band, band edges, both hemispheres, near a pole, the widest spindown
  const fs_point pts[] = {{0.1213, -4e-9, 2.1, 0.45},
                          {0.0004, -1e-8, 5.9, -1.2},
                          {0.2493, 0.0, 0.3, 1.52}};
  for (const fs_point &p : pts) {
    check_point_constants(g, det, p);
    const PointConst pc = point_constants(p, g, det);
    const FastConst fc = fast_const(pc, g);
    df32 fg[26] = {}, h2[46] = {}, h0[23] = {}, h1[23] = {};
    Ref r;
    for (int64_t k = 0; k < n; k++) {
      const FastSample s = fast_sample(fc, g, e64.data(), et, SC.data(), k);
      fg_sample(fc, s, fg);
      hess_sample<2>(fc, s, h2);
      hess_sample<0>(fc, s, h0);
      hess_sample<1>(fc, s, h1);
      ref_sample(pc, g, e64[k], x[k], k, r);
    }
    // F = c (|Sa|^2/<a^2> + |Sb|^2/<b^2>) is compared at 1e-9 relative, its gradient and
    // Hessian at 1e-7: the sums they are made of must stay well inside those bounds
    check("S", group_err(fg, r.fg, 0, 4), 1e-9);
    check("sum_a2_b2", group_err(fg, r.fg, 20, 22), 1e-9);
    check("dS_f0_f1", fmax(group_err(fg, r.fg, 4, 8), group_err(fg, r.fg, 12, 16)), 1e-8);
    check("dS_sky", fmax(group_err(fg, r.fg, 8, 12), group_err(fg, r.fg, 16, 20)), 1e-8);
    check("d2S_a", group_err(h2, r.h, 0, 20), 1e-8);
    check("d2S_b", group_err(h2, r.h, 20, 40), 1e-8);
    // sums of FP32 terms: they enter the gradient and the Hessian through <a^2>'s
    // derivatives, ~1e-6 of the phase-derivative terms
    check("sum_a_da", group_err(fg, r.fg, 22, 26), 1e-5);
    check("sum_da_da", group_err(h2, r.h, 40, 46), 1e-5);
    // one-signal layouts: the same operations, so the same bits
    int same = 1;
    for (int q = 0; q < 20; q++) {
      same &= h0[q].hi == h2[q].hi && h0[q].lo == h2[q].lo;
      same &= h1[q].hi == h2[20 + q].hi && h1[q].lo == h2[20 + q].lo;
    }
    for (int q = 0; q < 3; q++) {
      same &= h0[20 + q].hi == h2[40 + q].hi && h0[20 + q].lo == h2[40 + q].lo;
      same &= h1[20 + q].hi == h2[43 + q].hi && h1[20 + q].lo == h2[43 + q].lo;
    }
    check("one_signal_layout_mismatch", same ? 0.0 : 1.0, 0.0);
  }
  if (failures) {
    printf("FAILED %d\n", failures);
    return 1;
  }
  printf("OK\n");
  return 0;
}
