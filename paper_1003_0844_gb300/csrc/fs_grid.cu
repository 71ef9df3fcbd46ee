// Grid in the parameter space (Sec. IV), host code: the reduced Fisher matrix of
// the linear phase model (Eq. philin), the constrained lattice covering of
// Eqs. opt/opt2 built from A2* (Eq. A2gen) or A4* (Eq. gen), and the nodes of
// such a lattice in a band as continuous template points.
//
// Coordinates xi = (omega0, omega1, alpha1, alpha2) with m(t) = (t, t^2/2,
// mu1(t), mu2(t)), mu1 = (R_ES^y + R_E^y cos eps)/c, mu2 = (R_ES^x + R_E^x)/c,
// alpha1 = omega0 n0_y, alpha2 = omega0 n0_x in the ecliptic SSB frame (Eq. albe).
//
// Construction: x = M^-1 tau with M^T G M = I (the paper's M = U0 D0^-1, here from
// the unit-diagonal scaling of G for accuracy) turns the correlation ellipsoid
// into a sphere of radius R = sqrt(1 - C0); the A_n* lattice
// of covering radius R is shrunk along a lattice vector l (|l| >= |e0|, e0 =
// M^-1 a0) by mu = |e0|/|l| and expanded perpendicular to l by the nu >= 1 that
// brings its covering radius back to R (Eq. condition; solved by regula falsi);
// the l of largest mu nu^(n-1) is kept (one per length shell: A_n* is symmetric
// enough that equal lengths give congruent lattices); l is rotated onto e0 and,
// for the second constraint, a second lattice vector f is rotated about e0 into
// the directions without sky components; M^T maps back.  The returned basis
// starts with a0 and (second constraint) a vector without sky components.
#include <math.h>
#include <stdint.h>
#include <string.h>
#include <algorithm>
#include <array>
#include <vector>
#include "fs_internal.h"
#include "fs_model.cuh"

namespace {

constexpr int kMaxDim = 4;
typedef double Mat[kMaxDim][kMaxDim];

void mat_mul(int n, const Mat A, const Mat B, Mat C) {  // C = A B (C may not alias)
  for (int i = 0; i < n; i++)
    for (int j = 0; j < n; j++) {
      double s = 0.0;
      for (int k = 0; k < n; k++) s += A[i][k] * B[k][j];
      C[i][j] = s;
    }
}
void mat_copy(int n, const Mat A, Mat B) {
  for (int i = 0; i < n; i++)
    for (int j = 0; j < n; j++) B[i][j] = A[i][j];
}
void mat_transpose(int n, const Mat A, Mat B) {
  for (int i = 0; i < n; i++)
    for (int j = 0; j < n; j++) B[j][i] = A[i][j];
}
double dot(int n, const double *a, const double *b) {
  double s = 0.0;
  for (int i = 0; i < n; i++) s += a[i] * b[i];
  return s;
}
double vnorm(int n, const double *a) { return sqrt(dot(n, a, a)); }

// Solve A x = b (n <= 4) by Gaussian elimination with partial pivoting.
bool solve(int n, const Mat A_, const double *b, double *x) {
  double A[kMaxDim][kMaxDim + 1];
  for (int i = 0; i < n; i++) {
    for (int j = 0; j < n; j++) A[i][j] = A_[i][j];
    A[i][n] = b[i];
  }
  double scale = 0.0;
  for (int i = 0; i < n; i++)
    for (int j = 0; j < n; j++) scale = fmax(scale, fabs(A[i][j]));
  for (int c = 0; c < n; c++) {
    int p = c;
    for (int r = c + 1; r < n; r++)
      if (fabs(A[r][c]) > fabs(A[p][c])) p = r;
    if (!(fabs(A[p][c]) > 1e-12 * scale)) return false;
    if (p != c)
      for (int j = 0; j <= n; j++) std::swap(A[p][j], A[c][j]);
    for (int r = c + 1; r < n; r++) {
      const double f = A[r][c] / A[c][c];
      for (int j = c; j <= n; j++) A[r][j] -= f * A[c][j];
    }
  }
  for (int i = n - 1; i >= 0; i--) {
    double s = A[i][n];
    for (int j = i + 1; j < n; j++) s -= A[i][j] * x[j];
    x[i] = s / A[i][i];
  }
  return true;
}

double det(int n, const Mat A_) {
  Mat A;
  mat_copy(n, A_, A);
  double d = 1.0;
  for (int c = 0; c < n; c++) {
    int p = c;
    for (int r = c + 1; r < n; r++)
      if (fabs(A[r][c]) > fabs(A[p][c])) p = r;
    if (A[p][c] == 0.0) return 0.0;
    if (p != c) {
      for (int j = 0; j < n; j++) std::swap(A[p][j], A[c][j]);
      d = -d;
    }
    d *= A[c][c];
    for (int r = c + 1; r < n; r++) {
      const double f = A[r][c] / A[c][c];
      for (int j = c; j < n; j++) A[r][j] -= f * A[c][j];
    }
  }
  return d;
}

// Symmetric eigendecomposition by cyclic Jacobi rotations: G = V diag(w) V^T.
void jacobi_eig(int n, const Mat G, double *w, Mat V) {
  Mat A;
  mat_copy(n, G, A);
  for (int i = 0; i < n; i++)
    for (int j = 0; j < n; j++) V[i][j] = (i == j) ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 100; sweep++) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < n; i++)
      for (int j = 0; j < n; j++) {
        tot += A[i][j] * A[i][j];
        if (i != j) off += A[i][j] * A[i][j];
      }
    if (off <= 1e-30 * tot) break;
    for (int p = 0; p < n; p++)
      for (int q = p + 1; q < n; q++) {
        if (A[p][q] == 0.0) continue;
        const double theta = (A[q][q] - A[p][p]) / (2.0 * A[p][q]);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; k++) {  // A = J^T A J
          const double akp = A[k][p], akq = A[k][q];
          A[k][p] = c * akp - s * akq;
          A[k][q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; k++) {
          const double apk = A[p][k], aqk = A[q][k];
          A[p][k] = c * apk - s * aqk;
          A[q][k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; k++) {
          const double vkp = V[k][p], vkq = V[k][q];
          V[k][p] = c * vkp - s * vkq;
          V[k][q] = s * vkp + c * vkq;
        }
      }
  }
  for (int i = 0; i < n; i++) w[i] = A[i][i];
}

// Orthogonal matrix (columns) whose first column is the unit vector u
// (Gram-Schmidt on u and the unit vectors).
void frame(int n, const double *u, Mat Q) {
  double cols[kMaxDim][kMaxDim];
  int k = 0;
  for (int i = 0; i < n; i++) cols[0][i] = u[i];
  k = 1;
  for (int e = 0; e < n && k < n; e++) {
    double v[kMaxDim];
    for (int i = 0; i < n; i++) v[i] = (i == e) ? 1.0 : 0.0;
    for (int j = 0; j < k; j++) {
      const double p = dot(n, v, cols[j]);
      for (int i = 0; i < n; i++) v[i] -= p * cols[j][i];
    }
    const double nv = vnorm(n, v);
    if (nv < 1e-8) continue;
    for (int i = 0; i < n; i++) cols[k][i] = v[i] / nv;
    k++;
  }
  for (int i = 0; i < n; i++)
    for (int j = 0; j < n; j++) Q[i][j] = cols[j][i];
}

// LLL reduction (delta = 3/4) of the rows of B.
void lll(int n, Mat B) {
  auto gs = [&](Mat Bs, Mat mu) {
    for (int i = 0; i < n; i++) {
      for (int j = 0; j < n; j++) Bs[i][j] = B[i][j];
      for (int j = 0; j < i; j++) {
        mu[i][j] = dot(n, B[i], Bs[j]) / dot(n, Bs[j], Bs[j]);
        for (int c = 0; c < n; c++) Bs[i][c] -= mu[i][j] * Bs[j][c];
      }
    }
  };
  Mat Bs, mu;
  gs(Bs, mu);
  int k = 1, guard = 0;
  while (k < n && guard++ < 10000) {
    for (int j = k - 1; j >= 0; j--) {
      const double q = rint(mu[k][j]);
      if (q != 0.0) {
        for (int c = 0; c < n; c++) B[k][c] -= q * B[j][c];
        gs(Bs, mu);
      }
    }
    if (dot(n, Bs[k], Bs[k]) >= (0.75 - mu[k][k - 1] * mu[k][k - 1]) * dot(n, Bs[k - 1], Bs[k - 1])) {
      k++;
    } else {
      for (int c = 0; c < n; c++) std::swap(B[k][c], B[k - 1][c]);
      gs(Bs, mu);
      k = std::max(k - 1, 1);
    }
  }
}

// Lattice vectors sum k_i b_i with |k_i| <= kmax, nonzero.
void short_vectors(int n, const Mat B, int kmax, std::vector<std::array<double, kMaxDim>> &out,
                   std::vector<std::array<int64_t, kMaxDim>> *coef = nullptr) {
  out.clear();
  if (coef) coef->clear();
  int k[kMaxDim];
  for (int i = 0; i < n; i++) k[i] = -kmax;
  while (true) {
    bool zero = true;
    for (int i = 0; i < n; i++) zero = zero && k[i] == 0;
    if (!zero) {
      std::array<double, kMaxDim> v{};
      std::array<int64_t, kMaxDim> c{};
      for (int i = 0; i < n; i++) {
        c[i] = k[i];
        for (int j = 0; j < n; j++) v[j] += k[i] * B[i][j];
      }
      out.push_back(v);
      if (coef) coef->push_back(c);
    }
    int i = 0;
    while (i < n && k[i] == kmax) k[i++] = -kmax;
    if (i == n) break;
    k[i]++;
  }
}

// Covering radius of the lattice with generator rows gen: the largest distance of
// a Voronoi vertex (equidistant from the origin and n Voronoi-relevant vectors,
// inside every half-space x.v <= |v|^2/2).
double covering_radius(int n, const Mat gen) {
  Mat B;
  mat_copy(n, gen, B);
  lll(n, B);
  std::vector<std::array<double, kMaxDim>> V;
  short_vectors(n, B, 2, V);
  std::vector<double> h(V.size());
  for (size_t i = 0; i < V.size(); i++) h[i] = 0.5 * dot(n, V[i].data(), V[i].data());
  std::vector<int> rel;
  for (size_t i = 0; i < V.size(); i++) {
    bool ok = true;
    for (size_t j = 0; j < V.size() && ok; j++) {
      if (j == i) continue;
      ok = 0.5 * dot(n, V[j].data(), V[i].data()) <= h[j] + 1e-12 * 2.0 * h[i];
    }
    if (ok) rel.push_back((int)i);
  }
  double R2 = 0.0;
  const int r = (int)rel.size();
  int idx[kMaxDim];
  for (int i = 0; i < n; i++) idx[i] = i;
  if (r < n) return 0.0;
  while (true) {
    Mat A;
    double b[kMaxDim], x[kMaxDim];
    for (int i = 0; i < n; i++) {
      for (int j = 0; j < n; j++) A[i][j] = V[rel[idx[i]]][j];
      b[i] = h[rel[idx[i]]];
    }
    if (solve(n, A, b, x)) {
      const double xx = dot(n, x, x);
      if (xx > R2) {
        bool inside = true;
        for (size_t j = 0; j < V.size() && inside; j++)
          inside = dot(n, x, V[j].data()) <= h[j] + 1e-9 * (1.0 + xx);
        if (inside) R2 = xx;
      }
    }
    int i = n - 1;
    while (i >= 0 && idx[i] == r - n + i) i--;
    if (i < 0) break;
    idx[i]++;
    for (int j = i + 1; j < n; j++) idx[j] = idx[j - 1] + 1;
  }
  return sqrt(R2);
}

double thickness(int n, const Mat gen, double R) {
  const double vsph = pow(M_PI, 0.5 * n) / tgamma(0.5 * n + 1.0) * pow(R, n);
  return vsph / fabs(det(n, gen));
}

void a_star(int n, double R, Mat M0) {
  memset(M0, 0, sizeof(Mat));
  if (n == 2) {
    const double s = R * sqrt(3.0);
    M0[0][0] = s;
    M0[1][0] = 0.5 * s;
    M0[1][1] = 0.5 * sqrt(3.0) * s;
    return;
  }
  const double s2 = sqrt(2.0), s3 = sqrt(3.0), s5 = sqrt(5.0), s6 = sqrt(6.0), f = R * sqrt(2.5);
  const double m[4][4] = {{s2, 0, 0, 0},
                          {1 / s2, sqrt(2.0 / 3.0) + 1 / s6, 0, 0},
                          {1 / s2, 1 / s6, 1 / (2 * s3) + s3 / 2, 0},
                          {-1 / (5 * s2) - 2 * s2 / 5, 1 / (5 * s6) - s6 / 5, -1 / (5 * s3) - s3 / 10, -1 / (2 * s5)}};
  for (int i = 0; i < 4; i++)
    for (int j = 0; j < 4; j++) M0[i][j] = f * m[i][j];
}

// gen -> gen O diag(d0, d1, ...) O^T (rows scaled along the columns of O)
void scale_along(int n, const Mat gen, const Mat O, const double *d, Mat out) {
  Mat T1, T2, Ot, D = {};
  for (int i = 0; i < n; i++) D[i][i] = d[i];
  mat_transpose(n, O, Ot);
  mat_mul(n, O, D, T1);
  mat_mul(n, T1, Ot, T2);
  mat_mul(n, gen, T2, out);
}

// Column operations (extended Euclid) bringing the integer rows to unit vectors;
// returns U (det +-1) whose first rows are the given rows up to multiples of
// earlier ones, or false if they are not part of a basis.
bool unimodular_with_rows(int n, const int64_t rows[][kMaxDim], int nrows, int64_t U[][kMaxDim]) {
  int64_t V[kMaxDim][kMaxDim] = {};
  for (int i = 0; i < n; i++) V[i][i] = 1;
  for (int i = 0; i < nrows; i++) {
    int64_t r[kMaxDim] = {};
    for (int j = 0; j < n; j++)
      for (int k = 0; k < n; k++) r[j] += rows[i][k] * V[k][j];
    for (int j = n - 1; j > i; j--) {
      int guard = 0;
      while (r[j] != 0 && guard++ < 1000) {
        const int64_t q = (int64_t)floor((double)r[i] / (double)r[j]);
        for (int k = 0; k < n; k++) V[k][i] -= q * V[k][j];
        r[i] -= q * r[j];
        for (int k = 0; k < n; k++) std::swap(V[k][i], V[k][j]);
        std::swap(r[i], r[j]);
      }
    }
    if (r[i] != 1 && r[i] != -1) return false;
    if (r[i] < 0)
      for (int k = 0; k < n; k++) V[k][i] = -V[k][i];
  }
  // U = V^-1 (integer, det +-1)
  Mat Vd, Ud;
  for (int i = 0; i < n; i++)
    for (int j = 0; j < n; j++) Vd[i][j] = (double)V[i][j];
  for (int j = 0; j < n; j++) {
    double e[kMaxDim] = {}, col[kMaxDim];
    e[j] = 1.0;
    if (!solve(n, Vd, e, col)) return false;
    for (int i = 0; i < n; i++) Ud[i][j] = col[i];
  }
  for (int i = 0; i < n; i++)
    for (int j = 0; j < n; j++) U[i][j] = (int64_t)llrint(Ud[i][j]);
  return true;
}

bool int_coeffs(int n, const Mat gen, const double *v, int64_t *c) {
  Mat Gt;
  mat_transpose(n, gen, Gt);
  double x[kMaxDim];
  if (!solve(n, Gt, v, x)) return false;
  for (int i = 0; i < n; i++) {
    c[i] = llrint(x[i]);
    if (fabs(x[i] - (double)c[i]) > 1e-6) return false;
  }
  return true;
}

}  // namespace

extern "C" {

fs_status fs_linear_model_fisher(const fs_detector *det, int64_t n, double dt, double t0, double *G) {
  if (!det || !G || n < 2 || !(dt > 0.0) || !isfinite(t0)) return FS_ERR_ARG;
  fs::SegGeom g{};
  g.theta0 = fmod(det->theta_g0 + det->lon + fmod(fs::kOmegaR * t0, fs::kTwoPi), fs::kTwoPi);
  g.lambda0 = fmod(det->lambda_e0 + fmod(fs::kOmegaO * t0, fs::kTwoPi), fs::kTwoPi);
  double re, z;
  fs::site_radius(det->lat, &re, &z);
  const double ce = cos(det->eps);
  // means and second moments of m = (t, t^2/2, mu1, mu2), accumulated about
  // reference values (the means of the first samples' values) for accuracy
  double s1[4] = {}, s2[4][4] = {};
  double ref[4] = {0.0, 0.0, 0.0, 0.0};
  for (int64_t k = 0; k < n; k++) {
    const double t = (double)k * dt;
    const double lam = g.lambda0 + fs::kOmegaO * t, th = g.theta0 + fs::kOmegaR * t;
    const double mu1 = fs::kAUls * sin(lam) + (re / fs::kC) * sin(th) * ce;
    const double mu2 = fs::kAUls * cos(lam) + (re / fs::kC) * cos(th);
    double m[4] = {t, 0.5 * t * t, mu1, mu2};
    if (k == 0)
      for (int i = 0; i < 4; i++) ref[i] = m[i];
    for (int i = 0; i < 4; i++) m[i] -= ref[i];
    for (int i = 0; i < 4; i++) {
      s1[i] += m[i];
      for (int j = 0; j < 4; j++) s2[i][j] += m[i] * m[j];
    }
  }
  for (int i = 0; i < 4; i++)
    for (int j = 0; j < 4; j++) G[4 * i + j] = s2[i][j] / n - (s1[i] / n) * (s1[j] / n);
  return FS_OK;
}

fs_status fs_lattice(int32_t dim, const double *G_, double C0, double dp0, int32_t constraint2, double *basis,
                     double *theta) {
  if (!G_ || !basis || (dim != 2 && dim != 4) || !(C0 > 0.0 && C0 < 1.0) || !(dp0 > 0.0)) return FS_ERR_ARG;
  if (constraint2 && dim != 4) return FS_ERR_ARG;
  const int n = dim;
  const double R = sqrt(1.0 - C0);
  // tau = Mx x with Mx^T G Mx = I: eigendecomposition of the unit-diagonal
  // D^-1 G D^-1 (G's entries span many decades), Mx = D^-1 U0 diag(w)^-1/2
  Mat G, U0, Mx, Mxt;
  double dg[kMaxDim];
  for (int i = 0; i < n; i++) {
    if (!(G_[n * i + i] > 0.0)) return FS_ERR_ARG;
    dg[i] = sqrt(G_[n * i + i]);
  }
  for (int i = 0; i < n; i++)
    for (int j = 0; j < n; j++) G[i][j] = 0.5 * (G_[n * i + j] + G_[n * j + i]) / (dg[i] * dg[j]);
  double w[kMaxDim];
  jacobi_eig(n, G, w, U0);
  for (int i = 0; i < n; i++)
    if (!(w[i] > 0.0)) return FS_ERR_ARG;
  for (int i = 0; i < n; i++)
    for (int j = 0; j < n; j++) Mx[i][j] = U0[i][j] / (sqrt(w[j]) * dg[i]);
  double a0[kMaxDim] = {dp0, 0, 0, 0}, e0[kMaxDim];
  if (!solve(n, Mx, a0, e0)) return FS_ERR_ARG;
  const double le0 = vnorm(n, e0);
  Mat M0;
  a_star(n, R, M0);
  const double theta_min = thickness(n, M0, R);
  std::vector<std::array<double, kMaxDim>> vecs;
  std::vector<std::array<int64_t, kMaxDim>> coefs;
  short_vectors(n, M0, 3, vecs, &coefs);
  std::vector<int> order(vecs.size());
  for (size_t i = 0; i < order.size(); i++) order[i] = (int)i;
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return vnorm(n, vecs[a].data()) < vnorm(n, vecs[b].data()); });
  // candidates: one per length shell with |l| >= |e0|
  std::vector<int> cand;
  for (int i : order) {
    const double L = vnorm(n, vecs[i].data());
    if (L < le0 * (1 - 1e-12)) continue;
    bool dup = false;
    for (int c : cand) dup = dup || fabs(vnorm(n, vecs[c].data()) - L) <= 1e-9 * L;
    if (!dup) cand.push_back(i);
    if (cand.size() >= 4) break;
  }
  double best = -1.0, best_mu = 0, best_nu = 0;
  int best_l = -1;
  for (int ci : cand) {
    const double *l = vecs[ci].data();
    const double L = vnorm(n, l);
    double u[kMaxDim];
    for (int i = 0; i < n; i++) u[i] = l[i] / L;
    Mat O1, M1;
    frame(n, u, O1);
    const double mu = le0 / L;
    double d1[kMaxDim] = {mu, 1, 1, 1};
    scale_along(n, M0, O1, d1, M1);
    auto g = [&](double nu) {
      Mat Mn;
      double d[kMaxDim] = {1, nu, nu, nu};
      scale_along(n, M1, O1, d, Mn);
      return covering_radius(n, Mn) - R;
    };
    double lo = 1.0, hi = 2.0, glo = g(lo), ghi = g(hi);
    int guard = 0;
    while (ghi < 0 && guard++ < 40) {
      lo = hi;
      glo = ghi;
      hi *= 2.0;
      ghi = g(hi);
    }
    double mid = lo;
    int side = 0;
    for (int it = 0; it < 200; it++) {  // regula falsi, Illinois modification
      mid = (lo * ghi - hi * glo) / (ghi - glo);
      const double gm = g(mid);
      if (gm > 0) {
        hi = mid;
        ghi = gm;
        if (side == -1) glo *= 0.5;
        side = -1;
      } else {
        lo = mid;
        glo = gm;
        if (side == 1) ghi *= 0.5;
        side = 1;
      }
      if (hi - lo <= 1e-12 * hi || fabs(gm) <= 1e-15 * R) break;
    }
    const double detS = mu * pow(mid, n - 1);
    if (detS > best * (1 + 1e-12)) {
      best = detS;
      best_mu = mu;
      best_nu = mid;
      best_l = ci;
    }
  }
  if (best_l < 0) return FS_ERR_ARG;
  const double *l = vecs[best_l].data();
  const double L = vnorm(n, l);
  double u[kMaxDim], e0h[kMaxDim];
  for (int i = 0; i < n; i++) {
    u[i] = l[i] / L;
    e0h[i] = e0[i] / le0;
  }
  Mat O1, O2, O2t, S = {}, X, T1, T2;
  frame(n, u, O1);
  frame(n, e0h, O2);
  S[0][0] = best_mu;
  for (int i = 1; i < n; i++) S[i][i] = best_nu;
  mat_transpose(n, O2, O2t);
  mat_mul(n, M0, O1, T1);
  mat_mul(n, T1, S, T2);
  mat_mul(n, T2, O2t, X);  // rows: images of M0's rows in x
  int64_t rows[2][kMaxDim] = {};
  int nrows = 1;
  if (!int_coeffs(n, M0, l, rows[0])) return FS_ERR_ARG;
  if (constraint2) {
    // f: the shortest lattice vector not parallel to l that completes l to a basis
    int fi = -1;
    for (int i : order) {
      const double *v = vecs[i].data();
      if (fabs(fabs(dot(n, v, l)) - vnorm(n, v) * L) <= 1e-9 * dot(n, v, v)) continue;
      int64_t c2[2][kMaxDim], Ut[kMaxDim][kMaxDim];
      memcpy(c2[0], rows[0], sizeof(c2[0]));
      memcpy(c2[1], coefs[i].data(), sizeof(c2[1]));
      if (unimodular_with_rows(n, c2, 2, Ut)) {
        fi = i;
        break;
      }
    }
    if (fi < 0) return FS_ERR_ARG;
    memcpy(rows[1], coefs[fi].data(), sizeof(rows[1]));
    nrows = 2;
    // y_f = f O1 S O2^T (row); rotate its component orthogonal to e0 onto the
    // direction w of {x : (Mx x)_sky = 0} orthogonal to e0
    double yf[kMaxDim] = {};
    for (int j = 0; j < n; j++)
      for (int k = 0; k < n; k++) yf[j] += (double)rows[1][k] * X[k][j];
    // kernel of the sky rows of Mx: Gram-Schmidt complement of their span
    double s1[kMaxDim], s2[kMaxDim];
    for (int j = 0; j < n; j++) {
      s1[j] = Mx[2][j];
      s2[j] = Mx[3][j];
    }
    const double n1 = vnorm(n, s1);
    for (int j = 0; j < n; j++) s1[j] /= n1;
    const double p12 = dot(n, s2, s1);
    for (int j = 0; j < n; j++) s2[j] -= p12 * s1[j];
    const double n2 = vnorm(n, s2);
    for (int j = 0; j < n; j++) s2[j] /= n2;
    // w = the part of the kernel orthogonal to e0: project e0-orthogonal unit vectors
    double wv[kMaxDim] = {}, bestw = 0.0;
    for (int e = 0; e < n; e++) {
      double v[kMaxDim];
      for (int j = 0; j < n; j++) v[j] = (j == e) ? 1.0 : 0.0;
      const double a1 = dot(n, v, s1), a2 = dot(n, v, s2);
      for (int j = 0; j < n; j++) v[j] -= a1 * s1[j] + a2 * s2[j];
      const double ae = dot(n, v, e0h);
      for (int j = 0; j < n; j++) v[j] -= ae * e0h[j];
      const double nv = vnorm(n, v);
      if (nv > bestw) {
        bestw = nv;
        for (int j = 0; j < n; j++) wv[j] = v[j] / nv;
      }
    }
    double yp[kMaxDim];
    const double ye = dot(n, yf, e0h);
    for (int j = 0; j < n; j++) yp[j] = yf[j] - ye * e0h[j];
    const double nyp = vnorm(n, yp);
    double uu[kMaxDim];
    for (int j = 0; j < n; j++) uu[j] = yp[j] / nyp;
    const double c = fmax(-1.0, fmin(1.0, dot(n, uu, wv)));
    double v2[kMaxDim];
    for (int j = 0; j < n; j++) v2[j] = wv[j] - c * uu[j];
    const double nv2 = vnorm(n, v2);
    Mat O3, O3t, X2;
    for (int i = 0; i < n; i++)
      for (int j = 0; j < n; j++) O3[i][j] = (i == j) ? 1.0 : 0.0;
    if (nv2 > 1e-14) {
      for (int j = 0; j < n; j++) v2[j] /= nv2;
      const double s = sqrt(fmax(0.0, 1.0 - c * c));
      for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++)
          O3[i][j] += (c - 1.0) * (uu[i] * uu[j] + v2[i] * v2[j]) + s * (v2[i] * uu[j] - uu[i] * v2[j]);
    }
    mat_transpose(n, O3, O3t);
    mat_mul(n, X, O3t, X2);
    mat_copy(n, X2, X);
  }
  int64_t U[kMaxDim][kMaxDim];
  if (!unimodular_with_rows(n, rows, nrows, U)) return FS_ERR_ARG;
  Mat Ud, B1, B2;
  for (int i = 0; i < n; i++)
    for (int j = 0; j < n; j++) Ud[i][j] = (double)U[i][j];
  mat_transpose(n, Mx, Mxt);
  mat_mul(n, Ud, X, B1);
  mat_mul(n, B1, Mxt, B2);
  for (int i = 0; i < n; i++)
    for (int j = 0; j < n; j++) basis[n * i + j] = B2[i][j];
  // exact zeros where the constraints put them
  for (int j = 1; j < n; j++) basis[j] = 0.0;
  basis[0] = dp0;
  if (constraint2) basis[n + 2] = basis[n + 3] = 0.0;
  if (theta) *theta = theta_min / best;
  return FS_OK;
}

fs_status fs_lattice_nodes(const double *basis, const fs_detector *det, double fl, double f0_min, double f0_max,
                           double f1_min, double f1_max, fs_point *pts, int64_t cap, int64_t *count) {
  if (!basis || !det || !count || cap < 0 || (cap > 0 && !pts)) return FS_ERR_ARG;
  if (!(f0_max >= f0_min) || !(f1_max >= f1_min) || !(fl + f0_min > 0.0)) return FS_ERR_ARG;
  // the basis of fs_lattice with both constraints is triangular in its first two
  // rows: a0 = (dp0, 0, 0, 0), a1 = (a10, a11, 0, 0)
  const double *B0 = basis, *B1 = basis + 4, *B2 = basis + 8, *B3 = basis + 12;
  if (!(B0[0] > 0.0) || B0[1] != 0.0 || B0[2] != 0.0 || B0[3] != 0.0 || B1[1] == 0.0 || B1[2] != 0.0 ||
      B1[3] != 0.0)
    return FS_ERR_ARG;
  const double tp = 2.0 * M_PI;
  const double w0lo = tp * (fl + f0_min), w0hi = tp * (fl + f0_max);
  const double w1lo = tp * f1_min, w1hi = tp * f1_max;
  // sky nodes alpha = k2 s2 + k3 s3 with |alpha| <= w0hi: |k| <= w0hi |row of S^-1|
  const double s00 = B2[2], s01 = B2[3], s10 = B3[2], s11 = B3[3];
  const double dS = s00 * s11 - s01 * s10;
  if (dS == 0.0) return FS_ERR_ARG;
  // alpha^T = k^T S (rows s2, s3)  =>  k^T = alpha^T S^-1, S^-1 = [[s11, -s01], [-s10, s00]] / dS
  const double c2n = sqrt(s11 * s11 + s10 * s10) / fabs(dS), c3n = sqrt(s01 * s01 + s00 * s00) / fabs(dS);
  const int64_t k2r = (int64_t)ceil(w0hi * c2n) + 1, k3r = (int64_t)ceil(w0hi * c3n) + 1;
  if ((double)(2 * k2r + 1) * (double)(2 * k3r + 1) > 4e8) return FS_ERR_SHAPE;
  const double ce = cos(det->eps), se = sin(det->eps);
  int64_t cnt = 0;
  for (int64_t k2 = -k2r; k2 <= k2r; k2++)
    for (int64_t k3 = -k3r; k3 <= k3r; k3++) {
      const double a1 = k2 * B2[2] + k3 * B3[2], a2 = k2 * B2[3] + k3 * B3[3];
      if (a1 * a1 + a2 * a2 > w0hi * w0hi) continue;
      // spindown nodes: omega1 = k1 a11 + k2 B2[1] + k3 B3[1]
      const double c1 = k2 * B2[1] + k3 * B3[1];
      double lo1 = (w1lo - c1) / B1[1], hi1 = (w1hi - c1) / B1[1];
      if (lo1 > hi1) std::swap(lo1, hi1);
      for (int64_t k1 = (int64_t)ceil(lo1); (double)k1 <= hi1; k1++) {
        const double om1 = k1 * B1[1] + c1;
        if (om1 < w1lo || om1 > w1hi) continue;
        // frequency nodes: omega0 = k0 dp0 + k1 a10 + k2 B2[0] + k3 B3[0]
        const double c0 = k1 * B1[0] + k2 * B2[0] + k3 * B3[0];
        for (int64_t k0 = (int64_t)ceil((w0lo - c0) / B0[0]); (double)k0 * B0[0] + c0 <= w0hi; k0++) {
          const double om0 = k0 * B0[0] + c0;
          if (om0 < w0lo) continue;
          const double ny = a1 / om0, nx = a2 / om0;  // ecliptic n0_y, n0_x (Eq. albe)
          const double r2 = nx * nx + ny * ny;
          if (r2 > 1.0) continue;
          const double nz_abs = sqrt(fmax(0.0, 1.0 - r2));
          for (int h = 0; h < (nz_abs > 0.0 ? 2 : 1); h++) {
            const double nz = h ? -nz_abs : nz_abs;
            // equatorial components: n_eq = Rot(eps)^T n0
            const double ex = nx, ey = ce * ny - se * nz, ez = se * ny + ce * nz;
            double alpha = atan2(ey, ex);
            if (alpha < 0) alpha += tp;
            const double delta = asin(fmax(-1.0, fmin(1.0, ez)));
            if (cnt < cap) pts[cnt] = fs_point{om0 / tp - fl, om1 / tp, alpha, delta};
            cnt++;
          }
        }
      }
    }
  *count = cnt;
  return cnt > cap ? FS_ERR_CAPACITY : FS_OK;
}

fs_status fs_lattice_templates(const double *basis, const fs_detector *det, double fl, int64_t nfft, double dt,
                               double f1_min, double f1_max, const double *box, double *alpha, double *delta,
                               double *f1, double *offset, int64_t sky_cap, int32_t spin_cap, int64_t *nsky,
                               int32_t *nspin) {
  if (!basis || !det || !nsky || !nspin || sky_cap < 0 || spin_cap < 0) return FS_ERR_ARG;
  if (sky_cap > 0 && (!alpha || !delta || !f1 || !offset)) return FS_ERR_ARG;
  if (nfft < 2 || !(dt > 0.0) || !(f1_max >= f1_min) || !(fl > 0.0)) return FS_ERR_ARG;
  const double tp = 2.0 * M_PI;
  const double *B0 = basis, *B1 = basis + 4, *B2 = basis + 8, *B3 = basis + 12;
  // a0 must be the transform's Fourier spacing and a1 free of sky components
  // (zeros up to the rounding of the construction)
  const double dp0 = B0[0];
  if (!(fabs(dp0 - tp / ((double)nfft * dt)) <= 1e-9 * dp0)) return FS_ERR_ARG;
  double scale[4] = {0, 0, 0, 0};
  for (int r = 0; r < 4; r++)
    for (int c = 0; c < 4; c++) scale[c] = fmax(scale[c], fabs(basis[4 * r + c]));
  for (int c = 1; c < 4; c++)
    if (fabs(B0[c]) > 1e-9 * scale[c]) return FS_ERR_ARG;
  for (int c = 2; c < 4; c++)
    if (fabs(B1[c]) > 1e-9 * scale[c]) return FS_ERR_ARG;
  if (B1[1] == 0.0) return FS_ERR_ARG;
  const double bx[4] = {box ? box[0] : -1.0, box ? box[1] : 1.0, box ? box[2] : -1.0, box ? box[3] : 1.0};
  const double w_ref = tp * (fl + 0.5 / dt);  // sky positions at the band's upper edge (Eq. albe)
  const double w1lo = tp * f1_min, w1hi = tp * f1_max;
  const double s00 = B2[2], s01 = B2[3], s10 = B3[2], s11 = B3[3];
  const double dS = s00 * s11 - s01 * s10;
  if (dS == 0.0) return FS_ERR_ARG;
  // k^T = alpha^T S^-1 with S^-1 = [[s11, -s01], [-s10, s00]] / dS: |k_i| <= w_ref |column i|
  const int64_t k2r = (int64_t)ceil(w_ref * sqrt(s11 * s11 + s10 * s10) / fabs(dS)) + 1;
  const int64_t k3r = (int64_t)ceil(w_ref * sqrt(s01 * s01 + s00 * s00) / fabs(dS)) + 1;
  if ((double)(2 * k2r + 1) * (double)(2 * k3r + 1) > 4e8) return FS_ERR_SHAPE;
  const double ce = cos(det->eps), se = sin(det->eps);
  const double fl_bins = fl * (double)nfft * dt;
  std::vector<std::pair<double, double>> row;  // (f1, bin offset) of one line family
  int64_t ns = 0;
  int32_t nmax = 0;
  for (int pass = 0; pass < 2; pass++) {  // pass 0 sizes (skies, longest row), pass 1 writes
    ns = 0;
    for (int64_t k2 = -k2r; k2 <= k2r; k2++)
      for (int64_t k3 = -k3r; k3 <= k3r; k3++) {
        const double a1 = k2 * B2[2] + k3 * B3[2], a2 = k2 * B2[3] + k3 * B3[3];
        const double ny = a1 / w_ref, nx = a2 / w_ref;  // ecliptic n0_y, n0_x
        const double r2 = nx * nx + ny * ny;
        if (r2 > 1.0 || !(nx >= bx[0] && nx <= bx[1] && ny >= bx[2] && ny <= bx[3])) continue;
        const double c1 = k2 * B2[1] + k3 * B3[1];
        double lo = (w1lo - c1) / B1[1], hi = (w1hi - c1) / B1[1];
        if (lo > hi) std::swap(lo, hi);
        row.clear();
        for (int64_t k1 = (int64_t)ceil(lo); (double)k1 <= hi; k1++) {
          const double om1 = k1 * B1[1] + c1;
          if (om1 < w1lo || om1 > w1hi) continue;
          // the line omega0 = c0 + k0 dp0 sits on bins k shifted by the fraction xb - floor(xb)
          const double c0 = k1 * B1[0] + k2 * B2[0] + k3 * B3[0];
          const double xb = c0 / dp0 - fl_bins;
          double d = xb - floor(xb);
          if (d >= 1.0) d = 0.0;
          row.push_back({om1 / tp, d});
        }
        if (row.empty()) continue;
        const double nz_abs = sqrt(fmax(0.0, 1.0 - r2));
        const int nh = nz_abs > 0.0 ? 2 : 1;
        if (pass == 0) {
          nmax = std::max(nmax, (int32_t)row.size());
        } else {
          for (int h = 0; h < nh; h++) {
            const int64_t sk = ns + h;
            const double nz = h ? -nz_abs : nz_abs;
            const double ex = nx, ey = ce * ny - se * nz, ez = se * ny + ce * nz;  // n_eq = Rot(eps)^T n0
            double a = atan2(ey, ex);
            if (a < 0) a += tp;
            alpha[sk] = a;
            delta[sk] = asin(fmax(-1.0, fmin(1.0, ez)));
            for (int32_t q = 0; q < nmax; q++) {  // shorter rows repeat their last node
              const auto &e = row[std::min<size_t>((size_t)q, row.size() - 1)];
              f1[sk * nmax + q] = e.first;
              offset[sk * nmax + q] = e.second;
            }
          }
        }
        ns += nh;
      }
    if (pass == 0) {
      *nsky = ns;
      *nspin = nmax;
      if (sky_cap == 0 && spin_cap == 0) return FS_OK;  // size query
      if (ns > sky_cap || nmax > spin_cap) return FS_ERR_CAPACITY;
    }
  }
  return FS_OK;
}

}  // extern "C"
