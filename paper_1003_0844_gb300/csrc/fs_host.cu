// Host-side statistics of a search (no device work): the false-alarm
// probability of a threshold over a number of independent cells, its inverse,
// and the number of cells of a parameter-space volume (Sec. III).
#include <math.h>
#include "fs_internal.h"

extern "C" {

double fs_false_alarm_cell(double F0) {
  if (!(F0 > 0.0)) return 1.0;
  return (1.0 + F0) * exp(-F0);  // Eq. PF: 2F ~ chi^2 with 4 degrees of freedom
}

fs_status fs_false_alarm(double F0, double n_cells, double *alpha, double *n_false) {
  if (!alpha || !isfinite(F0) || !(n_cells > 0.0) || !isfinite(n_cells)) return FS_ERR_ARG;
  const double P = fs_false_alarm_cell(F0);
  // Eq. FP, 1 - (1 - P)^Nc, in a form that keeps its digits for tiny P
  *alpha = P < 1.0 ? -expm1(n_cells * log1p(-P)) : 1.0;
  if (n_false) *n_false = n_cells * P;  // Eq. NF
  return FS_OK;
}

fs_status fs_threshold(double alpha, double n_cells, double *F0) {
  if (!F0 || !(alpha > 0.0) || !(alpha < 1.0) || !(n_cells > 0.0) || !isfinite(n_cells)) return FS_ERR_ARG;
  // per-cell probability P = 1 - (1 - alpha)^(1/Nc), then (1 + F) exp(-F) = P
  const double P = -expm1(log1p(-alpha) / n_cells);
  if (P >= 1.0) {
    *F0 = 0.0;
    return FS_OK;
  }
  const double lp = log(P);
  // h(F) = log(1 + F) - F - log P is decreasing and concave on F > 0: Newton from
  // the right of the root (F = -log P + log(1 - log P) >= root) converges monotonically
  double F = -lp + log1p(-lp);
  for (int it = 0; it < 100; it++) {
    const double h = log1p(F) - F - lp;
    const double dh = -F / (1.0 + F);
    const double step = h / dh;
    F -= step;
    if (F < 0.0) F = 0.0;
    if (fabs(step) <= 1e-15 * (1.0 + F)) break;
  }
  *F0 = F;
  return FS_OK;
}

fs_status fs_cell_count(int32_t M, const double *G, double v_total, double *n_cells) {
  if (!G || !n_cells || M < 1 || M > 16 || !(v_total > 0.0)) return FS_ERR_ARG;
  // det G by Cholesky (G symmetric positive definite)
  double L[16][16] = {};
  double logdet = 0.0;
  for (int i = 0; i < M; i++) {
    for (int j = 0; j <= i; j++) {
      double v = G[i * M + j];
      for (int k = 0; k < j; k++) v -= L[i][k] * L[j][k];
      if (i == j) {
        if (!(v > 0.0)) return FS_ERR_ARG;
        L[i][i] = sqrt(v);
        logdet += 2.0 * log(L[i][i]);
      } else {
        L[i][j] = v / L[j][j];
      }
    }
  }
  // Eq. vc: V_cell = pi^(M/2) / (Gamma(M/2 + 1) sqrt(det G)); Eq. NT: Nc = V_total / V_cell
  const double log_vcell = 0.5 * M * log(M_PI) - lgamma(0.5 * M + 1.0) - 0.5 * logdet;
  *n_cells = v_total * exp(-log_vcell);
  return FS_OK;
}

}  // extern "C"
