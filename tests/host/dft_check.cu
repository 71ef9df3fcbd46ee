// Host-side check of the register DFTs of the transform kernels (fs_dft.cuh,
// compiled as host code): every size, zero-input pruning and output pruning the
// kernels instantiate, against a direct double-precision DFT of the same floats
// (Eq. eq:DFT, X_k = sum_l x_l exp(-2 pi i l k / n)).  Prints the worst error
// relative to the input norm per case and exits non-zero above the bound.
#include <cmath>
#include <cstdio>
#include <random>

#include "../../paper_1003_0844_gb300/csrc/fs_dft.cuh"

template <int N, int NZ, int NOUT>
static double worst_error(std::mt19937 &g) {
  std::normal_distribution<float> nd;
  double worst = 0;
  for (int rep = 0; rep < 200; rep++) {
    float2 v[N];
    double xr[N], xi[N], nrm = 0;
    for (int i = 0; i < N; i++) {
      v[i] = i < NZ ? make_float2(nd(g), nd(g)) : make_float2(0.f, 0.f);
      xr[i] = v[i].x;
      xi[i] = v[i].y;
      nrm += xr[i] * xr[i] + xi[i] * xi[i];
    }
    fs::dft_inplace<N, NZ, NOUT>(v);
    for (int k = 0; k < NOUT; k++) {
      double sr = 0, si = 0;
      for (int j = 0; j < N; j++) {
        const double a = -2.0 * M_PI * (double)((j * k) % N) / N;
        sr += xr[j] * std::cos(a) - xi[j] * std::sin(a);
        si += xr[j] * std::sin(a) + xi[j] * std::cos(a);
      }
      const double e = std::hypot(v[k].x - sr, v[k].y - si) / std::sqrt(nrm);
      if (e > worst) worst = e;
    }
  }
  return worst;
}

static int failures = 0;
template <int N, int NZ, int NOUT>
static void check(std::mt19937 &g) {
  // a few roundings of FP32 per stage: well below 1e-6 of the input norm
  const double e = worst_error<N, NZ, NOUT>(g), bound = 1e-6;
  printf("N=%2d NZ=%2d NOUT=%2d worst %.3e\n", N, NZ, NOUT, e);
  if (!(e < bound)) failures++;
}

int main() {
  std::mt19937 g(20100304);
  check<2, 2, 2>(g); check<2, 1, 2>(g); check<2, 2, 1>(g);
  check<4, 4, 4>(g); check<4, 2, 4>(g); check<4, 4, 2>(g); check<4, 1, 2>(g);
  check<8, 8, 8>(g); check<8, 4, 8>(g); check<8, 2, 8>(g); check<8, 8, 4>(g); check<8, 4, 4>(g);
  check<16, 16, 16>(g); check<16, 8, 16>(g); check<16, 4, 16>(g); check<16, 6, 16>(g);
  check<16, 16, 8>(g); check<16, 8, 8>(g); check<16, 3, 8>(g);
  check<32, 32, 32>(g); check<32, 16, 32>(g); check<32, 8, 32>(g); check<32, 5, 32>(g);
  check<32, 32, 16>(g); check<32, 16, 16>(g); check<32, 8, 16>(g);
  printf(failures ? "FAIL\n" : "OK\n");
  return failures ? 1 : 0;
}
