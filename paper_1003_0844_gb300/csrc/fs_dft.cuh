// Register-resident DFTs of small power-of-two sizes (FP32), fully unrolled at
// compile time.  Convention of Eq. (eq:DFT): X_k = sum_l x_l exp(-2 pi i l k / n).
#pragma once
#include <type_traits>
#include "fs_common.cuh"

namespace fs {

// Compile-time loop: calls f(std::integral_constant<int, I>) for I = B..E-1.
template <int B, int E, typename F>
__device__ __forceinline__ void sfor(F &&f) {
  if constexpr (B < E) {
    f(std::integral_constant<int, B>{});
    sfor<B + 1, E>(f);
  }
}

// cos and sin of k pi / 32 in double, evaluated at compile time: reduce to a
// quarter turn plus phi in [0, pi/2) and sum the Taylor series of phi.
constexpr double cx_pi = 3.14159265358979323846264338327950288;
constexpr double cx_sin_series(double x) {
  double x2 = x * x, term = x, sum = x;
  for (int n = 1; n < 14; n++) { term *= -x2 / ((2.0 * n) * (2.0 * n + 1.0)); sum += term; }
  return sum;
}
constexpr double cx_cos_series(double x) {
  double x2 = x * x, term = 1.0, sum = 1.0;
  for (int n = 1; n < 14; n++) { term *= -x2 / ((2.0 * n - 1.0) * (2.0 * n)); sum += term; }
  return sum;
}
constexpr double cx_cos64(int k) {  // cos(2 pi k / 64)
  int q = (k / 16) & 3, r = k % 16;
  double phi = r * cx_pi / 32.0;
  double c = cx_cos_series(phi), s = cx_sin_series(phi);
  return q == 0 ? c : q == 1 ? -s : q == 2 ? -c : s;
}
constexpr double cx_sin64(int k) {  // sin(2 pi k / 64)
  int q = (k / 16) & 3, r = k % 16;
  double phi = r * cx_pi / 32.0;
  double c = cx_cos_series(phi), s = cx_sin_series(phi);
  return q == 0 ? s : q == 1 ? c : q == 2 ? -s : -c;
}

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }

// z * exp(-2 pi i K / M), M a power of two dividing 64, 0 <= K < M/2.
template <int M, int K>
__device__ __forceinline__ float2 twmul(float2 z) {
  constexpr float r2 = 0.70710678118654752440f;
  if constexpr (K == 0) {
    return z;
  } else if constexpr (4 * K == M) {  // -i
    return make_float2(z.y, -z.x);
  } else if constexpr (8 * K == M) {  // (1 - i)/sqrt2
    return make_float2((z.x + z.y) * r2, (z.y - z.x) * r2);
  } else if constexpr (8 * K == 3 * M) {  // (-1 - i)/sqrt2
    return make_float2((z.y - z.x) * r2, -(z.x + z.y) * r2);
  } else {
    constexpr int k64 = K * (64 / M);
    constexpr float c = (float)cx_cos64(k64);
    constexpr float s = (float)(-cx_sin64(k64));
    return make_float2(fmaf(z.x, c, -z.y * s), fmaf(z.x, s, z.y * c));
  }
}

constexpr int cx_log2(int n) { return n <= 1 ? 0 : 1 + cx_log2(n / 2); }
constexpr int cx_bitrev(int i, int bits) {
  int r = 0;
  for (int b = 0; b < bits; b++) r |= ((i >> b) & 1) << (bits - 1 - b);
  return r;
}

// In-place DFT of v[0..N) (N = 2..32), natural order in and out: radix-2
// decimation in frequency, then a compile-time bit-reversal (register renaming).
// NZ: the inputs v[NZ..N) are known to be zero.  After each stage the nonzero
// entries of every group (2 span entries) stay at offsets below
// min(NZ, 2 span), so a pair whose both entries lie beyond that is left alone,
// and a pair whose second entry does reduces to a copy and a twiddle product.
// NOUT: only outputs X[0..NOUT) are needed (NOUT = N or N/2); with NOUT = N/2
// the last stage skips the differences (they land on odd bit-reversed positions).
template <int N, int NZ = N, int NOUT = N>
__device__ __forceinline__ void dft_inplace(float2 *v) {
  static_assert(NZ >= 1 && NZ <= N, "NZ leading inputs may be nonzero");
  static_assert(NOUT == N || 2 * NOUT == N, "output pruning keeps the lower half only");
  constexpr int LG = cx_log2(N);
  sfor<0, LG>([&](auto st) {
    constexpr int span = N >> (st + 1);
    constexpr int nz = NZ < 2 * span ? NZ : 2 * span;  // nonzero prefix of each group
    sfor<0, N / (2 * span)>([&](auto g) {
      sfor<0, span>([&](auto k) {
        constexpr int i0 = g * 2 * span + k;
        if constexpr (k >= nz) {
          // both entries are zero
        } else if constexpr (k + span >= nz) {
          const float2 a = v[i0];
          v[i0 + span] = twmul<2 * span, k>(a);
        } else if constexpr (st == LG - 1 && NOUT < N) {
          v[i0] = cadd(v[i0], v[i0 + span]);
        } else {
          float2 a = v[i0], b = v[i0 + span];
          v[i0] = cadd(a, b);
          v[i0 + span] = twmul<2 * span, k>(csub(a, b));
        }
      });
    });
  });
  float2 tmp[N];
  sfor<0, N>([&](auto i) { tmp[i] = v[cx_bitrev(i, LG)]; });
  sfor<0, N>([&](auto i) { v[i] = tmp[i]; });
}

}  // namespace fs
