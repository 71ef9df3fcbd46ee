// Register-resident DFTs of small power-of-two sizes (FP32), fully unrolled at
// compile time.  Convention of Eq. (eq:DFT): X_k = sum_l x_l exp(-2 pi i l k / n).
#pragma once
#include <type_traits>
#include "fs_common.cuh"

namespace fs {

// Compile-time loop: calls f(std::integral_constant<int, I>) for I = B..E-1.
template <int B, int E, typename F>
__host__ __device__ __forceinline__ void sfor(F &&f) {
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


// Packed FP32 pairs (the f32x2 forms of add, sub, mul and fma on sm_100 and later):
// both halves of a complex value in one instruction.  They do the same arithmetic at
// the same FP32 rate as two scalar instructions (measured: 69 TFLOP/s either way) but
// take half the issue slots, which bound the transform kernel; swapping the halves of
// an operand measured free.  The butterflies use them (3.5% faster on the 2-day grid,
// 7% on 2^21); complex products with a runtime twiddle measured slower packed (the
// broadcast and sign of the twiddle's halves cost more than they save).  Device code
// only; the host keeps the scalar forms (the butterflies round exactly as they do; a
// lone twiddle product rounds its two terms in another order).
#if defined(__CUDA_ARCH__)
#define FS_X2 1
__device__ __forceinline__ unsigned long long x2p(float2 a) {
  unsigned long long r; asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a.x), "f"(a.y)); return r;
}
__device__ __forceinline__ float2 x2u(unsigned long long v) {
  float2 a; asm("mov.b64 {%0, %1}, %2;" : "=f"(a.x), "=f"(a.y) : "l"(v)); return a;
}
__device__ __forceinline__ float2 x2add(float2 a, float2 b) {
  unsigned long long d; asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(x2p(a)), "l"(x2p(b))); return x2u(d);
}
__device__ __forceinline__ float2 x2sub(float2 a, float2 b) {
  unsigned long long d; asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(x2p(a)), "l"(x2p(b))); return x2u(d);
}
__device__ __forceinline__ float2 x2mul(float2 a, float2 b) {
  unsigned long long d; asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(x2p(a)), "l"(x2p(b))); return x2u(d);
}
__device__ __forceinline__ float2 x2fma(float2 a, float2 b, float2 c) {  // a * b + c by halves
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(x2p(a)), "l"(x2p(b)), "l"(x2p(c)));
  return x2u(d);
}
__device__ __forceinline__ float2 x2swap(float2 a) { return make_float2(a.y, a.x); }
#endif

__host__ __device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }

// z * exp(-2 pi i K / M), M a power of two dividing 64, 0 <= K < M/2.
template <int M, int K>
__host__ __device__ __forceinline__ float2 twmul(float2 z) {
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

// Radix-2 decimation in time with the butterflies written as fused multiply-adds.
// A butterfly (a, b) -> (a + w b, a - w b) with a general twiddle w = c + i s costs
// six FMAs instead of a complex product and four additions: w b is factored as
// c (u + i v) with u = b.x - (s/c) b.y, v = b.y + (s/c) b.x when |c| >= |s| (else
// as s (u + i v) with the ratio c/s), and a +- c u, a +- c v are FMAs (the
// "tangent" factorisation of Linzer and Feig for FMA machines).  w = 1 and
// w = -i need four additions.  The ratios and factors are rounded once at
// compile time from the double-precision table above.
template <int M, int K>
__host__ __device__ __forceinline__ void bfly_dit(float2 &a, float2 &b) {
#ifdef FS_X2
  if constexpr (K == 0) {
    const float2 t = b;
    b = x2sub(a, t);
    a = x2add(a, t);
  } else if constexpr (4 * K == M) {  // w = -i: w b = (b.y, -b.x)
    const float2 t = x2swap(b);
    b = x2fma(make_float2(-1.f, 1.f), t, a);
    a = x2fma(make_float2(1.f, -1.f), t, a);
  } else {
    constexpr int k64 = K * (64 / M);
    constexpr double c = cx_cos64(k64), s = -cx_sin64(k64);
    constexpr bool cbig = (c >= 0 ? c : -c) >= (s >= 0 ? s : -s);
    constexpr float f = (float)(cbig ? c : s);
    constexpr float r = (float)(cbig ? s / c : c / s);
    if constexpr (cbig) {
      const float2 uv = x2fma(make_float2(-r, r), x2swap(b), b);  // (b.x - r b.y, b.y + r b.x)
      b = x2fma(make_float2(-f, -f), uv, a);
      a = x2fma(make_float2(f, f), uv, a);
    } else {
      // (u, v) = (r b.x - b.y, r b.y + b.x) = (-v', u') with (u', v') = (b.x + r b.y, b.y - r b.x)
      const float2 vu = x2swap(x2fma(make_float2(r, -r), x2swap(b), b));
      b = x2fma(make_float2(f, -f), vu, a);
      a = x2fma(make_float2(-f, f), vu, a);
    }
  }
#else
  if constexpr (K == 0) {
    const float2 t = b;
    b = csub(a, t);
    a = cadd(a, t);
  } else if constexpr (4 * K == M) {  // w = -i: w b = (b.y, -b.x)
    const float2 t = b;
    b = make_float2(a.x - t.y, a.y + t.x);
    a = make_float2(a.x + t.y, a.y - t.x);
  } else {
    constexpr int k64 = K * (64 / M);
    constexpr double c = cx_cos64(k64), s = -cx_sin64(k64);
    constexpr bool cbig = (c >= 0 ? c : -c) >= (s >= 0 ? s : -s);
    constexpr float f = (float)(cbig ? c : s);
    constexpr float r = (float)(cbig ? s / c : c / s);
    float u, v;
    if constexpr (cbig) {
      u = fmaf(-r, b.y, b.x);
      v = fmaf(r, b.x, b.y);
    } else {
      u = fmaf(r, b.x, -b.y);
      v = fmaf(r, b.y, b.x);
    }
    b = make_float2(fmaf(-f, u, a.x), fmaf(-f, v, a.y));
    a = make_float2(fmaf(f, u, a.x), fmaf(f, v, a.y));
  }
#endif
}
// w b alone (the first operand of the butterfly is known to be zero).
template <int M, int K>
__host__ __device__ __forceinline__ float2 twmul_dit(float2 b) {
  if constexpr (K == 0) {
    return b;
  } else if constexpr (4 * K == M) {
    return make_float2(b.y, -b.x);
  } else {
    constexpr int k64 = K * (64 / M);
    constexpr float c = (float)cx_cos64(k64), s = (float)(-cx_sin64(k64));
#ifdef FS_X2
    return x2fma(make_float2(-s, s), x2swap(b), x2mul(make_float2(c, c), b));
#else
    return make_float2(fmaf(c, b.x, -s * b.y), fmaf(s, b.x, c * b.y));
#endif
  }
}

// Compile-time bookkeeping of the DIT stages: bit i of dit_nonzero(N, NZ, st) is set
// when working entry i may be nonzero after st stages, for inputs v[NZ..N) = 0
// (entry i starts as v[bitrev(i)]; a butterfly's outputs are nonzero when either
// input is).
constexpr unsigned dit_nonzero(int N, int NZ, int st) {
  const int LG = cx_log2(N);
  unsigned m = 0;
  for (int i = 0; i < N; i++)
    if (cx_bitrev(i, LG) < NZ) m |= 1u << i;
  for (int q = 0; q < st; q++) {
    const int h = 1 << q;
    unsigned r = 0;
    for (int i = 0; i < N; i++)
      if (((m >> i) & 1u) || ((m >> (i ^ h)) & 1u)) r |= 1u << i;
    m = r;
  }
  return m;
}

// In-place DFT of v[0..N) (N = 2..32), natural order in and out: the inputs are
// renamed into bit-reversed order at compile time, then log2 N DIT stages.
// NZ: the inputs v[NZ..N) are known to be zero (butterflies with a zero operand
// become copies or a single twiddle product).  NOUT: only X[0..NOUT) are needed
// (NOUT = N or N/2); with NOUT = N/2 the last stage forms the sums only.
template <int N, int NZ = N, int NOUT = N>
__host__ __device__ __forceinline__ void dft_inplace(float2 *v) {
  static_assert(NZ >= 1 && NZ <= N, "NZ leading inputs may be nonzero");
  static_assert(NOUT == N || 2 * NOUT == N, "output pruning keeps the lower half only");
  constexpr int LG = cx_log2(N);
  float2 u[N];
  sfor<0, N>([&](auto i) {
    if constexpr (cx_bitrev(i, LG) < NZ) u[i] = v[cx_bitrev(i, LG)];
  });
  sfor<0, LG>([&](auto st) {
    constexpr int h = 1 << st;
    constexpr unsigned m = dit_nonzero(N, NZ, st);
    sfor<0, N / (2 * h)>([&](auto g) {
      sfor<0, h>([&](auto k) {
        constexpr int i0 = g * 2 * h + k, i1 = i0 + h;
        constexpr bool z0 = !((m >> i0) & 1u), z1 = !((m >> i1) & 1u);
        constexpr bool last_pruned = (st == LG - 1) && (NOUT < N);
        if constexpr (z0 && z1) {
          // both zero
        } else if constexpr (z1) {
          if constexpr (!last_pruned) u[i1] = u[i0];
        } else if constexpr (z0) {
          const float2 t = twmul_dit<2 * h, k>(u[i1]);
          u[i0] = t;
          if constexpr (!last_pruned) u[i1] = make_float2(-t.x, -t.y);
        } else if constexpr (last_pruned) {
          const float2 t = twmul_dit<2 * h, k>(u[i1]);
#ifdef FS_X2
          u[i0] = x2add(u[i0], t);
#else
          u[i0] = cadd(u[i0], t);
#endif
        } else {
          bfly_dit<2 * h, k>(u[i0], u[i1]);
        }
      });
    });
  });
  sfor<0, NOUT>([&](auto i) { v[i] = u[i]; });
}

}  // namespace fs
