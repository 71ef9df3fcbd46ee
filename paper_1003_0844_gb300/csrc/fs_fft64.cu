// Stockham FFT in global memory: radix-16 passes (two radix-4 stages in
// registers), then one radix-4 and one radix-2 pass for the remaining factors,
// in FP64 (fft64: the plain all-FP64 form of the search, and the once-per-length
// plan of the upsampler) and in double-float arithmetic on the FP32 pipe (fftdf:
// the Bluestein transforms of the Fourier x2 upsampler on every segment load;
// ~1e-14 relative accuracy, and the FP64 pipe runs at 1/64 of the FP32 rate on
// this GPU).  Convention of Eq. (eq:DFT): X_k = sum_l x_l exp(-2 pi i l k / n),
// unnormalised; the inverse uses exp(+2 pi i l k / n), also unnormalised.
#include "fs_internal.h"
#include "fs_dfc.cuh"

namespace fs {

__global__ void k_twiddles64(double2 *tw, int64_t n) {
  int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q < n / 2) {
    double s, c;
    sincospi(2.0 * (double)q / (double)n, &s, &c);
    tw[q] = make_double2(c, -s);  // exp(-2 pi i q / n)
  }
}

// Stockham autosort stages (radix 2 and 4).  With p the product of the
// radices already applied, thread i < n/R reads u_q = x[i + q n/R], k = i mod p,
// multiplies u_q by W_{pR}^{q k}, takes the R-point DFT and writes
// y[(i - k) R + k + q p].  The twiddle table holds W_n^e for e < n/2.
__device__ inline double2 tw_get(const double2 *tw, int64_t e, int64_t half, int sign) {
  double2 w = (e < half) ? tw[e] : make_double2(-tw[e - half].x, -tw[e - half].y);
  if (sign > 0) w.y = -w.y;
  return w;
}

__global__ void k_stockham64_r2(const double2 *__restrict__ x, double2 *__restrict__ y,
                                const double2 *__restrict__ tw, int64_t n, int log2p, int sign, int batch) {
  const int64_t h = n >> 1;
  const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (gid >= h * batch) return;
  const int64_t b = gid / h, i = gid - b * h;
  const int64_t p = (int64_t)1 << log2p;
  const int64_t k = i & (p - 1);
  const double2 *xs = x + b * n;
  double2 *ys = y + b * n;
  const double2 u0 = xs[i];
  const double2 u1 = cmul(xs[i + h], tw_get(tw, k * (n >> (log2p + 1)), h, sign));
  const int64_t j = (i - k) * 2 + k;
  ys[j] = make_double2(u0.x + u1.x, u0.y + u1.y);
  ys[j + p] = make_double2(u0.x - u1.x, u0.y - u1.y);
}

__global__ void k_stockham64_r4(const double2 *__restrict__ x, double2 *__restrict__ y,
                                const double2 *__restrict__ tw, int64_t n, int log2p, int sign, int batch) {
  const int64_t q4 = n >> 2, h = n >> 1;
  const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (gid >= q4 * batch) return;
  const int64_t b = gid / q4, i = gid - b * q4;
  const int64_t p = (int64_t)1 << log2p;
  const int64_t k = i & (p - 1);
  const int64_t st = n >> (log2p + 2);
  const double2 *xs = x + b * n;
  double2 *ys = y + b * n;
  const double2 u0 = xs[i];
  const double2 u1 = cmul(xs[i + q4], tw_get(tw, k * st, h, sign));
  const double2 u2 = cmul(xs[i + 2 * q4], tw_get(tw, 2 * k * st, h, sign));
  const double2 u3 = cmul(xs[i + 3 * q4], tw_get(tw, 3 * k * st, h, sign));
  const double2 a0 = make_double2(u0.x + u2.x, u0.y + u2.y);
  const double2 a1 = make_double2(u0.x - u2.x, u0.y - u2.y);
  const double2 a2 = make_double2(u1.x + u3.x, u1.y + u3.y);
  const double2 d = make_double2(u1.x - u3.x, u1.y - u3.y);
  // forward: multiply by -i; inverse: by +i
  const double2 a3 = (sign < 0) ? make_double2(d.y, -d.x) : make_double2(-d.y, d.x);
  const int64_t j = (i - k) * 4 + k;
  ys[j] = make_double2(a0.x + a2.x, a0.y + a2.y);
  ys[j + p] = make_double2(a1.x + a3.x, a1.y + a3.y);
  ys[j + 2 * p] = make_double2(a0.x - a2.x, a0.y - a2.y);
  ys[j + 3 * p] = make_double2(a1.x - a3.x, a1.y - a3.y);
}

// Radix-4 butterfly on four values in place: v_c <- sum_q v_q W_4^{q c} (forward,
// sign < 0) or with W_4^{-q c} (inverse).
__device__ inline void bfly4(double2 &v0, double2 &v1, double2 &v2, double2 &v3, int sign) {
  const double2 a0 = make_double2(v0.x + v2.x, v0.y + v2.y);
  const double2 a1 = make_double2(v0.x - v2.x, v0.y - v2.y);
  const double2 a2 = make_double2(v1.x + v3.x, v1.y + v3.y);
  const double2 d = make_double2(v1.x - v3.x, v1.y - v3.y);
  const double2 a3 = (sign < 0) ? make_double2(d.y, -d.x) : make_double2(-d.y, d.x);
  v0 = make_double2(a0.x + a2.x, a0.y + a2.y);
  v1 = make_double2(a1.x + a3.x, a1.y + a3.y);
  v2 = make_double2(a0.x - a2.x, a0.y - a2.y);
  v3 = make_double2(a1.x - a3.x, a1.y - a3.y);
}

// exp(-2 pi i e / 16), e < 10 (the exponents b c of a radix-16 stage, b, c < 4)
__constant__ double2 kW16[10] = {
    {1.0, 0.0},
    {0.92387953251128675613, -0.38268343236508977173},
    {0.70710678118654752440, -0.70710678118654752440},
    {0.38268343236508977173, -0.92387953251128675613},
    {0.0, -1.0},
    {-0.38268343236508977173, -0.92387953251128675613},
    {-0.70710678118654752440, -0.70710678118654752440},
    {-0.92387953251128675613, -0.38268343236508977173},
    {-1.0, 0.0},
    {-0.92387953251128675613, 0.38268343236508977173}};

// Radix-16 Stockham stage (as the radix-4 one with R = 16): the 16-point DFT of
// the twiddled u_q, q = 4 a + b, is 4-point DFTs over a, the twiddles W_16^{b c}
// (c the first DFT's output), 4-point DFTs over b; output index c + 4 d.  (Four
// lanes per DFT with an exchange through shared memory measured no faster on a
// single transform and 9% slower on the batched transforms of the FP64 form.)
__global__ void __launch_bounds__(128) k_stockham64_r16(const double2 *__restrict__ x, double2 *__restrict__ y,
                                                        const double2 *__restrict__ tw, int64_t n, int log2p, int sign,
                                                        int batch) {
  const int64_t q16 = n >> 4, h = n >> 1;
  const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (gid >= q16 * batch) return;
  const int64_t b = gid / q16, i = gid - b * q16;
  const int64_t p = (int64_t)1 << log2p;
  const int64_t k = i & (p - 1);
  const int64_t st = n >> (log2p + 4);
  const double2 *xsrc = x + b * n;
  double2 *ydst = y + b * n;
  double2 u[16];
#pragma unroll
  for (int q = 0; q < 16; q++) {
    u[q] = xsrc[i + q * q16];
    if (q) u[q] = cmul(u[q], tw_get(tw, q * k * st, h, sign));
  }
#pragma unroll
  for (int bb = 0; bb < 4; bb++) {
    bfly4(u[bb], u[4 + bb], u[8 + bb], u[12 + bb], sign);  // over a: u[4 c + bb]
#pragma unroll
    for (int c = 1; c < 4; c++) {
      if (bb * c == 0) continue;
      double2 w = kW16[bb * c];  // W_16^{bb c}; the inverse conjugates
      if (sign > 0) w.y = -w.y;
      u[4 * c + bb] = cmul(u[4 * c + bb], w);
    }
  }
#pragma unroll
  for (int c = 0; c < 4; c++) bfly4(u[4 * c], u[4 * c + 1], u[4 * c + 2], u[4 * c + 3], sign);  // over b: u[4 c + d]
  const int64_t j = (i - k) * 16 + k;
#pragma unroll
  for (int c = 0; c < 4; c++)
#pragma unroll
    for (int d = 0; d < 4; d++) ydst[j + (c + 4 * d) * p] = u[4 * c + d];
}

// ------------------------------------------------------------------ double-float form
__global__ void k_to_df32(const double2 *in, float4 *out, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double2 v = in[i];  // read before the write: in and out may alias element by element
  const df32 r = df_from_double(v.x), m = df_from_double(v.y);
  out[i] = make_float4(r.hi, r.lo, m.hi, m.lo);
}

__device__ inline dfc twdf_get(const float4 *tw, int64_t e, int64_t half, int sign) {
  dfc w = (e < half) ? dfc_ld(tw[e]) : dfc_ld(tw[e - half]);
  if (e >= half) w = dfc{df_neg(w.re), df_neg(w.im)};
  if (sign > 0) w.im = df_neg(w.im);
  return w;
}

__global__ void k_stockham_df_r2(const float4 *__restrict__ x, float4 *__restrict__ y, const float4 *__restrict__ tw,
                                 int64_t n, int log2p, int sign, int batch) {
  const int64_t h = n >> 1;
  const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (gid >= h * batch) return;
  const int64_t b = gid / h, i = gid - b * h;
  const int64_t p = (int64_t)1 << log2p;
  const int64_t k = i & (p - 1);
  const float4 *xs = x + b * n;
  float4 *ys = y + b * n;
  const dfc u0 = dfc_ld(xs[i]);
  const dfc u1 = dfc_mul(dfc_ld(xs[i + h]), twdf_get(tw, k * (n >> (log2p + 1)), h, sign));
  const int64_t j = (i - k) * 2 + k;
  ys[j] = dfc_st(dfc_add(u0, u1));
  ys[j + p] = dfc_st(dfc_sub(u0, u1));
}

__device__ inline void bfly4_df(dfc &v0, dfc &v1, dfc &v2, dfc &v3, int sign) {
  const dfc a0 = dfc_add(v0, v2), a1 = dfc_sub(v0, v2), a2 = dfc_add(v1, v3);
  const dfc a3 = dfc_rot(dfc_sub(v1, v3), sign);
  v0 = dfc_add(a0, a2);
  v1 = dfc_add(a1, a3);
  v2 = dfc_sub(a0, a2);
  v3 = dfc_sub(a1, a3);
}

__global__ void k_stockham_df_r4(const float4 *__restrict__ x, float4 *__restrict__ y, const float4 *__restrict__ tw,
                                 int64_t n, int log2p, int sign, int batch) {
  const int64_t q4 = n >> 2, h = n >> 1;
  const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (gid >= q4 * batch) return;
  const int64_t b = gid / q4, i = gid - b * q4;
  const int64_t p = (int64_t)1 << log2p;
  const int64_t k = i & (p - 1);
  const int64_t st = n >> (log2p + 2);
  const float4 *xs = x + b * n;
  float4 *ys = y + b * n;
  dfc u0 = dfc_ld(xs[i]);
  dfc u1 = dfc_mul(dfc_ld(xs[i + q4]), twdf_get(tw, k * st, h, sign));
  dfc u2 = dfc_mul(dfc_ld(xs[i + 2 * q4]), twdf_get(tw, 2 * k * st, h, sign));
  dfc u3 = dfc_mul(dfc_ld(xs[i + 3 * q4]), twdf_get(tw, 3 * k * st, h, sign));
  bfly4_df(u0, u1, u2, u3, sign);
  const int64_t j = (i - k) * 4 + k;
  ys[j] = dfc_st(u0);
  ys[j + p] = dfc_st(u1);
  ys[j + 2 * p] = dfc_st(u2);
  ys[j + 3 * p] = dfc_st(u3);
}

// W_16^e (e < 10) as double-floats: the FP64 table's values split into hi + lo
#define FS_DF(v) (float)(v), (float)((v) - (double)(float)(v))
__constant__ float4 kW16df[10] = {
    {FS_DF(1.0), FS_DF(0.0)},
    {FS_DF(0.92387953251128675613), FS_DF(-0.38268343236508977173)},
    {FS_DF(0.70710678118654752440), FS_DF(-0.70710678118654752440)},
    {FS_DF(0.38268343236508977173), FS_DF(-0.92387953251128675613)},
    {FS_DF(0.0), FS_DF(-1.0)},
    {FS_DF(-0.38268343236508977173), FS_DF(-0.92387953251128675613)},
    {FS_DF(-0.70710678118654752440), FS_DF(-0.70710678118654752440)},
    {FS_DF(-0.92387953251128675613), FS_DF(-0.38268343236508977173)},
    {FS_DF(-1.0), FS_DF(0.0)},
    {FS_DF(-0.92387953251128675613), FS_DF(0.38268343236508977173)}};
#undef FS_DF

__global__ void __launch_bounds__(128) k_stockham_df_r16(const float4 *__restrict__ x, float4 *__restrict__ y,
                                                         const float4 *__restrict__ tw, int64_t n, int log2p, int sign,
                                                         int batch) {
  const int64_t q16 = n >> 4, h = n >> 1;
  const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (gid >= q16 * batch) return;
  const int64_t b = gid / q16, i = gid - b * q16;
  const int64_t p = (int64_t)1 << log2p;
  const int64_t k = i & (p - 1);
  const int64_t st = n >> (log2p + 4);
  const float4 *xsrc = x + b * n;
  float4 *ydst = y + b * n;
  dfc u[16];
#pragma unroll
  for (int q = 0; q < 16; q++) {
    u[q] = dfc_ld(xsrc[i + q * q16]);
    if (q) u[q] = dfc_mul(u[q], twdf_get(tw, q * k * st, h, sign));
  }
#pragma unroll
  for (int bb = 0; bb < 4; bb++) {
    bfly4_df(u[bb], u[4 + bb], u[8 + bb], u[12 + bb], sign);
#pragma unroll
    for (int c = 1; c < 4; c++) {
      if (bb * c == 0) continue;
      dfc w = dfc_ld(kW16df[bb * c]);
      if (sign > 0) w.im = df_neg(w.im);
      u[4 * c + bb] = dfc_mul(u[4 * c + bb], w);
    }
  }
#pragma unroll
  for (int c = 0; c < 4; c++) bfly4_df(u[4 * c], u[4 * c + 1], u[4 * c + 2], u[4 * c + 3], sign);
  const int64_t j = (i - k) * 16 + k;
#pragma unroll
  for (int c = 0; c < 4; c++)
#pragma unroll
    for (int d = 0; d < 4; d++) ydst[j + (c + 4 * d) * p] = dfc_st(u[4 * c + d]);
}

cudaError_t to_df32(const double2 *in, float4 *out, int64_t n, cudaStream_t st) {
  k_to_df32<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(in, out, n);
  return cudaGetLastError();
}

cudaError_t fftdf(float4 *buf, float4 *tmp, const float4 *twiddle, int64_t n, int batch, int sign, cudaStream_t st,
                  int64_t *launches) {
  int lg = 0;
  while (((int64_t)1 << lg) < n) lg++;
  float4 *src = buf, *dst = tmp;
  int log2p = 0;
  if (lg & 1) {
    const int64_t threads = (n / 2) * batch;
    k_stockham_df_r2<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(src, dst, twiddle, n, log2p, sign, batch);
    (*launches)++;
    float4 *sw = src; src = dst; dst = sw;
    log2p = 1;
  }
  if ((lg - log2p) % 4 == 2) {
    const int64_t threads4 = (n / 4) * batch;
    k_stockham_df_r4<<<(unsigned)((threads4 + 255) / 256), 256, 0, st>>>(src, dst, twiddle, n, log2p, sign, batch);
    (*launches)++;
    float4 *sw = src; src = dst; dst = sw;
    log2p += 2;
  }
  const int64_t threads16 = (n / 16) * batch;
  for (; log2p < lg; log2p += 4) {
    k_stockham_df_r16<<<(unsigned)((threads16 + 127) / 128), 128, 0, st>>>(src, dst, twiddle, n, log2p, sign, batch);
    (*launches)++;
    float4 *sw = src; src = dst; dst = sw;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (src != buf) e = cudaMemcpyAsync(buf, src, sizeof(float4) * n * batch, cudaMemcpyDeviceToDevice, st);
  return e;
}

cudaError_t fft64_twiddles(double2 *tw, int64_t n, cudaStream_t st) {
  int64_t h = n / 2;
  k_twiddles64<<<(unsigned)((h + 255) / 256), 256, 0, st>>>(tw, n);
  return cudaGetLastError();
}

cudaError_t fft64(double2 *buf, double2 *tmp, const double2 *twiddle, int64_t n, int batch, int sign,
                  cudaStream_t st, int64_t *launches) {
  int lg = 0;
  while (((int64_t)1 << lg) < n) lg++;
  double2 *src = buf, *dst = tmp;
  int log2p = 0;
  if (lg & 1) {
    const int64_t threads = (n / 2) * batch;
    k_stockham64_r2<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(src, dst, twiddle, n, log2p, sign, batch);
    (*launches)++;
    double2 *sw = src; src = dst; dst = sw;
    log2p = 1;
  }
  if ((lg - log2p) % 4 == 2) {
    const int64_t threads4 = (n / 4) * batch;
    k_stockham64_r4<<<(unsigned)((threads4 + 255) / 256), 256, 0, st>>>(src, dst, twiddle, n, log2p, sign, batch);
    (*launches)++;
    double2 *sw = src; src = dst; dst = sw;
    log2p += 2;
  }
  const int64_t threads16 = (n / 16) * batch;
  for (; log2p < lg; log2p += 4) {
    k_stockham64_r16<<<(unsigned)((threads16 + 127) / 128), 128, 0, st>>>(src, dst, twiddle, n, log2p, sign, batch);
    (*launches)++;
    double2 *sw = src; src = dst; dst = sw;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (src != buf) e = cudaMemcpyAsync(buf, src, sizeof(double2) * n * batch, cudaMemcpyDeviceToDevice, st);
  return e;
}

}  // namespace fs
