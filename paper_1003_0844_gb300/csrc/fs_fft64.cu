// FP64 Stockham FFT (radix 4, one radix-2 stage for odd log2 n) in global memory.
//
// Used where FP64 is wanted and the transform is off the per-template hot
// path: the Bluestein transforms of the Fourier x2 upsampler (once per
// segment) and the plain all-FP64 form of the search.  Convention of
// Eq. (eq:DFT): X_k = sum_l x_l exp(-2 pi i l k / n), unnormalised; the
// inverse uses exp(+2 pi i l k / n), also unnormalised.
#include "fs_internal.h"

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
  const int64_t threads4 = (n / 4) * batch;
  for (; log2p < lg; log2p += 2) {
    k_stockham64_r4<<<(unsigned)((threads4 + 255) / 256), 256, 0, st>>>(src, dst, twiddle, n, log2p, sign, batch);
    (*launches)++;
    double2 *sw = src; src = dst; dst = sw;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (src != buf) e = cudaMemcpyAsync(buf, src, sizeof(double2) * n * batch, cudaMemcpyDeviceToDevice, st);
  return e;
}

}  // namespace fs
