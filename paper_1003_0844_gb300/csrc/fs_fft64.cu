// FP64 radix-2 Stockham FFT in global memory.
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

// One Stockham autosort stage: l = n / 2^(t+1), m = 2^t.
//   y[k + 2 j m]     = x[k + j m] + x[k + j m + l m]
//   y[k + 2 j m + m] = W_{2l}^j (x[k + j m] - x[k + j m + l m]),  W_{2l}^j = tw[j m]
__global__ void k_stockham64(const double2 *__restrict__ x, double2 *__restrict__ y,
                             const double2 *__restrict__ tw, int64_t n, int log2m, int sign, int batch) {
  int64_t half = n >> 1;
  int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (gid >= half * batch) return;
  int64_t b = gid / half;
  int64_t idx = gid - b * half;
  int64_t m = (int64_t)1 << log2m;
  int64_t j = idx >> log2m;
  int64_t k = idx & (m - 1);
  const double2 *xs = x + b * n;
  double2 *ys = y + b * n;
  double2 c0 = xs[k + j * m];
  double2 c1 = xs[k + j * m + half];
  double2 w = tw[j * m];
  if (sign > 0) w.y = -w.y;
  double2 s = make_double2(c0.x + c1.x, c0.y + c1.y);
  double2 d = make_double2(c0.x - c1.x, c0.y - c1.y);
  ys[k + 2 * j * m] = s;
  ys[k + 2 * j * m + m] = cmul(w, d);
}

cudaError_t fft64_twiddles(double2 *tw, int64_t n, cudaStream_t st) {
  int64_t h = n / 2;
  k_twiddles64<<<(unsigned)((h + 255) / 256), 256, 0, st>>>(tw, n);
  return cudaGetLastError();
}

cudaError_t fft64(double2 *buf, double2 *tmp, const double2 *twiddle, int64_t n, int batch, int sign,
                  cudaStream_t st, int64_t *launches) {
  int p = 0;
  while (((int64_t)1 << p) < n) p++;
  double2 *src = buf, *dst = tmp;
  int64_t threads = (n / 2) * batch;
  unsigned blocks = (unsigned)((threads + 255) / 256);
  for (int t = 0; t < p; t++) {
    k_stockham64<<<blocks, 256, 0, st>>>(src, dst, twiddle, n, t, sign, batch);
    (*launches)++;
    double2 *sw = src; src = dst; dst = sw;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (src != buf) e = cudaMemcpyAsync(buf, src, sizeof(double2) * n * batch, cudaMemcpyDeviceToDevice, st);
  return e;
}

}  // namespace fs
