// Plain FP64 form of the search: every step in double, the analytic model (or
// the caller's position table) evaluated directly at each source time, the spline in double, and the
// zero-padded transform by the FP64 radix-2 Stockham FFT.  It is the
// all-FP64 comparison for the FP32 path on the same GPU.
#include "fs_internal.h"
#include "fs_model.cuh"

namespace fs {

constexpr unsigned kFull64 = 0xffffffffu;

// eph: NULL (analytic Earth) or the caller's position table of the segment.
__global__ void __launch_bounds__(256) k_demod64(SegGeom g, const SkyConst64 *sky, const dcoef4 *coef,
                                                 const double *x64, int interp, double2 *ya, double2 *yb,
                                                 double *qq, int64_t stride, double *partial, double *tsrc,
                                                 const dbl4 *eph) {
  const int s = blockIdx.y;
  const SkyConst64 K = sky[s];
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double a2 = 0.0, b2 = 0.0;
  if (j < g.n) {
    Geo64 geo;
    const double t = source_time64((double)j * g.dt, K, g, &geo, eph);
    double xr = 0.0;
    if (interp == FS_INTERP_SPLINE2X) {
      if (t >= 0.0 && t <= (double)(g.n - 1) * g.dt) {
        const double u = 2.0 * t / g.dt;
        int64_t i = (int64_t)floor(u);
        if (i > 2 * g.n - 2) i = 2 * g.n - 2;
        const double f = u - (double)i;
        const dcoef4 c = coef[i];
        xr = fma(f, fma(f, fma(f, c.w, c.z), c.y), c.x);
      }
    } else {
      const int64_t kk = (int64_t)rint(t / g.dt);
      if (kk >= 0 && kk < g.n) xr = x64[kk];
    }
    double av, bv;
    ab_eval64(K, geo.cx, geo.sx, &av, &bv);
    a2 = av * av;
    b2 = bv * bv;
    double cyc = g.fl * geo.phi;
    cyc -= floor(cyc);
    double sp, cp;
    sincospi(2.0 * cyc, &sp, &cp);
    ya[s * stride + j] = make_double2(xr * av * cp, -xr * av * sp);
    yb[s * stride + j] = make_double2(xr * bv * cp, -xr * bv * sp);
    qq[s * stride + j] = t * (0.5 * t + geo.phi);
    if (tsrc && s == 0) tsrc[j] = t;
  }
  for (int o = 16; o > 0; o >>= 1) {
    a2 += __shfl_down_sync(kFull64, a2, o);
    b2 += __shfl_down_sync(kFull64, b2, o);
  }
  __shared__ double wa[8], wb[8];
  if ((threadIdx.x & 31) == 0) { wa[threadIdx.x >> 5] = a2; wb[threadIdx.x >> 5] = b2; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sa = 0.0, sb = 0.0;
    for (int w = 0; w < 8; w++) { sa += wa[w]; sb += wb[w]; }
    double *p = partial + ((int64_t)s * gridDim.x + blockIdx.x) * 2;
    p[0] = sa;
    p[1] = sb;
  }
}

__global__ void k_finalize64(const double *partial, int nb, int64_t n, double dt, double S0, double2 *norm,
                             double2 *ab2) {
  const int s = blockIdx.x;
  double sa = 0.0, sb = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) {
    sa += partial[((int64_t)s * nb + i) * 2];
    sb += partial[((int64_t)s * nb + i) * 2 + 1];
  }
  __shared__ double ra[256], rb[256];
  ra[threadIdx.x] = sa;
  rb[threadIdx.x] = sb;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) { ra[threadIdx.x] += ra[threadIdx.x + o]; rb[threadIdx.x] += rb[threadIdx.x + o]; }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double ma = ra[0] / (double)n, mb = rb[0] / (double)n;
    double cF = 2.0 * dt / (S0 * (double)n);
    if (norm) norm[s] = make_double2(cF / ma, cF / mb);
    if (ab2) ab2[s] = make_double2(ma, mb);
  }
}

// buf[(m*2 + sig)][k] = y^sig_k exp(-2 pi i f1_m Q_k) for k < n, 0 up to nfft; with
// lattice templates (offset non-NULL) also exp(-2 pi i d_m k / nfft), which moves bin
// j of the transform to the frequency (j + d_m) / (nfft dt)
__global__ void k_modulate64(const double2 *ya, const double2 *yb, const double *qq, const double *f1,
                             const double *offset, int nspin, int64_t n, int64_t nfft, double2 *buf) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int m = blockIdx.y;
  if (k >= nfft || m >= nspin) return;
  double2 va = make_double2(0.0, 0.0), vb = va;
  if (k < n) {
    double cyc = f1[m] * qq[k];
    cyc -= floor(cyc);
    if (offset) {
      cyc += offset[m] * ((double)k / (double)nfft);
      cyc -= floor(cyc);
    }
    double sp, cp;
    sincospi(2.0 * cyc, &sp, &cp);
    const double2 c = make_double2(cp, -sp);
    va = cmul(ya[k], c);
    vb = cmul(yb[k], c);
  }
  buf[(2 * (int64_t)m) * nfft + k] = va;
  buf[(2 * (int64_t)m + 1) * nfft + k] = vb;
}

// F on bin k < nbins; with interbinning (ib) on the half-bin grid: output j
// takes X(j/2) for even j and (X(j/2+1) - X(j/2))/sqrt(2) for odd j (Eq. intbin).
__global__ void k_fstat64(const double2 *buf, int nspin, int64_t nfft, int64_t nbins, const double2 *nrmp, double *F,
                          int sky, float thr, fs_candidate *cand, int64_t cap, unsigned long long *ncand,
                          uint32_t *flags, int ib) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int m = blockIdx.y;
  const int lane = threadIdx.x & 31;
  double Fv = 0.0;
  const bool ok = (k < nbins);
  const double2 nrm = *nrmp;
  if (ok) {
    const double2 *ba = buf + (2 * (int64_t)m) * nfft, *bb = ba + nfft;
    const int64_t q = ib ? (k >> 1) : k;
    double2 xa = ba[q], xb = bb[q];
    if (ib && (k & 1)) {
      const double2 ya = ba[q + 1], yb = bb[q + 1];
      xa = make_double2((ya.x - xa.x) * 0.70710678118654752440, (ya.y - xa.y) * 0.70710678118654752440);
      xb = make_double2((yb.x - xb.x) * 0.70710678118654752440, (yb.y - xb.y) * 0.70710678118654752440);
    }
    Fv = (xa.x * xa.x + xa.y * xa.y) * nrm.x + (xb.x * xb.x + xb.y * xb.y) * nrm.y;
    if (F) F[(int64_t)m * nbins + k] = Fv;
  }
  const bool hit = ok && Fv > (double)thr;
  const unsigned msk = __ballot_sync(kFull64, hit);
  if (msk) {
    const int leader = __ffs(msk) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(ncand, (unsigned long long)__popc(msk));
    base = __shfl_sync(kFull64, base, leader);
    if (hit) {
      const unsigned long long idx = base + __popc(msk & ((1u << lane) - 1u));
      if ((long long)idx < cap) {
        fs_candidate c;
        c.sky = (uint32_t)sky;
        c.spin = (uint32_t)m;
        c.bin = (uint32_t)k;
        c.F = (float)Fv;
        cand[idx] = c;
      } else {
        atomicOr(flags, ERRF_CAPACITY);
      }
    }
  }
}

struct Ws64 {
  SkyConst64 *skyc;
  double2 *ya, *yb, *norm, *ab2, *buf, *tmp, *tw;
  double *qq, *partial;
  int nblk;
};

static size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

static fs_status workspace64(fs_ctx *ctx, const fs_seg *seg, int nspin, cudaStream_t st, Ws64 *w) {
  const int64_t n = seg->g.n, nfft = seg->g.nfft;
  const int nblk = (int)((n + 255) / 256);
  size_t off = 0;
  size_t o_sky = off; off = al256(off + sizeof(SkyConst64));
  size_t o_ya = off; off = al256(off + sizeof(double2) * n);
  size_t o_yb = off; off = al256(off + sizeof(double2) * n);
  size_t o_qq = off; off = al256(off + sizeof(double) * n);
  size_t o_nm = off; off = al256(off + sizeof(double2));
  size_t o_ab = off; off = al256(off + sizeof(double2));
  size_t o_pa = off; off = al256(off + sizeof(double) * 2 * nblk);
  size_t o_bf = off; off = al256(off + sizeof(double2) * 2 * (size_t)nspin * nfft);
  size_t o_tm = off; off = al256(off + sizeof(double2) * 2 * (size_t)nspin * nfft);
  size_t o_tw = off; off = al256(off + sizeof(double2) * (size_t)(nfft / 2));
  fs_status s = ensure_buffer(&ctx->ws64, &ctx->ws64_bytes, off, st);
  if (s != FS_OK) return s;
  char *b = (char *)ctx->ws64;
  w->skyc = (SkyConst64 *)(b + o_sky);
  w->ya = (double2 *)(b + o_ya);
  w->yb = (double2 *)(b + o_yb);
  w->qq = (double *)(b + o_qq);
  w->norm = (double2 *)(b + o_nm);
  w->ab2 = (double2 *)(b + o_ab);
  w->partial = (double *)(b + o_pa);
  w->buf = (double2 *)(b + o_bf);
  w->tmp = (double2 *)(b + o_tm);
  w->tw = (double2 *)(b + o_tw);
  w->nblk = nblk;
  return FS_OK;
}

// offset non-NULL: lattice templates, f1 and offset [nsky][nspin] (row sk for sky sk)
fs_status search64(fs_ctx *ctx, fs_seg *seg, const double *alpha, const double *delta, int nsky,
                   const double *f1, int nspin, float thr, double *F, int64_t nbins, fs_candidate *cand,
                   int64_t cap, int64_t *ncand, cudaStream_t st, const double *offset) {
  const int64_t n = seg->g.n, nfft = seg->g.nfft;
  Ws64 w;
  fs_status s = workspace64(ctx, seg, nspin, st, &w);
  if (s != FS_OK) return s;
  if (cudaMemsetAsync(ncand, 0, sizeof(int64_t), st) != cudaSuccess) return FS_ERR_CUDA;
  if (fft64_twiddles(w.tw, nfft, st) != cudaSuccess) return FS_ERR_CUDA;
  ctx->launches += 1;
  for (int sk = 0; sk < nsky; sk++) {
    if (sky_constants64(alpha + sk, delta + sk, 1, seg->g, ctx->det, w.skyc, st) != cudaSuccess) return FS_ERR_CUDA;
    k_demod64<<<dim3(w.nblk, 1), 256, 0, st>>>(seg->g, w.skyc, (const dcoef4 *)seg->coef, seg->x64,
                                                seg->d.interp, w.ya, w.yb, w.qq, 0, w.partial, nullptr,
                                                seg->eph);
    k_finalize64<<<1, 256, 0, st>>>(w.partial, w.nblk, n, seg->g.dt, seg->g.S0, w.norm, w.ab2);
    ctx->launches += 5;  // sky constants, demodulation, finalize, modulation, F epilogue
    const double *f1s = offset ? f1 + (int64_t)sk * nspin : f1;
    const double *ds = offset ? offset + (int64_t)sk * nspin : nullptr;
    k_modulate64<<<dim3((unsigned)((nfft + 255) / 256), nspin), 256, 0, st>>>(w.ya, w.yb, w.qq, f1s, ds, nspin, n,
                                                                              nfft, w.buf);
    if (fft64(w.buf, w.tmp, w.tw, nfft, 2 * nspin, -1, st, &ctx->launches) != cudaSuccess) return FS_ERR_CUDA;
    k_fstat64<<<dim3((unsigned)((nbins + 255) / 256), nspin), 256, 0, st>>>(
        w.buf, nspin, nfft, nbins, w.norm, F ? F + (int64_t)sk * nspin * nbins : nullptr, sk, thr, cand, cap,
        (unsigned long long *)ncand, ctx->d_flags, (seg->d.options & FS_OPT_INTERBIN) ? 1 : 0);
  }
  return cuda_status(cudaGetLastError());
}

__global__ void k_copy_pairs(const double2 *y, double *o, int64_t n) {
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j < n) { o[2 * j] = y[j].x; o[2 * j + 1] = y[j].y; }
}

fs_status demod64_debug(fs_ctx *ctx, fs_seg *seg, double alpha, double delta, double *ya, double *yb,
                        double *tsrc, double *ab2, cudaStream_t st) {
  const int64_t n = seg->g.n;
  Ws64 w;
  fs_status s = workspace64(ctx, seg, 1, st, &w);
  if (s != FS_OK) return s;
  double hd[2] = {alpha, delta};
  double *dd = (double *)w.ab2;
  if (cudaMemcpyAsync(dd, hd, sizeof(hd), cudaMemcpyHostToDevice, st) != cudaSuccess) return FS_ERR_CUDA;
  if (sky_constants64(dd, dd + 1, 1, seg->g, ctx->det, w.skyc, st) != cudaSuccess) return FS_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return FS_ERR_CUDA;
  k_demod64<<<dim3(w.nblk, 1), 256, 0, st>>>(seg->g, w.skyc, (const dcoef4 *)seg->coef, seg->x64,
                                              seg->d.interp, w.ya, w.yb, w.qq, 0, w.partial, tsrc,
                                              seg->eph);
  k_finalize64<<<1, 256, 0, st>>>(w.partial, w.nblk, n, seg->g.dt, seg->g.S0, nullptr, (double2 *)ab2);
  k_copy_pairs<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(w.ya, ya, n);
  k_copy_pairs<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(w.yb, yb, n);
  return cuda_status(cudaGetLastError());
}

}  // namespace fs
