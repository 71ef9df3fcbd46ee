// The coarse search's F at continuous template points and its gradient (the
// adjoint of the search), for gradient-driven refinement of coarse candidates.
//
// For theta = (f0, f1, alpha, delta) and the barycentric output grid tau_j = j dt:
//   t_j, x~_j = x(t_j), a_j, b_j, phi_m(t_j), Q_j = t_j (t_j/2 + phi_m(t_j))  (Sec. VI.A,
//   Eq. eq:Bt: the resampling of the coarse search, resample_sample),
//   Psi_j = fl phi_m(t_j) + f1 Q_j + f0 tau_j                                 [cycles]
//   Sa = sum_j x~_j a_j exp(-2 pi i Psi_j), Sb likewise,
//   F = 2 dt / (S0 N) (|Sa|^2 / <a^2> + |Sb|^2 / <b^2>)                      (Eqs. ia, Fab, OS)
// At f0 = k / (Nfft dt) this is the search's F at bin k (the zero-padded DFT of
// Eq. eq:DFT), between bins the same sum off the Fourier grid.
//
// The gradient recomputes the resampled series sample by sample (nothing is stored
// between the forward and the backward call).  With tau_j fixed, t_j moves with the
// sky: dt_j/dsky = -(d phi_m/dsky) / (1 + d phi_m/dt) (Eq. eq:Bt differentiated), so
//   d x~_j = x~'(t_j) dt_j (the spline's slope),
//   da_j/dalpha = a_x (1 - Omega_r dt_j/dalpha), da_j/ddelta = a_delta - Omega_r a_x dt_j/ddelta,
//   dPsi_j/dsky = dt_j/dsky (f1 phi_m(t_j) - fl), dPsi_j/df0 = tau_j, dPsi_j/df1 = Q_j,
//   dSa = sum_j [d(x~ a)_j - 2 pi i x~_j a_j dPsi_j] exp(-2 pi i Psi_j),
//   dF = c [2 Re(conj(Sa) dSa) / <a^2> - |Sa|^2 d<a^2> / <a^2>^2 + (same for b)].
// Arithmetic as in the coarse search: FP32, with the phase terms as double-floats
// reduced to fractions of a cycle; per-thread FP32 sums over a block's samples,
// combined in FP64 across warps in a fixed order.
#include <algorithm>
#include "fs_internal.h"
#include "fs_model.cuh"
#include "fs_demod.cuh"
#include "fs_refine_df.cuh"

namespace fs {

constexpr int kAdjThreads = 256;
// Samples per thread per block: at most 192 (measured fastest for the gradient over
// 32..192 with 1024 points; the forward kernel, 3% faster at 64, keeps the same blocks
// so that both calls sum F in the same order), fewer when the points alone leave the
// GPU short of blocks, 8 at least; blocks of equal size (adj_block_range).
constexpr int kAdjSamplesMax = 192;
constexpr int kAdjSamplesMin = 8;

__device__ __forceinline__ void adj_block_range(int64_t n, int64_t *k0, int64_t *k1) {
  const int64_t per = ((n + gridDim.y - 1) / gridDim.y + kAdjThreads - 1) / kAdjThreads * kAdjThreads;
  *k0 = (int64_t)blockIdx.y * per;
  *k1 = min(n, *k0 + per);
}

// Per-point constants: the coarse search's sky constants, the sky derivatives of
// the delay's and of a, b's coefficients, and the phase coefficients.
struct ResPointConst {
  SkyConst32 k;
  float nx_a, nyp_a, nx_d, nyp_d, rcd_d, zsd_d;
  float ea_d[5], eb_d[4];
  df32 f0dt, f1;  // f0 dt (cycles per output sample), f1
  float f1f;
};

__global__ void k_res_constants(const fs_point *pts, int npt, SegGeom g, fs_detector det, ResPointConst *out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npt) return;
  const fs_point p = pts[i];
  SkyConst64 k;
  sky_constants(p.alpha, p.delta, det.eps, det.lat, det.gamma, g, &k);
  const PointConst pc = point_constants(p, g, det);
  ResPointConst c;
  c.k.nx = df_from_double(k.nx);  // the tables carry the factor AU/c
  c.k.nyp = df_from_double(k.nyp);
  c.k.nz = df_from_double(k.nz);
  c.k.ca = (float)k.ca;
  c.k.sa = (float)k.sa;
  c.k.rcd = (float)k.rcd;
  c.k.zsd = (float)k.zsd;
  for (int q = 0; q < 5; q++) {
    c.k.ea[q] = (float)k.ea[q];
    c.ea_d[q] = (float)pc.ea_d[q];
  }
  for (int q = 0; q < 4; q++) {
    c.k.eb[q] = (float)k.eb[q];
    c.eb_d[q] = (float)pc.eb_d[q];
  }
  c.nx_a = (float)pc.nx_a;
  c.nyp_a = (float)pc.nyp_a;
  c.nx_d = (float)pc.nx_d;
  c.nyp_d = (float)pc.nyp_d;
  c.rcd_d = (float)pc.rcd_d;
  c.zsd_d = (float)pc.zsd_d;
  c.f0dt = df_from_double(p.f0 * g.dt);
  c.f1 = df_from_double(p.f1);
  c.f1f = (float)p.f1;
  out[i] = c;
}

// Sums per point (NQ = 6 for F, 26 with the gradient):
//  [0, 4) Sa, Sb (re, im); [4, 6) sum a^2, b^2;
//  [6, 14) dSa/dtheta_i (re, im), i = f0, f1, alpha, delta; [14, 22) the same for Sb;
//  [22, 26) sum a da/dalpha, a da/ddelta, b db/dalpha, b db/ddelta.
template <bool GRAD>
__global__ void __launch_bounds__(kAdjThreads) k_resampled(DemodArgs A, const ResPointConst *pcs, double *partial) {
  constexpr int NQ = GRAD ? 26 : 6;
  __shared__ ResPointConst c;
  __shared__ double red[kAdjThreads / 32][NQ];
  const int pt = blockIdx.x;
  if (threadIdx.x == 0) c = pcs[pt];
  __syncthreads();
  float acc[NQ];
#pragma unroll
  for (int q = 0; q < NQ; q++) acc[q] = 0.f;
  int64_t k0, k1;
  adj_block_range(A.g.n, &k0, &k1);
  // two samples in flight for the gradient (2.5% faster); the forward kernel is faster
  // with one (24% slower at two: its loads already overlap across warps)
  constexpr int UNROLL = GRAD ? 2 : 1;
#pragma unroll UNROLL
  for (int64_t j = k0 + threadIdx.x; j < k1; j += kAdjThreads) {
    const ResampledSample r = resample_sample<FS_INTERP_SPLINE2X, false>(A, c.k, j);
    // exp(-2 pi i Psi_j): each term reduced to a fraction of a cycle (j < 2^24 is exact)
    float f = df_mul_frac(A.fl, r.phim) + df_mul_frac(c.f1, r.Q) + df_mul_frac(c.f0dt, df32{(float)j, 0.f});
    f -= rintf(f);
    const float2 e = expm2pi(f);
    const float ua = r.xr * r.av, ub = r.xr * r.bv;
    acc[0] = fmaf(ua, e.x, acc[0]);
    acc[1] = fmaf(ua, e.y, acc[1]);
    acc[2] = fmaf(ub, e.x, acc[2]);
    acc[3] = fmaf(ub, e.y, acc[3]);
    acc[4] = fmaf(r.av, r.av, acc[4]);
    acc[5] = fmaf(r.bv, r.bv, acc[5]);
    if constexpr (GRAD) {
      // the spline's slope d x~/dt (zero outside the data: spl_c is zero there)
      const float sf = r.spl_f;
      const float xp = fmaf(sf, fmaf(3.f * sf, r.spl_c.w, 2.f * r.spl_c.z), r.spl_c.y) * A.two_over_dt;
      // sky derivatives of the delay at t_j with t fixed, then of t_j itself
      const float phi_a = fmaf(c.nx_a, r.U0.x, c.nyp_a * r.U0.z) - c.k.rcd * r.sx;
      const float phi_d = fmaf(c.nx_d, r.U0.x, fmaf(c.nyp_d, r.U0.z, fmaf(c.rcd_d, r.cx, c.zsd_d)));
      const float den = 1.f / (1.f + r.phidot);
      const float t_a = -phi_a * den, t_d = -phi_d * den;
      // a, b: through x = alpha - theta(t_j) and the delta dependence of the coefficients
      const float cx = r.cx, sx = r.sx;
      const float c2 = fmaf(cx, cx, -sx * sx), s2 = 2.f * sx * cx;
      const float a_x = 2.f * (c.k.ea[1] * c2 - c.k.ea[0] * s2) - c.k.ea[2] * sx + c.k.ea[3] * cx;
      const float b_x = 2.f * (c.k.eb[1] * c2 - c.k.eb[0] * s2) - c.k.eb[2] * sx + c.k.eb[3] * cx;
      const float a_dl = c.ea_d[0] * c2 + c.ea_d[1] * s2 + c.ea_d[2] * cx + c.ea_d[3] * sx + c.ea_d[4];
      const float b_dl = c.eb_d[0] * c2 + c.eb_d[1] * s2 + c.eb_d[2] * cx + c.eb_d[3] * sx;
      const float wr = (float)kOmegaR;
      const float a_a = a_x * (1.f - wr * t_a), a_d = a_dl - wr * a_x * t_d;
      const float b_a = b_x * (1.f - wr * t_a), b_d = b_dl - wr * b_x * t_d;
      // phase derivatives [cycles per unit]
      const float gsky = fmaf(c.f1f, r.phim.hi, -A.fl.hi);  // f1 phi_m - fl
      const float dpsi[4] = {(float)j * A.dt, r.Q.hi, t_a * gsky, t_d * gsky};
      const float rea[4] = {0.f, 0.f, fmaf(xp * t_a, r.av, r.xr * a_a), fmaf(xp * t_d, r.av, r.xr * a_d)};
      const float reb[4] = {0.f, 0.f, fmaf(xp * t_a, r.bv, r.xr * b_a), fmaf(xp * t_d, r.bv, r.xr * b_d)};
      constexpr float m2pi = -6.283185307179586f;
#pragma unroll
      for (int i = 0; i < 4; i++) {
        // (re - 2 pi i u dPsi_i) (e.x + i e.y)
        const float ima = m2pi * ua * dpsi[i], imb = m2pi * ub * dpsi[i];
        acc[6 + 2 * i] += fmaf(rea[i], e.x, -ima * e.y);
        acc[7 + 2 * i] += fmaf(rea[i], e.y, ima * e.x);
        acc[14 + 2 * i] += fmaf(reb[i], e.x, -imb * e.y);
        acc[15 + 2 * i] += fmaf(reb[i], e.y, imb * e.x);
      }
      acc[22] = fmaf(r.av, a_a, acc[22]);
      acc[23] = fmaf(r.av, a_d, acc[23]);
      acc[24] = fmaf(r.bv, b_a, acc[24]);
      acc[25] = fmaf(r.bv, b_d, acc[25]);
    }
  }
  // the block's sums: a pairwise FP32 tree within each warp (5 roundings), then the
  // warps in FP64 in a fixed order (an FP64 tree here kept the 1/64-rate FP64 pipe 60%
  // busy)
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NQ; q++) {
    float v = acc[q];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) red[wp][q] = (double)v;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < NQ; q += kAdjThreads) {
    double v = 0.0;
    for (int w2 = 0; w2 < kAdjThreads / 32; w2++) v += red[w2][q];
    partial[((int64_t)pt * gridDim.y + blockIdx.y) * NQ + q] = v;
  }
}

// F and (GRAD) gF_i dF_i/dtheta per point from the blocks' sums, in block order.
template <bool GRAD>
__global__ void k_resampled_final(const double *partial, int nblk, int npt, int64_t n, double dt, double S0,
                                  const double *gF, double *F, double *grad) {
  constexpr int NQ = GRAD ? 26 : 6;
  const int pt = blockIdx.x * blockDim.x + threadIdx.x;
  if (pt >= npt) return;
  double s[NQ];
  for (int q = 0; q < NQ; q++) s[q] = 0.0;
  for (int b = 0; b < nblk; b++)
    for (int q = 0; q < NQ; q++) s[q] += partial[((int64_t)pt * nblk + b) * NQ + q];
  const double cF = 2.0 * dt / (S0 * (double)n);
  const double A2 = s[4] / (double)n, B2 = s[5] / (double)n;
  const double Pa = s[0] * s[0] + s[1] * s[1], Pb = s[2] * s[2] + s[3] * s[3];
  if (F) F[pt] = cF * (Pa / A2 + Pb / B2);
  if constexpr (GRAD) {
    const double g = gF ? gF[pt] : 1.0;
    for (int i = 0; i < 4; i++) {
      const double ta = 2.0 * (s[0] * s[6 + 2 * i] + s[1] * s[7 + 2 * i]) / A2;
      const double tb = 2.0 * (s[2] * s[14 + 2 * i] + s[3] * s[15 + 2 * i]) / B2;
      const double dA2 = i >= 2 ? 2.0 * s[20 + i] / (double)n : 0.0;
      const double dB2 = i >= 2 ? 2.0 * s[22 + i] / (double)n : 0.0;
      grad[4 * pt + i] = g * cF * (ta - Pa * dA2 / (A2 * A2) + tb - Pb * dB2 / (B2 * B2));
    }
  }
}

fs_status fstat_resampled(fs_ctx *ctx, fs_seg *seg, const fs_point *pts, int npt, const double *gF, double *F,
                          double *grad, cudaStream_t st) {
  if (seg->d.precision != FS_PREC_F32 || seg->d.interp != FS_INTERP_SPLINE2X || seg->eph) return FS_ERR_UNSUPPORTED;
  ProfScope ps(ctx, PROF_OTHER, st);
  const bool g = grad != nullptr;
  const int NQ = g ? 26 : 6;
  int nsm = 0;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device) != cudaSuccess) return FS_ERR_CUDA;
  const int64_t n = seg->g.n;
  const int64_t lo = (n + (int64_t)kAdjThreads * kAdjSamplesMax - 1) / ((int64_t)kAdjThreads * kAdjSamplesMax);
  const int64_t hi = (n + (int64_t)kAdjThreads * kAdjSamplesMin - 1) / ((int64_t)kAdjThreads * kAdjSamplesMin);
  const int64_t want = (4 * (int64_t)nsm + npt - 1) / npt;  // blocks per point for ~2 waves
  const int nblk = (int)std::min(hi, std::max(lo, want));  // <= 65535 for n <= 2^27
  const size_t o_pa = (sizeof(ResPointConst) * (size_t)npt + 255) & ~(size_t)255;
  fs_status s = ensure_buffer(&ctx->aws, &ctx->aws_bytes, o_pa + sizeof(double) * NQ * (size_t)nblk * npt, st);
  if (s != FS_OK) return s;
  ResPointConst *pc = (ResPointConst *)ctx->aws;
  double *partial = (double *)((char *)ctx->aws + o_pa);
  DemodArgs A{};
  A.g = seg->g;
  A.dt2 = df_from_double(seg->g.dt);
  A.dt = (float)seg->g.dt;
  A.inv_dt = (float)(1.0 / seg->g.dt);
  A.two_over_dt = (float)(2.0 / seg->g.dt);
  A.fl = df_from_double(seg->g.fl);
  A.tab0 = seg->tab0;
  A.tab1 = seg->tab1;
  A.coef = (const float4 *)seg->coef;
  k_res_constants<<<(unsigned)((npt + 127) / 128), 128, 0, st>>>(pts, npt, seg->g, ctx->det, pc);
  const dim3 grid((unsigned)npt, (unsigned)nblk);
  if (g) {
    k_resampled<true><<<grid, kAdjThreads, 0, st>>>(A, pc, partial);
    k_resampled_final<true><<<(unsigned)((npt + 127) / 128), 128, 0, st>>>(partial, nblk, npt, seg->g.n, seg->g.dt,
                                                                          seg->g.S0, gF, F, grad);
  } else {
    k_resampled<false><<<grid, kAdjThreads, 0, st>>>(A, pc, partial);
    k_resampled_final<false><<<(unsigned)((npt + 127) / 128), 128, 0, st>>>(partial, nblk, npt, seg->g.n, seg->g.dt,
                                                                           seg->g.S0, gF, F, grad);
  }
  ctx->launches += 3;
  return cuda_status(cudaGetLastError());
}

}  // namespace fs
