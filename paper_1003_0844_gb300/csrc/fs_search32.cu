// FP32 search path with compensated (double-float) phases.
//
// Per sky (A1, k_demod32): source times t_j of Eq. (eq:Bt) by one Newton
// step from a first delay estimate, the spline value x~_j (Sec. VI.A),
// a_j, b_j (Sec. II), the heterodyne factor exp(-2 pi i fl phi_m(t_j)) and
// the spindown phase argument Q_j = t_j^2/2 + t_j phi_m(t_j) (Eq. phas) kept
// as a double-float.  Output per sky: y^a_j, y^b_j (float2) and Q_j.
//
// Per template (sky, f1), the zero-padded transform of length
// Nfft = N1 * N2 runs in two passes (index n = N2 n1 + n2, bin k = k1 + N1 k2):
//  pass 1 (k_pass1): multiply by the chirp exp(-2 pi i f1 Q_j), DFTs of
//    length N1 over n1 for a tile of 16 columns n2 (both signals a and b),
//    twiddle exp(-2 pi i n2 k1 / Nfft), write Z[k1][n2];
//  pass 2 (k_pass2): DFTs of length N2 over n2 for 16 or 32 rows k1, then
//    F_k = 2/(S0 To) (|Fa_k|^2/<a^2> + |Fb_k|^2/<b^2>) (Eq. OS), threshold
//    compaction, and a transposed store of F in natural bin order.
// Each length-L DFT (L = P Q) is itself two register stages (DFT_P over the
// stride-Q samples, twiddle exp(-2 pi i b c / L), DFT_Q) with one exchange
// through shared memory.
#include <stdio.h>
#include <mutex>
#include "fs_internal.h"
#include "fs_model.cuh"
#include "fs_dft.cuh"

namespace fs {

constexpr unsigned kFull = 0xffffffffu;

// ------------------------------------------------------------------ per-sky constants
__global__ void k_skyconst(const double *alpha, const double *delta, int nsky, SegGeom g, double eps,
                           double lat, double gamma, SkyConst32 *out32, SkyConst64 *out64) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nsky) return;
  SkyConst64 k;
  sky_constants(alpha[s], delta[s], eps, lat, gamma, g, &k);
  if (out64) out64[s] = k;
  if (out32) {
    SkyConst32 c;
    c.nx = df_from_double(k.nx);  // the tables carry the factor AU/c
    c.nyp = df_from_double(k.nyp);
    c.ca = (float)k.ca;
    c.sa = (float)k.sa;
    c.rcd = (float)k.rcd;
    c.zsd = (float)k.zsd;
    for (int i = 0; i < 5; i++) c.ea[i] = (float)k.ea[i];
    for (int i = 0; i < 4; i++) c.eb[i] = (float)k.eb[i];
    out32[s] = c;
  }
}

cudaError_t sky_constants32(const double *alpha, const double *delta, int nsky, const SegGeom &g,
                            const fs_detector &det, SkyConst32 *out, cudaStream_t st) {
  k_skyconst<<<(nsky + 127) / 128, 128, 0, st>>>(alpha, delta, nsky, g, det.eps, det.lat, det.gamma, out,
                                                  nullptr);
  return cudaGetLastError();
}
cudaError_t sky_constants64(const double *alpha, const double *delta, int nsky, const SegGeom &g,
                            const fs_detector &det, SkyConst64 *out, cudaStream_t st) {
  k_skyconst<<<(nsky + 127) / 128, 128, 0, st>>>(alpha, delta, nsky, g, det.eps, det.lat, det.gamma,
                                                  nullptr, out);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ A1: resample + demodulate one sky
struct DemodArgs {
  SegGeom g;
  df32 dt2;            // dt as double-float
  float dt, inv_dt, two_over_dt;
  df32 fl;
  const SkyConst32 *sky;
  const float4 *tab0, *tab1;  // indexed by m + margin
  const float4 *coef;         // spline intervals [2n]
  const float *x32;           // data, nearest-neighbour path
  float2 *ya, *yb, *qq;       // [nsky][stride]
  int64_t stride, npad;
  double *partial;            // [nsky][gridDim.x][2]
  double *tsrc;               // optional [n] (first sky only)
};

template <int INTERP>
__global__ void __launch_bounds__(256) k_demod32(DemodArgs A) {
  const int s = blockIdx.y;
  const SkyConst32 K = A.sky[s];
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  float a2 = 0.f, b2 = 0.f;
  if (j < A.npad) {
    float2 oa = make_float2(0.f, 0.f), ob = oa, oq = oa;
    if (j < A.g.n) {
      const int64_t M = A.g.margin;
      // 1) delay at the output time t_b = j dt, plain FP32 (only seeds the solve)
      const float4 T0 = A.tab0[j + M], T1 = A.tab1[j + M];
      const float phi0 = fmaf(K.nx.hi, T0.x, K.nyp.hi * T0.z) + fmaf(K.rcd, K.ca * T1.x + K.sa * T1.y, K.zsd);
      // 2) first source time t1 = m1 dt + tau1 with t1 - t_b = -phi0 (up to rounding)
      const float kf = rintf(-phi0 * A.inv_dt);
      const int k1 = (int)kf;
      const df32 kd = two_prod(kf, A.dt2.hi);  // k1 dt as an exact pair (plus kf * dt.lo)
      const float kdlo = fmaf(kf, A.dt2.lo, kd.lo);
      const float tau1 = (-phi0 - kd.hi) - kdlo;
      const int64_t m1 = j + k1;
      const float4 U0 = A.tab0[m1 + M], U1 = A.tab1[m1 + M];
      // 3) delay at t1: orbit term as double-float at the grid point, rotated by Omega_o tau1
      df32 P = df_add(df_mul(K.nx, df32{U0.x, U0.y}), df_mul(K.nyp, df32{U0.z, U0.w}));
      const float eo = (float)kOmegaO * tau1;
      const float Qo = fmaf(-K.nx.hi, U0.z, K.nyp.hi * U0.x);  // d(orbit)/d(lambda)
      const float orb = fmaf(eo, Qo, -0.5f * eo * eo * P.hi);
      const float er = (float)kOmegaR * tau1;
      const float ce = 1.f - 0.5f * er * er, se = er - er * er * er * (1.f / 6.f);
      const float cth = fmaf(U1.x, ce, -U1.y * se), sth = fmaf(U1.y, ce, U1.x * se);
      float cx = fmaf(K.ca, cth, K.sa * sth);   // cos(alpha - theta(t1))
      float sx = fmaf(K.sa, cth, -K.ca * sth);  // sin(alpha - theta(t1))
      const float rot = fmaf(K.rcd, cx, K.zsd);
      const float phidot = fmaf((float)kOmegaO, Qo, K.rcd * (float)kOmegaR * sx);
      // 4) Newton step on g(t) = t + phi_m(t) - t_b at t1
      const df32 Ah = two_sum(kd.hi, P.hi);
      const float gres = ((Ah.hi + tau1) + (Ah.lo + kdlo)) + ((P.lo + orb) + rot);
      const float delta = -gres / (1.f + phidot);
      const float tau = tau1 + delta;  // t_j = m1 dt + tau
      const float small = ((P.lo + orb) + rot) + phidot * delta;
      const df32 phim = quick_two_sum(P.hi, small);  // phi_m(t_j)
      const float eta = (float)kOmegaR * delta;
      const float cxj = fmaf(sx, eta, cx), sxj = fmaf(-cx, eta, sx);
      cx = cxj;
      sx = sxj;
      // 5) data at the source time
      float xr = 0.f;
      if (INTERP == FS_INTERP_SPLINE2X) {
        const float v = tau * A.two_over_dt;
        const float fv = floorf(v);
        const int64_t i = 2 * m1 + (int64_t)fv;
        const float f = v - fv;
        const int64_t ilast = 2 * A.g.n - 2;
        if ((i >= 0 && i < ilast) || (i == ilast && f == 0.f)) {
          const float4 c = A.coef[i];
          xr = fmaf(f, fmaf(f, fmaf(f, c.w, c.z), c.y), c.x);
        }
      } else {
        const int64_t kk = m1 + (int64_t)rintf(tau * A.inv_dt);
        if (kk >= 0 && kk < A.g.n) xr = A.x32[kk];
      }
      // 6) amplitude modulation at t_j
      const float c2 = fmaf(cx, cx, -sx * sx), s2 = 2.f * sx * cx;
      const float av = fmaf(K.ea[0], c2, fmaf(K.ea[1], s2, fmaf(K.ea[2], cx, fmaf(K.ea[3], sx, K.ea[4]))));
      const float bv = fmaf(K.eb[0], c2, fmaf(K.eb[1], s2, fmaf(K.eb[2], cx, K.eb[3] * sx)));
      a2 = av * av;
      b2 = bv * bv;
      // 7) heterodyne exp(-2 pi i fl phi_m(t_j))
      const float2 h = expm2pi(df_mul_frac(A.fl, phim));
      oa = make_float2(xr * av * h.x, xr * av * h.y);
      ob = make_float2(xr * bv * h.x, xr * bv * h.y);
      // 8) Q_j = t_j (t_j/2 + phi_m(t_j)) as double-float
      const df32 tj = df_add_f(df32{U1.z, U1.w}, tau);
      const df32 U = df_add(df32{0.5f * tj.hi, 0.5f * tj.lo}, phim);
      const df32 Q = df_mul(tj, U);
      oq = make_float2(Q.hi, Q.lo);
      if (A.tsrc && s == 0) A.tsrc[j] = (double)m1 * A.g.dt + (double)tau;
    }
    A.ya[s * A.stride + j] = oa;
    A.yb[s * A.stride + j] = ob;
    A.qq[s * A.stride + j] = oq;
  }
  // deterministic block sums of a^2, b^2: FP32 within a warp (32 terms), FP64 beyond
  for (int o = 16; o > 0; o >>= 1) {
    a2 += __shfl_down_sync(kFull, a2, o);
    b2 += __shfl_down_sync(kFull, b2, o);
  }
  const double da = a2, db = b2;
  __shared__ double wa[8], wb[8];
  if ((threadIdx.x & 31) == 0) { wa[threadIdx.x >> 5] = da; wb[threadIdx.x >> 5] = db; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sa = 0.0, sb = 0.0;
    for (int w = 0; w < 8; w++) { sa += wa[w]; sb += wb[w]; }
    double *p = A.partial + ((int64_t)s * gridDim.x + blockIdx.x) * 2;
    p[0] = sa;
    p[1] = sb;
  }
}

// <a^2>, <b^2> over the n output samples and the per-sky F normalisation
// (cF / <a^2>, cF / <b^2>) with cF = 2 dt^2 / (S0 To) = 2 dt / (S0 n).
__global__ void k_demod_finalize(const double *partial, int nb, int64_t n, double dt, double S0, float2 *norm,
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
    if (norm) norm[s] = make_float2((float)(cF / ma), (float)(cF / mb));
    if (ab2) ab2[s] = make_double2(ma, mb);
  }
}

// ------------------------------------------------------------------ pass 1
struct Pass1Args {
  const float2 *ya, *yb, *qq;
  int64_t sky_stride;
  const double *f1;
  int nspin, tmpl0;
  int N2, n1max;
  int64_t nfft;
  float2 *Z;  // [batch][2][N1][N2]
};

// CW columns per CTA; a warp holds CW columns x 2 signals x TPW sub-DFT threads.
// AM: rows n1 = Q a + b with a >= AM are zero for every column (AM = P when the
// data may fill the column, P/2 when n1max <= L/2, i.e. N <= Nfft/2).
__device__ __forceinline__ float2 chirp_cycles(float f) {
  // exp(-2 pi i f), |f| <= 1/2: hardware sine/cosine (absolute error < 1e-6 on [-pi, pi])
  float s, c;
  __sincosf(6.283185307179586f * f, &s, &c);
  return make_float2(c, -s);
}

// One pass-1 work item: template tm (index within the group) and its column
// tile, writing Z slot zs.  Needs P * 2 * CW threads; xch holds L * 2 * CW
// float2, twL the table W_L^q (q < L).  The caller synchronises before and after.
template <int P, int Q, int CW, int AM>
__device__ __forceinline__ void pass1_item(const Pass1Args &A, int tm, int zs, int tile, float2 *xch,
                                           const float2 *twL) {
  constexpr int L = P * Q;
  constexpr int S = Q / P;
  constexpr int CS = 2 * CW;     // (column, signal) pairs
  constexpr int TPW = 32 / CS;   // sub-DFT threads per warp
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int cs = lane % CS, col = cs % CW, sig = cs / CW;
  const int t = w * TPW + lane / CS;
  const int sky = tm / A.nspin, spin = tm - sky * A.nspin;
  const int n2 = tile * CW + col;
  const float2 *y = (sig ? A.yb : A.ya) + sky * A.sky_stride;
  const float2 *qq = A.qq + sky * A.sky_stride;
  const df32 f1 = df_from_double(A.f1[spin]);
  const int n1max = A.n1max;
  const int64_t N2 = A.N2;

  float2 v[Q];
  // load y_j and the chirp exp(-2 pi i f1 Q_j); the two signal lanes of a
  // column share the chirp: each computes every other one and swaps.  All
  // loads of a b-slot are issued before any of them is used.
  sfor<0, S>([&](auto s) {
    const int b = t + P * s;
    float2 qv[AM / 2];
    sfor<0, AM / 2>([&](auto ap) {
      const int my = Q * (2 * ap + sig) + b;
      qv[ap] = (my < n1max) ? qq[my * N2 + n2] : make_float2(0.f, 0.f);
    });
    sfor<0, P>([&](auto a) {
      const int na = Q * a + b;
      if constexpr (a < AM) v[s * P + a] = (na < n1max) ? y[na * N2 + n2] : make_float2(0.f, 0.f);
      else v[s * P + a] = make_float2(0.f, 0.f);
    });
    sfor<0, AM / 2>([&](auto ap) {
      constexpr int a0 = 2 * ap, a1 = 2 * ap + 1;
      const int my = Q * (a0 + sig) + b;
      float2 cm = make_float2(0.f, 0.f);
      if (my < n1max) cm = chirp_cycles(df_mul_frac(f1, df32{qv[ap].x, qv[ap].y}));
      float2 cp;
      cp.x = __shfl_xor_sync(kFull, cm.x, CW);
      cp.y = __shfl_xor_sync(kFull, cm.y, CW);
      const float2 c0 = sig ? cp : cm, c1 = sig ? cm : cp;
      v[s * P + a0] = cmul(v[s * P + a0], c0);
      v[s * P + a1] = cmul(v[s * P + a1], c1);
    });
  });
  sfor<0, S>([&](auto s) {
    const int b = t + P * s;
    dft_inplace<P, AM>(v + s * P);
    sfor<1, P>([&](auto c) { v[s * P + c] = cmul(v[s * P + c], twL[(b * c) & (L - 1)]); });
    sfor<0, P>([&](auto c) { xch[(b * P + c) * CS + cs] = v[s * P + c]; });
  });
  __syncthreads();
  sfor<0, Q>([&](auto bb) { v[bb] = xch[(bb * P + t) * CS + cs]; });
  dft_inplace<Q>(v);  // v[d] = X[k1 = t + P d] of column n2
  // inter-pass twiddle exp(-2 pi i n2 k1 / Nfft): anchors every 16 d from the
  // hardware sine/cosine (argument reduced to half a turn), and an exactly
  // rounded step for the recurrence between anchors so errors do not build up
  const int64_t nf = A.nfft;
  const float inv_nf = 1.0f / (float)nf;
  const float2 step = expm2pi((float)(((int64_t)n2 * P) & (nf - 1)) * inv_nf);
  float2 wt = make_float2(1.f, 0.f);
  sfor<0, Q>([&](auto d) {
    if constexpr (d % 16 == 0) {
      const float f = (float)(((int64_t)n2 * (t + P * d)) & (nf - 1)) * inv_nf;
      wt = chirp_cycles(f > 0.5f ? f - 1.0f : f);
    } else {
      wt = cmul(wt, step);
    }
    v[d] = cmul(v[d], wt);
  });
  float2 *Zs = A.Z + ((int64_t)zs * 2 + sig) * nf;
  sfor<0, Q>([&](auto d) { Zs[(int64_t)(t + P * d) * N2 + n2] = v[d]; });
}

template <int P, int Q, int CW, int AM>
__global__ void __launch_bounds__(P * 2 * CW, 2) k_pass1(Pass1Args A) {
  constexpr int L = P * Q;
  extern __shared__ float2 smem[];
  float2 *xch = smem;               // [Q][P][2 CW]
  float2 *twL = smem + L * 2 * CW;  // W_L^q
  const int tiles = A.N2 / CW;
  const int bt = blockIdx.x / tiles, tile = blockIdx.x - bt * tiles;
  for (int q = threadIdx.x; q < L; q += blockDim.x) twL[q] = expm2pi((float)q * (1.0f / L));
  __syncthreads();
  pass1_item<P, Q, CW, AM>(A, A.tmpl0 + bt, bt, tile, xch, twL);
}

// ------------------------------------------------------------------ pass 2 + F epilogue
struct Pass2Args {
  const float2 *Z;
  int N1, N2;
  int64_t nfft;
  const float2 *norm;  // per sky of the group
  int nspin, tmpl0;
  int sky_base;        // global index of the group's first sky
  float *F;            // NULL or F_out + (global template of the group's first template) * nbins
  int64_t nbins;
  float thr;
  fs_candidate *cand;
  int64_t cap;
  unsigned long long *ncand;
  uint32_t *flags;
};

// One pass-2 work item: template tm (within the group), row tile rt, reading Z
// slot zs.  Needs 32 * WARPS threads; work holds the exchange and F tile areas
// (pass2_work_floats2), twM the matrix W_L^{b c} stored by c then b.  Z is read
// past L1 (it may have been rewritten since an earlier item on this SM).
// Exchange layout of one sub-DFT: element (c, b) at c * PITCH + col(c, b).  For
// 16- and 32-thread sub-DFTs the row pitch is Q and the column is XOR-swizzled
// by c (conflict-free, no padding); otherwise rows are padded to Q + 1.
template <int P, int Q>
struct Xch2 {
  static constexpr bool SWZ = (P >= 16);
  static constexpr int PITCH = SWZ ? Q : Q + 1;
  static constexpr int SIZE = P * PITCH;
  static __device__ __forceinline__ int at(int c, int b) { return c * PITCH + (SWZ ? (b ^ (c & 15)) : b); }
};

// Pass-2 work item for 32-thread row DFTs (N2 = 1024): a warp holds one signal of
// one row (warps 2r, 2r+1: signals a, b of row r), so an item covers WARPS/2
// rows; the two signals' |X|^2 terms meet through the F tile.
template <int Q, int WARPS, bool FULLBINS>
__device__ __forceinline__ void pass2_item_wide(const Pass2Args &A, int tm, int zs, int rt, float2 *work,
                                                const float2 *twM) {
  constexpr int P = 32, R = WARPS / 2, S = Q / P;
  constexpr int D = FULLBINS ? Q : Q / 2;
  using X = Xch2<P, Q>;
  constexpr int XW = X::SIZE;
  constexpr int K2 = D * P;
  float *Fs = (float *)work;  // [K2][R + 1], aliased over the exchange area
  const int t = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int sig = w & 1, row = w >> 1;
  const int k1 = rt * R + row;
  const int sky = tm / A.nspin, spin = tm - sky * A.nspin;
  const float2 *z = A.Z + ((int64_t)zs * 2 + sig) * A.nfft + (int64_t)k1 * A.N2;
  float2 v[Q];
  sfor<0, S>([&](auto s) { sfor<0, P>([&](auto a) { v[s * P + a] = __ldcg(z + Q * a + t + P * s); }); });
  float2 *xw = work + w * XW;
  sfor<0, S>([&](auto s) {
    const int b = t + P * s;
    dft_inplace<P>(v + s * P);
    sfor<1, P>([&](auto c) { v[s * P + c] = cmul(v[s * P + c], twM[c * Q + b]); });
    sfor<0, P>([&](auto c) { xw[X::at(c, b)] = v[s * P + c]; });
  });
  __syncwarp();
  sfor<0, Q>([&](auto bb) { v[bb] = xw[X::at(t, bb)]; });
  __syncthreads();  // every warp is done with the exchange area (reused for the F tile)
  dft_inplace<Q, Q, D>(v);  // v[d] = X[k2 = t + P d] of row k1 (d < D)
  const float2 nrm = A.norm[sky];
  if (sig == 0) {
    sfor<0, D>([&](auto d) { Fs[(t + P * d) * (R + 1) + row] = fmaf(v[d].x, v[d].x, v[d].y * v[d].y) * nrm.x; });
  }
  __syncthreads();
  const unsigned lt_mask = (1u << t) - 1u;
  if (sig == 1) {
    sfor<0, D>([&](auto d) {
      const int k2 = t + P * d;
      float *fp = Fs + k2 * (R + 1) + row;
      const float Fv = *fp + fmaf(v[d].x, v[d].x, v[d].y * v[d].y) * nrm.y;
      *fp = Fv;
      const bool hit = Fv > A.thr;
      const unsigned m = __ballot_sync(kFull, hit);
      if (m) {
        const int leader = __ffs(m) - 1;
        unsigned long long base = 0;
        if (t == leader) base = atomicAdd(A.ncand, (unsigned long long)__popc(m));
        base = __shfl_sync(kFull, base, leader);
        if (hit) {
          const unsigned long long idx = base + __popc(m & lt_mask);
          if ((long long)idx < A.cap) {
            fs_candidate c;
            c.sky = (uint32_t)(A.sky_base + sky);
            c.spin = (uint32_t)spin;
            c.bin = (uint32_t)(k1 + A.N1 * k2);
            c.F = Fv;
            A.cand[idx] = c;
          } else {
            atomicOr(A.flags, ERRF_CAPACITY);
          }
        }
      }
    });
  }
  if (A.F == nullptr) return;
  __syncthreads();
  float *Fo = A.F + (int64_t)tm * A.nbins + rt * R;
  for (int idx = threadIdx.x; idx < K2 * R; idx += blockDim.x) {
    const int k2 = idx / R, r = idx - k2 * R;
    __stcs(Fo + r + (int64_t)A.N1 * k2, Fs[k2 * (R + 1) + r]);
  }
}

// ALIAS_F: the F tile reuses the exchange area (one more barrier, less shared memory).
template <int P, int Q, int WARPS, bool FULLBINS, bool ALIAS_F = false>
__device__ __forceinline__ void pass2_item(const Pass2Args &A, int tm, int zs, int rt, float2 *work,
                                           const float2 *twM) {
  if constexpr (P == 32) {
    pass2_item_wide<Q, WARPS, FULLBINS>(A, tm, zs, rt, work, twM);
    return;
  }
  constexpr int T = P, G = (P <= 16 ? 16 / P : 1), R = WARPS * G, S = Q / P;
  constexpr int D = FULLBINS ? Q : Q / 2;  // d values with k2 = t + P d in the output band
  using X = Xch2<P, Q>;
  constexpr int XW = X::SIZE;              // exchange float2s per sub-DFT
  float *Fs = (float *)(ALIAS_F ? work : work + WARPS * 2 * G * XW);  // [D*P][R+1]
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int t = lane % T, sig = (lane / T) & 1, gr = lane / (2 * T);
  const int row = w * G + gr;
  const int k1 = rt * R + row;
  const int sky = tm / A.nspin, spin = tm - sky * A.nspin;
  const float2 *z = A.Z + ((int64_t)zs * 2 + sig) * A.nfft + (int64_t)k1 * A.N2;
  float2 v[Q];
  sfor<0, S>([&](auto s) { sfor<0, P>([&](auto a) { v[s * P + a] = __ldcg(z + Q * a + t + P * s); }); });
  float2 *xw = work + (w * 2 * G + (sig + 2 * gr)) * XW;
  sfor<0, S>([&](auto s) {
    const int b = t + P * s;
    dft_inplace<P>(v + s * P);
    // W_L^{b c} stored by c then b: lanes read consecutive entries (no bank conflicts)
    sfor<1, P>([&](auto c) { v[s * P + c] = cmul(v[s * P + c], twM[c * Q + b]); });
    sfor<0, P>([&](auto c) { xw[X::at(c, b)] = v[s * P + c]; });
  });
  __syncwarp();
  sfor<0, Q>([&](auto bb) { v[bb] = xw[X::at(t, bb)]; });
  if constexpr (ALIAS_F) __syncthreads();  // every warp is done with the exchange area
  dft_inplace<Q, Q, (FULLBINS ? Q : Q / 2)>(v);  // v[d] = X[k2 = t + P d] of row k1 (d < D)
  const float2 nrm = A.norm[sky];
  const float myn = sig ? nrm.y : nrm.x;
  float p[D];
  sfor<0, D>([&](auto d) { p[d] = fmaf(v[d].x, v[d].x, v[d].y * v[d].y) * myn; });
  const unsigned lt_mask = (1u << lane) - 1u;
  sfor<0, D / 2>([&](auto dp) {
    const float send = sig ? p[dp] : p[dp + D / 2];
    const float mine = sig ? p[dp + D / 2] : p[dp];
    const float Fv = mine + __shfl_xor_sync(kFull, send, T);
    const int d = dp + sig * (D / 2);
    const int k2 = t + P * d;
    Fs[k2 * (R + 1) + row] = Fv;
    const bool hit = Fv > A.thr;
    const unsigned m = __ballot_sync(kFull, hit);
    if (m) {
      const int leader = __ffs(m) - 1;
      unsigned long long base = 0;
      if (lane == leader) base = atomicAdd(A.ncand, (unsigned long long)__popc(m));
      base = __shfl_sync(kFull, base, leader);
      if (hit) {
        const unsigned long long idx = base + __popc(m & lt_mask);
        if ((long long)idx < A.cap) {
          fs_candidate c;
          c.sky = (uint32_t)(A.sky_base + sky);
          c.spin = (uint32_t)spin;
          c.bin = (uint32_t)(k1 + A.N1 * k2);
          c.F = Fv;
          A.cand[idx] = c;
        } else {
          atomicOr(A.flags, ERRF_CAPACITY);
        }
      }
    }
  });
  if (A.F == nullptr) return;
  __syncthreads();
  float *Fo = A.F + (int64_t)tm * A.nbins + rt * R;
  constexpr int K2 = D * P;
  for (int idx = threadIdx.x; idx < K2 * R; idx += blockDim.x) {
    const int k2 = idx / R, r = idx - k2 * R;
    __stcs(Fo + r + (int64_t)A.N1 * k2, Fs[k2 * (R + 1) + r]);
  }
}

template <int P, int Q, int WARPS, bool FULLBINS, bool ALIAS_F = false>
constexpr size_t pass2_work_floats2() {
  constexpr int G = P <= 16 ? 16 / P : 1;
  constexpr int R = P <= 16 ? WARPS * G : WARPS / 2, D = FULLBINS ? Q : Q / 2;
  constexpr size_t xch = P <= 16 ? (size_t)WARPS * 2 * G * Xch2<P, Q>::SIZE : (size_t)WARPS * Xch2<P, Q>::SIZE;
  constexpr size_t ftile = ((size_t)D * P * (R + 1) + 1) / 2;
  return (ALIAS_F || P == 32) ? (xch > ftile ? xch : ftile) : xch + ftile;
}

__device__ __forceinline__ void twiddle_matrix(float2 *twM, int P, int Q) {
  const int L = P * Q;
  for (int q = threadIdx.x; q < L; q += blockDim.x) {
    const int c = q / Q, b = q - c * Q;
    twM[q] = expm2pi((float)((b * c) & (L - 1)) * (1.0f / L));
  }
}

template <int P, int Q, int WARPS, bool FULLBINS>
__global__ void __launch_bounds__(32 * WARPS, 2) k_pass2(Pass2Args A) {
  constexpr int R = P <= 16 ? WARPS * (16 / P) : WARPS / 2;
  extern __shared__ float2 smem[];
  float2 *twM = smem;
  float2 *work = smem + P * Q;
  const int rtiles = A.N1 / R;
  const int bt = blockIdx.x / rtiles, rt = blockIdx.x - bt * rtiles;
  twiddle_matrix(twM, P, Q);
  __syncthreads();
  pass2_item<P, Q, WARPS, FULLBINS>(A, A.tmpl0 + bt, bt, rt, work, twM);
}

// ------------------------------------------------------------------ persistent pass kernel
// One launch runs both passes for every template of a sky group from a work
// queue.  Round r holds the pass-1 items of template r and the pass-2 items of
// template r - lag.  A pass-2 item waits until all pass-1 items of its template
// have completed; a pass-1 item of template t waits until the pass-2 items of
// template t - slots (the previous user of its Z slot) have completed.  Items
// are taken in queue order, so every wait is on earlier items held by running
// CTAs.  Waits are bounded: on exhaustion the kernel latches ERRF_TIMEOUT and
// continues (results are then invalid, the device stays responsive).
struct QueueArgs {
  int ntm, tiles1, tiles2, lag, slots;
  int kr;             // templates per round: a round holds the pass-1 items of kr templates,
                      // then the pass-2 items of the kr templates lag rounds earlier
  unsigned *counter;  // [1 + 2 ntm]: next item, pass-1 done per template, pass-2 done per template
};

constexpr long kSpinLimit = 20000000;  // ~100 ns per poll: a few seconds at most

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void red_release_add(unsigned *p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
// Called by one thread: wait until *p >= target (bounded).
__device__ inline void wait_at_least(const unsigned *p, unsigned target, uint32_t *flags) {
  for (long it = 0; ld_acquire(p) < target; it++) {
    if (it > kSpinLimit) {
      atomicOr(flags, ERRF_TIMEOUT);
      return;
    }
    __nanosleep(100);
  }
}

template <int P1, int Q1, int AM, int P2, int Q2, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB) k_passes(Pass1Args A1, Pass2Args A2, QueueArgs Qa) {
  constexpr int CW = NT / (2 * P1);
  constexpr int L1 = P1 * Q1, L2 = P2 * Q2;
  extern __shared__ float2 smem[];
  float2 *twL = smem;            // W_{L1}^q
  float2 *twM = smem + L1;       // W_{L2}^{b c} by c then b
  float2 *work = smem + L1 + L2; // union of the pass-1 exchange and the pass-2 work areas
  for (int q = threadIdx.x; q < L1; q += blockDim.x) twL[q] = expm2pi((float)q * (1.0f / L1));
  twiddle_matrix(twM, P2, Q2);
  unsigned *next = Qa.counter;
  unsigned *done1 = Qa.counter + 1;
  unsigned *done2 = Qa.counter + 1 + Qa.ntm;
  const int kr = Qa.kr;
  const int ipr = kr * (Qa.tiles1 + Qa.tiles2);
  const int total = ((Qa.ntm + kr - 1) / kr + Qa.lag) * ipr;
  // Items are decoded identically by every thread; thread 0 takes the next item
  // from the queue while the current one runs, checks whether the next item's
  // dependency is already met, and publishes both through ping-pong slots before
  // the end-of-item barrier (the slot it writes was last read before the previous
  // end-of-item barrier).  A ready item then needs no extra barrier.
  struct Item {
    int tm, j;
    bool is1, valid;
  };
  auto decode = [&](int it) {
    Item d;
    const int r = it / ipr;
    const int jr = it - r * ipr;
    d.is1 = jr < kr * Qa.tiles1;
    if (d.is1) {
      const int k = jr / Qa.tiles1;
      d.j = jr - k * Qa.tiles1;
      d.tm = r * kr + k;
    } else {
      const int j2 = jr - kr * Qa.tiles1;
      const int k = j2 / Qa.tiles2;
      d.j = Qa.tiles1 + (j2 - k * Qa.tiles2);
      d.tm = (r - Qa.lag) * kr + k;
    }
    d.valid = it < total && d.tm >= 0 && d.tm < Qa.ntm;
    return d;
  };
  auto dep_met = [&](const Item &d) {  // thread 0 only
    if (!d.valid) return true;
    if (d.is1) return d.tm < Qa.slots || ld_acquire(done2 + (d.tm - Qa.slots)) >= (unsigned)Qa.tiles2;
    return ld_acquire(done1 + d.tm) >= (unsigned)Qa.tiles1;
  };
  __shared__ int s_next[2], s_ready[2];
  if (threadIdx.x == 0) {
    s_next[0] = (int)atomicAdd(next, 1u);
    s_ready[0] = 0;
  }
  __syncthreads();
  int buf = 0;
  int cur = s_next[0], ready = s_ready[0];
  while (cur < total) {
    int nxt = 0;
    if (threadIdx.x == 0) nxt = (int)atomicAdd(next, 1u);
    const Item d = decode(cur);
    if (d.valid) {
      if (!ready) {
        if (threadIdx.x == 0) {
          if (d.is1) {
            if (d.tm >= Qa.slots) wait_at_least(done2 + (d.tm - Qa.slots), Qa.tiles2, A2.flags);
          } else {
            wait_at_least(done1 + d.tm, Qa.tiles1, A2.flags);
          }
        }
        __syncthreads();
      }
      if (d.is1) pass1_item<P1, Q1, CW, AM>(A1, d.tm, d.tm % Qa.slots, d.j, work, twL);
      else pass2_item<P2, Q2, NT / 32, false, true>(A2, d.tm, d.tm % Qa.slots, d.j - Qa.tiles1, work, twM);
    }
    if (threadIdx.x == 0) {
      s_next[buf ^ 1] = nxt;
      s_ready[buf ^ 1] = dep_met(decode(nxt)) ? 1 : 0;
    }
    __syncthreads();  // item complete: global writes done, shared memory free, next item published
    if (threadIdx.x == 0 && d.valid) red_release_add((d.is1 ? done1 : done2) + d.tm, 1u);
    buf ^= 1;
    cur = s_next[buf];
    ready = s_ready[buf];
  }
}

// ------------------------------------------------------------------ host orchestration
struct FftShape {
  int N1, N2;
};
static bool fft_shape(int64_t nfft, FftShape *s) {
  int p = 0;
  while (((int64_t)1 << p) < nfft) p++;
  if (((int64_t)1 << p) != nfft || p < 12 || p > 20) return false;
  s->N1 = 1 << ((p + 1) / 2);
  s->N2 = 1 << (p / 2);
  return true;
}

constexpr int kPass2Warps = 8;  // warps per pass-2 CTA

template <int P, int Q>
static size_t pass1_smem() { return sizeof(float2) * ((size_t)P * Q * 2 * (256 / (2 * P)) + (size_t)P * Q); }
template <int P, int Q, bool FULL>
static size_t pass2_smem() {
  return sizeof(float2) * ((size_t)P * Q + pass2_work_floats2<P, Q, kPass2Warps, FULL>());
}

template <int P, int Q>
static cudaError_t launch_pass1(const Pass1Args &a, int nb, cudaStream_t st) {
  size_t sm = pass1_smem<P, Q>();
  constexpr int CW = 256 / (2 * P);
  auto kern = (a.n1max <= P * Q / 2) ? k_pass1<P, Q, CW, P / 2> : k_pass1<P, Q, CW, P>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  kern<<<nb * (a.N2 / CW), P * 2 * CW, sm, st>>>(a);
  return cudaGetLastError();
}
template <int P, int Q, bool FULL>
static cudaError_t launch_pass2(const Pass2Args &a, int nb, cudaStream_t st) {
  size_t sm = pass2_smem<P, Q, FULL>();
  auto kern = k_pass2<P, Q, kPass2Warps, FULL>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  constexpr int R = P <= 16 ? kPass2Warps * (16 / P) : kPass2Warps / 2;
  kern<<<nb * (a.N1 / R), 32 * kPass2Warps, sm, st>>>(a);
  return cudaGetLastError();
}

static cudaError_t dispatch_pass1(int N1, const Pass1Args &a, int nb, cudaStream_t st) {
  switch (N1) {
    case 64: return launch_pass1<8, 8>(a, nb, st);
    case 128: return launch_pass1<8, 16>(a, nb, st);
    case 256: return launch_pass1<16, 16>(a, nb, st);
    case 512: return launch_pass1<16, 32>(a, nb, st);
    case 1024: return launch_pass1<32, 32>(a, nb, st);
  }
  return cudaErrorInvalidValue;
}
static cudaError_t dispatch_pass2(int N2, bool full, const Pass2Args &a, int nb, cudaStream_t st) {
  switch (N2 * 2 + (full ? 1 : 0)) {
    case 128: return launch_pass2<8, 8, false>(a, nb, st);
    case 129: return launch_pass2<8, 8, true>(a, nb, st);
    case 256: return launch_pass2<8, 16, false>(a, nb, st);
    case 257: return launch_pass2<8, 16, true>(a, nb, st);
    case 512: return launch_pass2<16, 16, false>(a, nb, st);
    case 513: return launch_pass2<16, 16, true>(a, nb, st);
    case 1024: return launch_pass2<16, 32, false>(a, nb, st);
    case 1025: return launch_pass2<16, 32, true>(a, nb, st);
    case 2048: return launch_pass2<32, 32, false>(a, nb, st);
    case 2049: return launch_pass2<32, 32, true>(a, nb, st);
  }
  return cudaErrorInvalidValue;
}

// Persistent pass kernel: shapes (N1 x N2) -> (P1, Q1, P2, Q2), pruning AM.
#ifndef FS_PERSIST_MINB
#define FS_PERSIST_MINB 3
#endif
constexpr int kPersistMinBlocks = FS_PERSIST_MINB;  // CTAs per SM the kernel is compiled for

template <int P1, int Q1, int P2, int Q2, int NT>
constexpr size_t persist_smem() {
  constexpr int CW = NT / (2 * P1);
  constexpr size_t w1 = (size_t)P1 * Q1 * 2 * CW;
  constexpr size_t w2 = pass2_work_floats2<P2, Q2, NT / 32, false, true>();
  return sizeof(float2) * ((size_t)P1 * Q1 + (size_t)P2 * Q2 + (w1 > w2 ? w1 : w2));
}
// CTAs per SM the kernel is compiled for: 3 when three fit in shared memory.
template <int P1, int Q1, int P2, int Q2, int NT>
constexpr int persist_minb() { return persist_smem<P1, Q1, P2, Q2, NT>() <= 74 * 1024 ? kPersistMinBlocks : 2; }

template <int P1, int Q1, int AM, int P2, int Q2, int NT>
static cudaError_t launch_passes_t(const Pass1Args &a1, const Pass2Args &a2, const QueueArgs &qa, cudaStream_t st) {
  constexpr int MINB = persist_minb<P1, Q1, P2, Q2, NT>();
  const size_t sm = persist_smem<P1, Q1, P2, Q2, NT>();
  auto kern = k_passes<P1, Q1, AM, P2, Q2, NT, MINB>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  int dev = 0, nsm = 0, occ = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, NT, sm);
  if (e != cudaSuccess) return e;
  if (occ < 1) occ = 1;
  const long total = (long)((qa.ntm + qa.kr - 1) / qa.kr + qa.lag) * qa.kr * (qa.tiles1 + qa.tiles2);
  long grid = (long)occ * nsm;
  if (grid > total) grid = total;
  kern<<<(unsigned)grid, NT, sm, st>>>(a1, a2, qa);
  return cudaGetLastError();
}

template <int P1, int Q1, int P2, int Q2, int NT>
static cudaError_t launch_passes_am(const Pass1Args &a1, const Pass2Args &a2, const QueueArgs &qa, cudaStream_t st) {
  if (a1.n1max <= P1 * Q1 / 2) return launch_passes_t<P1, Q1, P1 / 2, P2, Q2, NT>(a1, a2, qa, st);
  return launch_passes_t<P1, Q1, P1, P2, Q2, NT>(a1, a2, qa, st);
}

template <int NT>
static cudaError_t dispatch_passes_nt(int N1, int N2, const Pass1Args &a1, const Pass2Args &a2,
                                      const QueueArgs &qa, cudaStream_t st) {
  switch (N1 * 4096 + N2) {
    case 64 * 4096 + 64: return launch_passes_am<8, 8, 8, 8, NT>(a1, a2, qa, st);
    case 128 * 4096 + 64: return launch_passes_am<8, 16, 8, 8, NT>(a1, a2, qa, st);
    case 128 * 4096 + 128: return launch_passes_am<8, 16, 8, 16, NT>(a1, a2, qa, st);
    case 256 * 4096 + 128: return launch_passes_am<16, 16, 8, 16, NT>(a1, a2, qa, st);
    case 256 * 4096 + 256: return launch_passes_am<16, 16, 16, 16, NT>(a1, a2, qa, st);
    case 512 * 4096 + 256: return launch_passes_am<16, 32, 16, 16, NT>(a1, a2, qa, st);
    case 512 * 4096 + 512: return launch_passes_am<16, 32, 16, 32, NT>(a1, a2, qa, st);
    case 1024 * 4096 + 512: return launch_passes_am<32, 32, 16, 32, NT>(a1, a2, qa, st);
    case 1024 * 4096 + 1024: return launch_passes_am<32, 32, 32, 32, NT>(a1, a2, qa, st);
  }
  return cudaErrorInvalidValue;
}

// Work-item geometry of the persistent kernel for NT threads per CTA.
static void queue_tiles(int N1, int N2, int NT, int *tiles1, int *tiles2) {
  const int P1 = N1 <= 128 ? 8 : (N1 <= 512 ? 16 : 32);
  const int P2 = N2 <= 128 ? 8 : (N2 <= 512 ? 16 : 32);
  *tiles1 = N2 / (NT / (2 * P1));
  *tiles2 = N1 / (P2 <= 16 ? (NT / 32) * (16 / P2) : (NT / 32) / 2);
}

// 256 threads (2 CTAs per SM): measured faster than 128 threads with half-size items.
constexpr int kPersistThreads = 256;
static cudaError_t dispatch_passes(int N1, int N2, const Pass1Args &a1, const Pass2Args &a2,
                                   const QueueArgs &qa, cudaStream_t st) {
  return dispatch_passes_nt<kPersistThreads>(N1, N2, a1, a2, qa, st);
}

struct Ws32 {
  SkyConst32 *skyc;
  float2 *ya, *yb, *qq, *norm;
  double2 *ab2;
  double *partial;
  float2 *Z;
  unsigned *counters;
  int64_t stride;
  int nblk_a1;
};

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

static fs_status workspace32(fs_ctx *ctx, const fs_seg *seg, int G, int B, int64_t npad, int nsky,
                             int nspin, cudaStream_t st, Ws32 *w) {
  int64_t stride = (npad + 63) & ~(int64_t)63;
  int nblk = (int)((npad + 255) / 256);
  size_t off = 0;
  size_t o_sky = off; off = align256(off + sizeof(SkyConst32) * (nsky > G ? nsky : G));
  size_t o_ya = off; off = align256(off + sizeof(float2) * stride * G);
  size_t o_yb = off; off = align256(off + sizeof(float2) * stride * G);
  size_t o_qq = off; off = align256(off + sizeof(float2) * stride * G);
  size_t o_nm = off; off = align256(off + sizeof(float2) * G);
  size_t o_ab = off; off = align256(off + sizeof(double2) * G);
  size_t o_pa = off; off = align256(off + sizeof(double) * 2 * (size_t)nblk * G);
  size_t o_z = off; off = align256(off + sizeof(float2) * 2 * (size_t)seg->g.nfft * B);
  size_t o_ct = off; off = align256(off + sizeof(unsigned) * (1 + 2 * (size_t)G * nspin));
  fs_status s = ensure_buffer(&ctx->ws, &ctx->ws_bytes, off, st);
  if (s != FS_OK) return s;
  char *base = (char *)ctx->ws;
  w->skyc = (SkyConst32 *)(base + o_sky);
  w->ya = (float2 *)(base + o_ya);
  w->yb = (float2 *)(base + o_yb);
  w->qq = (float2 *)(base + o_qq);
  w->norm = (float2 *)(base + o_nm);
  w->ab2 = (double2 *)(base + o_ab);
  w->partial = (double *)(base + o_pa);
  w->Z = (float2 *)(base + o_z);
  w->counters = (unsigned *)(base + o_ct);
  w->stride = stride;
  w->nblk_a1 = nblk;
  return FS_OK;
}

static DemodArgs demod_args(const fs_seg *seg, const Ws32 &w, int64_t npad) {
  DemodArgs A{};
  A.g = seg->g;
  A.dt2 = df_from_double(seg->g.dt);
  A.dt = (float)seg->g.dt;
  A.inv_dt = (float)(1.0 / seg->g.dt);
  A.two_over_dt = (float)(2.0 / seg->g.dt);
  A.fl = df_from_double(seg->g.fl);
  A.sky = w.skyc;
  A.tab0 = seg->tab0;
  A.tab1 = seg->tab1;
  A.coef = (const float4 *)seg->coef;
  A.x32 = seg->x32;
  A.ya = w.ya;
  A.yb = w.yb;
  A.qq = w.qq;
  A.stride = w.stride;
  A.npad = npad;
  A.partial = w.partial;
  A.tsrc = nullptr;
  return A;
}

static cudaError_t launch_demod(const DemodArgs &A, int nsky, int nblk, int interp, cudaStream_t st) {
  dim3 grid(nblk, nsky);
  if (interp == FS_INTERP_NEAREST) k_demod32<FS_INTERP_NEAREST><<<grid, 256, 0, st>>>(A);
  else k_demod32<FS_INTERP_SPLINE2X><<<grid, 256, 0, st>>>(A);
  return cudaGetLastError();
}

// Shape of the persistent queue: templates per round, lag (rounds) and Z slots.
struct QueueShape {
  int kr, lag, slots, tiles1, tiles2;
};
static QueueShape queue_shape(const fs_ctx *ctx, const FftShape &sh) {
  QueueShape q{};
  queue_tiles(sh.N1, sh.N2, kPersistThreads, &q.tiles1, &q.tiles2);
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int ctas = (sh.N1 * sh.N2 >= (1 << 19) ? 2 : kPersistMinBlocks) * (nsm > 0 ? nsm : 1);
  q.kr = ctx->queue_round > 0 ? ctx->queue_round : (int)(0.85 * ctas / q.tiles1 + 0.5);
  if (q.kr < 1) q.kr = 1;
  q.lag = ctx->queue_lag > 0 ? ctx->queue_lag : 1;
  const int need = (q.lag + 2) * q.kr;
  q.slots = ctx->z_slots > need ? ctx->z_slots : need;
  return q;
}

fs_status search32(fs_ctx *ctx, fs_seg *seg, const double *alpha, const double *delta, int nsky,
                   const double *f1, int nspin, float thr, float *F, int64_t nbins, fs_candidate *cand,
                   int64_t cap, int64_t *ncand, cudaStream_t st) {
  FftShape sh;
  if (!fft_shape(seg->g.nfft, &sh)) return FS_ERR_SHAPE;
  const int64_t n = seg->g.n;
  const int n1max = (int)((n + sh.N2 - 1) / sh.N2);
  const int64_t npad = (int64_t)n1max * sh.N2;
  const int G = ctx->group_skies < nsky ? ctx->group_skies : nsky;
  const bool full = (nbins == seg->g.nfft);
  const bool persistent = !full && ctx->persistent;
  const QueueShape qs = queue_shape(ctx, sh);
  const int B = persistent ? qs.slots : ctx->batch_templates;  // Z slots of the workspace
  Ws32 w;
  fs_status s = workspace32(ctx, seg, G, B, npad, nsky, nspin, st, &w);
  if (s != FS_OK) return s;
  if (cudaMemsetAsync(ncand, 0, sizeof(int64_t), st) != cudaSuccess) return FS_ERR_CUDA;
  DemodArgs DA = demod_args(seg, w, npad);
  {
    ProfScope ps(ctx, PROF_OTHER, st);
    if (sky_constants32(alpha, delta, nsky, seg->g, ctx->det, w.skyc, st) != cudaSuccess) return FS_ERR_CUDA;
    ctx->launches += 1;
  }
  for (int g0 = 0; g0 < nsky; g0 += G) {
    const int gs = (nsky - g0) < G ? (nsky - g0) : G;
    DA.sky = w.skyc + g0;
    {
      ProfScope ps(ctx, PROF_DEMOD, st);
      if (launch_demod(DA, gs, w.nblk_a1, seg->d.interp, st) != cudaSuccess) return FS_ERR_CUDA;
    }
    {
      ProfScope ps(ctx, PROF_OTHER, st);
      k_demod_finalize<<<gs, 256, 0, st>>>(w.partial, w.nblk_a1, n, seg->g.dt, seg->g.S0, w.norm, w.ab2);
    }
    ctx->launches += 2;
    const int ntm = gs * nspin;
    Pass1Args p1{};
    p1.ya = w.ya;
    p1.yb = w.yb;
    p1.qq = w.qq;
    p1.sky_stride = w.stride;
    p1.f1 = f1;
    p1.nspin = nspin;
    p1.N2 = sh.N2;
    p1.n1max = n1max;
    p1.nfft = seg->g.nfft;
    p1.Z = w.Z;
    Pass2Args p2{};
    p2.Z = w.Z;
    p2.N1 = sh.N1;
    p2.N2 = sh.N2;
    p2.nfft = seg->g.nfft;
    p2.norm = w.norm;
    p2.nspin = nspin;
    p2.sky_base = g0;
    p2.F = F ? F + (int64_t)g0 * nspin * nbins : nullptr;
    p2.nbins = nbins;
    p2.thr = thr;
    p2.cand = cand;
    p2.cap = cap;
    p2.ncand = (unsigned long long *)ncand;
    p2.flags = ctx->d_flags;
    if (persistent) {
      QueueArgs qa{};
      qa.ntm = ntm;
      qa.tiles1 = qs.tiles1;
      qa.tiles2 = qs.tiles2;
      qa.kr = qs.kr;
      qa.lag = qs.lag;
      qa.slots = qs.slots;
      qa.counter = w.counters;
      if (cudaMemsetAsync(w.counters, 0, sizeof(unsigned) * (1 + 2 * (size_t)ntm), st) != cudaSuccess)
        return FS_ERR_CUDA;
      {
        ProfScope ps(ctx, PROF_PASS2, st);
        if (dispatch_passes(sh.N1, sh.N2, p1, p2, qa, st) != cudaSuccess) return FS_ERR_CUDA;
      }
      ctx->launches += 1;
      continue;
    }
    for (int b0 = 0; b0 < ntm; b0 += B) {
      const int nb = (ntm - b0) < B ? (ntm - b0) : B;
      p1.tmpl0 = b0;
      p2.tmpl0 = b0;
      {
        ProfScope ps(ctx, PROF_PASS1, st);
        if (dispatch_pass1(sh.N1, p1, nb, st) != cudaSuccess) return FS_ERR_CUDA;
      }
      {
        ProfScope ps(ctx, PROF_PASS2, st);
        if (dispatch_pass2(sh.N2, full, p2, nb, st) != cudaSuccess) return FS_ERR_CUDA;
      }
      ctx->launches += 2;
    }
  }
  return FS_OK;
}

// Stage access: A1 for one sky, widened to double.
__global__ void k_widen(const float2 *ya, const float2 *yb, double *oa, double *ob, int64_t n) {
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= n) return;
  oa[2 * j] = ya[j].x;
  oa[2 * j + 1] = ya[j].y;
  ob[2 * j] = yb[j].x;
  ob[2 * j + 1] = yb[j].y;
}

fs_status demod32_debug(fs_ctx *ctx, fs_seg *seg, double alpha, double delta, double *ya, double *yb,
                        double *tsrc, double *ab2, cudaStream_t st) {
  const int64_t n = seg->g.n;
  Ws32 w;
  fs_status s = workspace32(ctx, seg, 1, 1, n, 1, 1, st, &w);
  if (s != FS_OK) return s;
  // alpha/delta are host values: stage them through the partial buffer's tail is not
  // possible before allocation, so use a small device copy.
  double hd[2] = {alpha, delta};
  double *dd = (double *)w.ab2;  // 16 bytes, overwritten by finalize afterwards
  if (cudaMemcpyAsync(dd, hd, sizeof(hd), cudaMemcpyHostToDevice, st) != cudaSuccess) return FS_ERR_CUDA;
  if (sky_constants32(dd, dd + 1, 1, seg->g, ctx->det, w.skyc, st) != cudaSuccess) return FS_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return FS_ERR_CUDA;  // hd is on the stack
  DemodArgs A = demod_args(seg, w, n);
  A.tsrc = tsrc;
  if (launch_demod(A, 1, w.nblk_a1, seg->d.interp, st) != cudaSuccess) return FS_ERR_CUDA;
  k_demod_finalize<<<1, 256, 0, st>>>(w.partial, w.nblk_a1, n, seg->g.dt, seg->g.S0, nullptr, (double2 *)ab2);
  k_widen<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(w.ya, w.yb, ya, yb, n);
  return cuda_status(cudaGetLastError());
}

// ------------------------------------------------------------------ allocation-free search
// The working memory of fs_search_noalloc: one fixed array per device, alive
// until the process exits.  Host code never dereferences the symbol; it looks up
// the array's device address once per device and passes that address on.
static __device__ __align__(256) unsigned char g_noalloc_scratch[FS_NOALLOC_SCRATCH_BYTES];

static std::mutex g_noalloc_mu;
static unsigned char *g_noalloc_addr[256];

static fs_status noalloc_scratch(unsigned char **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return FS_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return FS_ERR_CUDA;
    }
    g_noalloc_addr[dev] = (unsigned char *)p;
  }
  *out = g_noalloc_addr[dev];
  return FS_OK;
}

fs_status search32_noalloc(fs_ctx *ctx, fs_seg *seg, const double *alpha, const double *delta, int nsky,
                           const double *f1, int nspin, float thr, float *F, int64_t nbins, fs_candidate *cand,
                           int64_t cap, int64_t *ncand, cudaStream_t st) {
  if (seg->d.precision != FS_PREC_F32 || nbins != seg->g.nfft / 2) return FS_ERR_UNSUPPORTED;
  FftShape sh;
  if (!fft_shape(seg->g.nfft, &sh)) return FS_ERR_SHAPE;
  const int64_t n = seg->g.n;
  const int n1max = (int)((n + sh.N2 - 1) / sh.N2);
  const int64_t npad = (int64_t)n1max * sh.N2;
  const int64_t stride = (npad + 63) & ~(int64_t)63;
  const int nblk = (int)((npad + 255) / 256);
  const int lag = 4, slots = 6;  // one sky per launch: a short ring suffices
  // layout inside the fixed array (one sky at a time)
  size_t off = 0;
  const size_t o_sky = off; off = align256(off + sizeof(SkyConst32));
  const size_t o_ya = off; off = align256(off + sizeof(float2) * stride);
  const size_t o_yb = off; off = align256(off + sizeof(float2) * stride);
  const size_t o_qq = off; off = align256(off + sizeof(float2) * stride);
  const size_t o_nm = off; off = align256(off + sizeof(float2));
  const size_t o_ab = off; off = align256(off + sizeof(double2));
  const size_t o_pa = off; off = align256(off + sizeof(double) * 2 * (size_t)nblk);
  const size_t o_z = off; off = align256(off + sizeof(float2) * 2 * (size_t)seg->g.nfft * slots);
  const size_t o_ct = off; off = align256(off + sizeof(unsigned) * (1 + 2 * (size_t)nspin));
  if (off > (size_t)FS_NOALLOC_SCRATCH_BYTES) return FS_ERR_SCRATCH;
  unsigned char *base = nullptr;
  fs_status s = noalloc_scratch(&base);
  if (s != FS_OK) return s;
  Ws32 w{};
  w.skyc = (SkyConst32 *)(base + o_sky);
  w.ya = (float2 *)(base + o_ya);
  w.yb = (float2 *)(base + o_yb);
  w.qq = (float2 *)(base + o_qq);
  w.norm = (float2 *)(base + o_nm);
  w.ab2 = (double2 *)(base + o_ab);
  w.partial = (double *)(base + o_pa);
  w.Z = (float2 *)(base + o_z);
  w.counters = (unsigned *)(base + o_ct);
  w.stride = stride;
  w.nblk_a1 = nblk;
  if (cudaMemsetAsync(ncand, 0, sizeof(int64_t), st) != cudaSuccess) return FS_ERR_CUDA;
  DemodArgs DA = demod_args(seg, w, npad);
  for (int g0 = 0; g0 < nsky; g0++) {
    if (sky_constants32(alpha + g0, delta + g0, 1, seg->g, ctx->det, w.skyc, st) != cudaSuccess) return FS_ERR_CUDA;
    if (launch_demod(DA, 1, nblk, seg->d.interp, st) != cudaSuccess) return FS_ERR_CUDA;
    k_demod_finalize<<<1, 256, 0, st>>>(w.partial, nblk, n, seg->g.dt, seg->g.S0, w.norm, w.ab2);
    Pass1Args p1{};
    p1.ya = w.ya;
    p1.yb = w.yb;
    p1.qq = w.qq;
    p1.sky_stride = w.stride;
    p1.f1 = f1;
    p1.nspin = nspin;
    p1.N2 = sh.N2;
    p1.n1max = n1max;
    p1.nfft = seg->g.nfft;
    p1.Z = w.Z;
    Pass2Args p2{};
    p2.Z = w.Z;
    p2.N1 = sh.N1;
    p2.N2 = sh.N2;
    p2.nfft = seg->g.nfft;
    p2.norm = w.norm;
    p2.nspin = nspin;
    p2.sky_base = g0;
    p2.F = F ? F + (int64_t)g0 * nspin * nbins : nullptr;
    p2.nbins = nbins;
    p2.thr = thr;
    p2.cand = cand;
    p2.cap = cap;
    p2.ncand = (unsigned long long *)ncand;
    p2.flags = ctx->d_flags;
    QueueArgs qa{};
    qa.ntm = nspin;
    queue_tiles(sh.N1, sh.N2, kPersistThreads, &qa.tiles1, &qa.tiles2);
    qa.kr = 1;
    qa.lag = lag;
    qa.slots = slots;
    qa.counter = w.counters;
    // the array keeps the previous call's contents: the queue counters start at zero
    if (cudaMemsetAsync(w.counters, 0, sizeof(unsigned) * (1 + 2 * (size_t)nspin), st) != cudaSuccess)
      return FS_ERR_CUDA;
    if (dispatch_passes(sh.N1, sh.N2, p1, p2, qa, st) != cudaSuccess) return FS_ERR_CUDA;
    ctx->launches += 4;
  }
  return FS_OK;
}

}  // namespace fs
