// Transform passes of the FP32 search path (device code and launch templates),
// shared by the translation units that instantiate them per transform shape.
//
// Per template (sky, f1), the zero-padded transform of length
// Nfft = N1 * N2 runs in two passes (index n = N2 n1 + n2, bin k = k1 + N1 k2):
//  pass 1: multiply by the chirp exp(-2 pi i f1 Q_j), DFTs of length N1 over
//    n1 for a tile of columns n2 (both signals a and b), twiddle
//    exp(-2 pi i n2 k1 / Nfft), write Z[k1][n2];
//  pass 2: DFTs of length N2 over n2 for a tile of rows k1, then
//    F_k = 2/(S0 To) (|Fa_k|^2/<a^2> + |Fb_k|^2/<b^2>) (Eq. OS), threshold
//    compaction, and a transposed store of F in natural bin order.
// Each length-L DFT (L = P Q) is itself two register stages (DFT_P over the
// stride-Q samples, twiddle exp(-2 pi i b c / L), DFT_Q) with one exchange
// through shared memory.  Both passes run either as separate per-batch launches
// (k_pass1, k_pass2) or from one persistent work queue (k_passes).
#pragma once
#include "fs_internal.h"
#include "fs_model.cuh"
#include "fs_dft.cuh"

namespace fs {

constexpr unsigned kFull = 0xffffffffu;

// Division by a runtime divisor d through one 64-bit multiply: q = (n m) >> 48
// with m = ceil(2^48 / d) is exact for n < 2^31 and 1 <= d < 2^17 (the error
// n (m - 2^48/d) / 2^48 < 2^-17 < 1/d never reaches the next integer); larger d
// fall back to plain division.
struct FastDiv {
  uint32_t d;
  uint64_t m;  // 0: use plain division
};
inline FastDiv make_fastdiv(uint32_t d) {
  FastDiv f{d, 0};
  if (d >= 1 && d < (1u << 17)) f.m = ((uint64_t(1) << 48) + d - 1) / d;
  return f;
}
__device__ __forceinline__ int fdiv(int n, const FastDiv &f) {
  return f.m ? (int)(((uint64_t)(uint32_t)n * f.m) >> 48) : (int)((uint32_t)n / f.d);
}

// W_L^{b c} (L = P Q) stored by c then b, c < P, b < Q.
__device__ __forceinline__ void twiddle_matrix(float2 *twM, int P, int Q) {
  const int L = P * Q;
  for (int q = threadIdx.x; q < L; q += blockDim.x) {
    const int c = q / Q, b = q - c * Q;
    twM[q] = expm2pi((float)((b * c) & (L - 1)) * (1.0f / L));
  }
}

// ------------------------------------------------------------------ pass 1
struct Pass1Args {
  const float2 *ya, *yb, *qq;
  int64_t sky_stride;
  const float2 *f1df;  // spindowns as double-floats (hi, lo), converted once per search
  int nspin, tmpl0;
  FastDiv nspin_fd;  // division by nspin
  int N2, n1max;
  int64_t nfft;  // sub-transform length N1 N2
  // A template's transform of length Nfft = nfft << vshift (data no longer than
  // nfft) is split into 2^vshift sub-transforms of length nfft: sub-transform
  // s takes the samples times exp(-2 pi i s j / Nfft) and gives the bins
  // k = (m << vshift) + s (decimation in frequency).  Work items carry the
  // virtual template index (template << vshift) + s.
  int vshift;
  float inv_nfft_total;  // 1 / Nfft
  float2 *Z;  // [batch][2][N1][N2]
  // lattice templates (LAT items): f1df and the bin offset d per template of the group
  // (index sky * nspin + spin); the chirp gains exp(-2 pi i d j / Nfft)
  const double *bin_offset;
  // extents checked by debug builds: Z ring and per-sky series (elements), error flags
  int64_t z_elems, yq_elems;
  uint32_t *flags;
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
// N2T: N2 at compile time (0: A.N2 at run time); the sub-transform length is then P Q N2T.
// LAT: lattice templates (own f1 and bin offset per template, Pass1Args::bin_offset).
template <int P, int Q, int CW, int AM, int VS = 0, int N2T = 0, bool LAT = false>
__device__ __forceinline__ void pass1_item(const Pass1Args &A, int tm, int zs, int tile, float2 *xch,
                                           const float2 *twL) {
  constexpr int L = P * Q;
  constexpr int S = Q / P;
  constexpr int CS = 2 * CW;     // (column, signal) pairs
  static_assert(AM >= 2 && AM <= P && AM % 2 == 0, "rows with data come in chirp pairs");
  constexpr int TPW = 32 / CS;   // sub-DFT threads per warp
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int cs = lane % CS, col = cs % CW, sig = cs / CW;
  const int t = w * TPW + lane / CS;
  const int tr = tm >> VS, par = tm & ((1 << VS) - 1);
  const int sky = fdiv(tr, A.nspin_fd), spin = tr - sky * A.nspin;
  const int n2 = tile * CW + col;
  const float2 *y = (sig ? A.yb : A.ya) + sky * A.sky_stride;
  const float2 *qq = A.qq + sky * A.sky_stride;
  const float2 f1v = A.f1df[LAT ? tr : spin];
  const df32 f1{f1v.x, f1v.y};
  const float boff = LAT ? (float)A.bin_offset[tr] : 0.f;
  const int n1max = A.n1max;
  const int64_t N2 = N2T ? (int64_t)N2T : (int64_t)A.N2;

  float2 v[Q];
  // load y_j and the chirp exp(-2 pi i f1 Q_j); the two signal lanes of a
  // column share the chirp: each computes every other one and swaps.  All
  // loads of a b-slot are issued before any of them is used.
  sfor<0, S>([&](auto s) {
    const int b = t + P * s;
    float2 qv[AM / 2];
    sfor<0, AM / 2>([&](auto ap) {
      const int my = Q * (2 * ap + sig) + b;
      qv[ap] = (my < n1max && dbg_in(sky * A.sky_stride + my * N2 + n2, A.yq_elems, A.flags)) ? qq[my * N2 + n2]
                                                                                            : make_float2(0.f, 0.f);
    });
    sfor<0, P>([&](auto a) {
      const int na = Q * a + b;
      if constexpr (a < AM)
        v[s * P + a] = (na < n1max && dbg_in(sky * A.sky_stride + na * N2 + n2, A.yq_elems, A.flags))
                           ? y[na * N2 + n2]
                           : make_float2(0.f, 0.f);
      else v[s * P + a] = make_float2(0.f, 0.f);
    });
    sfor<0, AM / 2>([&](auto ap) {
      constexpr int a0 = 2 * ap, a1 = 2 * ap + 1;
      const int my = Q * (a0 + sig) + b;
      float2 cm = make_float2(0.f, 0.f);
      if (my < n1max) {
        float f = df_mul_frac(f1, df32{qv[ap].x, qv[ap].y});
        if (VS > 0 && par) {  // sub-transform shift: exact fraction (j < 2^24)
          f += (float)(par * (my * N2 + n2)) * A.inv_nfft_total;
          f -= rintf(f);
        }
        if constexpr (LAT) {  // bin offset d: d j / Nfft < 1 cycle, error ~ 1e-7 cycles
          f = fmaf(boff * (float)(my * N2 + n2), A.inv_nfft_total, f);
          f -= rintf(f);
        }
        cm = chirp_cycles(f);
      }
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
    // (a [c][b] table with compile-time offsets measured 5% slower here)
    sfor<1, P>([&](auto c) { v[s * P + c] = cmul(v[s * P + c], twL[(b * c) & (L - 1)]); });
    sfor<0, P>([&](auto c) { xch[(b * P + c) * CS + cs] = v[s * P + c]; });
  });
  __syncthreads();
  sfor<0, Q>([&](auto bb) { v[bb] = xch[(bb * P + t) * CS + cs]; });
  dft_inplace<Q>(v);  // v[d] = X[k1 = t + P d] of column n2
  // inter-pass twiddle exp(-2 pi i n2 k1 / Nfft): anchors every 16 d from the
  // hardware sine/cosine (argument reduced to half a turn), and an exactly
  // rounded step for the recurrence between anchors so errors do not build up
  const int64_t nf = N2T ? (int64_t)L * N2T : A.nfft;
  const float inv_nf = 1.0f / (float)nf;
  const float2 step = expm2pi((float)(((int64_t)n2 * P) & (nf - 1)) * inv_nf);
#ifdef FS_X2
  // 512-point columns (16 x 32): the twiddle w kept as (w.x, w.x) and (-w.y, w.y), so
  // that v w and the step w' = w step are two packed FP32 instructions per product.
  // Measured per shape: 0.9% faster on the 2-day transform and 1.5% on the lattice
  // search, but 2.1% slower for 1024-point columns and 0.4% for 256-point ones (a table
  // of twiddles kept that way measured slower everywhere).
  constexpr bool kPackedTw = P == 16 && Q == 32;
#else
  constexpr bool kPackedTw = false;
#endif
  if constexpr (kPackedTw) {
#ifdef FS_X2
    float2 wc, ws;
    const float2 sr = make_float2(step.x, step.x), sk = make_float2(step.y, -step.y);
    sfor<0, Q>([&](auto d) {
      if constexpr (d % 16 == 0) {
        const float f = (float)(((int64_t)n2 * (t + P * d)) & (nf - 1)) * inv_nf;
        const float2 w0 = chirp_cycles(f > 0.5f ? f - 1.0f : f);
        wc = make_float2(w0.x, w0.x);
        ws = make_float2(-w0.y, w0.y);
      } else {
        const float2 c1 = x2mul(wc, sr), s1 = x2mul(ws, sr), wc0 = wc;
        wc = x2fma(ws, sk, c1);           // (w'.x, w'.x)
        ws = x2fma(wc0, x2swap(sk), s1);  // (-w'.y, w'.y)
      }
      v[d] = x2fma(ws, x2swap(v[d]), x2mul(wc, v[d]));
    });
#endif
  } else {
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
  }
  float2 *Zs = A.Z + ((int64_t)zs * 2 + sig) * nf;
  sfor<0, Q>([&](auto d) {
    if (dbg_in(((int64_t)zs * 2 + sig) * nf + (int64_t)(t + P * d) * N2 + n2, A.z_elems, A.flags))
      Zs[(int64_t)(t + P * d) * N2 + n2] = v[d];
  });
}

template <int P, int Q, int CW, int AM, int VS>
__global__ void __launch_bounds__(P * 2 * CW, 2) k_pass1(Pass1Args A) {
  constexpr int L = P * Q;
  extern __shared__ float2 smem[];
  float2 *xch = smem;               // [Q][P][2 CW]
  float2 *twL = smem + L * 2 * CW;  // W_L^q
  const int tiles = A.N2 / CW;
  const int bt = blockIdx.x / tiles, tile = blockIdx.x - bt * tiles;
  for (int q = threadIdx.x; q < L; q += blockDim.x) twL[q] = expm2pi((float)q * (1.0f / L));
  __syncthreads();
  pass1_item<P, Q, CW, AM, VS>(A, A.tmpl0 + bt, bt, tile, xch, twL);
}

// ------------------------------------------------------------------ pass 2 + F epilogue
struct Pass2Args {
  const float2 *Z;
  int N1, N2;
  int64_t nfft;
  const float2 *norm;  // per sky of the group
  int nspin, tmpl0;
  FastDiv nspin_fd;    // division by nspin
  int vshift;          // sub-transforms per template (see Pass1Args)
  int sky_base;        // global index of the group's first sky
  float *F;            // NULL or F_out + (global template of the group's first template) * nbins
  int64_t nbins;       // F row length of one template (all its sub-transforms)
  float2 *X;           // XOUT items: complex bins [batch][2][nfft] in natural order;
                       // interbinning items: edge rows, eb_stride per template (pass2_item_ib)
  int64_t eb_stride;
  float thr;
  fs_candidate *cand;
  int64_t cap;
  unsigned long long *ncand;
  uint32_t *flags;
  // extents checked by debug builds: Z ring and F from A.F (elements)
  int64_t z_elems, f_elems;
};

// One pass-2 work item: template tm (within the group), row tile rt, reading Z
// slot zs.  Needs 32 * WARPS threads; work holds the exchange and F tile areas
// (pass2_work_floats2), twM the matrix W_L^{b c} stored by c then b.  Z is read
// past L1 (it may have been rewritten since an earlier item on this SM).
// Exchange layout of one sub-DFT: element (c, b) at c * (Q + 1) + b.  Writers
// (lanes along b) and readers (lanes along c: a stride of Q + 1 float2) both hit
// distinct banks, and every address is a per-thread base plus a compile-time
// offset.  (An XOR swizzle without padding saves 4% of the area but costs an
// integer operation per element and measured 2.3% slower on the 2-day transform.)
template <int P, int Q>
struct Xch2 {
  static constexpr int PITCH = Q + 1;
  static constexpr int SIZE = P * PITCH;
  static __device__ __forceinline__ int at(int c, int b) { return c * PITCH + b; }
};

// Drop the 128-byte L2 lines of one consumed Z row without writing them back to
// DRAM: the slot is rewritten by a later template before anything reads it
// again.  Called after a warp barrier that follows the first use of the loaded
// values (every lane's loads from the row have completed).
template <int L2, int T>
__device__ __forceinline__ void discard_row(const float2 *row, int t) {
  constexpr int LINES = L2 / 16;
  const char *rb = (const char *)row;
  for (int i = t; i < LINES; i += T) asm volatile("discard.global.L2 [%0], 128;" ::"l"(rb + 128 * i) : "memory");
}

// Pass-2 work item for 32-thread row DFTs (N2 = 1024): a warp holds one signal of
// one row (warps 2r, 2r+1: signals a, b of row r), so an item covers WARPS/2
// rows; the two signals' |X|^2 terms meet through the F tile.
template <int Q, int WARPS, bool FULLBINS, int VS, bool XOUT = false, int N1T = 0>
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
  const int tr = tm >> VS, par = tm & ((1 << VS) - 1);
  const int sky = fdiv(tr, A.nspin_fd), spin = tr - sky * A.nspin;
  constexpr int L2 = P * Q;
  const int64_t N1 = N1T ? (int64_t)N1T : (int64_t)A.N1;
  const int64_t nfft = N1T ? (int64_t)N1T * L2 : A.nfft;
  const int64_t zoff = ((int64_t)zs * 2 + sig) * nfft + (int64_t)k1 * L2;
  const float2 *z = A.Z + zoff;
  float2 v[Q];
  sfor<0, S>([&](auto s) {
    sfor<0, P>([&](auto a) {
      v[s * P + a] = dbg_in(zoff + Q * a + t + P * s, A.z_elems, A.flags) ? __ldcg(z + Q * a + t + P * s)
                                                                          : make_float2(0.f, 0.f);
    });
  });
  float2 *xw = work + w * XW;
  sfor<0, S>([&](auto s) {
    const int b = t + P * s;
    dft_inplace<P>(v + s * P);
    sfor<1, P>([&](auto c) { v[s * P + c] = cmul(v[s * P + c], twM[c * Q + b]); });
    sfor<0, P>([&](auto c) { xw[X::at(c, b)] = v[s * P + c]; });
  });
  __syncwarp();
  if constexpr (!XOUT) {
    if (dbg_in(zoff + L2 - 1, A.z_elems, A.flags)) discard_row<L2, 32>(z, t);
  }
  sfor<0, Q>([&](auto bb) { v[bb] = xw[X::at(t, bb)]; });
  __syncthreads();  // every warp is done with the exchange area (reused for the F tile)
  dft_inplace<Q, Q, D>(v);  // v[d] = X[k2 = t + P d] of row k1 (d < D)
  if constexpr (XOUT) {
    float2 *Xo = A.X + ((int64_t)zs * 2 + sig) * nfft + k1;
    sfor<0, D>([&](auto d) { Xo[N1 * (t + P * d)] = v[d]; });
    return;
  }
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
            c.bin = (uint32_t)(((k1 + N1 * k2) << VS) + par);
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
  // VS = 0: template row plus the item's first row; VS > 0: interleaved sub-transform bins
  float *Fo = VS == 0 ? A.F + (int64_t)tm * A.nbins + rt * R : A.F + (int64_t)tr * A.nbins + par;
  for (int idx = threadIdx.x; idx < K2 * R; idx += blockDim.x) {
    const int k2 = idx / R, r = idx - k2 * R;
    const int64_t fo = VS == 0 ? r + N1 * k2 : ((rt * R + r + N1 * k2) << VS);
    if (dbg_in((Fo - A.F) + fo, A.f_elems, A.flags)) __stcs(Fo + fo, Fs[k2 * (R + 1) + r]);
  }
}

// ALIAS_F: the F tile reuses the exchange area (one more barrier, less shared memory).
// N1T: N1 at compile time (0: A.N1 at run time); the sub-transform length is then N1T P Q.
template <int P, int Q, int WARPS, bool FULLBINS, bool ALIAS_F = false, int VS = 0, bool XOUT = false, int N1T = 0>
__device__ __forceinline__ void pass2_item(const Pass2Args &A, int tm, int zs, int rt, float2 *work,
                                           const float2 *twM) {
  if constexpr (P == 32) {
    pass2_item_wide<Q, WARPS, FULLBINS, VS, XOUT, N1T>(A, tm, zs, rt, work, twM);
    return;
  }
  constexpr int T = P, G = (P <= 16 ? 16 / P : 1), R = WARPS * G, S = Q / P;
  constexpr int D = FULLBINS ? Q : Q / 2;  // d values with k2 = t + P d in the output band
  using X = Xch2<P, Q>;
  constexpr int XW = X::SIZE;              // exchange float2s per sub-DFT
  constexpr int FPITCH = R + 1;  // odd pitch: conflict-free column writes
  float *Fs = (float *)(ALIAS_F ? work : work + WARPS * 2 * G * XW);  // [D*P][FPITCH]
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int t = lane % T, sig = (lane / T) & 1, gr = lane / (2 * T);
  const int row = w * G + gr;
  const int k1 = rt * R + row;
  const int tr = tm >> VS, par = tm & ((1 << VS) - 1);
  const int sky = fdiv(tr, A.nspin_fd), spin = tr - sky * A.nspin;
  constexpr int L2 = P * Q;
  const int64_t N1 = N1T ? (int64_t)N1T : (int64_t)A.N1;
  const int64_t nfft = N1T ? (int64_t)N1T * L2 : A.nfft;
  const int64_t zoff = ((int64_t)zs * 2 + sig) * nfft + (int64_t)k1 * L2;
  const float2 *z = A.Z + zoff;
  float2 v[Q];
  sfor<0, S>([&](auto s) {
    sfor<0, P>([&](auto a) {
      v[s * P + a] = dbg_in(zoff + Q * a + t + P * s, A.z_elems, A.flags) ? __ldcg(z + Q * a + t + P * s)
                                                                          : make_float2(0.f, 0.f);
    });
  });
  float2 *xw = work + (w * 2 * G + (sig + 2 * gr)) * XW;
  sfor<0, S>([&](auto s) {
    const int b = t + P * s;
    dft_inplace<P>(v + s * P);
    // W_L^{b c} stored by c then b: lanes read consecutive entries (no bank conflicts)
    sfor<1, P>([&](auto c) { v[s * P + c] = cmul(v[s * P + c], twM[c * Q + b]); });
    sfor<0, P>([&](auto c) { xw[X::at(c, b)] = v[s * P + c]; });
  });
  __syncwarp();
  if constexpr (!XOUT) {
    if (dbg_in(zoff + L2 - 1, A.z_elems, A.flags)) discard_row<L2, T>(z, t);
  }
  sfor<0, Q>([&](auto bb) { v[bb] = xw[X::at(t, bb)]; });
  if constexpr (ALIAS_F) __syncthreads();  // every warp is done with the exchange area
  dft_inplace<Q, Q, (FULLBINS ? Q : Q / 2)>(v);  // v[d] = X[k2 = t + P d] of row k1 (d < D)
  if constexpr (XOUT) {
    float2 *Xo = A.X + ((int64_t)zs * 2 + sig) * nfft + k1;
    sfor<0, D>([&](auto d) { Xo[N1 * (t + P * d)] = v[d]; });
    return;
  }
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
    Fs[k2 * FPITCH + row] = Fv;
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
          c.bin = (uint32_t)(((k1 + N1 * k2) << VS) + par);
          c.F = Fv;
          A.cand[idx] = c;
        } else {
          atomicOr(A.flags, ERRF_CAPACITY);
        }
      }
    }
  });
  // (storing each warp's F values directly, without the tile and its two barriers,
  // measured 16% slower: scattered 4-byte stores)
  if (A.F == nullptr) return;
  __syncthreads();
  // VS = 0: template row plus the item's first row; VS > 0: interleaved sub-transform bins
  float *Fo = VS == 0 ? A.F + (int64_t)tm * A.nbins + rt * R : A.F + (int64_t)tr * A.nbins + par;
  constexpr int K2 = D * P;
  for (int idx = threadIdx.x; idx < K2 * R; idx += blockDim.x) {
    const int k2 = idx / R, r = idx - k2 * R;
    const int64_t fo = VS == 0 ? r + N1 * k2 : ((rt * R + r + N1 * k2) << VS);
    if (dbg_in((Fo - A.F) + fo, A.f_elems, A.flags)) __stcs(Fo + fo, Fs[k2 * FPITCH + r]);
  }
}

// Interbinning pass-2 work item (Eq. intbin, Sec. VI.B) for P <= 16: F on the
// half-bin grid j = 2k, 2k + 1 of the band k < Nfft/2 for the R rows k1 of tile
// rt.  Even j from X(k); odd j from (X(k+1) - X(k)) / sqrt 2, where X(k+1) sits in
// row k1 + 1 of the same k2 (k = k1 + N1 k2).  The tile's last row pairs with the
// next tile's first row (the last tile's with row 0 at k2 + 1), so every item
// stores its first and last rows in A.X (per template, eb_stride float2:
// [tiles2][first a, first b, last a, last b][N2/2], then X(Nfft/2) of a and b)
// and k_interbin_edges forms those odd bins after the launch.  X(Nfft/2) =
// sum_n2 Z[0][n2] (-1)^n2 comes from row 0 before its transform.
// For P = 32 (1024-point rows) a warp holds one signal of one row, as in
// pass2_item_wide: warps 2r, 2r + 1 hold signals a, b of row r.
template <int P, int Q, int WARPS>
__device__ __forceinline__ void pass2_item_ib(const Pass2Args &A, int tm, int zs, int rt, float2 *work,
                                              const float2 *twM) {
  constexpr bool WIDE = (P == 32);
  constexpr int T = P, G = WIDE ? 1 : 16 / P, R = WIDE ? WARPS / 2 : WARPS * G, S = Q / P, D = Q / 2, DP = D * P,
                FP = 2 * R + 1;
  using X = Xch2<P, Q>;
  constexpr int XW = X::SIZE;
  static_assert(DP >= 32 && (DP & (DP - 1)) == 0, "a warp's F items share one row");
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int t = WIDE ? lane : lane % T;
  const int sig = WIDE ? (w & 1) : (lane / T) & 1;
  const int gr = WIDE ? 0 : lane / (2 * T);
  const int row = WIDE ? (w >> 1) : w * G + gr;
  const int k1 = rt * R + row;
  const int sky = fdiv(tm, A.nspin_fd), spin = tm - sky * A.nspin;
  constexpr int L2 = P * Q;
  const int64_t N1 = A.N1, nfft = A.nfft;
  const int tiles2 = (int)(N1 / R);
  const int64_t zoff = ((int64_t)zs * 2 + sig) * nfft + (int64_t)k1 * L2;
  const float2 *z = A.Z + zoff;
  float2 v[Q];
  sfor<0, S>([&](auto s) {
    sfor<0, P>([&](auto a) {
      v[s * P + a] = dbg_in(zoff + Q * a + t + P * s, A.z_elems, A.flags) ? __ldcg(z + Q * a + t + P * s)
                                                                          : make_float2(0.f, 0.f);
    });
  });
  float2 *eb = A.X + (int64_t)tm * A.eb_stride;
  if (rt == 0 && (WIDE ? w < 2 : w == 0)) {  // row k1 = 0 (gr = 0): X(Nfft/2); n2 = Q a + t + P s has t's parity
    float2 sum = make_float2(0.f, 0.f);
    sfor<0, Q>([&](auto i) { sum = cadd(sum, v[i]); });
    if (t & 1) sum = make_float2(-sum.x, -sum.y);
    for (int o = T / 2; o > 0; o >>= 1) {
      sum.x += __shfl_xor_sync(kFull, sum.x, o);
      sum.y += __shfl_xor_sync(kFull, sum.y, o);
    }
    if (gr == 0 && t == 0) eb[(int64_t)tiles2 * 4 * DP + sig] = sum;
  }
  float2 *xw = WIDE ? work + w * XW : work + (w * 2 * G + (sig + 2 * gr)) * XW;
  sfor<0, S>([&](auto s) {
    const int b = t + P * s;
    dft_inplace<P>(v + s * P);
    sfor<1, P>([&](auto c) { v[s * P + c] = cmul(v[s * P + c], twM[c * Q + b]); });
    sfor<0, P>([&](auto c) { xw[X::at(c, b)] = v[s * P + c]; });
  });
  __syncwarp();
  if (dbg_in(zoff + L2 - 1, A.z_elems, A.flags)) discard_row<L2, T>(z, t);
  sfor<0, Q>([&](auto bb) { v[bb] = xw[X::at(t, bb)]; });
  __syncthreads();  // every warp is done with the exchange area (reused for the rows and the F tile)
  dft_inplace<Q, Q, D>(v);  // v[d] = X[k2 = t + P d] of row k1 (d < D)
  float2 *Xs = work;                         // [R][2][DP]
  float *Fs = (float *)(work + 2 * R * DP);  // [DP][FP]: even and odd F of the tile's rows
  sfor<0, D>([&](auto d) { Xs[(row * 2 + sig) * DP + t + P * d] = v[d]; });
  __syncthreads();
  for (int i = threadIdx.x; i < 2 * DP; i += blockDim.x) {
    eb[(int64_t)rt * 4 * DP + i] = Xs[i];
    eb[(int64_t)rt * 4 * DP + 2 * DP + i] = Xs[(R - 1) * 2 * DP + i];
  }
  const float2 nrm = A.norm[sky];
  const unsigned lt_mask = (1u << lane) - 1u;
  auto emit = [&](bool hit, float Fv, uint32_t bin) {  // warp-uniform call: ballot compaction
    const unsigned m = __ballot_sync(kFull, hit);
    if (!m) return;
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
        c.bin = bin;
        c.F = Fv;
        A.cand[idx] = c;
      } else {
        atomicOr(A.flags, ERRF_CAPACITY);
      }
    }
  };
  static_assert((R * DP) % 32 == 0, "whole warps per F loop");
  for (int idx = threadIdx.x; idx < R * DP; idx += blockDim.x) {
    const int r = idx / DP, k2 = idx - r * DP;  // r is the same across a warp
    const float2 a0 = Xs[(r * 2) * DP + k2], b0 = Xs[(r * 2 + 1) * DP + k2];
    const float Fe = fmaf(a0.x, a0.x, a0.y * a0.y) * nrm.x + fmaf(b0.x, b0.x, b0.y * b0.y) * nrm.y;
    Fs[k2 * FP + 2 * r] = Fe;
    const uint32_t j = 2u * (uint32_t)(rt * R + r + N1 * k2);
    emit(Fe > A.thr, Fe, j);
    if (r < R - 1) {
      const float2 a1 = Xs[(r * 2 + 2) * DP + k2], b1 = Xs[(r * 2 + 3) * DP + k2];
      const float dax = a1.x - a0.x, day = a1.y - a0.y, dbx = b1.x - b0.x, dby = b1.y - b0.y;
      const float Fo = 0.5f * (fmaf(dax, dax, day * day) * nrm.x + fmaf(dbx, dbx, dby * dby) * nrm.y);
      Fs[k2 * FP + 2 * r + 1] = Fo;
      emit(Fo > A.thr, Fo, j + 1u);
    }
  }
  if (A.F == nullptr) return;
  __syncthreads();
  // bins j = 2 rt R + q + 2 N1 k2, q < 2R: runs of 2R floats; the last odd one is the edge kernel's
  float *Fout = A.F + (int64_t)tm * A.nbins + 2 * rt * R;
  for (int idx = threadIdx.x; idx < 2 * R * DP; idx += blockDim.x) {
    const int k2 = idx / (2 * R), q = idx - k2 * (2 * R);
    if (q != 2 * R - 1 && dbg_in((Fout - A.F) + q + 2 * N1 * k2, A.f_elems, A.flags))
      __stcs(Fout + q + 2 * N1 * k2, Fs[k2 * FP + q]);
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


template <int P, int Q, int WARPS, bool FULLBINS, int VS, bool XOUT = false>
__global__ void __launch_bounds__(32 * WARPS, 2) k_pass2(Pass2Args A) {
  constexpr int R = P <= 16 ? WARPS * (16 / P) : WARPS / 2;
  extern __shared__ float2 smem[];
  float2 *twM = smem;
  float2 *work = smem + P * Q;
  const int rtiles = A.N1 / R;
  const int bt = blockIdx.x / rtiles, rt = blockIdx.x - bt * rtiles;
  twiddle_matrix(twM, P, Q);
  __syncthreads();
  pass2_item<P, Q, WARPS, FULLBINS, false, VS, XOUT>(A, A.tmpl0 + bt, bt, rt, work, twM);
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
  FastDiv ipr_fd, slots_fd;  // division by kr (tiles1 + tiles2) and by slots
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

// IB: pass-2 items are interbinning items (pass2_item_ib); LAT: pass-1 items of
// lattice templates.
template <int P1, int Q1, int AM, int P2, int Q2, int NT, int MINB, int VS, bool IB = false, bool LAT = false>
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
  // items per template of each pass, fixed by the shape (the host's queue_tiles agrees)
  constexpr int T1 = (P2 * Q2) / CW;
  constexpr int T2 = (P1 * Q1) / (P2 <= 16 ? (NT / 32) * (16 / P2) : (NT / 32) / 2);
  const int ipr = kr * (T1 + T2);
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
    const int r = fdiv(it, Qa.ipr_fd);
    const int jr = it - r * ipr;
    d.is1 = jr < kr * T1;
    if (d.is1) {
      const int k = jr / T1;
      d.j = jr - k * T1;
      d.tm = r * kr + k;
    } else {
      const int j2 = jr - kr * T1;
      const int k = j2 / T2;
      d.j = T1 + (j2 - k * T2);
      d.tm = (r - Qa.lag) * kr + k;
    }
    d.valid = it < total && d.tm >= 0 && d.tm < Qa.ntm;
    return d;
  };
  auto dep_met = [&](const Item &d) {  // thread 0 only
    if (!d.valid) return true;
    if (d.is1) return d.tm < Qa.slots || ld_acquire(done2 + (d.tm - Qa.slots)) >= (unsigned)T2;
    return ld_acquire(done1 + d.tm) >= (unsigned)T1;
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
            if (d.tm >= Qa.slots) wait_at_least(done2 + (d.tm - Qa.slots), T2, A2.flags);
          } else {
            wait_at_least(done1 + d.tm, T1, A2.flags);
          }
        }
        __syncthreads();
      }
      const int zs = d.tm - fdiv(d.tm, Qa.slots_fd) * Qa.slots;
      // N1 compiled into the second pass (0.5% faster); N2 in the first pass measured slower
      constexpr int N1C = P1 * Q1;
      if (d.is1) pass1_item<P1, Q1, CW, AM, VS, 0, LAT>(A1, d.tm, zs, d.j, work, twL);
      else if constexpr (IB) pass2_item_ib<P2, Q2, NT / 32>(A2, d.tm, zs, d.j - T1, work, twM);
      else pass2_item<P2, Q2, NT / 32, false, true, VS, false, N1C>(A2, d.tm, zs, d.j - T1, work, twM);
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

// ------------------------------------------------------------------ launch templates
constexpr int kPass2Warps = 8;  // warps per pass-2 CTA

template <int P, int Q>
static size_t pass1_smem() { return sizeof(float2) * ((size_t)P * Q * 2 * (256 / (2 * P)) + (size_t)P * Q); }
template <int P, int Q, bool FULL>
static size_t pass2_smem() {
  return sizeof(float2) * ((size_t)P * Q + pass2_work_floats2<P, Q, kPass2Warps, FULL>());
}

template <int P, int Q, int VS = 0>
static cudaError_t launch_pass1(const Pass1Args &a, int nb, cudaStream_t st) {
  size_t sm = pass1_smem<P, Q>();
  constexpr int CW = 256 / (2 * P);
  auto kern = (a.n1max <= P * Q / 2) ? k_pass1<P, Q, CW, P / 2, VS> : k_pass1<P, Q, CW, P, VS>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  kern<<<nb * (a.N2 / CW), P * 2 * CW, sm, st>>>(a);
  return cudaGetLastError();
}
template <int P, int Q, bool FULL, int VS = 0, bool XOUT = false>
static cudaError_t launch_pass2(const Pass2Args &a, int nb, cudaStream_t st) {
  size_t sm = pass2_smem<P, Q, FULL>();
  auto kern = k_pass2<P, Q, kPass2Warps, FULL, VS, XOUT>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  constexpr int R = P <= 16 ? kPass2Warps * (16 / P) : kPass2Warps / 2;
  kern<<<nb * (a.N1 / R), 32 * kPass2Warps, sm, st>>>(a);
  return cudaGetLastError();
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

template <int P1, int Q1, int AM, int P2, int Q2, int NT, int VS, bool IB = false, bool LAT = false>
static cudaError_t launch_passes_t(const Pass1Args &a1, const Pass2Args &a2, const QueueArgs &qa, cudaStream_t st) {
  constexpr int MINB = persist_minb<P1, Q1, P2, Q2, NT>();
  const size_t sm = persist_smem<P1, Q1, P2, Q2, NT>();
  auto kern = k_passes<P1, Q1, AM, P2, Q2, NT, MINB, VS, IB, LAT>;
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

// VS: sub-transforms per template (2^VS) compiled in; only the 2^20 split is
// built with VS = 1 (the 2^21 transform).
// AMQ > 0: also build the variant for data in the rows n1 < AMQ Q1 (AMQ even, < P1/2),
// whose first-pass DFTs skip the pairs known to be zero.
template <int P1, int Q1, int P2, int Q2, int NT, int VS = 0, bool IB = false, bool LAT = false, int AMQ = 0>
static cudaError_t launch_passes_am(const Pass1Args &a1, const Pass2Args &a2, const QueueArgs &qa, cudaStream_t st) {
  if (a1.vshift != VS) return cudaErrorInvalidValue;
  if constexpr (AMQ > 0) {
    static_assert(AMQ % 2 == 0 && 2 * AMQ < P1, "a pruned variant below the half");
    if (a1.n1max <= AMQ * Q1) return launch_passes_t<P1, Q1, AMQ, P2, Q2, NT, VS, IB, LAT>(a1, a2, qa, st);
  }
  if (a1.n1max <= P1 * Q1 / 2) return launch_passes_t<P1, Q1, P1 / 2, P2, Q2, NT, VS, IB, LAT>(a1, a2, qa, st);
  return launch_passes_t<P1, Q1, P1, P2, Q2, NT, VS, IB, LAT>(a1, a2, qa, st);
}

// Work-item geometry of the persistent kernel for NT threads per CTA.
static inline void queue_tiles(int N1, int N2, int NT, int *tiles1, int *tiles2) {
  const int P1 = N1 <= 128 ? 8 : (N1 <= 512 ? 16 : 32);
  const int P2 = N2 <= 128 ? 8 : (N2 <= 512 ? 16 : 32);
  *tiles1 = N2 / (NT / (2 * P1));
  *tiles2 = N1 / (P2 <= 16 ? (NT / 32) * (16 / P2) : (NT / 32) / 2);
}

// 256 threads (2 CTAs per SM): measured faster than 128 threads with half-size items.
constexpr int kPersistThreads = 256;

// Per-shape dispatch, one translation unit per group of shapes.
cudaError_t dispatch_pass1(int N1, const Pass1Args &a, int nb, cudaStream_t st);
cudaError_t dispatch_pass2(int N2, bool full, const Pass2Args &a, int nb, cudaStream_t st);
// Pass 2 storing the complex bins (all Nfft, natural order) in a.X instead of F.
cudaError_t dispatch_pass2x(int N2, const Pass2Args &a, int nb, cudaStream_t st);
// Interbinning epilogue (Eq. intbin) over nb templates of a batch from a.X.
cudaError_t launch_interbin(const Pass2Args &a, int nb, cudaStream_t st);
// Persistent launch with interbinning items for the default split N1 x N2 of
// 2^12 .. 2^20 (also 256 x 512), and the edge bins after it (k_interbin_edges);
// cudaErrorInvalidValue for another split (passes_ib_instantiated is false).
cudaError_t dispatch_passes_ib(int N1, int N2, const Pass1Args &a1, const Pass2Args &a2, const QueueArgs &qa,
                               cudaStream_t st);
bool passes_ib_instantiated(int N1, int N2);
// Persistent launch of lattice templates (LAT items) for the default split of
// 2^12 .. 2^20; cudaErrorInvalidValue for another split.
cudaError_t dispatch_passes_lat(int N1, int N2, const Pass1Args &a1, const Pass2Args &a2, const QueueArgs &qa,
                                cudaStream_t st);
bool passes_lat_instantiated(int N1, int N2);
// Per-template stride (float2) of the interbinning items' edge rows.
inline int64_t ib_edge_stride(int N1, int N2, int NT) {
  const int P2 = N2 <= 128 ? 8 : (N2 <= 512 ? 16 : 32);
  const int R = P2 == 32 ? (NT / 32) / 2 : (NT / 32) * (16 / P2);
  return (int64_t)(N1 / R) * 4 * (N2 / 2) + 2;
}
// Persistent launch for an N1 x N2 split; cudaErrorInvalidValue for a split
// the library does not instantiate (split_instantiated is false).
cudaError_t dispatch_passes(int N1, int N2, const Pass1Args &a1, const Pass2Args &a2, const QueueArgs &qa,
                            cudaStream_t st);
cudaError_t dispatch_passes_small(int N1, int N2, const Pass1Args &a1, const Pass2Args &a2, const QueueArgs &qa,
                                  cudaStream_t st);
cudaError_t dispatch_passes_mid(int N1, int N2, const Pass1Args &a1, const Pass2Args &a2, const QueueArgs &qa,
                                cudaStream_t st);
cudaError_t dispatch_passes_large(int N1, int N2, const Pass1Args &a1, const Pass2Args &a2, const QueueArgs &qa,
                                  cudaStream_t st);
bool split_instantiated(int N1, int N2);
// CTAs per SM the persistent kernel of a split is compiled for (0: not instantiated).
int passes_blocks_per_sm(int N1, int N2);
int passes_blocks_per_sm_small(int N1, int N2);
int passes_blocks_per_sm_mid(int N1, int N2);
int passes_blocks_per_sm_large(int N1, int N2);

// ------------------------------------------------------------------ host-side configuration
struct FftShape {
  int N1, N2;
};
// Shape of the persistent queue: templates per round, lag (rounds) and Z slots.
struct QueueShape {
  int kr, lag, slots, tiles1, tiles2;
};
// Resolved launch configuration of one FP32 search of one segment.
struct Cfg32 {
  FftShape sh;     // split of the sub-transform
  int vshift;      // 2^vshift sub-transforms per template
  int64_t nsub;    // sub-transform length N1 N2
  int n1max;       // rows n1 that hold data
  int64_t npad;    // n1max N2: per-sky series length
  int G;           // skies per group
  bool full;       // F on all Nfft bins (per-batch launches)
  bool persistent; // both passes from one work queue
  bool interbin;   // F on the half-bin grid by interbinning (per-batch launches)
  QueueShape qs;
  int B;           // Z slots of the workspace
};
struct Ws32 {
  SkyConst32 *skyc;
  float2 *ya, *yb, *qq, *norm;
  double2 *ab2;
  float2 *partial; // per-block sums of a^2, b^2 of the demodulation
  float2 *f1df;    // spindowns (per template for lattice searches) as double-floats
  float2 *Z;
  float2 *X;       // interbinning: complex bins of a batch [B][2][nsub]
  unsigned *counters;
  int64_t stride;
  int nblk_a1;
  // debug builds: guard words before and after the Z ring and after the counters
  uint32_t *guard[3];
};
fs_status config32(const fs_ctx *ctx, const fs_seg *seg, int nsky, int64_t nbins, Cfg32 *c);
// Lay out (and, if may_alloc, grow) context workspace `slot` for a search.
fs_status workspace32(fs_ctx *ctx, int slot, const fs_seg *seg, const Cfg32 &c, int nsky, int nspin,
                      bool may_alloc, cudaStream_t st, Ws32 *w);
// Enqueue one search on `st` with a laid-out workspace; allocates nothing.
// lat_offset: NULL, or lattice templates (f1 and lat_offset per template, nsky x nspin).
fs_status search32_run(fs_ctx *ctx, fs_seg *seg, const Cfg32 &c, const Ws32 &w, const double *alpha,
                       const double *delta, int nsky, const double *f1, int nspin, float thr, float *F,
                       int64_t nbins, fs_candidate *cand, int64_t cap, int64_t *ncand, cudaStream_t st,
                       const double *lat_offset = nullptr);

}  // namespace fs
