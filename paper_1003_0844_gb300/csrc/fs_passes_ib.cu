// Persistent transform launches with interbinning items (Eq. intbin, Sec. VI.B)
// for the default split of each transform length 2^12 .. 2^20 (and the other
// near-square split of 2^17), followed by the odd bins of the tile edges.
#include "fs_pass32.cuh"

namespace fs {

// Odd bins of the tile edges for the interbinning items: boundary b pairs the last
// row of tile b with the first row of tile b + 1 (for the last tile: row 0 at
// k2 + 1, or X(Nfft/2)); one thread per (template, boundary, k2).
__global__ void __launch_bounds__(256) k_interbin_edges(Pass2Args A, int ntm, int R, int tiles2) {
  const int64_t DP = A.N2 / 2;
  const int64_t total = (int64_t)ntm * tiles2 * DP;
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const bool ok = idx < total;
  float Fv = 0.f;
  uint32_t bin = 0;
  int sky = 0, spin = 0;
  if (ok) {
    const int tm = (int)(idx / (tiles2 * DP));
    const int64_t rem = idx - (int64_t)tm * tiles2 * DP;
    const int b = (int)(rem / DP);
    const int64_t k2 = rem - (int64_t)b * DP;
    sky = tm / A.nspin;
    spin = tm - sky * A.nspin;
    const float2 *eb = A.X + (int64_t)tm * A.eb_stride;
    const float2 la = eb[(int64_t)b * 4 * DP + 2 * DP + k2], lb = eb[(int64_t)b * 4 * DP + 3 * DP + k2];
    float2 ra, rb;
    if (b + 1 < tiles2) {
      ra = eb[(int64_t)(b + 1) * 4 * DP + k2];
      rb = eb[(int64_t)(b + 1) * 4 * DP + DP + k2];
    } else if (k2 + 1 < DP) {
      ra = eb[k2 + 1];
      rb = eb[DP + k2 + 1];
    } else {
      ra = eb[(int64_t)tiles2 * 4 * DP];
      rb = eb[(int64_t)tiles2 * 4 * DP + 1];
    }
    const float2 nrm = A.norm[sky];
    const float dax = ra.x - la.x, day = ra.y - la.y, dbx = rb.x - lb.x, dby = rb.y - lb.y;
    Fv = 0.5f * (fmaf(dax, dax, day * day) * nrm.x + fmaf(dbx, dbx, dby * dby) * nrm.y);
    bin = 2u * (uint32_t)((int64_t)b * R + R - 1 + A.N1 * k2) + 1u;
    if (A.F) A.F[(int64_t)tm * A.nbins + bin] = Fv;
  }
  const bool hit = ok && Fv > A.thr;
  const unsigned m = __ballot_sync(kFull, hit);
  if (!m) return;
  const int leader = __ffs(m) - 1;
  unsigned long long base = 0;
  if (lane == leader) base = atomicAdd(A.ncand, (unsigned long long)__popc(m));
  base = __shfl_sync(kFull, base, leader);
  if (hit) {
    const unsigned long long i = base + __popc(m & ((1u << lane) - 1u));
    if ((long long)i < A.cap) {
      fs_candidate c;
      c.sky = (uint32_t)(A.sky_base + sky);
      c.spin = (uint32_t)spin;
      c.bin = bin;
      c.F = Fv;
      A.cand[i] = c;
    } else {
      atomicOr(A.flags, ERRF_CAPACITY);
    }
  }
}

template <int P1, int Q1, int P2, int Q2>
static cudaError_t launch_ib(const Pass1Args &a1, const Pass2Args &a2, const QueueArgs &qa, cudaStream_t st) {
  constexpr int NT = kPersistThreads;
  constexpr int R = P2 == 32 ? (NT / 32) / 2 : (NT / 32) * (16 / P2), DP = P2 * Q2 / 2;
  // the item's rows (float2 [R][2][DP]) and F tile (float [DP][2R + 1]) fit the work area
  static_assert(2 * R * DP + (DP * (2 * R + 1) + 1) / 2 <=
                    persist_smem<P1, Q1, P2, Q2, NT>() / sizeof(float2) - P1 * Q1 - P2 * Q2,
                "interbinning tile exceeds the work area");
  cudaError_t e = launch_passes_am<P1, Q1, P2, Q2, NT, 0, true>(a1, a2, qa, st);
  if (e != cudaSuccess) return e;
  const int tiles2 = a2.N1 / R;
  const int64_t total = (int64_t)qa.ntm * tiles2 * (a2.N2 / 2);
  k_interbin_edges<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(a2, qa.ntm, R, tiles2);
  return cudaGetLastError();
}

cudaError_t dispatch_passes_ib(int N1, int N2, const Pass1Args &a1, const Pass2Args &a2, const QueueArgs &qa,
                               cudaStream_t st) {
  if (a1.vshift) return cudaErrorInvalidValue;
  switch (N1 * 4096 + N2) {
    case 64 * 4096 + 64: return launch_ib<8, 8, 8, 8>(a1, a2, qa, st);
    case 128 * 4096 + 64: return launch_ib<8, 16, 8, 8>(a1, a2, qa, st);
    case 128 * 4096 + 128: return launch_ib<8, 16, 8, 16>(a1, a2, qa, st);
    case 256 * 4096 + 128: return launch_ib<16, 16, 8, 16>(a1, a2, qa, st);
    case 256 * 4096 + 256: return launch_ib<16, 16, 16, 16>(a1, a2, qa, st);
    case 512 * 4096 + 256: return launch_ib<16, 32, 16, 16>(a1, a2, qa, st);
    case 256 * 4096 + 512: return launch_ib<16, 16, 16, 32>(a1, a2, qa, st);
    case 512 * 4096 + 512: return launch_ib<16, 32, 16, 32>(a1, a2, qa, st);
    case 1024 * 4096 + 512: return launch_ib<32, 32, 16, 32>(a1, a2, qa, st);
    case 1024 * 4096 + 1024: return launch_ib<32, 32, 32, 32>(a1, a2, qa, st);
  }
  return cudaErrorInvalidValue;
}

bool passes_ib_instantiated(int N1, int N2) {
  switch (N1 * 4096 + N2) {
    case 64 * 4096 + 64:
    case 128 * 4096 + 64:
    case 128 * 4096 + 128:
    case 256 * 4096 + 128:
    case 256 * 4096 + 256:
    case 512 * 4096 + 256:
    case 256 * 4096 + 512:
    case 512 * 4096 + 512:
    case 1024 * 4096 + 512:
    case 1024 * 4096 + 1024:
      return true;
  }
  return false;
}

}  // namespace fs
