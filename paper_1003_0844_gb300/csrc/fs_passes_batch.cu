// Per-batch launches of the two transform passes (used when F is wanted on
// all Nfft bins).
#include "fs_pass32.cuh"

namespace fs {

// Sub-transforms (vshift = 1) exist only for the 2^20 split 1024 x 1024.
cudaError_t dispatch_pass1(int N1, const Pass1Args &a, int nb, cudaStream_t st) {
  if (a.vshift) return (a.vshift == 1 && N1 == 1024) ? launch_pass1<32, 32, 1>(a, nb, st) : cudaErrorInvalidValue;
  switch (N1) {
    case 64: return launch_pass1<8, 8>(a, nb, st);
    case 128: return launch_pass1<8, 16>(a, nb, st);
    case 256: return launch_pass1<16, 16>(a, nb, st);
    case 512: return launch_pass1<16, 32>(a, nb, st);
    case 1024: return launch_pass1<32, 32>(a, nb, st);
  }
  return cudaErrorInvalidValue;
}
cudaError_t dispatch_pass2(int N2, bool full, const Pass2Args &a, int nb, cudaStream_t st) {
  if (a.vshift) {
    if (a.vshift != 1 || N2 != 1024) return cudaErrorInvalidValue;
    return full ? launch_pass2<32, 32, true, 1>(a, nb, st) : launch_pass2<32, 32, false, 1>(a, nb, st);
  }
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

cudaError_t dispatch_pass2x(int N2, const Pass2Args &a, int nb, cudaStream_t st) {
  if (a.vshift) return cudaErrorInvalidValue;
  switch (N2) {
    case 64: return launch_pass2<8, 8, true, 0, true>(a, nb, st);
    case 128: return launch_pass2<8, 16, true, 0, true>(a, nb, st);
    case 256: return launch_pass2<16, 16, true, 0, true>(a, nb, st);
    case 512: return launch_pass2<16, 32, true, 0, true>(a, nb, st);
    case 1024: return launch_pass2<32, 32, true, 0, true>(a, nb, st);
  }
  return cudaErrorInvalidValue;
}

// F on the half-bin grid j < Nfft of template tmpl0 + blockIdx.y: even j = 2k from
// X(k), odd j = 2k + 1 from X(k + 1/2) ~ (X(k+1) - X(k)) / sqrt(2) (Eq. intbin),
// then the threshold compaction with bin index j.
__global__ void __launch_bounds__(256) k_interbin(Pass2Args A) {
  const int bt = blockIdx.y;
  const int tm = A.tmpl0 + bt;
  const int sky = tm / A.nspin, spin = tm - sky * A.nspin;
  const int64_t nb = A.nfft / 2;
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const float2 nrm = A.norm[sky];
  float Fe = 0.f, Fo = 0.f;
  const bool ok = k < nb;
  if (ok) {
    const float2 *Xa = A.X + (int64_t)bt * 2 * A.nfft, *Xb = Xa + A.nfft;
    const float2 a0 = Xa[k], a1 = Xa[k + 1], b0 = Xb[k], b1 = Xb[k + 1];
    const float dax = a1.x - a0.x, day = a1.y - a0.y, dbx = b1.x - b0.x, dby = b1.y - b0.y;
    Fe = fmaf(a0.x, a0.x, a0.y * a0.y) * nrm.x + fmaf(b0.x, b0.x, b0.y * b0.y) * nrm.y;
    Fo = 0.5f * (fmaf(dax, dax, day * day) * nrm.x + fmaf(dbx, dbx, dby * dby) * nrm.y);
    if (A.F) reinterpret_cast<float2 *>(A.F + (int64_t)tm * A.nbins)[k] = make_float2(Fe, Fo);
  }
  for (int par = 0; par < 2; par++) {
    const float Fv = par ? Fo : Fe;
    const bool hit = ok && Fv > A.thr;
    const unsigned m = __ballot_sync(kFull, hit);
    if (!m) continue;
    const int leader = __ffs(m) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(A.ncand, (unsigned long long)__popc(m));
    base = __shfl_sync(kFull, base, leader);
    if (hit) {
      const unsigned long long idx = base + __popc(m & ((1u << lane) - 1u));
      if ((long long)idx < A.cap) {
        fs_candidate c;
        c.sky = (uint32_t)(A.sky_base + sky);
        c.spin = (uint32_t)spin;
        c.bin = (uint32_t)(2 * k + par);
        c.F = Fv;
        A.cand[idx] = c;
      } else {
        atomicOr(A.flags, ERRF_CAPACITY);
      }
    }
  }
}

cudaError_t launch_interbin(const Pass2Args &a, int nb, cudaStream_t st) {
  const int64_t nbins = a.nfft / 2;
  k_interbin<<<dim3((unsigned)((nbins + 255) / 256), nb), 256, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace fs
