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

}  // namespace fs
