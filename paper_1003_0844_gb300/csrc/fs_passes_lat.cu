// Persistent transform launches for lattice templates (Sec. IV: lines of the
// constrained lattice along a0, each with its own spindown and bin offset) for the
// default split of each transform length 2^12 .. 2^20; 2^21 in fs_passes_lat_wide.cu.
#include "fs_pass32.cuh"

namespace fs {

// the 2^21 transform, two 2^20 sub-transforms per template (fs_passes_lat_wide.cu)
cudaError_t dispatch_passes_lat_wide(int N1, int N2, const Pass1Args &a1, const Pass2Args &a2, const QueueArgs &qa,
                                     cudaStream_t st);

cudaError_t dispatch_passes_lat(int N1, int N2, const Pass1Args &a1, const Pass2Args &a2, const QueueArgs &qa,
                                cudaStream_t st) {
  constexpr int NT = kPersistThreads;
  if (!a1.bin_offset) return cudaErrorInvalidValue;
  if (a1.vshift) return dispatch_passes_lat_wide(N1, N2, a1, a2, qa, st);
  switch (N1 * 4096 + N2) {
    case 64 * 4096 + 64: return launch_passes_am<8, 8, 8, 8, NT, 0, false, true>(a1, a2, qa, st);
    case 128 * 4096 + 64: return launch_passes_am<8, 16, 8, 8, NT, 0, false, true>(a1, a2, qa, st);
    case 128 * 4096 + 128: return launch_passes_am<8, 16, 8, 16, NT, 0, false, true>(a1, a2, qa, st);
    case 256 * 4096 + 128: return launch_passes_am<16, 16, 8, 16, NT, 0, false, true>(a1, a2, qa, st);
    case 256 * 4096 + 256: return launch_passes_am<16, 16, 16, 16, NT, 0, false, true>(a1, a2, qa, st);
    case 512 * 4096 + 256: return launch_passes_am<16, 32, 16, 16, NT, 0, false, true>(a1, a2, qa, st);
    case 512 * 4096 + 512: return launch_passes_am<16, 32, 16, 32, NT, 0, false, true>(a1, a2, qa, st);
    case 1024 * 4096 + 512: return launch_passes_am<32, 32, 16, 32, NT, 0, false, true>(a1, a2, qa, st);
    case 1024 * 4096 + 1024: return launch_passes_am<32, 32, 32, 32, NT, 0, false, true>(a1, a2, qa, st);
  }
  return cudaErrorInvalidValue;
}

bool passes_lat_instantiated(int N1, int N2) {
  switch (N1 * 4096 + N2) {
    case 64 * 4096 + 64:
    case 128 * 4096 + 64:
    case 128 * 4096 + 128:
    case 256 * 4096 + 128:
    case 256 * 4096 + 256:
    case 512 * 4096 + 256:
    case 512 * 4096 + 512:
    case 1024 * 4096 + 512:
    case 1024 * 4096 + 1024:
      return true;
  }
  return false;
}

}  // namespace fs
