// Persistent transform launch for lattice templates (Sec. IV) on the 2^21
// transform: two 2^20 sub-transforms per template (the 1024 x 1024 split), the
// bin offset d of each line applied on the full 2^21 frequency grid.
#include "fs_pass32.cuh"

namespace fs {

cudaError_t dispatch_passes_lat_wide(int N1, int N2, const Pass1Args &a1, const Pass2Args &a2, const QueueArgs &qa,
                                     cudaStream_t st) {
  if (a1.vshift != 1 || !a1.bin_offset || N1 != 1024 || N2 != 1024) return cudaErrorInvalidValue;
  return launch_passes_am<32, 32, 32, 32, kPersistThreads, 1, false, true>(a1, a2, qa, st);
}

}  // namespace fs
