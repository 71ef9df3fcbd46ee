// Persistent transform launches for Nfft = 2^19 .. 2^20.
#include "fs_pass32.cuh"

namespace fs {

cudaError_t dispatch_passes_large(int N1, int N2, const Pass1Args &a1, const Pass2Args &a2, const QueueArgs &qa,
                                cudaStream_t st) {
  constexpr int NT = kPersistThreads;
  switch (N1 * 4096 + N2) {
    case 1024 * 4096 + 512: return launch_passes_am<32, 32, 16, 32, NT>(a1, a2, qa, st);
    case 512 * 4096 + 1024: return launch_passes_am<16, 32, 32, 32, NT>(a1, a2, qa, st);
    case 1024 * 4096 + 1024:
      if (a1.vshift == 1) return launch_passes_am<32, 32, 32, 32, NT, 1>(a1, a2, qa, st);
      // data in a quarter of the rows (6 days at 2 s padded to 2^20) prunes two stages
      return launch_passes_am<32, 32, 32, 32, NT, 0, false, false, 8>(a1, a2, qa, st);
  }
  return cudaErrorInvalidValue;
}

int passes_blocks_per_sm_large(int N1, int N2) {
  constexpr int NT = kPersistThreads;
  switch (N1 * 4096 + N2) {
    case 1024 * 4096 + 512: return persist_minb<32, 32, 16, 32, NT>();
    case 512 * 4096 + 1024: return persist_minb<16, 32, 32, 32, NT>();
    case 1024 * 4096 + 1024: return persist_minb<32, 32, 32, 32, NT>();
  }
  return 0;
}

}  // namespace fs
