// (sigma, pi) counting kernels, z line of sight (Sec. 2.1 Eq. 2).
#include "count_impl.cuh"

namespace cute {
cudaError_t launch_count_sigpi(const KParams &p, bool periodic, int acc, int hp, int blocks,
                               int threads, size_t smem, cudaStream_t st) {
  if (periodic) return launch_count_acc<KSIGPI, true>(p, acc, hp, blocks, threads, smem, st);
  return launch_count_acc<KSIGPI, false>(p, acc, hp, blocks, threads, smem, st);
}
}  // namespace cute
