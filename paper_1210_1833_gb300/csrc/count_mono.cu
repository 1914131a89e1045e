// Monopole and chord (theta) counting kernels: d^2 = |x_j - x_i|^2
// (Sec. 2.2 Eq. 11; Sec. 3.4 angular correlation on chords).
#include "count_impl.cuh"

namespace cute {
cudaError_t launch_count_mono(const KParams &p, bool periodic, int acc, int hp, int blocks,
                              int threads, size_t smem, cudaStream_t st) {
  if (periodic) return launch_count_acc<KMONO, true>(p, acc, hp, blocks, threads, smem, st);
  return launch_count_acc<KMONO, false>(p, acc, hp, blocks, threads, smem, st);
}
}  // namespace cute
