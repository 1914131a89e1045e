// Monopole and chord (theta) counting kernels: d^2 = |x_j - x_i|^2
// (Sec. 2.2 Eq. 11; Sec. 3.4 angular correlation on chords).
#include "count_impl.cuh"

namespace cute {
cudaError_t launch_count_mono(const KParams &p, bool periodic, int hp, int blocks, int threads,
                              size_t smem, cudaStream_t st) {
  if (periodic) {
    if (hp == 2) return launch_count_t<KMONO, true, 2>(p, blocks, threads, smem, st);
    return launch_count_t<KMONO, true, 4>(p, blocks, threads, smem, st);
  }
  if (hp == 2) return launch_count_t<KMONO, false, 2>(p, blocks, threads, smem, st);
  return launch_count_t<KMONO, false, 4>(p, blocks, threads, smem, st);
}
}  // namespace cute
