// (sigma, pi) counting kernels, z line of sight (Sec. 2.1 Eq. 2).
#include "count_impl.cuh"

namespace cute {
cudaError_t launch_count_sigpi(const KParams &p, bool periodic, int hp, int blocks, int threads,
                               size_t smem, cudaStream_t st) {
  if (periodic) {
    if (hp == 2) return launch_count_t<KSIGPI, true, 2>(p, blocks, threads, smem, st);
    return launch_count_t<KSIGPI, true, 4>(p, blocks, threads, smem, st);
  }
  if (hp == 2) return launch_count_t<KSIGPI, false, 2>(p, blocks, threads, smem, st);
  return launch_count_t<KSIGPI, false, 4>(p, blocks, threads, smem, st);
}
}  // namespace cute
