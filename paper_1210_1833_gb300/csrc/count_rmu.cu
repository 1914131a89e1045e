// (r, mu) counting kernels with the midpoint line of sight (Sec. 2.1
// Eq. 2-3), open (light-cone) catalogs.
#include "count_impl.cuh"

namespace cute {
cudaError_t launch_count_rmu(const KParams &p, int acc, int hp, int blocks, int threads,
                             size_t smem, cudaStream_t st) {
  return launch_count_acc<KRMU, false>(p, acc, hp, blocks, threads, smem, st);
}
}  // namespace cute
