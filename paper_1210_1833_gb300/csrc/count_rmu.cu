// (r, mu) counting kernels with the midpoint line of sight (Sec. 2.1
// Eq. 2-3), open (light-cone) catalogs.
#include "count_impl.cuh"

namespace cute {
cudaError_t launch_count_rmu(const KParams &p, int hp, int blocks, int threads, size_t smem,
                             cudaStream_t st) {
  if (hp == 2) return launch_count_t<KRMU, false, 2>(p, blocks, threads, smem, st);
  return launch_count_t<KRMU, false, 4>(p, blocks, threads, smem, st);
}
}  // namespace cute
