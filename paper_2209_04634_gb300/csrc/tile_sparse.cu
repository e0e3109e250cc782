// The batch-persistent tile kernel, sparse (Sec. III-B) instances: every combination
// of reference mode, threshold maps and intensity table, in 64x16 and 64x8
// tiles.
#include "tile.cuh"

namespace evsim {

cudaError_t launch_sparse(const SimParams& p, const BatchArg& b, cudaStream_t st) {
  if (p.xtime) return launch_xtime_sparse(p, b, st);
  return launch_tile_mode<true>(p, b, st);
}

cudaError_t configure_sparse_kernels(int n_max) {
  return set_mode_attrs<true>(n_max);
}

}  // namespace evsim
