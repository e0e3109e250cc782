// The batch-persistent tile kernel, dense (Sec. III-A) instances: every combination
// of reference mode, threshold maps and intensity table, in 64x16 and 64x8
// tiles.
#include "tile.cuh"

namespace evsim {

cudaError_t launch_dense(const SimParams& p, const BatchArg& b, cudaStream_t st) {
  if (p.xtime) return launch_xtime_dense(p, b, st);
  return launch_tile_mode<false>(p, b, st);
}

cudaError_t configure_dense_kernels(int n_max) {
  return set_mode_attrs<false>(n_max);
}

}  // namespace evsim
