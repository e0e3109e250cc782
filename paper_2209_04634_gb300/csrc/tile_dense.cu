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
  set_tile_attr<false, false, false, false>(n_max);
  set_tile_attr<false, true, false, false>(n_max);
  set_tile_attr<false, false, true, false>(n_max);
  set_tile_attr<false, true, true, false>(n_max);
  set_tile_attr<true, false, false, false>(n_max);
  set_tile_attr<true, true, false, false>(n_max);
  set_tile_attr<true, false, true, false>(n_max);
  set_tile_attr<true, true, true, false>(n_max);
  return cudaGetLastError();
}

}  // namespace evsim
