// The tile kernel with per-crossing event times (SIM_TIME_CROSSING), sparse
// instances, 64x16 tiles: every pixel runs the dense row mapping (sparse:
// inactive pixels masked) and every row with an event stages its events,
// each at the time the line between the values of consecutive substeps meets
// the level it crosses.
#include "tile.cuh"

namespace evsim {

cudaError_t launch_xtime_sparse(const SimParams& p, const BatchArg& b, cudaStream_t st) {
  return launch_tile_shape<true, 16, true>(p, b, st);
}

cudaError_t configure_xtime_sparse_kernels(int n_max) {
  return set_mode_attrs<true, true>(n_max);
}

}  // namespace evsim
