// Private header of the evsim host runtime: the handle structure and the
// helpers that the single-stream API (runtime.cu) and the multi-stream group
// API (group.cu) share.  Not part of the C ABI.
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "../../include/evsim.h"
#include "internal.h"

using evsim::Ctl;
using evsim::Ev;

struct ProfRec {
  int kind;
  cudaEvent_t a, b;
};

struct sim_s {
  sim_config cfg{};
  int W = 0, H = 0, ch = 1;
  long long P = 0;
  int n_max = 0;
  int tiles_x = 0, tiles_y = 0;
  int tile_h = 16;             // batch kernel tile height (8 or 16; 1: the row kernel)
  int block_order = 0;         // batch kernel tile order: 0 linear, 1 serpentine, 2 balanced
  unsigned int* d_tile_cost = nullptr;  // balanced order: estimated cost per tile of the batch
  int* d_tile_order = nullptr;          // balanced order: tile of each block
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int device = 0;
  int sms = 1;

  int* d_lut = nullptr;
  unsigned short* d_cpmap = nullptr;
  unsigned short* d_cnmap = nullptr;
  unsigned char* d_ring[2] = {nullptr, nullptr};
  unsigned char* d_ring2[2] = {nullptr, nullptr};  // difference mode: frame i-2
  int* d_R[2] = {nullptr, nullptr};
  Ctl* d_ctl = nullptr;
  unsigned long long* d_maxf2 = nullptr;
  Ev* d_staging = nullptr;
  Ev* d_events = nullptr;
  evsim::Seg* d_seg = nullptr;
  unsigned char* d_segflag = nullptr;       // row kernel: per (frame, row unit) written flags
  int* d_units = nullptr;                   // per frame: its flagged units (order kernel)
  int* d_unit_count = nullptr;              // [bmax] flagged units per frame
  unsigned long long* d_tdone = nullptr;    // per tile progress words
  unsigned long long* d_order_status = nullptr;
  evsim::FrameDesc* d_desc = nullptr;       // bmax descriptors of the batch in flight
  unsigned char* d_stage_frames = nullptr;  // host batches: staged frames and flows
  float2* d_stage_flows = nullptr;
  long long stage_frames = 0;               // frames the host staging holds
  // host batches: chunks are copied on copy_stream into two alternating
  // staging slots while the previous chunk simulates on `stream`
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t slot_copied[2] = {nullptr, nullptr};  // a slot's copies are done
  cudaEvent_t slot_free[2] = {nullptr, nullptr};    // a slot's kernels are done
  cudaEvent_t stage_ready = nullptr;                // earlier work on `stream` is done
  long long event_cap = 0;
  long long stage_cap = 0;     // staging events (event capacity plus chunk slack)
  long long segs_per_k = 0;
  int bmax = 1;
  int order_grid = 1;

  // host shadow of the stream
  bool have_first = false;
  long long t0 = 0, t_last = 0;
  long long pushed = 0;
  unsigned serial = 0;
  long long popped = 0;
  long long popped_total = 0;

  bool prof = false;
  std::vector<ProfRec> pending;
  std::vector<cudaEvent_t> pool;
  double prof_ms[SIM_K_COUNT] = {};
  long long prof_n[SIM_K_COUNT] = {};
};

namespace evsim_rt {

template <class T>
cudaError_t dalloc(T** p, size_t count) {
  *p = nullptr;
  if (count == 0) return cudaSuccess;
  return cudaMalloc((void**)p, count * sizeof(T));
}

// Kernel parameters of a handle.
evsim::SimParams make_params(const sim_t* s);
// cudaError_t -> SIM_* code (records the error for sim_last_cuda_error).
int cuda_rc(cudaError_t e);
// Frame 0 of a stream: frame ring and reference (enqueued on s->stream).
int push_first(sim_t* s, const void* frame, long long pitch, int64_t t_us, int32_t mem);
// Wait for the handle's stream and read its control block.
int read_ctl(sim_t* s, Ctl* c);
// After a device-side failure: clear the error and the per-batch scratch and
// roll the host shadow back to the last committed frame.
int recover(sim_t* s, Ctl* c);
// Device bytes sim_create allocates for a configuration (before host staging grows).
long long state_bytes(const sim_config& c);
// The autotuner's tile height for a configuration, if its table has one.
bool tuned_tile_height(const sim_config& c, int* th, int* order);

}  // namespace evsim_rt
