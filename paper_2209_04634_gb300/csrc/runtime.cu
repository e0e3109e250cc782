// Host runtime and C ABI of the evsim library: handle state, device
// allocation, the per-batch launch sequence, event pop, error recovery and
// per-kernel profiling.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "handle.h"

namespace evsim_rt {

thread_local cudaError_t g_last_cuda = cudaSuccess;

// Sizes of a handle's device buffers.
struct Sizing {
  int n_max, tiles_x;
  long long P, cap, stage, segs_per_k, seg_cap, ochunks;
  int bmax;
};

Sizing sizing(const sim_config& c) {
  Sizing z{};
  z.P = (long long)c.width * c.height;
  z.n_max = c.substeps > 0 ? c.substeps : c.max_substeps;
  z.tiles_x = (c.width + evsim::TW - 1) / evsim::TW;
  long long cap = c.event_capacity > 0 ? c.event_capacity : std::max<long long>(1LL << 20, 8 * z.P);
  z.cap = std::min<long long>(cap, evsim::MAX_EVENTS);
  // staging: the events of multi-crossing rows, taken in per-warp chunks
  // (at most a third wasted, plus one chunk per warp)
  const long long warps = (long long)z.tiles_x * ((c.height + evsim::TH - 1) / evsim::TH) *
                          (evsim::NTD / 32);
  z.stage = z.cap + z.cap / 3 + (warps + 1) * evsim::STAGE_CHUNK;
  z.segs_per_k = (long long)c.height * z.tiles_x;  // one segment per tile row
  // frames per batch: the requested cap, else what a 512 MB segment table holds
  const long long seg_bytes_per_frame = z.segs_per_k * z.n_max * (long long)sizeof(evsim::Seg);
  const long long bm = c.max_batch > 0
                           ? c.max_batch
                           : std::max(1LL, (512LL << 20) / std::max(1LL, seg_bytes_per_frame));
  z.bmax = (int)std::min<long long>(bm, SIM_MAX_BATCH);
  z.seg_cap = (long long)z.bmax * z.n_max * z.segs_per_k;
  z.ochunks = std::max(1LL, (z.seg_cap + evsim::OCHUNK - 1) / evsim::OCHUNK);
  return z;
}

long long state_bytes(const sim_config& c) {
  const Sizing z = sizing(c);
  long long b = 256 * 4 + 2 * z.P + (long long)sizeof(Ctl) + 8LL * z.bmax;
  if (c.ref_mode == SIM_REF_ACCUM && c.mode != SIM_DIFF) b += 8 * z.P;
  if (c.mode == SIM_DIFF) b += 2 * z.P;  // the second frame ring
  b += (z.stage + z.cap) * (long long)sizeof(Ev);       // staging + events
  b += z.seg_cap * (long long)sizeof(evsim::Seg) + 8 * z.ochunks;
  b += (long long)z.bmax * z.segs_per_k * 5 + 4LL * z.bmax;  // segment flags, flagged units
  b += 8LL * z.tiles_x * ((c.height + 7) / 8);                     // tile progress words
  b += (long long)z.bmax * sizeof(evsim::FrameDesc);
  b += z.P * c.pixel_format;                             // host-frame staging (one frame)
  if (c.c_pos_map) b += 4 * z.P;
  return b;
}

void build_lut(int intensity, int lut[256]) {
  for (int v = 0; v < 256; ++v) {
    if (intensity == SIM_LINEAR)
      lut[v] = v * 65536;
    else
      lut[v] = (int)std::nearbyint(65536.0 * std::log((double)v + 1.0));
  }
}

void free_all(sim_t* s) {
  cudaFree(s->d_lut);
  cudaFree(s->d_cpmap);
  cudaFree(s->d_cnmap);
  cudaFree(s->d_ring[0]);
  cudaFree(s->d_ring[1]);
  cudaFree(s->d_ring2[0]);
  cudaFree(s->d_ring2[1]);
  cudaFree(s->d_R[0]);
  cudaFree(s->d_R[1]);
  cudaFree(s->d_ctl);
  cudaFree(s->d_maxf2);
  cudaFree(s->d_tile_cost);
  cudaFree(s->d_tile_order);
  cudaFree(s->d_staging);
  cudaFree(s->d_events);
  cudaFree(s->d_seg);
  cudaFree(s->d_segflag);
  cudaFree(s->d_units);
  cudaFree(s->d_unit_count);
  cudaFree(s->d_tdone);
  cudaFree(s->d_order_status);
  cudaFree(s->d_desc);
  cudaFree(s->d_stage_frames);
  cudaFree(s->d_stage_flows);
  for (auto& r : s->pending) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (auto e : s->pool) cudaEventDestroy(e);
  for (int k = 0; k < 2; ++k) {
    if (s->slot_copied[k]) cudaEventDestroy(s->slot_copied[k]);
    if (s->slot_free[k]) cudaEventDestroy(s->slot_free[k]);
  }
  if (s->stage_ready) cudaEventDestroy(s->stage_ready);
  if (s->copy_stream) cudaStreamDestroy(s->copy_stream);
  if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
}

evsim::SimParams make_params(const sim_t* s) {
  evsim::SimParams p{};
  p.W = s->W;
  p.H = s->H;
  p.ch = s->ch;
  p.tiles_x = s->tiles_x;
  p.tiles_y = s->tiles_y;
  p.tile_h = s->tile_h;
  p.sms = s->sms;
  p.block_order = s->block_order;
  p.tile_cost = s->block_order == 2 ? s->d_tile_cost : nullptr;
  p.tile_order = s->d_tile_order;
  // segment flags: the row kernel, and the dense tile kernel (which skips
  // rows whose pixels are all quiet)
  p.segflag = s->d_segflag;
  p.units = s->d_units;
  p.unit_count = s->d_unit_count;
  p.xtime = s->cfg.event_time == SIM_TIME_CROSSING;
  p.mode = s->cfg.mode;
  p.ref_mode = s->cfg.ref_mode;
  p.intensity = s->cfg.intensity;
  p.n_fixed = s->cfg.substeps;
  p.n_max = s->n_max;
  p.cp = s->cfg.c_pos_q16;
  p.cn = s->cfg.c_neg_q16;
  p.cact = s->cfg.c_act_q16;
  p.bmax = s->bmax;
  p.cpmap = s->d_cpmap;
  p.cnmap = s->d_cnmap;
  p.lut = s->d_lut;
  p.ring0 = s->d_ring[0];
  p.ring1 = s->d_ring[1];
  p.ring2_0 = s->d_ring2[0];
  p.ring2_1 = s->d_ring2[1];
  p.R0 = s->d_R[0];
  p.R1 = s->d_R[1];
  p.ctl = s->d_ctl;
  p.maxf2 = s->d_maxf2;
  p.staging = s->d_staging;
  p.stage_cap = s->stage_cap;
  p.stage_chunk = evsim::STAGE_CHUNK;
  p.seg = s->d_seg;
  p.tdone = s->d_tdone;
  p.segs_per_k = s->segs_per_k;
  p.seg_cap = (long long)s->bmax * s->n_max * s->segs_per_k;
  p.order_status = s->d_order_status;
  p.events = s->d_events;
  p.event_cap = s->event_cap;
  return p;
}

int cuda_rc(cudaError_t e) {
  if (e == cudaSuccess) return SIM_OK;
  g_last_cuda = e;
  if (e == cudaErrorMemoryAllocation) return SIM_ERR_OOM;
  if (e == cudaErrorNoDevice || e == cudaErrorInsufficientDriver || e == cudaErrorNoKernelImageForDevice)
    return SIM_ERR_NO_DEVICE;
  return SIM_ERR_CUDA;
}

cudaEvent_t pool_get(sim_t* s) {
  if (!s->pool.empty()) {
    cudaEvent_t e = s->pool.back();
    s->pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Launch wrapper: records a CUDA event pair around the launch when profiling.
template <class F>
cudaError_t timed(sim_t* s, int kind, F&& launch) {
  if (!s->prof) return launch();
  ProfRec r{kind, pool_get(s), pool_get(s)};
  cudaEventRecord(r.a, s->stream);
  cudaError_t e = launch();
  cudaEventRecord(r.b, s->stream);
  s->pending.push_back(r);
  return e;
}

void prof_collect(sim_t* s) {
  if (s->pending.empty()) return;
  cudaStreamSynchronize(s->stream);
  for (auto& r : s->pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      s->prof_ms[r.kind] += ms;
      s->prof_n[r.kind] += 1;
    }
    s->pool.push_back(r.a);
    s->pool.push_back(r.b);
  }
  s->pending.clear();
}

// Read the control block (after the stream is idle).
int read_ctl(sim_t* s, Ctl* c) {
  // on the handle's stream: a copy on the legacy default stream would also
  // wait for other streams' work
  cudaError_t e = cudaMemcpyAsync(c, s->d_ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  return cuda_rc(e);
}

// After a device-side failure: clear the error and the per-batch scratch, and
// roll the host shadow back to the last committed frame.
int recover(sim_t* s, Ctl* c) {
  c->err = 0;
  c->batch_fail = 0;
  c->active = 0;
  c->active_n = 0;
  c->stage_top = 0;
  c->order_ticket = 0;
  c->order_done = 0;
  c->order_exit = 0;
  s->t_last = s->t0 + c->t_prev;
  cudaError_t e = cudaMemcpy(s->d_ctl, c, sizeof(Ctl), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(s->d_maxf2, 0, s->bmax * sizeof(unsigned long long));
  return cuda_rc(e);
}

int push_first(sim_t* s, const void* frame, long long pitch, int64_t t_us, int32_t mem) {
  const long long row = (long long)s->W * s->ch;
  evsim::FrameDesc f{};
  f.frame = (const unsigned char*)frame;
  f.pitch = pitch;
  cudaError_t e = cudaSuccess;
  if (mem == SIM_HOST) {
    e = cudaMemcpy2DAsync(s->d_stage_frames, row, frame, pitch, row, s->H, cudaMemcpyHostToDevice,
                          s->stream);
    if (e != cudaSuccess) return cuda_rc(e);
    f.frame = s->d_stage_frames;
    f.pitch = row;
  }
  const evsim::SimParams p = make_params(s);
  e = timed(s, SIM_K_INIT, [&] { return evsim::launch_init(p, f, s->stream); });
  if (e != cudaSuccess) return cuda_rc(e);
  Ctl c{};
  c.committed = 1;
  e = cudaMemcpyAsync(s->d_ctl, &c, sizeof(Ctl), cudaMemcpyHostToDevice, s->stream);
  if (e != cudaSuccess) return cuda_rc(e);
  // the source is a stack object: make sure the copy has left it
  e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_rc(e);
  s->have_first = true;
  s->t0 = t_us;
  s->t_last = t_us;
  s->pushed += 1;
  return SIM_OK;
}

// Enqueue one batch whose descriptors are already in d_desc.
cudaError_t enqueue_batch(sim_t* s, int n, bool host_mapped) {
  const evsim::SimParams p = make_params(s);
  evsim::BatchArg b{};
  b.frames = s->d_desc;
  b.count = n;
  b.serial = ++s->serial;
  b.host_mapped = host_mapped ? 1 : 0;
  cudaError_t e;
  const bool adaptive = s->cfg.substeps == 0;
  if (s->cfg.mode == SIM_DENSE || s->cfg.mode == SIM_DIFF) {
    if (adaptive) {
      e = timed(s, SIM_K_FLOWMAX, [&] { return evsim::launch_flowmax(p, b, s->stream); });
      if (e != cudaSuccess) return e;
    }
    if (s->block_order == 2 && s->cfg.mode != SIM_DIFF && s->tile_h != SIM_TILE_ROWS) {
      e = evsim::launch_plan(p, b, s->stream);  // the balanced order of this batch's tiles
      if (e != cudaSuccess) return e;
    }
    if (s->cfg.mode == SIM_DIFF)
      e = timed(s, SIM_K_DENSE, [&] { return evsim::launch_diff(p, b, s->stream); });
    else if (s->tile_h == SIM_TILE_ROWS)
      e = timed(s, SIM_K_DENSE, [&] { return evsim::launch_rows(p, b, s->stream); });
    else
      e = timed(s, SIM_K_DENSE, [&] { return evsim::launch_dense(p, b, s->stream); });
  } else {
    if (adaptive) {
      e = timed(s, SIM_K_MASK, [&] { return evsim::launch_sparse_pre(p, b, s->stream); });
      if (e != cudaSuccess) return e;
    }
    if (s->block_order == 2 && s->tile_h != SIM_TILE_ROWS) {
      e = evsim::launch_plan(p, b, s->stream);
      if (e != cudaSuccess) return e;
    }
    if (s->tile_h == SIM_TILE_ROWS)
      e = timed(s, SIM_K_SPARSE, [&] { return evsim::launch_rows(p, b, s->stream); });
    else if (p.segflag && !p.xtime)  // the dense tile kernel with activity masks
      e = timed(s, SIM_K_SPARSE, [&] { return evsim::launch_dense(p, b, s->stream); });
    else
      e = timed(s, SIM_K_SPARSE, [&] { return evsim::launch_sparse(p, b, s->stream); });
  }
  if (e != cudaSuccess) return e;
  return timed(s, SIM_K_ORDER, [&] { return evsim::launch_order(p, b, s->stream, s->order_grid); });
}

}  // namespace evsim_rt

using namespace evsim_rt;

void evsim::note_cuda_error(cudaError_t e) { g_last_cuda = e; }

extern "C" {

const char* sim_version(void) { return "0.2.0"; }

const char* sim_last_cuda_error(void) { return cudaGetErrorString(g_last_cuda); }

const char* sim_strerror(int code) {
  switch (code) {
    case SIM_OK: return "ok";
    case SIM_MORE: return "more events remain";
    case SIM_ERR_ARG: return "invalid argument";
    case SIM_ERR_CUDA: return "CUDA runtime error";
    case SIM_ERR_OOM: return "out of memory";
    case SIM_ERR_TIME: return "timestamp not strictly increasing";
    case SIM_ERR_TIME_RANGE: return "timestamp more than 2^32-1 us after the first frame";
    case SIM_ERR_EVENT_OVERFLOW: return "event buffer overflow; batch not committed";
    case SIM_ERR_DEVICE_TIMEOUT: return "device-side wait timed out";
    case SIM_ERR_STATE: return "call not valid in this state";
    case SIM_ERR_ADMIT: return "admission refused";
    case SIM_ERR_NO_DEVICE: return "no usable CUDA device";
    case SIM_ERR_TOO_LARGE: return "problem too large for the fixed scratch array";
    case SIM_ERR_BOUNDS: return "a kernel index left its buffer (debug build bounds check)";
    default: return "unknown error";
  }
}

int32_t sim_threshold_q16(double c) {
  if (!std::isfinite(c)) return SIM_ERR_ARG;
  const double q = std::nearbyint(std::fabs(c) * 65536.0);  // ties to even
  if (q >= 1073741824.0) return SIM_ERR_ARG;
  return (int32_t)q;
}

int sim_config_default(sim_config* cfg, int32_t width, int32_t height) {
  if (!cfg) return SIM_ERR_ARG;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->width = width;
  cfg->height = height;
  cfg->pixel_format = SIM_LUMA8;
  cfg->mode = SIM_DENSE;
  cfg->substeps = 8;
  cfg->max_substeps = 16;
  cfg->intensity = SIM_LOG;
  cfg->ref_mode = SIM_REF_ACCUM;
  cfg->c_pos_q16 = 13107;
  cfg->c_neg_q16 = 13107;
  cfg->c_act_q16 = -1;
  return SIM_OK;
}

int sim_create(const sim_config* cfg, sim_t** out) {
  if (!cfg || !out) return SIM_ERR_ARG;
  const sim_config& c = *cfg;
  if (c.width < 1 || c.height < 1 || c.width > SIM_MAX_DIM || c.height > SIM_MAX_DIM) return SIM_ERR_ARG;
  if (c.pixel_format != SIM_LUMA8 && c.pixel_format != SIM_RGB8) return SIM_ERR_ARG;
  if (c.mode != SIM_DENSE && c.mode != SIM_SPARSE && c.mode != SIM_DIFF) return SIM_ERR_ARG;
  if (c.intensity != SIM_LOG && c.intensity != SIM_LINEAR) return SIM_ERR_ARG;
  if (c.ref_mode != SIM_REF_ACCUM && c.ref_mode != SIM_REF_RESET) return SIM_ERR_ARG;
  if (c.substeps < 0 || c.substeps > SIM_MAX_SUBSTEPS) return SIM_ERR_ARG;
  if (c.substeps == 0 && (c.max_substeps < 1 || c.max_substeps > SIM_MAX_SUBSTEPS)) return SIM_ERR_ARG;
  if (c.event_capacity < 0 || c.event_capacity > evsim::MAX_EVENTS) return SIM_ERR_ARG;
  if (c.max_batch < 0 || c.max_batch > SIM_MAX_BATCH) return SIM_ERR_ARG;
  if (c.tile_height != SIM_TILE_AUTO && c.tile_height != SIM_TILE_TUNE && c.tile_height != 8 &&
      c.tile_height != 16 && c.tile_height != SIM_TILE_ROWS)
    return SIM_ERR_ARG;
  if (c.event_time != SIM_TIME_SUBSTEP && c.event_time != SIM_TIME_CROSSING) return SIM_ERR_ARG;
  if (c.host_inputs != SIM_HOST_STAGE && c.host_inputs != SIM_HOST_MAPPED) return SIM_ERR_ARG;
  const bool xtime = c.event_time == SIM_TIME_CROSSING;
  if (xtime && c.mode == SIM_DIFF) return SIM_ERR_ARG;  // no crossings: no reference

  int lut[256];
  build_lut(c.intensity, lut);
  // Thresholds: >= 1, < 2^30; accumulate mode also bounds the events of one
  // pixel-substep to 32767 (they are counted in 16 bits).
  const long long range = (long long)lut[255] - lut[0];
  const bool accum = c.ref_mode == SIM_REF_ACCUM && c.mode != SIM_DIFF;
  const long long cmin = accum ? (range + 32765) / 32766 : 1;
  auto bad_c = [&](long long v) { return v < cmin || v >= (1LL << 30); };
  const long long P = (long long)c.width * c.height;
  if (!c.c_pos_map && bad_c(c.c_pos_q16)) return SIM_ERR_ARG;
  if (!c.c_neg_map && bad_c(c.c_neg_q16)) return SIM_ERR_ARG;
  if ((c.c_pos_map == nullptr) != (c.c_neg_map == nullptr)) return SIM_ERR_ARG;
  if (c.c_pos_map) {
    for (long long i = 0; i < P; ++i)
      if (bad_c(c.c_pos_map[i]) || bad_c(c.c_neg_map[i])) return SIM_ERR_ARG;
  }

  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) return SIM_ERR_NO_DEVICE;

  // tile shape: fixed, or the autotuner's choice for this configuration
  int th = c.tile_height, order = 0, tth = 16, torder = 0;
  const bool tuned = !xtime && tuned_tile_height(c, &tth, &torder);
  if (xtime || (c.mode == SIM_DIFF && th == SIM_TILE_ROWS)) {
    th = 16;  // the per-crossing-time and difference kernels have the 64 x 16 shape only
  } else if (th != 8 && th != 16 && th != SIM_TILE_ROWS) {
    if (tuned) {
      th = tth;
      order = torder;
    } else {
      th = 16;
      if (c.tile_height == SIM_TILE_TUNE) {
        int32_t t = 16;
        const int rc = sim_autotune(&c, 8, &t, nullptr);
        if (rc) return rc;
        tuned_tile_height(c, &tth, &torder);
        th = t;
        order = torder;
      }
    }
  } else if (tuned && tth == th) {
    order = torder;  // a fixed shape keeps the tuned order for that shape
  }

  sim_t* s = new (std::nothrow) sim_t();
  if (!s) return SIM_ERR_OOM;
  s->cfg = c;
  if (c.mode == SIM_DIFF) s->cfg.ref_mode = SIM_REF_RESET;  // no reference state
  s->cfg.c_pos_map = nullptr;
  s->cfg.c_neg_map = nullptr;
  s->W = c.width;
  s->H = c.height;
  s->ch = c.pixel_format;
  s->P = P;
  s->n_max = c.substeps > 0 ? c.substeps : c.max_substeps;
  s->tiles_x = (c.width + evsim::TW - 1) / evsim::TW;
  s->tile_h = th;
  s->block_order = order;
  s->tiles_y = (c.height + th - 1) / th;
  cudaGetDevice(&s->device);
  s->sms = std::max(1, evsim::device_sm_count());

  const Sizing z = sizing(c);
  const long long cap = z.cap;
  s->event_cap = cap;
  s->stage_cap = z.stage;
  s->segs_per_k = z.segs_per_k;
  s->bmax = z.bmax;
  const long long seg_cap = z.seg_cap;
  const long long ochunks = z.ochunks;

  cudaError_t e = cudaSuccess;
  auto chk = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
  if (c.cuda_stream) {
    s->stream = (cudaStream_t)c.cuda_stream;
  } else {
    chk(cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking));
    s->own_stream = true;
  }
  chk(dalloc(&s->d_lut, 256));
  chk(dalloc(&s->d_ring[0], P));
  chk(dalloc(&s->d_ring[1], P));
  if (c.mode == SIM_DIFF) {
    chk(dalloc(&s->d_ring2[0], P));
    chk(dalloc(&s->d_ring2[1], P));
  }
  if (s->cfg.ref_mode == SIM_REF_ACCUM) {
    chk(dalloc(&s->d_R[0], P));
    chk(dalloc(&s->d_R[1], P));
  }
  chk(dalloc(&s->d_ctl, 1));
  {
    // balanced block order: per-tile cost estimates of the batch and the
    // plan made from them before each batch
    const int T = s->tiles_x * s->tiles_y;
    if (T <= evsim::PLAN_MAX_TILES) {
      chk(dalloc(&s->d_tile_cost, T));
      chk(dalloc(&s->d_tile_order, T));
      if (e == cudaSuccess) {
        std::vector<int> id(T);
        for (int t = 0; t < T; ++t) id[t] = t;
        chk(cudaMemcpy(s->d_tile_order, id.data(), T * sizeof(int), cudaMemcpyHostToDevice));
        chk(cudaMemset(s->d_tile_cost, 0, T * sizeof(unsigned)));
      }
    } else if (s->block_order == 2) {
      s->block_order = 0;
    }
  }
  chk(dalloc(&s->d_maxf2, s->bmax));
  chk(dalloc(&s->d_staging, z.stage));
  chk(dalloc(&s->d_events, cap));
  chk(dalloc(&s->d_seg, seg_cap));
  // segment flags (row kernel; tile kernel with substep times)
  if (th == SIM_TILE_ROWS || (c.mode != SIM_DIFF && !xtime)) {
    chk(dalloc(&s->d_segflag, (size_t)s->bmax * s->segs_per_k));
    // the order pass walks the flagged units only (its 32-bit segment
    // counts need a table below 2^31 segments)
    if (seg_cap < (1LL << 31)) {
      chk(dalloc(&s->d_units, (size_t)s->bmax * s->segs_per_k));
      chk(dalloc(&s->d_unit_count, (size_t)s->bmax));
    }
  }
  chk(dalloc(&s->d_tdone, (size_t)s->tiles_x * s->tiles_y));
  chk(dalloc(&s->d_order_status, ochunks));
  chk(dalloc(&s->d_desc, s->bmax));
  chk(dalloc(&s->d_stage_frames, P * s->ch));
  if (c.c_pos_map) {
    chk(dalloc(&s->d_cpmap, P));
    chk(dalloc(&s->d_cnmap, P));
    if (e == cudaSuccess) {
      chk(cudaMemcpy(s->d_cpmap, c.c_pos_map, P * 2, cudaMemcpyHostToDevice));
      chk(cudaMemcpy(s->d_cnmap, c.c_neg_map, P * 2, cudaMemcpyHostToDevice));
    }
  }
  if (e == cudaSuccess) {
    chk(cudaMemcpy(s->d_lut, lut, sizeof(lut), cudaMemcpyHostToDevice));
    chk(cudaMemset(s->d_ctl, 0, sizeof(Ctl)));
    chk(cudaMemset(s->d_maxf2, 0, s->bmax * sizeof(unsigned long long)));
    chk(cudaMemset(s->d_order_status, 0, ochunks * sizeof(unsigned long long)));
    chk(cudaMemset(s->d_tdone, 0, (size_t)s->tiles_x * s->tiles_y * sizeof(unsigned long long)));
  }
  if (e == cudaSuccess) {
    chk(evsim::raise_kernel_limits(s->n_max, false));
  }
  if (e != cudaSuccess) {
    const int rc = cuda_rc(e);
    free_all(s);
    delete s;
    return rc;
  }
  s->order_grid = (int)std::min<long long>(ochunks, (long long)s->sms * 8);
  *out = s;
  return SIM_OK;
}

int sim_push_frames(sim_t* s, int32_t count, const void* const* frames, int64_t pitch_bytes,
                    const float* const* flows, const int64_t* t_us, int32_t mem) {
  if (!s || count < 0 || (count > 0 && (!frames || !t_us))) return SIM_ERR_ARG;
  if (mem != SIM_HOST && mem != SIM_DEVICE) return SIM_ERR_ARG;
  const long long row = (long long)s->W * s->ch;
  if (pitch_bytes < row) return SIM_ERR_ARG;
  // validate the whole batch first
  long long tl = s->t_last, t0 = s->have_first ? s->t0 : (count > 0 ? t_us[0] : 0);
  for (int i = 0; i < count; ++i) {
    if (!frames[i]) return SIM_ERR_ARG;
    if (!s->have_first && i == 0) {
      tl = t_us[0];
      continue;
    }
    if (!flows || !flows[i]) return SIM_ERR_ARG;
    if (t_us[i] <= tl) return SIM_ERR_TIME;
    if (t_us[i] - t0 > 4294967295LL) return SIM_ERR_TIME_RANGE;
    tl = t_us[i];
  }
  int i0 = 0;
  if (!s->have_first && count > 0) {
    const int rc = push_first(s, frames[0], pitch_bytes, t_us[0], mem);
    if (rc) return rc;
    i0 = 1;
  }
  cudaError_t e = cudaSuccess;
  std::vector<evsim::FrameDesc> desc;
  // SIM_HOST_MAPPED: pinned host buffers are read in place through their
  // device mapping - the kernels pull the bytes over the host link as they
  // stage each frame, so no copy precedes the kernels.
  std::vector<const void*> mfr;
  std::vector<const float*> mfl;
  bool host_mapped = false;
  if (mem == SIM_HOST && s->cfg.host_inputs == SIM_HOST_MAPPED && i0 < count) {
    bool mapped = true;
    mfr.assign(count, nullptr);
    mfl.assign(count, nullptr);
    for (int i = i0; i < count && mapped; ++i) {
      void* dp[2] = {nullptr, nullptr};
      const void* hp[2] = {frames[i], flows[i]};
      for (int k = 0; k < 2 && mapped; ++k) {
        cudaPointerAttributes a;
        if (cudaPointerGetAttributes(&a, hp[k]) != cudaSuccess) {
          cudaGetLastError();  // an unregistered pointer is not an error here
          mapped = false;
        } else if (a.type != cudaMemoryTypeHost || !a.devicePointer) {
          mapped = false;
        } else {
          dp[k] = a.devicePointer;
        }
      }
      mfr[i] = dp[0];
      mfl[i] = (const float*)dp[1];
    }
    if (mapped) {
      frames = mfr.data();
      flows = mfl.data();
      mem = SIM_DEVICE;
      host_mapped = true;
    }
  }
  // Host frames go through device staging in chunks of m frames (about an
  // eighth of the call, at least 4, at most a device batch), each chunk a
  // device batch of its own: chunk j + 1 is copied on the copy stream into
  // the other of two staging slots while chunk j simulates, so the copies
  // overlap the kernels.  Device frames are read in place, in device batches
  // of max_batch frames.
  const int rest = count - i0;
  const int m = mem == SIM_HOST ? std::min(s->bmax, std::max(4, (rest + 7) / 8)) : s->bmax;
  if (mem == SIM_HOST && rest > 0) {
    if (!s->copy_stream) {
      e = cudaStreamCreateWithFlags(&s->copy_stream, cudaStreamNonBlocking);
      for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
        e = cudaEventCreateWithFlags(&s->slot_copied[k], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->slot_free[k], cudaEventDisableTiming);
      }
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->stage_ready, cudaEventDisableTiming);
      if (e != cudaSuccess) return cuda_rc(e);
    }
    const int slots = std::min(2 * m, 2 * rest);
    if (s->stage_frames < slots) {
      // earlier batches may still read the old area
      e = cudaStreamSynchronize(s->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s->copy_stream);
      if (e != cudaSuccess) return cuda_rc(e);
      cudaFree(s->d_stage_frames);
      cudaFree(s->d_stage_flows);
      s->d_stage_frames = nullptr;
      s->d_stage_flows = nullptr;
      s->stage_frames = 0;
      e = dalloc(&s->d_stage_frames, (size_t)slots * s->P * s->ch);
      if (e == cudaSuccess) e = dalloc(&s->d_stage_flows, (size_t)slots * s->P);
      if (e != cudaSuccess) return cuda_rc(e);
      s->stage_frames = slots;
    }
    // the copies wait for whatever the handle's stream did with the staging
    // area before this call (a first frame, earlier batches)
    e = cudaEventRecord(s->stage_ready, s->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s->copy_stream, s->stage_ready, 0);
    if (e != cudaSuccess) return cuda_rc(e);
  }
  int slot = 0;
  while (i0 < count) {
    const int n = std::min(count - i0, m);
    desc.assign(n, evsim::FrameDesc{});
    if (mem == SIM_HOST) {
      // the slot's previous chunk must have been simulated before it is overwritten
      e = cudaStreamWaitEvent(s->copy_stream, s->slot_free[slot], 0);
      if (e != cudaSuccess) return cuda_rc(e);
    }
    for (int j = 0; j < n; ++j) {
      const int i = i0 + j;
      evsim::FrameDesc& d = desc[j];
      if (mem == SIM_HOST) {
        const size_t f = (size_t)slot * m + j;
        unsigned char* fd = s->d_stage_frames + f * s->P * s->ch;
        float2* fl = s->d_stage_flows + f * s->P;
        e = cudaMemcpy2DAsync(fd, row, frames[i], pitch_bytes, row, s->H, cudaMemcpyHostToDevice,
                              s->copy_stream);
        if (e == cudaSuccess)
          e = cudaMemcpyAsync(fl, flows[i], s->P * sizeof(float2), cudaMemcpyHostToDevice,
                              s->copy_stream);
        if (e != cudaSuccess) return cuda_rc(e);
        d.frame = fd;
        d.pitch = row;
        d.flow = fl;
      } else {
        d.frame = (const unsigned char*)frames[i];
        d.pitch = pitch_bytes;
        d.flow = (const float2*)flows[i];
      }
      d.t_rel = t_us[i] - s->t0;
    }
    if (mem == SIM_HOST) {
      e = cudaEventRecord(s->slot_copied[slot], s->copy_stream);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(s->stream, s->slot_copied[slot], 0);
      if (e != cudaSuccess) return cuda_rc(e);
    }
    e = cudaMemcpyAsync(s->d_desc, desc.data(), n * sizeof(evsim::FrameDesc),
                        cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = enqueue_batch(s, n, host_mapped);
    if (e == cudaSuccess && mem == SIM_HOST) e = cudaEventRecord(s->slot_free[slot], s->stream);
    if (e != cudaSuccess) return cuda_rc(e);
    s->t_last = t_us[i0 + n - 1];
    s->pushed += n;
    i0 += n;
    slot ^= 1;
  }
  return SIM_OK;
}

int sim_push_frame(sim_t* s, const void* frame, int64_t pitch_bytes, const float* flow,
                   int64_t t_us, int32_t mem) {
  return sim_push_frames(s, 1, &frame, pitch_bytes, &flow, &t_us, mem);
}

int sim_sync(sim_t* s) {
  if (!s) return SIM_ERR_ARG;
  Ctl c;
  int rc = read_ctl(s, &c);
  if (rc) return rc;
  if (c.err) {
    const int err = c.err;
    rc = recover(s, &c);
    return rc ? rc : err;
  }
  return SIM_OK;
}

int sim_pop_events(sim_t* s, sim_event* out, int64_t cap, int64_t* n_out, int32_t mem) {
  if (!s || !n_out || cap < 0 || (cap > 0 && !out)) return SIM_ERR_ARG;
  if (mem != SIM_HOST && mem != SIM_DEVICE) return SIM_ERR_ARG;
  *n_out = 0;
  Ctl c;
  int rc = read_ctl(s, &c);
  if (rc) return rc;
  if (c.err) {
    // report the failure first; the committed events stay for the next pop
    const int err = c.err;
    rc = recover(s, &c);
    return rc ? rc : err;
  }
  int status = SIM_OK;
  const long long avail = c.cursor - s->popped;
  const long long m = std::min<long long>(avail, cap);
  // the copies run on the handle's stream (not the legacy default stream,
  // which would also wait for other streams' work) and are waited for here
  if (m > 0) {
    cudaError_t e = cudaMemcpyAsync(out, s->d_events + s->popped, (size_t)m * sizeof(Ev),
                                    mem == SIM_HOST ? cudaMemcpyDeviceToHost
                                                    : cudaMemcpyDeviceToDevice,
                                    s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_rc(e);
  }
  s->popped += m;
  s->popped_total += m;
  *n_out = m;
  if (s->popped == c.cursor && c.cursor > 0) {
    const long long zero = 0;
    cudaError_t e = cudaMemcpyAsync(&s->d_ctl->cursor, &zero, sizeof(zero),
                                    cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_rc(e);
    s->popped = 0;
  }
  if (avail > m) status = SIM_MORE;
  return status;
}

int sim_get_stats(sim_t* s, sim_stats* st) {
  if (!s || !st) return SIM_ERR_ARG;
  Ctl c;
  int rc = read_ctl(s, &c);
  if (rc) return rc;
  std::memset(st, 0, sizeof(*st));
  st->frames_pushed = s->pushed;
  st->frames_committed = c.committed;
  st->events_pending = c.cursor - s->popped;
  st->events_popped = s->popped_total;
  st->last_active = c.last_active;
  st->last_batch_events = c.batch_events;
  st->flow_clamped = (int64_t)c.clamped;
  st->last_substeps = c.last_n;
  st->max_batch = s->bmax;
  st->pixel_substeps = c.work_px;
  st->active_substeps = c.work_active;
  st->active_pixels = c.work_pixels;
  st->tile_height = s->tile_h;
  st->block_order = s->block_order;
  return SIM_OK;
}

int sim_get_reference(sim_t* s, int32_t* out_host) {
  if (!s || !out_host) return SIM_ERR_ARG;
  if (s->cfg.ref_mode != SIM_REF_ACCUM) return SIM_ERR_STATE;
  Ctl c;
  int rc = read_ctl(s, &c);
  if (rc) return rc;
  const int* src = (c.sel & 1) ? s->d_R[1] : s->d_R[0];
  cudaError_t e = cudaMemcpy(out_host, src, s->P * sizeof(int), cudaMemcpyDeviceToHost);
  return cuda_rc(e);
}

int sim_set_profiling(sim_t* s, int32_t enable) {
  if (!s) return SIM_ERR_ARG;
  if (!enable) prof_collect(s);
  s->prof = enable != 0;
  return SIM_OK;
}

int sim_kernel_time(sim_t* s, int32_t kind, double* ms, int64_t* launches, int32_t reset) {
  if (!s || kind < 0 || kind >= SIM_K_COUNT) return SIM_ERR_ARG;
  prof_collect(s);
  if (ms) *ms = s->prof_ms[kind];
  if (launches) *launches = s->prof_n[kind];
  if (reset) {
    s->prof_ms[kind] = 0;
    s->prof_n[kind] = 0;
  }
  return SIM_OK;
}

int sim_accumulate(const sim_event* events, int64_t n, int32_t width, int32_t height,
                   int64_t t_begin, int64_t t_end, int32_t* frame, void* cuda_stream) {
  if (n < 0 || (n > 0 && !events) || !frame || width < 1 || height < 1 ||
      width > SIM_MAX_DIM || height > SIM_MAX_DIM)
    return SIM_ERR_ARG;
  cudaError_t e = evsim::launch_accumulate((const Ev*)events, n, width, height, t_begin, t_end,
                                           frame, (cudaStream_t)cuda_stream);
  return cuda_rc(e);
}

int sim_reset(sim_t* s) {
  if (!s) return SIM_ERR_ARG;
  cudaError_t e = cudaStreamSynchronize(s->stream);
  if (e == cudaSuccess) e = cudaMemset(s->d_ctl, 0, sizeof(Ctl));
  if (e == cudaSuccess) e = cudaMemset(s->d_maxf2, 0, s->bmax * sizeof(unsigned long long));
  if (e != cudaSuccess) return cuda_rc(e);
  s->have_first = false;
  s->t0 = s->t_last = 0;
  s->pushed = 0;
  s->popped = 0;
  return SIM_OK;
}

int sim_destroy(sim_t* s) {
  if (!s) return SIM_ERR_ARG;
  cudaStreamSynchronize(s->stream);
  free_all(s);
  delete s;
  return SIM_OK;
}

}  // extern "C"
