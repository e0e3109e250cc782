// sim_step_pair_static: one frame pair through the simulation kernels with
// every scratch buffer carved out of a fixed, file-scope device array, so the
// call itself allocates no memory.
//
// Who needs it: callers that may not allocate device memory once they are
// running.  A process whose device memory is owned by another framework's
// caching allocator (cudaMalloc outside that pool can fail or fragment it,
// and cudaFree synchronises the whole device, stalling every other stream); a
// frame-rate pipeline with a no-allocation rule after start-up, because
// cudaMalloc / cudaFree have unbounded latency; a plug-in that receives device
// buffers from its host application and is not allowed to allocate its own.
// Such callers own their frames, flow, reference and event buffers and pass
// them in; everything else lives in g_scratch.
//
// The array is shared by every call on a device: it is re-initialised at the
// start of each call (control block, tile progress words, look-back words
// and flow maxima are cleared there), and two calls whose GPU work overlaps
// race on it.  An accumulate step that updates its reference in place (or
// starts one) builds the new reference in the array and copies it out only
// after the step has been checked, so a failed step leaves the caller's
// reference as it was.
#include <cuda_runtime.h>

#include <cmath>
#include <cstddef>
#include <cstring>
#include <mutex>

#include "../../include/evsim.h"
#include "internal.h"

namespace {

using evsim::Ctl;
using evsim::Ev;
using evsim::FrameDesc;
using evsim::Seg;

static __device__ __align__(256) unsigned char g_scratch[SIM_STATIC_SCRATCH_BYTES];

constexpr int MAX_DEVICES = 256;
std::mutex g_setup_mu;

// Set-up of one device, valid for one CUDA context on it: the array's address
// in that context and the tile kernels' shared-memory permission.  A context
// is recognised by its unique id (cuCtxGetId, reached through the runtime's
// driver entry points), so a cudaDeviceReset, or another context made current
// on the same device, leads to a fresh set-up instead of a stale address.
struct DeviceSetup {
  unsigned long long ctx_id;  // 0: not set up
  unsigned char* base;        // address of g_scratch in that context
};
DeviceSetup g_dev[MAX_DEVICES] = {};

typedef int (*CtxGetCurrentFn)(void** ctx);
typedef int (*CtxGetIdFn)(void* ctx, unsigned long long* id);
CtxGetCurrentFn g_ctx_current = nullptr;
CtxGetIdFn g_ctx_id = nullptr;
bool g_ctx_fns_tried = false;

// Unique id of the calling thread's current context, or 0 when it cannot be
// told (no current context, or a driver without the query).  Call under
// g_setup_mu.
unsigned long long current_context_id() {
  if (!g_ctx_fns_tried) {
    g_ctx_fns_tried = true;
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      g_ctx_current = (CtxGetCurrentFn)f;
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      g_ctx_id = (CtxGetIdFn)f;
  }
  if (!g_ctx_current || !g_ctx_id) return 0;
  void* ctx = nullptr;
  unsigned long long id = 0;
  if (g_ctx_current(&ctx) != 0 || !ctx) return 0;
  if (g_ctx_id(ctx, &id) != 0) return 0;
  return id;
}

// Start of the array: uploaded by every call in one copy.
struct alignas(256) Header {
  Ctl ctl;
  unsigned char pad0[256 - sizeof(Ctl) % 256];
  int lut[256];
  FrameDesc desc;
};
static_assert(sizeof(Ctl) < 256, "control block fits the first 256 bytes");
static_assert(offsetof(Header, lut) % 16 == 0, "table alignment");

constexpr long long align256(long long v) { return (v + 255) & ~255LL; }
constexpr long long STAGE_MIN = 1LL << 20;  // bytes of staging a call must have at least

// Byte offsets of the parts of g_scratch for one problem size.
struct Layout {
  long long zero;      // maxf2 (one frame), tile progress words, look-back words: cleared per call
  long long zero_len;
  long long tdone;
  long long status;
  long long ring0, ring1;
  long long rnew;      // in-place or new-stream accumulate steps: the new reference (4 P)
  long long seg;
  long long staging;
  long long stage_events;
  long long need;      // bytes up to and including the minimum staging
};

Layout layout(long long P, long long nseg, long long tiles, bool rnew) {
  Layout l{};
  const long long nchunks = (nseg + evsim::OCHUNK - 1) / evsim::OCHUNK;
  l.zero = align256(sizeof(Header));
  l.tdone = l.zero + 256;
  l.status = align256(l.tdone + tiles * 8);
  l.zero_len = l.status - l.zero + nchunks * 8;
  l.ring0 = align256(l.zero + l.zero_len);
  l.ring1 = align256(l.ring0 + P);
  l.rnew = align256(l.ring1 + P);
  l.seg = align256(l.rnew + (rnew ? 4 * P : 0));
  l.staging = align256(l.seg + nseg * (long long)sizeof(Seg));
  l.need = l.staging + STAGE_MIN;
  l.stage_events = (SIM_STATIC_SCRATCH_BYTES - l.staging) / (long long)sizeof(Ev);
  return l;
}

int fail(cudaError_t e) {
  evsim::note_cuda_error(e);
  return e == cudaErrorNoDevice || e == cudaErrorInsufficientDriver ||
                 e == cudaErrorNoKernelImageForDevice
             ? SIM_ERR_NO_DEVICE
             : SIM_ERR_CUDA;
}

// With device `dev` current: the array's address in the current context and
// the kernels' shared-memory permission, set up once per device and context
// (again after a cudaDeviceReset).  Every return code is checked.
int device_setup(int dev, unsigned char** out) {
  std::lock_guard<std::mutex> g(g_setup_mu);
  unsigned long long id = current_context_id();
  if (id != 0 && g_dev[dev].ctx_id == id) {
    *out = g_dev[dev].base;
    return SIM_OK;
  }
  void* ptr = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&ptr, g_scratch);  // creates the context if needed
  if (e != cudaSuccess) return fail(e);
  // shared-memory permission of the tile kernels, at the largest substep cap
  // (never below what any handle needs)
  e = evsim::raise_kernel_limits(SIM_MAX_SUBSTEPS, true);
  if (e != cudaSuccess) return fail(e);
  if (id == 0) id = current_context_id();
  g_dev[dev] = DeviceSetup{id, (unsigned char*)ptr};  // id 0: set up again next call
  *out = (unsigned char*)ptr;
  return SIM_OK;
}

bool misaligned(const void* p, unsigned a) { return ((size_t)p & (a - 1)) != 0; }

}  // namespace

extern "C" int sim_step_pair_static(const sim_config* cfg, const void* prev_frame,
                                    int64_t prev_pitch, const void* frame, int64_t pitch,
                                    const float* flow, int64_t t_prev_us, int64_t t_us,
                                    const int32_t* ref_in, int32_t* ref_out, sim_event* events,
                                    int64_t event_capacity, int64_t* n_events) {
  if (!cfg || !n_events) return SIM_ERR_ARG;
  *n_events = 0;
  const sim_config& c = *cfg;
  if (c.width < 1 || c.height < 1 || c.width > SIM_MAX_DIM || c.height > SIM_MAX_DIM) return SIM_ERR_ARG;
  if (c.pixel_format != SIM_LUMA8 && c.pixel_format != SIM_RGB8) return SIM_ERR_ARG;
  if (c.mode != SIM_DENSE && c.mode != SIM_SPARSE) return SIM_ERR_ARG;
  if (c.intensity != SIM_LOG && c.intensity != SIM_LINEAR) return SIM_ERR_ARG;
  if (c.ref_mode != SIM_REF_ACCUM && c.ref_mode != SIM_REF_RESET) return SIM_ERR_ARG;
  if (c.substeps < 0 || c.substeps > SIM_MAX_SUBSTEPS) return SIM_ERR_ARG;
  if (c.substeps == 0 && (c.max_substeps < 1 || c.max_substeps > SIM_MAX_SUBSTEPS)) return SIM_ERR_ARG;
  if (c.c_pos_map || c.c_neg_map) return SIM_ERR_ARG;  // threshold maps: sim_create only
  if (c.event_time != SIM_TIME_SUBSTEP) return SIM_ERR_ARG;  // per-crossing times: sim_create only
  if (event_capacity < 0 || event_capacity > evsim::MAX_EVENTS) return SIM_ERR_ARG;
  if (!prev_frame || !frame || !flow || (event_capacity > 0 && !events)) return SIM_ERR_ARG;
  if (misaligned(flow, 8) || misaligned(events, 8)) return SIM_ERR_ARG;
  const bool accum = c.ref_mode == SIM_REF_ACCUM;
  if (accum && (!ref_out || misaligned(ref_out, 4) || misaligned(ref_in, 4))) return SIM_ERR_ARG;
  const long long row = (long long)c.width * c.pixel_format;
  if (prev_pitch < row || pitch < row) return SIM_ERR_ARG;
  if (t_prev_us < 0) return SIM_ERR_TIME_RANGE;
  if (t_us <= t_prev_us) return SIM_ERR_TIME;
  if (t_us > 4294967295LL) return SIM_ERR_TIME_RANGE;

  Header h;
  std::memset(&h, 0, sizeof(h));
  for (int v = 0; v < 256; ++v)
    h.lut[v] = c.intensity == SIM_LINEAR ? v * 65536 : (int)std::nearbyint(65536.0 * std::log(v + 1.0));
  const long long range = (long long)h.lut[255] - h.lut[0];
  const long long cmin = accum ? (range + 32765) / 32766 : 1;
  if (c.c_pos_q16 < cmin || c.c_pos_q16 >= (1 << 30)) return SIM_ERR_ARG;
  if (c.c_neg_q16 < cmin || c.c_neg_q16 >= (1 << 30)) return SIM_ERR_ARG;

  const int tiles_x = (c.width + evsim::TW - 1) / evsim::TW;
  const int tiles_y = (c.height + evsim::TH - 1) / evsim::TH;
  const int n_max = c.substeps > 0 ? c.substeps : c.max_substeps;
  const long long P = (long long)c.width * c.height;
  const long long segs_per_k = (long long)c.height * tiles_x;
  const long long nseg = (long long)n_max * segs_per_k;
  // The reference is replaced only when the step succeeds: with ref_in given
  // and distinct from ref_out the kernels read ref_in and write ref_out
  // directly; in place (ref_in == ref_out) or with a fresh reference
  // (ref_in = NULL), the new reference goes to the array first and is copied
  // to ref_out after the step has been checked.
  const bool staged_ref = accum && (!ref_in || ref_in == ref_out);
  const Layout L = layout(P, nseg, (long long)tiles_x * tiles_y, staged_ref);
  if (L.need > SIM_STATIC_SCRATCH_BYTES) return SIM_ERR_TOO_LARGE;

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(e);
  if (dev < 0 || dev >= MAX_DEVICES) return SIM_ERR_NO_DEVICE;
  unsigned char* base = nullptr;
  const int rc = device_setup(dev, &base);
  if (rc) return rc;
  const int sms = evsim::device_sm_count();
  cudaStream_t st = c.cuda_stream ? (cudaStream_t)c.cuda_stream : cudaStreamLegacy;

  evsim::SimParams p{};
  p.W = c.width;
  p.H = c.height;
  p.ch = c.pixel_format;
  p.tiles_x = tiles_x;
  p.tiles_y = tiles_y;
  p.tile_h = evsim::TH;
  p.sms = evsim::device_sm_count();
  p.mode = c.mode;
  p.ref_mode = c.ref_mode;
  p.intensity = c.intensity;
  p.n_fixed = c.substeps;
  p.n_max = n_max;
  p.cp = c.c_pos_q16;
  p.cn = c.c_neg_q16;
  p.cact = c.c_act_q16;
  p.bmax = 1;
  p.lut = (const int*)(base + offsetof(Header, lut));
  p.ring0 = base + L.ring0;
  p.ring1 = base + L.ring1;
  p.ctl = (Ctl*)(base + offsetof(Header, ctl));
  p.maxf2 = (unsigned long long*)(base + L.zero);
  p.staging = (Ev*)(base + L.staging);
  p.stage_cap = L.stage_events;
  p.seg = (Seg*)(base + L.seg);
  p.segs_per_k = segs_per_k;
  p.seg_cap = nseg;
  p.order_status = (unsigned long long*)(base + L.status);
  p.tdone = (unsigned long long*)(base + L.tdone);
  p.events = (Ev*)events;
  p.event_cap = event_capacity;

  // control block (zero, t of frame i-1), table and the frame descriptor
  h.ctl.t_prev = t_prev_us;
  h.desc.frame = (const unsigned char*)frame;
  h.desc.pitch = pitch;
  h.desc.flow = (const float2*)flow;
  h.desc.t_rel = t_us;
  e = cudaMemcpyAsync(base, &h, sizeof(h), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(base + L.zero, 0, L.zero_len, st);
  if (e != cudaSuccess) return fail(e);

  // frame i-1: its luma into the ring; with no reference given (accumulate
  // mode), also the reference R = LUT[luma], written to ref_out
  evsim::SimParams pi = p;
  FrameDesc f0{};
  f0.frame = (const unsigned char*)prev_frame;
  f0.pitch = prev_pitch;
  int32_t* rstage = (int32_t*)(base + L.rnew);
  if (accum && !ref_in) {
    pi.R0 = rstage;
  } else {
    pi.ref_mode = SIM_REF_RESET;  // ring only
  }
  e = evsim::launch_init(pi, f0, st);
  if (e != cudaSuccess) return fail(e);
  if (accum) {
    p.R0 = ref_in ? const_cast<int32_t*>(ref_in) : rstage;  // read (sel = 0)
    p.R1 = staged_ref ? rstage : ref_out;                   // written
  }

  evsim::BatchArg b{};
  b.frames = (const FrameDesc*)(base + offsetof(Header, desc));
  b.count = 1;
  b.serial = 1;  // the look-back words were cleared above
  const bool adaptive = c.substeps == 0;
  if (c.mode == SIM_DENSE) {
    if (adaptive) e = evsim::launch_flowmax(p, b, st);
    if (e == cudaSuccess) e = evsim::launch_dense(p, b, st);
  } else {
    if (adaptive) e = evsim::launch_sparse_pre(p, b, st);
    if (e == cudaSuccess) e = evsim::launch_sparse(p, b, st);
  }
  const long long ochunks = (nseg + evsim::OCHUNK - 1) / evsim::OCHUNK;
  const int grid = (int)(ochunks < (long long)sms * 8 ? ochunks : (long long)sms * 8);
  if (e == cudaSuccess) e = evsim::launch_order(p, b, st, grid > 0 ? grid : 1);
  if (e != cudaSuccess) return fail(e);

  Ctl out;
  e = cudaMemcpyAsync(&out, p.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(e);
  if (out.err) return out.err;
  if (staged_ref) {
    e = cudaMemcpyAsync(ref_out, rstage, (size_t)(4 * P), cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(e);
  }
  *n_events = out.cursor;
  return SIM_OK;
}
