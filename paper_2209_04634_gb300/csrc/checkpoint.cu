// State checkpoint and restore of a stream (sim_state_size, sim_get_state,
// sim_set_state): what continuing the simulation needs - the committed frame
// count and times, the last frame's luma (and, in the difference mode, the
// frame before it), the reference (accumulate mode) and the statistics.
// Events not yet popped are output, not state: they stay with the source.
#include <cuda_runtime.h>

#include <cstring>

#include "../../include/evsim.h"
#include "handle.h"
#include "internal.h"

namespace {

struct CkHeader {
  char magic[8];
  int32_t version;
  int32_t W, H, ch, mode, intensity, ref_mode, substeps, max_substeps;
  int32_t c_pos, c_neg, c_act, maps;
  int32_t have_first, last_n;
  int64_t t0, committed, t_prev, pushed, work_px, work_active, batch_events, work_pixels;
  uint64_t clamped;
  int64_t ring_bytes, ring2_bytes, ref_bytes;
};

constexpr char kMagic[8] = {'E', 'V', 'S', 'I', 'M', 'C', 'K', '1'};

long long ring2_bytes(const sim_t* s) { return s->cfg.mode == SIM_DIFF ? s->P : 0; }
long long ref_bytes(const sim_t* s) {
  return s->cfg.ref_mode == SIM_REF_ACCUM ? s->P * (long long)sizeof(int) : 0;
}
long long total_bytes(const sim_t* s) {
  return (long long)sizeof(CkHeader) + s->P + ring2_bytes(s) + ref_bytes(s);
}

bool same_config(const CkHeader& h, const sim_t* s) {
  const sim_config& c = s->cfg;
  return h.W == s->W && h.H == s->H && h.ch == s->ch && h.mode == c.mode &&
         h.intensity == c.intensity && h.ref_mode == c.ref_mode && h.substeps == c.substeps &&
         (c.substeps > 0 || h.max_substeps == c.max_substeps) && h.c_pos == c.c_pos_q16 &&
         h.c_neg == c.c_neg_q16 && h.c_act == c.c_act_q16 &&
         h.maps == (s->d_cpmap != nullptr ? 1 : 0);
}

}  // namespace

using namespace evsim_rt;

extern "C" {

int sim_state_size(const sim_t* s, int64_t* bytes) {
  if (!s || !bytes) return SIM_ERR_ARG;
  *bytes = total_bytes(s);
  return SIM_OK;
}

int sim_get_state(sim_t* s, void* buf, int64_t bytes) {
  if (!s || !buf || bytes != total_bytes(s)) return SIM_ERR_ARG;
  Ctl c;
  int rc = read_ctl(s, &c);
  if (rc) return rc;
  if (c.err) return SIM_ERR_STATE;  // a failed batch must be reported (sim_sync) first
  CkHeader h;
  std::memset(&h, 0, sizeof(h));
  std::memcpy(h.magic, kMagic, sizeof(kMagic));
  h.version = 2;  // 2: the header carries the simulated-pixel count
  h.W = s->W;
  h.H = s->H;
  h.ch = s->ch;
  h.mode = s->cfg.mode;
  h.intensity = s->cfg.intensity;
  h.ref_mode = s->cfg.ref_mode;
  h.substeps = s->cfg.substeps;
  h.max_substeps = s->cfg.max_substeps;
  h.c_pos = s->cfg.c_pos_q16;
  h.c_neg = s->cfg.c_neg_q16;
  h.c_act = s->cfg.c_act_q16;
  h.maps = s->d_cpmap != nullptr ? 1 : 0;
  h.have_first = s->have_first ? 1 : 0;
  h.last_n = c.last_n;
  h.t0 = s->t0;
  h.committed = c.committed;
  h.t_prev = c.t_prev;
  h.pushed = s->pushed;
  h.work_px = c.work_px;
  h.work_active = c.work_active;
  h.work_pixels = c.work_pixels;
  h.batch_events = c.batch_events;
  h.clamped = c.clamped;
  h.ring_bytes = s->P;
  h.ring2_bytes = ring2_bytes(s);
  h.ref_bytes = ref_bytes(s);
  unsigned char* out = (unsigned char*)buf;
  std::memcpy(out, &h, sizeof(h));
  out += sizeof(h);
  if (!s->have_first) {  // nothing simulated yet: no frame, no reference
    std::memset(out, 0, (size_t)(bytes - (long long)sizeof(h)));
    return SIM_OK;
  }
  cudaError_t e = cudaMemcpy(out, (c.sel & 2) ? s->d_ring[1] : s->d_ring[0], s->P,
                             cudaMemcpyDeviceToHost);
  out += s->P;
  if (e == cudaSuccess && h.ring2_bytes)
    e = cudaMemcpy(out, (c.sel & 2) ? s->d_ring2[1] : s->d_ring2[0], s->P,
                   cudaMemcpyDeviceToHost);
  out += h.ring2_bytes;
  if (e == cudaSuccess && h.ref_bytes)
    e = cudaMemcpy(out, (c.sel & 1) ? s->d_R[1] : s->d_R[0], h.ref_bytes,
                   cudaMemcpyDeviceToHost);
  return cuda_rc(e);
}

int sim_set_state(sim_t* s, const void* buf, int64_t bytes) {
  if (!s || !buf || bytes != total_bytes(s)) return SIM_ERR_ARG;
  CkHeader h;
  std::memcpy(&h, buf, sizeof(h));
  if (std::memcmp(h.magic, kMagic, sizeof(kMagic)) != 0 || h.version != 2) return SIM_ERR_ARG;
  if (!same_config(h, s) || h.ring_bytes != s->P || h.ring2_bytes != ring2_bytes(s) ||
      h.ref_bytes != ref_bytes(s) || h.committed < 0 || h.t_prev < 0)
    return SIM_ERR_ARG;
  cudaError_t e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_rc(e);
  Ctl c;
  std::memset(&c, 0, sizeof(c));
  c.sel = 0;
  c.last_n = h.last_n;
  c.t_prev = h.t_prev;
  c.committed = h.committed;
  c.work_px = h.work_px;
  c.work_active = h.work_active;
  c.work_pixels = h.work_pixels;
  c.batch_events = h.batch_events;
  c.clamped = h.clamped;
  const unsigned char* in = (const unsigned char*)buf + sizeof(h);
  e = cudaMemcpy(s->d_ctl, &c, sizeof(c), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(s->d_maxf2, 0, s->bmax * sizeof(unsigned long long));
  if (e == cudaSuccess && h.have_first) {
    e = cudaMemcpy(s->d_ring[0], in, s->P, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && h.ring2_bytes)
      e = cudaMemcpy(s->d_ring2[0], in + s->P, s->P, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && h.ref_bytes)
      e = cudaMemcpy(s->d_R[0], in + s->P + h.ring2_bytes, h.ref_bytes, cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) return cuda_rc(e);
  s->have_first = h.have_first != 0;
  s->t0 = h.t0;
  s->t_last = h.t0 + h.t_prev;
  s->pushed = h.pushed;
  s->popped = 0;
  return SIM_OK;
}

}  // extern "C"
