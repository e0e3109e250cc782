// Multi-stream group (simb_*): member streams are sim_t handles on the
// group's CUDA stream; a step advances all members with queued frames with
// one launch per kernel (k_pre_multi, k_tile_multi per tile class,
// k_order_multi), optionally replayed from a CUDA graph captured once per
// member set.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "handle.h"

using evsim::FrameDesc;
using evsim::GroupArg;
using evsim::GroupCtl;
using evsim::GroupStream;
using evsim::GroupTotals;
using evsim::StreamStep;
using evsim_rt::cuda_rc;

namespace {

struct Pending {
  FrameDesc d;
  long long t_us;
};

struct Member {
  sim_t* s = nullptr;
  int id = -1;
  long long bytes = 0;
  int cls = 0;
  int tiles = 0;
  bool adaptive = false;
  int pre_blocks = 0;
  std::vector<Pending> q;
  long long one = 1;  // source of the committed-frame count set by the first frame
};

}  // namespace

struct simb_s {
  simb_config cfg{};
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int sms = 1;
  int fmax = 1;
  std::vector<Member*> members;  // dense, in table order
  std::vector<int> id_slot;      // id -> index in members (-1: free)
  long long bytes_used = 0;

  // device tables: [GroupTotals][StreamStep x max][FrameDesc x max x fmax]
  unsigned char* d_step = nullptr;
  unsigned char* h_step = nullptr;  // pinned mirror
  size_t step_bytes = 0;
  GroupStream* d_gs = nullptr;
  GroupCtl* d_gctl = nullptr;
  int* d_block_map = nullptr;
  size_t block_map_cap = 0;
  cudaEvent_t copy_done = nullptr;
  bool copy_pending = false;

  // launch plan of the current member set
  bool dirty = true;
  int cls_off[evsim::TILE_CLASSES] = {};
  int cls_tiles[evsim::TILE_CLASSES] = {};
  size_t cls_smem[evsim::TILE_CLASSES] = {};
  int n_classes = 0;
  bool any_adaptive = false;
  int order_grid = 1;
  int pre_grid = 1;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;

  simb_stats st{};
};

namespace {

size_t off_steps() { return 256; }
size_t off_desc(const simb_t* g) {
  return (off_steps() + sizeof(StreamStep) * g->cfg.max_streams + 255) & ~(size_t)255;
}
GroupTotals* d_tot(const simb_t* g) { return (GroupTotals*)g->d_step; }
StreamStep* d_steps(const simb_t* g) { return (StreamStep*)(g->d_step + off_steps()); }
FrameDesc* d_desc(const simb_t* g) { return (FrameDesc*)(g->d_step + off_desc(g)); }
GroupTotals* h_tot(const simb_t* g) { return (GroupTotals*)g->h_step; }
StreamStep* h_steps(const simb_t* g) { return (StreamStep*)(g->h_step + off_steps()); }
FrameDesc* h_desc(const simb_t* g) { return (FrameDesc*)(g->h_step + off_desc(g)); }

int order_chunks(const sim_t* s, int count) {
  const long long nseg = (long long)count * s->n_max * s->segs_per_k;
  return (int)std::max(1LL, (nseg + evsim::OCHUNK - 1) / evsim::OCHUNK);
}

void drop_graph(simb_t* g) {
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  g->exec = nullptr;
  g->graph = nullptr;
}

// Rebuild the member table, the tile block maps and the launch plan after a
// change of members (the group's stream is idle).
int rebuild(simb_t* g) {
  drop_graph(g);
  const int n = (int)g->members.size();
  std::vector<GroupStream> gs(n);
  std::fill(std::begin(g->cls_tiles), std::end(g->cls_tiles), 0);
  std::fill(std::begin(g->cls_smem), std::end(g->cls_smem), 0);
  g->any_adaptive = false;
  long long max_chunks = 0;
  for (int i = 0; i < n; ++i) {
    const Member* m = g->members[i];
    g->cls_tiles[m->cls] += m->tiles;
    g->cls_smem[m->cls] = std::max(g->cls_smem[m->cls], evsim::tile_smem_bytes(m->s->n_max));
    g->any_adaptive |= m->adaptive;
    max_chunks += order_chunks(m->s, g->fmax);
  }
  int total = 0;
  g->n_classes = 0;
  for (int c = 0; c < evsim::TILE_CLASSES; ++c) {
    g->cls_off[c] = total;
    total += g->cls_tiles[c];
    if (g->cls_tiles[c]) ++g->n_classes;
  }
  std::vector<int> map(std::max(total, 1));
  int fill[evsim::TILE_CLASSES];
  std::memcpy(fill, g->cls_off, sizeof(fill));
  for (int i = 0; i < n; ++i) {
    const Member* m = g->members[i];
    gs[i].p = evsim_rt::make_params(m->s);
    gs[i].frames = d_desc(g) + (size_t)i * g->fmax;
    gs[i].tile_begin = fill[m->cls] - g->cls_off[m->cls];
    gs[i].pre_blocks = m->pre_blocks;
    for (int t = 0; t < m->tiles; ++t) map[fill[m->cls] + t] = i;
    fill[m->cls] += m->tiles;
  }
  cudaError_t e = cudaSuccess;
  if ((size_t)map.size() > g->block_map_cap) {
    cudaFree(g->d_block_map);
    g->d_block_map = nullptr;
    g->block_map_cap = 0;
    e = evsim_rt::dalloc(&g->d_block_map, map.size() * 2);
    if (e != cudaSuccess) return cuda_rc(e);
    g->block_map_cap = map.size() * 2;
  }
  e = cudaMemcpy(g->d_block_map, map.data(), map.size() * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && n > 0)
    e = cudaMemcpy(g->d_gs, gs.data(), n * sizeof(GroupStream), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    size_t smax = 0;
    for (size_t v : g->cls_smem) smax = std::max(smax, v);
    if (smax) e = evsim::configure_group_kernels(smax);
  }
  if (e != cudaSuccess) return cuda_rc(e);
  g->order_grid = (int)std::max(1LL, std::min<long long>(max_chunks, (long long)g->sms * 8));
  g->pre_grid = g->sms * 4;
  g->st.tile_classes = g->n_classes;
  g->dirty = false;
  return SIM_OK;
}

// The step's launches (also what a graph captures).
cudaError_t launch_step(simb_t* g, int* launches) {
  GroupArg a{};
  a.gs = g->d_gs;
  a.steps = d_steps(g);
  a.tot = d_tot(g);
  a.gctl = g->d_gctl;
  a.n = (int)g->members.size();
  int k = 0;
  cudaError_t e = cudaSuccess;
  if (g->any_adaptive) {
    e = evsim::launch_pre_multi(a, g->pre_grid, g->stream);
    ++k;
  }
  for (int c = 0; c < evsim::TILE_CLASSES && e == cudaSuccess; ++c) {
    if (!g->cls_tiles[c]) continue;
    e = evsim::launch_tile_multi(a, c, g->d_block_map + g->cls_off[c], g->cls_tiles[c],
                                 g->cls_smem[c], g->stream);
    ++k;
  }
  if (e == cudaSuccess) {
    e = evsim::launch_order_multi(a, g->order_grid, g->stream);
    ++k;
  }
  *launches = k;
  return e;
}

Member* member(simb_t* g, int id) {
  if (!g || id < 0 || id >= (int)g->id_slot.size() || g->id_slot[id] < 0) return nullptr;
  return g->members[g->id_slot[id]];
}

void free_group(simb_t* g) {
  drop_graph(g);
  for (Member* m : g->members) {
    sim_destroy(m->s);
    delete m;
  }
  g->members.clear();
  cudaFree(g->d_step);
  cudaFreeHost(g->h_step);
  cudaFree(g->d_gs);
  cudaFree(g->d_gctl);
  cudaFree(g->d_block_map);
  if (g->copy_done) cudaEventDestroy(g->copy_done);
  if (g->own_stream && g->stream) cudaStreamDestroy(g->stream);
}

sim_config member_config(const simb_t* g, const sim_config& c) {
  sim_config mc = c;
  mc.cuda_stream = g->stream;
  mc.max_batch = g->fmax;
  return mc;
}

}  // namespace

extern "C" {

int simb_config_default(simb_config* cfg) {
  if (!cfg) return SIM_ERR_ARG;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->max_streams = 64;
  cfg->frames_per_step = 4;
  cfg->hbm_budget_bytes = 8LL << 30;
  cfg->use_graphs = 1;
  return SIM_OK;
}

int simb_create(const simb_config* cfg, simb_t** out) {
  if (!cfg || !out) return SIM_ERR_ARG;
  if (cfg->max_streams < 1 || cfg->max_streams > SIM_MAX_GROUP) return SIM_ERR_ARG;
  if (cfg->frames_per_step < 1 || cfg->frames_per_step > SIM_MAX_SUBSTEPS) return SIM_ERR_ARG;
  if (cfg->hbm_budget_bytes < 0) return SIM_ERR_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) return SIM_ERR_NO_DEVICE;
  simb_t* g = new (std::nothrow) simb_t();
  if (!g) return SIM_ERR_OOM;
  g->cfg = *cfg;
  if (!g->cfg.hbm_budget_bytes) g->cfg.hbm_budget_bytes = 8LL << 30;
  g->fmax = cfg->frames_per_step;
  g->sms = std::max(1, evsim::device_sm_count());
  g->st.budget = g->cfg.hbm_budget_bytes;
  g->id_slot.assign(cfg->max_streams, -1);
  cudaError_t e = cudaSuccess;
  auto chk = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
  if (cfg->cuda_stream) {
    g->stream = (cudaStream_t)cfg->cuda_stream;
    // the legacy and per-thread default streams cannot be captured
    if (g->stream == cudaStreamLegacy || g->stream == cudaStreamPerThread) g->cfg.use_graphs = 0;
  } else {
    chk(cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking));
    g->own_stream = true;
  }
  g->step_bytes = off_desc(g) + sizeof(FrameDesc) * (size_t)cfg->max_streams * g->fmax;
  chk(evsim_rt::dalloc(&g->d_step, g->step_bytes));
  chk(cudaMallocHost((void**)&g->h_step, g->step_bytes));
  chk(evsim_rt::dalloc(&g->d_gs, (size_t)cfg->max_streams));
  chk(evsim_rt::dalloc(&g->d_gctl, 1));
  chk(cudaEventCreateWithFlags(&g->copy_done, cudaEventDisableTiming));
  if (e == cudaSuccess) {
    std::memset(g->h_step, 0, g->step_bytes);
    chk(cudaMemset(g->d_step, 0, g->step_bytes));
    chk(cudaMemset(g->d_gctl, 0, sizeof(GroupCtl)));
  }
  if (e != cudaSuccess) {
    const int rc = cuda_rc(e);
    free_group(g);
    delete g;
    return rc;
  }
  *out = g;
  return SIM_OK;
}

int simb_state_bytes(const simb_t* g, const sim_config* cfg, int64_t* bytes) {
  if (!g || !cfg || !bytes) return SIM_ERR_ARG;
  const sim_config mc = member_config(g, *cfg);
  const long long P = (long long)cfg->width * cfg->height;
  // host-frame staging holds frames_per_step frames and flows
  *bytes = evsim_rt::state_bytes(mc) + (long long)(g->fmax - 1) * P * cfg->pixel_format +
           (long long)g->fmax * P * 8;
  return SIM_OK;
}

int simb_admit(simb_t* g, const sim_config* cfg, int32_t* id) {
  if (!g || !cfg || !id) return SIM_ERR_ARG;
  int64_t bytes = 0;
  int rc = simb_state_bytes(g, cfg, &bytes);
  if (rc) return rc;
  int slot = -1;
  for (int i = 0; i < (int)g->id_slot.size(); ++i)
    if (g->id_slot[i] < 0) { slot = i; break; }
  if (slot < 0 || g->bytes_used + bytes > g->cfg.hbm_budget_bytes) {
    g->st.admit_refused += 1;
    return SIM_ERR_ADMIT;
  }
  cudaError_t e = cudaStreamSynchronize(g->stream);
  if (e != cudaSuccess) return cuda_rc(e);
  const sim_config mc = member_config(g, *cfg);
  sim_t* s = nullptr;
  rc = sim_create(&mc, &s);
  if (rc) return rc;
  // host-frame staging for a full step, allocated now rather than in a push
  const long long P = s->P;
  cudaFree(s->d_stage_frames);
  s->d_stage_frames = nullptr;
  e = evsim_rt::dalloc(&s->d_stage_frames, (size_t)g->fmax * P * s->ch);
  if (e == cudaSuccess) e = evsim_rt::dalloc(&s->d_stage_flows, (size_t)g->fmax * P);
  if (e != cudaSuccess) {
    sim_destroy(s);
    return cuda_rc(e);
  }
  s->stage_frames = g->fmax;
  Member* m = new (std::nothrow) Member();
  if (!m) {
    sim_destroy(s);
    return SIM_ERR_OOM;
  }
  const evsim::SimParams p = evsim_rt::make_params(s);
  m->s = s;
  m->id = slot;
  m->bytes = bytes;
  m->cls = evsim::tile_class(p);
  m->tiles = s->tiles_x * s->tiles_y;
  m->adaptive = s->cfg.substeps == 0;
  m->pre_blocks = (int)std::max(1LL, (P + evsim::NT * 8 - 1) / (evsim::NT * 8));
  m->q.reserve(g->fmax);
  g->id_slot[slot] = (int)g->members.size();
  g->members.push_back(m);
  g->bytes_used += bytes;
  g->st.members = (int)g->members.size();
  g->st.bytes_used = g->bytes_used;
  g->dirty = true;
  *id = slot;
  return SIM_OK;
}

int simb_push(simb_t* g, int32_t id, const void* frame, int64_t pitch_bytes, const float* flow,
              int64_t t_us, int32_t mem) {
  Member* m = member(g, id);
  if (!m || !frame) return SIM_ERR_ARG;
  if (mem != SIM_HOST && mem != SIM_DEVICE) return SIM_ERR_ARG;
  sim_t* s = m->s;
  const long long row = (long long)s->W * s->ch;
  if (pitch_bytes < row) return SIM_ERR_ARG;
  if (!s->have_first) {
    // frame 0: ring and reference now; the control block starts at zero
    // with one committed frame
    cudaError_t e = cudaMemsetAsync(s->d_ctl, 0, sizeof(Ctl), g->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(&s->d_ctl->committed, &m->one, sizeof(long long),
                          cudaMemcpyHostToDevice, g->stream);
    if (e != cudaSuccess) return cuda_rc(e);
    FrameDesc f{};
    f.frame = (const unsigned char*)frame;
    f.pitch = pitch_bytes;
    if (mem == SIM_HOST) {
      e = cudaMemcpy2DAsync(s->d_stage_frames, row, frame, pitch_bytes, row, s->H,
                            cudaMemcpyHostToDevice, g->stream);
      if (e != cudaSuccess) return cuda_rc(e);
      f.frame = s->d_stage_frames;
      f.pitch = row;
    }
    e = evsim::launch_init(evsim_rt::make_params(s), f, g->stream);
    if (e != cudaSuccess) return cuda_rc(e);
    s->have_first = true;
    s->t0 = s->t_last = t_us;
    s->pushed = 1;
    return SIM_OK;
  }
  if (!flow) return SIM_ERR_ARG;
  const long long tl = m->q.empty() ? s->t_last : m->q.back().t_us;
  if (t_us <= tl) return SIM_ERR_TIME;
  if (t_us - s->t0 > 4294967295LL) return SIM_ERR_TIME_RANGE;
  if ((int)m->q.size() >= g->fmax) return SIM_ERR_STATE;
  Pending pd{};
  pd.t_us = t_us;
  pd.d.t_rel = t_us - s->t0;
  if (mem == SIM_HOST) {
    const int j = (int)m->q.size();
    unsigned char* fd = s->d_stage_frames + (size_t)j * s->P * s->ch;
    float2* fl = s->d_stage_flows + (size_t)j * s->P;
    cudaError_t e = cudaMemcpy2DAsync(fd, row, frame, pitch_bytes, row, s->H,
                                      cudaMemcpyHostToDevice, g->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(fl, flow, s->P * sizeof(float2), cudaMemcpyHostToDevice, g->stream);
    if (e != cudaSuccess) return cuda_rc(e);
    pd.d.frame = fd;
    pd.d.pitch = row;
    pd.d.flow = fl;
  } else {
    pd.d.frame = (const unsigned char*)frame;
    pd.d.pitch = pitch_bytes;
    pd.d.flow = (const float2*)flow;
  }
  m->q.push_back(pd);
  return SIM_OK;
}

int simb_step(simb_t* g, int64_t* frames) {
  if (!g) return SIM_ERR_ARG;
  if (frames) *frames = 0;
  cudaError_t e = cudaSuccess;
  if (g->dirty) {
    e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess) return cuda_rc(e);
    const int rc = rebuild(g);
    if (rc) return rc;
  }
  // the previous step's table upload must have left the pinned mirror
  if (g->copy_pending) {
    e = cudaEventSynchronize(g->copy_done);
    if (e != cudaSuccess) return cuda_rc(e);
    g->copy_pending = false;
  }
  const int n = (int)g->members.size();
  StreamStep* hs = h_steps(g);
  FrameDesc* hd = h_desc(g);
  int chunks = 0, pre = 0;
  long long nf = 0;
  for (int i = 0; i < n; ++i) {
    Member* m = g->members[i];
    const int cnt = (int)m->q.size();
    StreamStep& st = hs[i];
    st.count = cnt;
    st.serial = cnt ? ++m->s->serial : 0;
    st.chunk_begin = chunks;
    st.pre_begin = pre;
    if (!cnt) continue;
    chunks += order_chunks(m->s, cnt);
    if (m->adaptive) pre += cnt * m->pre_blocks;
    for (int j = 0; j < cnt; ++j) hd[(size_t)i * g->fmax + j] = m->q[j].d;
    nf += cnt;
  }
  if (nf == 0) return SIM_OK;
  h_tot(g)->chunks = chunks;
  h_tot(g)->pre_items = pre;
  const size_t bytes = off_desc(g) + sizeof(FrameDesc) * (size_t)n * g->fmax;
  e = cudaMemcpyAsync(g->d_step, g->h_step, bytes, cudaMemcpyHostToDevice, g->stream);
  if (e == cudaSuccess) e = cudaEventRecord(g->copy_done, g->stream);
  if (e != cudaSuccess) return cuda_rc(e);
  g->copy_pending = true;

  int launches = 0;
  if (g->cfg.use_graphs) {
    if (!g->exec) {
      e = cudaStreamBeginCapture(g->stream, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) return cuda_rc(e);
      cudaError_t le = launch_step(g, &launches);
      cudaGraph_t graph = nullptr;
      e = cudaStreamEndCapture(g->stream, &graph);
      if (le != cudaSuccess) e = le;
      if (e == cudaSuccess) e = cudaGraphInstantiate(&g->exec, graph, 0);
      if (e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        g->exec = nullptr;
        return cuda_rc(e);
      }
      g->graph = graph;
      g->st.graph_captures += 1;
    }
    e = cudaGraphLaunch(g->exec, g->stream);
    if (e != cudaSuccess) return cuda_rc(e);
    g->st.graph_launches += 1;
    launches = 1 + (g->any_adaptive ? 1 : 0) + g->n_classes;
  } else {
    e = launch_step(g, &launches);
    if (e != cudaSuccess) return cuda_rc(e);
  }
  for (Member* m : g->members) {
    if (m->q.empty()) continue;
    m->s->t_last = m->q.back().t_us;
    m->s->pushed += (long long)m->q.size();
    m->q.clear();
  }
  g->st.steps += 1;
  g->st.frames_stepped += nf;
  g->st.kernel_launches += launches;
  if (frames) *frames = nf;
  return SIM_OK;
}

int simb_pop(simb_t* g, int32_t id, sim_event* out, int64_t cap, int64_t* n_out, int32_t mem) {
  Member* m = member(g, id);
  if (!m) return SIM_ERR_ARG;
  const int rc = sim_pop_events(m->s, out, cap, n_out, mem);
  // a device failure rolled the member back to its last committed frame:
  // frames queued after the failure are dropped as well
  if (rc == SIM_ERR_EVENT_OVERFLOW || rc == SIM_ERR_DEVICE_TIMEOUT) m->q.clear();
  return rc;
}

int simb_stream_stats(simb_t* g, int32_t id, sim_stats* st) {
  Member* m = member(g, id);
  if (!m) return SIM_ERR_ARG;
  return sim_get_stats(m->s, st);
}

int simb_evict(simb_t* g, int32_t id) {
  Member* m = member(g, id);
  if (!m) return SIM_ERR_ARG;
  cudaError_t e = cudaStreamSynchronize(g->stream);
  if (e != cudaSuccess) return cuda_rc(e);
  const int idx = g->id_slot[id];
  sim_destroy(m->s);
  g->bytes_used -= m->bytes;
  delete m;
  g->members.erase(g->members.begin() + idx);
  g->id_slot[id] = -1;
  for (int i = 0; i < (int)g->members.size(); ++i) g->id_slot[g->members[i]->id] = i;
  g->st.members = (int)g->members.size();
  g->st.bytes_used = g->bytes_used;
  g->dirty = true;
  return SIM_OK;
}

int simb_sync(simb_t* g) {
  if (!g) return SIM_ERR_ARG;
  return cuda_rc(cudaStreamSynchronize(g->stream));
}

int simb_get_stats(simb_t* g, simb_stats* st) {
  if (!g || !st) return SIM_ERR_ARG;
  *st = g->st;
  return SIM_OK;
}

int simb_destroy(simb_t* g) {
  if (!g) return SIM_ERR_ARG;
  cudaStreamSynchronize(g->stream);
  free_group(g);
  delete g;
  return SIM_OK;
}

}  // extern "C"
