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

  // per-step device table: [GroupTotals][StreamStep x max][ActiveTile x max]
  // [FrameDesc x max x fmax], uploaded in one copy from a pinned mirror
  unsigned char* d_step = nullptr;
  unsigned char* h_step = nullptr;
  size_t step_bytes = 0;
  GroupStream* d_gs = nullptr;
  GroupCtl* d_gctl = nullptr;
  cudaEvent_t copy_done = nullptr;
  bool copy_pending = false;

  // launch plan of the current member set
  bool dirty = true;
  int cls_moff[evsim::TILE_CLASSES] = {};   // first work-list slot of each class
  int cls_tiles[evsim::TILE_CLASSES] = {};  // tiles of all members of the class
  int cls_grid[evsim::TILE_CLASSES] = {};
  size_t cls_smem[evsim::TILE_CLASSES] = {};
  int n_classes = 0;
  bool any_adaptive = false;
  int order_grid = 1;
  int pre_grid = 1;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;

  // delivery areas (serving form of a step), alternating
  struct Area {
    unsigned char* host = nullptr;   // pinned, mapped: events, table, total
    evsim::Ev* h_events = nullptr;
    evsim::Delivery* h_table = nullptr;
    long long* h_total = nullptr;
    evsim::Ev* d_events = nullptr;   // device views of the same memory
    evsim::Delivery* d_table = nullptr;
    long long* d_total = nullptr;
    cudaEvent_t done = nullptr;
    int n = 0;
  };
  Area area[2];
  bool delivering = false;
  int next_area = 0;
  int oldest = 0;
  int inflight = 0;
  long long deliv_cap = 0;
  int* d_ids = nullptr;              // member ids in table order

  simb_stats st{};
};

namespace {

static_assert(sizeof(GroupTotals) <= 512, "totals fit their slot");
size_t off_steps() { return 512; }
size_t off_act(const simb_t* g) {
  return (off_steps() + sizeof(StreamStep) * g->cfg.max_streams + 255) & ~(size_t)255;
}
size_t off_desc(const simb_t* g) {
  return (off_act(g) + sizeof(evsim::ActiveTile) * g->cfg.max_streams + 255) & ~(size_t)255;
}
GroupTotals* d_tot(const simb_t* g) { return (GroupTotals*)g->d_step; }
StreamStep* d_steps(const simb_t* g) { return (StreamStep*)(g->d_step + off_steps()); }
evsim::ActiveTile* d_act(const simb_t* g) { return (evsim::ActiveTile*)(g->d_step + off_act(g)); }
FrameDesc* d_desc(const simb_t* g) { return (FrameDesc*)(g->d_step + off_desc(g)); }
GroupTotals* h_tot(const simb_t* g) { return (GroupTotals*)g->h_step; }
StreamStep* h_steps(const simb_t* g) { return (StreamStep*)(g->h_step + off_steps()); }
evsim::ActiveTile* h_act(const simb_t* g) { return (evsim::ActiveTile*)(g->h_step + off_act(g)); }
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

// Rebuild the member table and the launch plan after a change of members
// (the group's stream is idle).
int rebuild(simb_t* g) {
  drop_graph(g);
  const int n = (int)g->members.size();
  std::vector<GroupStream> gs(n);
  int cls_members[evsim::TILE_CLASSES] = {};
  std::fill(std::begin(g->cls_tiles), std::end(g->cls_tiles), 0);
  std::fill(std::begin(g->cls_smem), std::end(g->cls_smem), 0);
  g->any_adaptive = false;
  long long max_chunks = 0;
  for (int i = 0; i < n; ++i) {
    const Member* m = g->members[i];
    g->cls_tiles[m->cls] += m->tiles;
    cls_members[m->cls] += 1;
    g->cls_smem[m->cls] =
        std::max(g->cls_smem[m->cls], evsim::tile_smem_bytes(m->s->n_max, m->s->tile_h));
    g->any_adaptive |= m->adaptive;
    max_chunks += order_chunks(m->s, g->fmax);
    gs[i].p = evsim_rt::make_params(m->s);
    gs[i].p.segflag = nullptr;  // group tile launches write every segment
    gs[i].p.units = nullptr;
    gs[i].frames = d_desc(g) + (size_t)i * g->fmax;
    gs[i].pre_blocks = m->pre_blocks;
  }
  g->n_classes = 0;
  int moff = 0;
  for (int c = 0; c < evsim::TILE_CLASSES; ++c) {
    g->cls_moff[c] = moff;
    moff += cls_members[c];
    // persistent tile grid: the kernel's residency per SM (two 512-thread
    // blocks of 64 x 16 tiles, four 256-thread blocks of 64 x 8)
    const int per_sm = (c & evsim::TILE_TH8) ? 4 : 2;
    g->cls_grid[c] = std::min(g->cls_tiles[c] * g->fmax, per_sm * g->sms);
    if (g->cls_tiles[c]) ++g->n_classes;
  }
  std::vector<int> ids(std::max(n, 1));
  for (int i = 0; i < n; ++i) ids[i] = g->members[i]->id;
  cudaError_t e = cudaMemcpy(g->d_ids, ids.data(), ids.size() * sizeof(int), cudaMemcpyHostToDevice);
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

GroupArg group_arg(const simb_t* g) {
  GroupArg a{};
  a.gs = g->d_gs;
  a.steps = d_steps(g);
  a.tot = d_tot(g);
  a.gctl = g->d_gctl;
  a.n = (int)g->members.size();
  return a;
}

// Pinned, mapped delivery areas (allocated at the first delivery).
int alloc_areas(simb_t* g) {
  const size_t ev = (size_t)g->deliv_cap * sizeof(evsim::Ev);
  const size_t tab = (size_t)g->cfg.max_streams * sizeof(evsim::Delivery);
  for (auto& a : g->area) {
    if (a.host) continue;
    cudaError_t e = cudaHostAlloc((void**)&a.host, ev + tab + 64, cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&a.done, cudaEventDisableTiming);
    unsigned char* d = nullptr;
    if (e == cudaSuccess) e = cudaHostGetDevicePointer((void**)&d, a.host, 0);
    if (e != cudaSuccess) return cuda_rc(e);
    a.h_events = (evsim::Ev*)a.host;
    a.h_table = (evsim::Delivery*)(a.host + ev);
    a.h_total = (long long*)(a.host + ev + tab);
    a.d_events = (evsim::Ev*)d;
    a.d_table = (evsim::Delivery*)(d + ev);
    a.d_total = (long long*)(d + ev + tab);
  }
  return SIM_OK;
}

// The step's launches (also what a graph captures).
cudaError_t launch_step(simb_t* g, int* launches) {
  const GroupArg a = group_arg(g);
  int k = 0;
  cudaError_t e = cudaSuccess;
  if (g->any_adaptive) {
    e = evsim::launch_pre_multi(a, g->pre_grid, g->stream);
    ++k;
  }
  for (int c = 0; c < evsim::TILE_CLASSES && e == cudaSuccess; ++c) {
    if (!g->cls_tiles[c]) continue;
    e = evsim::launch_tile_multi(a, c, d_act(g) + g->cls_moff[c], g->cls_grid[c],
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
  cudaFree(g->d_ids);
  for (auto& a : g->area) {
    if (a.host) cudaFreeHost(a.host);
    if (a.done) cudaEventDestroy(a.done);
  }
  if (g->copy_done) cudaEventDestroy(g->copy_done);
  if (g->own_stream && g->stream) cudaStreamDestroy(g->stream);
}

// A member's configuration: its tile shape is the one asked for (8 or 16),
// else the autotuner table's choice for its configuration when that is a
// tile shape, else 64 x 16 (the group's tile kernel has the two tile shapes;
// the row kernel and block orders do not apply to its ticketed launches).
sim_config member_config(const simb_t* g, const sim_config& c) {
  sim_config mc = c;
  mc.cuda_stream = g->stream;
  mc.max_batch = g->fmax;
  int th = 16, order = 0;
  if (c.tile_height == 8 || c.tile_height == 16)
    th = c.tile_height;
  else if (evsim_rt::tuned_tile_height(c, &th, &order) && th != 8 && th != 16)
    th = 16;
  mc.tile_height = th;
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
  if (cfg->delivery_events < 0 || cfg->delivery_events > evsim::MAX_EVENTS) return SIM_ERR_ARG;
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
  chk(evsim_rt::dalloc(&g->d_ids, (size_t)cfg->max_streams));
  g->deliv_cap = cfg->delivery_events > 0 ? cfg->delivery_events : (1LL << 23);
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
  // single handles only
  if (cfg->mode == SIM_DIFF || cfg->event_time != SIM_TIME_SUBSTEP) return SIM_ERR_ARG;
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
  // pre-pass blocks per frame: dense flow maximum over NT * 8 pixels per
  // block, sparse activity + flow maximum one warp per row
  m->pre_blocks = s->cfg.mode == SIM_SPARSE
                      ? (s->H + evsim::NWARP - 1) / evsim::NWARP
                      : (int)std::max(1LL, (P + evsim::NT * 8 - 1) / (evsim::NT * 8));
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
  evsim::ActiveTile* ha = h_act(g);
  GroupTotals* ht = h_tot(g);
  std::memset(ht, 0, sizeof(GroupTotals));
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
    evsim::ActiveTile& a = ha[g->cls_moff[m->cls] + ht->active[m->cls]++];
    a.member = i;
    a.tile_begin = ht->tiles[m->cls];
    ht->tiles[m->cls] += cnt * m->tiles;  // (frame, tile) items
    chunks += order_chunks(m->s, cnt);
    if (m->adaptive) pre += cnt * m->pre_blocks;
    for (int j = 0; j < cnt; ++j) hd[(size_t)i * g->fmax + j] = m->q[j].d;
    nf += cnt;
  }
  if (nf == 0) return SIM_OK;
  ht->chunks = chunks;
  ht->pre_items = pre;
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

int simb_step_deliver(simb_t* g, int64_t* frames) {
  if (!g) return SIM_ERR_ARG;
  if (frames) *frames = 0;
  if (g->inflight == 2) return SIM_ERR_STATE;
  int rc = alloc_areas(g);
  if (rc) return rc;
  g->delivering = true;
  rc = simb_step(g, frames);
  if (rc) return rc;
  auto& A = g->area[g->next_area];
  evsim::DrainArg d{};
  d.events = A.d_events;
  d.cap = g->deliv_cap;
  d.table = A.d_table;
  d.total = A.d_total;
  d.ids = g->d_ids;
  d.done = &g->d_gctl->drain_done;
  cudaError_t e = evsim::launch_drain(group_arg(g), d, g->sms * 2, g->stream);
  if (e == cudaSuccess) e = cudaEventRecord(A.done, g->stream);
  if (e != cudaSuccess) return cuda_rc(e);
  g->st.kernel_launches += 1;
  A.n = (int)g->members.size();
  g->next_area ^= 1;
  g->inflight += 1;
  return SIM_OK;
}

int simb_collect(simb_t* g, const simb_delivery** table, int32_t* n, const sim_event** events,
                 int64_t* n_events) {
  if (!g || !table || !n || !events || !n_events) return SIM_ERR_ARG;
  if (!g->inflight) return SIM_ERR_STATE;
  auto& A = g->area[g->oldest];
  cudaError_t e = cudaEventSynchronize(A.done);
  if (e != cudaSuccess) return cuda_rc(e);
  bool synced = false;
  for (int i = 0; i < A.n; ++i) {
    if (!A.h_table[i].status) continue;
    Member* m = member(g, A.h_table[i].id);
    if (!m) continue;
    if (!synced) {
      e = cudaStreamSynchronize(g->stream);
      if (e != cudaSuccess) return cuda_rc(e);
      synced = true;
    }
    Ctl c;
    int rc = evsim_rt::read_ctl(m->s, &c);
    if (rc) return rc;
    if (!c.err) continue;  // already rolled back by an earlier collect
    rc = evsim_rt::recover(m->s, &c);
    if (rc) return rc;
    m->q.clear();
  }
  static_assert(sizeof(simb_delivery) == sizeof(evsim::Delivery), "delivery layout");
  *table = (const simb_delivery*)A.h_table;
  *n = A.n;
  *events = (const sim_event*)A.h_events;
  *n_events = *A.h_total;
  g->oldest ^= 1;
  g->inflight -= 1;
  return SIM_OK;
}

int simb_delivery_ready(simb_t* g) {
  if (!g) return SIM_ERR_ARG;
  if (!g->inflight) return SIM_ERR_STATE;
  const cudaError_t e = cudaEventQuery(g->area[g->oldest].done);
  if (e == cudaSuccess) return 1;
  if (e == cudaErrorNotReady) return 0;
  return cuda_rc(e);
}

int simb_pop(simb_t* g, int32_t id, sim_event* out, int64_t cap, int64_t* n_out, int32_t mem) {
  Member* m = member(g, id);
  if (!m) return SIM_ERR_ARG;
  if (g->delivering) return SIM_ERR_STATE;
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
  if (g->inflight) return SIM_ERR_STATE;  // collect the deliveries first
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
