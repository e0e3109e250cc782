// Serving loop (sim_serve_run): a Poisson arrival trace of camera streams
// served either by continuous batching over a group (simb_step_deliver /
// simb_collect) or by one sim_t and CUDA stream per camera.  Host code only;
// every simulation step runs in the library's kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <thread>
#include <vector>

#include "handle.h"

namespace {

using clk = std::chrono::steady_clock;

// SplitMix64 (Steele, Lea and Flood 2014): the arrival trace's generator.
struct Mix {
  uint64_t x;
  uint64_t next() {
    uint64_t z = (x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
  double uniform() { return (double)(next() >> 11) * (1.0 / 9007199254740992.0); }
};

struct Req {
  int sid;
  double arrive;  // s; warm-start streams arrive at 0
  double dur;     // s from admission
  int pool, fps, phase;
};

std::vector<Req> make_trace(const sim_serve_config& c) {
  Mix m{c.seed};
  std::vector<Req> out;
  const double t0 = c.warm_start ? -c.dur_max_s : 0.0;
  double t = t0;
  for (;;) {
    t += -std::log(1.0 - m.uniform()) / c.rate_per_s;
    if (t >= c.horizon_s) break;
    Req r{};
    r.pool = (int)(m.uniform() * c.n_pools) % c.n_pools;
    r.fps = c.fps[(int)(m.uniform() * c.n_fps) % c.n_fps];
    r.dur = c.dur_min_s + (c.dur_max_s - c.dur_min_s) * m.uniform();
    r.arrive = t;
    if (t < 0) {  // arrived before the window: present at 0 with what remains
      if (t + r.dur <= 0) continue;
      r.dur += t;
      r.arrive = 0;
    }
    r.sid = (int)out.size();
    const int U = c.pools[r.pool].frames;
    r.phase = r.sid % (2 * (U - 1));
    out.push_back(r);
  }
  std::stable_sort(out.begin(), out.end(),
                   [](const Req& a, const Req& b) { return a.arrive < b.arrive; });
  return out;
}

// Pool frame played at position t of a forward-backward replay of U frames.
int pp_at(long long t, int U) {
  const long long period = 2LL * (U - 1);
  const long long p = t % period;
  return (int)(p < U ? p : period - p);
}

struct FrameIn {
  const void* frame;
  const float* flow;
};

// Frame j of a stream (j >= 1: with the flow from frame j-1).
FrameIn frame_of(const sim_serve_pool& pl, int phase, long long j) {
  const int U = pl.frames;
  const int b = pp_at(j + phase, U);
  FrameIn f{pl.frame[b], nullptr};
  if (j > 0) {
    const int a = pp_at(j - 1 + phase, U);
    f.flow = b == a + 1 ? pl.flow[b] : pl.flow_back[a];
  }
  return f;
}

long long t_of(long long j, int fps) { return (long long)std::llround((double)j * 1e6 / fps); }

sim_config stream_config(const sim_serve_config& c, const sim_serve_pool& pl) {
  sim_config sc;
  sim_config_default(&sc, pl.width, pl.height);
  sc.mode = c.mode;
  sc.substeps = pl.substeps;
  sc.max_substeps = pl.max_substeps;
  sc.c_pos_q16 = pl.c_pos_q16;
  sc.c_neg_q16 = pl.c_neg_q16;
  sc.c_pos_map = pl.c_pos_map;
  sc.c_neg_map = pl.c_neg_map;
  sc.event_capacity = std::max<long long>(1 << 16, c.events_per_pixel * pl.width * pl.height);
  sc.max_batch = c.frames_per_step;
  return sc;
}

// Device bytes charged for a stream (the group's admission formula: state,
// plus host-frame staging for a full step).
long long stream_bytes(const sim_serve_config& c, const sim_config& sc) {
  const long long P = (long long)sc.width * sc.height;
  return evsim_rt::state_bytes(sc) + (long long)(c.frames_per_step - 1) * P +
         (long long)c.frames_per_step * P * 8;
}

struct Live {
  Req r;
  int id = -1;          // group member id
  sim_t* sim = nullptr; // per-stream handle
  long long bytes = 0;
  double start = 0;
  long long next = 1;   // next frame to release
  long long total = 1;  // frames released in all (frame 0 included)
  std::deque<std::pair<long long, double>> inflight;  // (frame, release time)
  int queued = 0;       // group: frames pushed since the last step
  long long delivered = 1;
  long long events = 0;
  long long work = 0;
  uint64_t digest = 0;
  int status = SIM_OK;
  bool done = false;
};

// Order-sensitive digest of an event stream: Horner's rule over the events
// as 64-bit words, h = h * M + e (mod 2^64).
constexpr uint64_t DIGEST_M = 0x9E3779B97F4A7C15ull;
void digest(uint64_t& h, const sim_event* e, size_t n) {
  for (size_t i = 0; i < n; ++i) {
    uint64_t w;
    std::memcpy(&w, e + i, 8);
    h = h * DIGEST_M + w;
  }
}

struct Loop {
  const sim_serve_config& c;
  sim_serve_result& res;
  std::vector<Req> trace;
  std::vector<Live> live;  // by trace index (only admitted ones are used)
  std::vector<int> active;
  std::deque<int> waitq;
  size_t ai = 0;
  long long used = 0;
  std::vector<double> lat, wait;
  clk::time_point t0;
  double last_delivery = 0;

  Loop(const sim_serve_config& cfg, sim_serve_result& r) : c(cfg), res(r) {}

  double now() const { return std::chrono::duration<double>(clk::now() - t0).count(); }

  double release_time(const Live& s, long long j) const { return s.start + (double)j / s.r.fps; }

  void complete(Live& s, long long upto, double t) {
    // frames with index < upto are delivered
    while (!s.inflight.empty() && s.inflight.front().first < upto) {
      const double rel = s.inflight.front().second;
      if (rel >= c.warmup_s) lat.push_back((t - rel) * 1e3);
      s.inflight.pop_front();
      res.frames_completed += 1;
    }
    s.delivered = std::max(s.delivered, upto);
  }

  void arrivals(double t) {
    while (ai < trace.size() && trace[ai].arrive <= t) {
      waitq.push_back((int)ai++);
      res.arrived += 1;
    }
  }

  void record(const Live& s) {
    if (!c.streams || res.streams_written >= c.streams_cap) return;
    sim_serve_stream& o = c.streams[res.streams_written++];
    const sim_serve_pool& pl = c.pools[s.r.pool];
    o.sid = s.r.sid;
    o.width = pl.width;
    o.height = pl.height;
    o.fps = s.r.fps;
    o.pool = s.r.pool;
    o.phase = s.r.phase;
    o.frames = (int32_t)s.delivered;
    o.status = s.status;
    o.events = s.events;
    o.digest = s.digest;
  }

  // frames of a stream admitted at `start`: released while both its duration
  // and the horizon last
  long long frames_total(const Req& r, double start) const {
    const double end = std::min(start + r.dur, c.horizon_s);
    if (end <= start) return 1;
    return 1 + (long long)std::floor((end - start) * r.fps - 1e-9);
  }

  void finish_stats(double t_end) {
    res.wall_s = t_end;
    std::sort(lat.begin(), lat.end());
    auto pct = [](const std::vector<double>& v, double q) {
      if (v.empty()) return 0.0;
      const size_t i = std::min(v.size() - 1, (size_t)std::ceil(q * v.size()) - (q > 0 ? 1 : 0));
      return v[i];
    };
    res.latencies = (int64_t)lat.size();
    res.lat_p50_ms = pct(lat, 0.50);
    res.lat_p90_ms = pct(lat, 0.90);
    res.lat_p99_ms = pct(lat, 0.99);
    res.lat_max_ms = lat.empty() ? 0 : lat.back();
    double sum = 0;
    for (double v : lat) sum += v;
    res.lat_mean_ms = lat.empty() ? 0 : sum / lat.size();
    if (c.latency_ms) {
      const size_t n = std::min<size_t>(lat.size(), (size_t)std::max<int64_t>(0, c.latency_cap));
      std::memcpy(c.latency_ms, lat.data(), n * sizeof(double));
    }
    std::sort(wait.begin(), wait.end());
    res.admit_wait_p50_ms = pct(wait, 0.50);
    res.admit_wait_p99_ms = pct(wait, 0.99);
    res.never_admitted = (int64_t)waitq.size() + (int64_t)(trace.size() - ai);
    res.gpix_substeps_per_s = t_end > 0 ? res.pixel_substeps / t_end / 1e9 : 0;
    res.events_per_s = t_end > 0 ? res.events / t_end : 0;
  }

  // sleep until the next arrival or release (at most `cap` seconds)
  void idle(double t, double cap) {
    double next = t + cap;
    if (ai < trace.size()) next = std::min(next, trace[ai].arrive);
    for (int k : active) {
      const Live& s = live[k];
      if (s.next < s.total) next = std::min(next, release_time(s, s.next));
    }
    const double dt = next - t;
    if (dt > 2e-5) std::this_thread::sleep_for(std::chrono::duration<double>(std::min(dt, cap)));
  }
};

int run_group(Loop& L) {
  const sim_serve_config& c = L.c;
  simb_config gc;
  simb_config_default(&gc);
  gc.max_streams = c.max_streams;
  gc.frames_per_step = c.frames_per_step;
  gc.hbm_budget_bytes = c.hbm_budget_bytes + (1LL << 30);  // the loop applies the budget
  gc.use_graphs = 1;
  gc.delivery_events = 1LL << 24;
  simb_t* g = nullptr;
  int rc = simb_create(&gc, &g);
  if (rc) return rc;
  std::vector<int> id2k(c.max_streams, -1);
  int inflight = 0;
  std::vector<int> finishing;

  auto collect = [&]() -> int {
    const simb_delivery* tab = nullptr;
    int32_t n = 0;
    const sim_event* ev = nullptr;
    int64_t ne = 0;
    int r = simb_collect(g, &tab, &n, &ev, &ne);
    if (r) return r;
    --inflight;
    const double t = L.now();
    L.last_delivery = t;
    for (int i = 0; i < n; ++i) {
      const simb_delivery& d = tab[i];
      const int k = id2k[d.id];
      if (k < 0) continue;
      Live& s = L.live[k];
      if (d.count > 0) digest(s.digest, ev + d.first, (size_t)d.count);
      s.events += d.count;
      L.res.events += d.count;
      L.res.pixel_substeps += d.pixel_substeps - s.work;
      s.work = d.pixel_substeps;
      if (d.status) {
        if (s.status == SIM_OK) s.status = d.status;
        L.res.frames_failed += (long long)s.inflight.size();
        s.inflight.clear();
        s.next = s.total;  // a failed stream releases nothing more
      } else {
        L.complete(s, d.frames_committed, t);
      }
    }
    return SIM_OK;
  };
  auto drain_all = [&]() -> int {
    while (inflight) {
      int r = collect();
      if (r) return r;
    }
    return SIM_OK;
  };

  L.t0 = clk::now();
  for (;;) {
    double t = L.now();
    bool did = false;
    L.arrivals(t);
    // leave: streams whose frames are all delivered (ids are reused, so no
    // delivery may be in flight)
    if (!finishing.empty()) {
      if ((rc = drain_all())) break;
      for (int k : finishing) {
        Live& s = L.live[k];
        L.record(s);
        simb_evict(g, s.id);
        id2k[s.id] = -1;
        L.used -= s.bytes;
        L.active.erase(std::find(L.active.begin(), L.active.end(), k));
      }
      finishing.clear();
      did = true;
    }
    // admission, first come first served
    while (!L.waitq.empty() && t < c.horizon_s && (int)L.active.size() < c.max_streams) {
      const Req& r = L.trace[L.waitq.front()];
      const sim_serve_pool& pl = c.pools[r.pool];
      const sim_config sc = stream_config(c, pl);
      const long long b = stream_bytes(c, sc);
      if (L.used + b > c.hbm_budget_bytes) break;
      int32_t id = -1;
      if ((rc = simb_admit(g, &sc, &id))) break;
      Live& s = L.live[r.sid];
      s.r = r;
      s.id = id;
      s.bytes = b;
      t = L.now();
      s.start = t;
      s.total = L.frames_total(r, t);
      id2k[id] = r.sid;
      L.used += b;
      L.wait.push_back((t - r.arrive) * 1e3);
      const FrameIn f0 = frame_of(pl, r.phase, 0);
      if ((rc = simb_push(g, id, f0.frame, pl.width, nullptr, 0, SIM_DEVICE))) break;
      L.active.push_back(r.sid);
      L.waitq.pop_front();
      L.res.admitted += 1;
      L.res.peak_streams = std::max<int64_t>(L.res.peak_streams, (int64_t)L.active.size());
      did = true;
    }
    if (rc) break;
    // release the frames that have arrived
    bool queued = false;
    for (int k : L.active) {
      Live& s = L.live[k];
      while (s.next < s.total && s.queued < c.frames_per_step &&
             (int)s.inflight.size() < 2 * c.frames_per_step && L.release_time(s, s.next) <= t) {
        const sim_serve_pool& pl = c.pools[s.r.pool];
        const FrameIn f = frame_of(pl, s.r.phase, s.next);
        if ((rc = simb_push(g, s.id, f.frame, pl.width, f.flow, t_of(s.next, s.r.fps),
                            SIM_DEVICE)))
          break;
        s.inflight.emplace_back(s.next, L.release_time(s, s.next));
        s.next += 1;
        s.queued += 1;
        L.res.frames_released += 1;
        queued = true;
      }
      if (rc) break;
    }
    if (rc) break;
    // collect a finished step without waiting
    if (inflight && simb_delivery_ready(g) == 1) {
      if ((rc = collect())) break;
      did = true;
    }
    if (queued) {
      if (inflight == 2 && (rc = collect())) break;
      int64_t nf = 0;
      if ((rc = simb_step_deliver(g, &nf))) break;
      ++inflight;
      L.res.steps += 1;
      for (int k : L.active) L.live[k].queued = 0;
      did = true;
    }
    for (int k : L.active) {
      Live& s = L.live[k];
      if (!s.done && s.next >= s.total && s.inflight.empty()) {
        s.done = true;
        finishing.push_back(k);
      }
    }
    const bool more = L.ai < L.trace.size() && t < c.horizon_s;
    if (!more && L.active.empty() && finishing.empty() && !inflight) break;
    // nothing done: sleep briefly (shorter while a step is in flight, so that
    // its events are collected soon after it ends)
    if (!did) L.idle(t, inflight ? 2e-5 : 2e-4);
  }
  if (!rc) rc = drain_all();
  for (int k : L.active) L.record(L.live[k]);
  simb_stats gs{};
  simb_get_stats(g, &gs);
  L.res.kernel_launches = gs.kernel_launches;
  simb_destroy(g);
  L.finish_stats(L.last_delivery);
  return rc;
}

int run_per_stream(Loop& L) {
  const sim_serve_config& c = L.c;
  long long bufcap = 1;
  for (int i = 0; i < c.n_pools; ++i)
    bufcap = std::max<long long>(bufcap, stream_config(c, c.pools[i]).event_capacity);
  sim_event* buf = nullptr;
  cudaError_t e = cudaMallocHost((void**)&buf, (size_t)bufcap * sizeof(sim_event));
  if (e != cudaSuccess) return evsim_rt::cuda_rc(e);
  int rc = SIM_OK;
  long long launches = 0;

  auto pop = [&](Live& s) -> int {
    int64_t n = 0;
    int r;
    do {
      r = sim_pop_events(s.sim, buf, bufcap, &n, SIM_HOST);
      if (r < 0) break;
      if (n > 0) digest(s.digest, buf, (size_t)n);
      s.events += n;
      L.res.events += n;
    } while (r == SIM_MORE);
    const double t = L.now();
    L.last_delivery = t;
    if (r < 0) {
      if (s.status == SIM_OK) s.status = r;
      L.res.frames_failed += (long long)s.inflight.size();
      s.inflight.clear();
      s.next = s.total;
      return SIM_OK;
    }
    L.complete(s, s.next, t);
    return SIM_OK;
  };
  auto leave = [&](int k) {
    Live& s = L.live[k];
    sim_stats st{};
    if (sim_get_stats(s.sim, &st) == SIM_OK) L.res.pixel_substeps += st.pixel_substeps;
    L.record(s);
    sim_destroy(s.sim);
    s.sim = nullptr;
    L.used -= s.bytes;
  };

  L.t0 = clk::now();
  for (;;) {
    double t = L.now();
    bool did = false;
    L.arrivals(t);
    while (!L.waitq.empty() && t < c.horizon_s && (int)L.active.size() < c.max_streams) {
      const Req& r = L.trace[L.waitq.front()];
      const sim_serve_pool& pl = c.pools[r.pool];
      const sim_config sc = stream_config(c, pl);
      const long long b = stream_bytes(c, sc);
      if (L.used + b > c.hbm_budget_bytes) break;
      Live& s = L.live[r.sid];
      if ((rc = sim_create(&sc, &s.sim))) break;
      s.r = r;
      s.bytes = b;
      t = L.now();
      s.start = t;
      s.total = L.frames_total(r, t);
      L.used += b;
      L.wait.push_back((t - r.arrive) * 1e3);
      const FrameIn f0 = frame_of(pl, r.phase, 0);
      if ((rc = sim_push_frame(s.sim, f0.frame, pl.width, nullptr, 0, SIM_DEVICE))) break;
      launches += 1;
      L.active.push_back(r.sid);
      L.waitq.pop_front();
      L.res.admitted += 1;
      L.res.peak_streams = std::max<int64_t>(L.res.peak_streams, (int64_t)L.active.size());
      did = true;
    }
    if (rc) break;
    // push every frame that has arrived, on its camera's own stream
    std::vector<int> pushed;
    for (int k : L.active) {
      Live& s = L.live[k];
      bool any = false;
      while (s.next < s.total && (int)s.inflight.size() < c.frames_per_step &&
             L.release_time(s, s.next) <= t) {
        const sim_serve_pool& pl = c.pools[s.r.pool];
        const FrameIn f = frame_of(pl, s.r.phase, s.next);
        if ((rc = sim_push_frame(s.sim, f.frame, pl.width, f.flow, t_of(s.next, s.r.fps),
                                 SIM_DEVICE)))
          break;
        launches += pl.substeps == 0 ? 3 : 2;
        s.inflight.emplace_back(s.next, L.release_time(s, s.next));
        s.next += 1;
        L.res.frames_released += 1;
        any = true;
      }
      if (rc) break;
      if (any) pushed.push_back(k);
    }
    if (rc) break;
    for (int k : pushed) {
      if ((rc = pop(L.live[k]))) break;
      did = true;
    }
    if (rc) break;
    for (size_t i = 0; i < L.active.size();) {
      const int k = L.active[i];
      Live& s = L.live[k];
      if (s.next >= s.total && s.inflight.empty()) {
        leave(k);
        L.active.erase(L.active.begin() + i);
        did = true;
      } else {
        ++i;
      }
    }
    const bool more = L.ai < L.trace.size() && t < c.horizon_s;
    if (!more && L.active.empty()) break;
    if (!did) L.idle(t, 2e-4);
  }
  for (int k : L.active) leave(k);
  cudaFreeHost(buf);
  L.res.kernel_launches = launches;
  L.res.steps = 0;
  L.finish_stats(L.last_delivery);
  return rc;
}

}  // namespace

extern "C" int sim_serve_run(const sim_serve_config* cfg, sim_serve_result* res) {
  if (!cfg || !res) return SIM_ERR_ARG;
  const sim_serve_config& c = *cfg;
  if (c.policy != SIM_SERVE_GROUP && c.policy != SIM_SERVE_PER_STREAM) return SIM_ERR_ARG;
  if (c.mode != SIM_DENSE && c.mode != SIM_SPARSE) return SIM_ERR_ARG;
  if (!(c.horizon_s > 0) || !(c.rate_per_s > 0) || c.dur_min_s < 0 || c.dur_max_s < c.dur_min_s)
    return SIM_ERR_ARG;
  if (c.n_pools < 1 || !c.pools || c.n_fps < 1 || !c.fps) return SIM_ERR_ARG;
  if (c.max_streams < 1 || c.max_streams > SIM_MAX_GROUP) return SIM_ERR_ARG;
  if (c.frames_per_step < 1 || c.frames_per_step > SIM_MAX_SUBSTEPS) return SIM_ERR_ARG;
  if (c.hbm_budget_bytes <= 0 || c.events_per_pixel < 1) return SIM_ERR_ARG;
  for (int i = 0; i < c.n_fps; ++i)
    if (c.fps[i] < 1 || c.fps[i] > 1000) return SIM_ERR_ARG;
  for (int i = 0; i < c.n_pools; ++i) {
    const sim_serve_pool& p = c.pools[i];
    if (p.frames < 2 || !p.frame || !p.flow || !p.flow_back) return SIM_ERR_ARG;
  }
  std::memset(res, 0, sizeof(*res));
  Loop L(c, *res);
  L.trace = make_trace(c);
  L.live.resize(L.trace.size());
  return c.policy == SIM_SERVE_GROUP ? run_group(L) : run_per_stream(L);
}
