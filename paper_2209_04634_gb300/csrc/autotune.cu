// Autotuner of the batch kernel's tile shape (sim_autotune): both tile shapes
// and the row kernel run the same frames, the fastest is recorded per
// configuration in a process-wide table that sim_create consults.  The paper has no
// counterpart; the choice changes only how the work is launched, never the
// events (both shapes compute the same integer arithmetic).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "../../include/evsim.h"
#include "handle.h"
#include "internal.h"

namespace {

using Key = std::tuple<int, int, int, int, int, int, int, int, int>;

struct Entry {
  int th, order;
  double us16, us8;  // best per-frame time of each tile shape over the block orders
  double us_rows;    // per-frame time of the row kernel (0: not timed)
};

std::mutex g_tune_mu;
constexpr double kMargin = 0.95;  // another choice than 64x16 / linear only when 5 % faster
std::map<Key, Entry> g_table;

Key key_of(const sim_config& c) {
  // max_substeps matters only for adaptive N
  return Key{c.width, c.height, c.pixel_format, c.mode, c.substeps,
             c.substeps == 0 ? c.max_substeps : 0, c.intensity, c.ref_mode,
             c.c_pos_map != nullptr ? 1 : 0};
}

// Probe frame j of a moving sinusoidal texture (the same content for both
// shapes), and a constant flow of (3.0, -2.0) px per frame.
__global__ void k_probe(unsigned char* frames, float2* flows, int W, int H, int ch, int F) {
  const long long P = (long long)W * H;
  const long long total = P * F;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(i / P);
    const long long r = i - (long long)j * P;
    const int y = (int)(r / W), x = (int)(r - (long long)y * W);
    const float u = x - 3.0f * j, v = y + 2.0f * j;
    const float a = 128.f + 70.f * __sinf(0.09f * u + 0.6f * __sinf(0.031f * v)) +
                    40.f * __sinf(0.13f * v - 0.05f * u);
    const int g = min(255, max(0, (int)a));
    for (int c = 0; c < ch; ++c) frames[i * ch + c] = (unsigned char)min(255, g + 9 * c);
    flows[i] = make_float2(3.0f, -2.0f);
  }
}

int rc_of(cudaError_t e) { return evsim_rt::cuda_rc(e); }

// Per-frame time (us) of the simulation kernel of a stream with tile height th
// on frames[0..count): frame 0 starts the stream, frames 1.. form one batch;
// run twice (the first pass warms up), the second pass's tile launch timed.
int time_shape(const sim_config& c, int th, int order, int count, const void* const* frames,
               int64_t pitch, const float* const* flows, const int64_t* t_us, int32_t mem,
               double* us) {
  sim_config tc = c;
  tc.tile_height = th;
  tc.event_time = SIM_TIME_SUBSTEP;  // the table serves the substep-time kernels only
  tc.cuda_stream = nullptr;
  tc.max_batch = count - 1;
  tc.event_capacity = std::min<long long>((long long)c.width * c.height * 2 * count, 1LL << 27);
  sim_t* s = nullptr;
  int rc = sim_create(&tc, &s);
  if (rc) return rc;
  s->block_order = order;
  const int kind = c.mode == SIM_SPARSE ? SIM_K_SPARSE : SIM_K_DENSE;
  // An event overflow only means the batch did not commit: its kernels ran
  // in full and were timed.
  auto ok = [](int r) { return r == SIM_OK || r == SIM_ERR_EVENT_OVERFLOW ? SIM_OK : r; };
  for (int pass = 0; pass < 2 && !rc; ++pass) {
    if (pass == 1) {
      rc = sim_reset(s);
      if (!rc) rc = sim_set_profiling(s, 1);
    }
    if (!rc) rc = sim_push_frames(s, count, frames, pitch, flows, t_us, mem);
    if (!rc) rc = ok(sim_sync(s));
  }
  double ms = 0;
  int64_t n = 0;
  if (!rc) rc = sim_kernel_time(s, kind, &ms, &n, 1);
  const int rd = sim_destroy(s);
  if (!rc) rc = rd;
  if (!rc && n < 1) rc = SIM_ERR_STATE;
  if (!rc) *us = ms * 1e3 / (count - 1);
  return rc;
}

int valid_cfg(const sim_config& c) {
  if (c.width < 1 || c.height < 1 || c.width > SIM_MAX_DIM || c.height > SIM_MAX_DIM)
    return SIM_ERR_ARG;
  if (c.pixel_format != SIM_LUMA8 && c.pixel_format != SIM_RGB8) return SIM_ERR_ARG;
  return SIM_OK;
}

// Time both shapes in each block order (linear, serpentine, balanced) on the
// frames and record the fastest; the default (64x16, linear order) unless
// another choice is at least 5 % faster (a sample's timings scatter by a few
// percent).  The balanced order plans each batch from samples of its own
// flows, as in a stream.
int tune(const sim_config& c, int count, const void* const* frames, int64_t pitch,
         const float* const* flows, const int64_t* t_us, int32_t mem, int32_t* th_out,
         double* us_out) {
  const int shapes[2] = {16, 8};
  // the row kernel serves dense and sparse interpolation
  double us_rows = 0;
  if (c.mode != SIM_DIFF) {
    const int rc = time_shape(c, SIM_TILE_ROWS, 0, count, frames, pitch, flows, t_us, mem,
                              &us_rows);
    if (rc) return rc;
  }
  const long long T16 = ((c.width + 63) / 64) * (long long)((c.height + 15) / 16);
  const int norders = T16 * 2 <= evsim::PLAN_MAX_TILES ? 3 : 2;  // balanced needs a plan
  double us[2][3] = {{0, 0, 0}, {0, 0, 0}};
  for (int a = 0; a < 2; ++a)
    for (int o = 0; o < norders; ++o) {
      const int rc = time_shape(c, shapes[a], o, count, frames, pitch, flows, t_us, mem, &us[a][o]);
      if (rc) return rc;
    }
  int ba = 0, bo = 0;
  for (int a = 0; a < 2; ++a)
    for (int o = 0; o < norders; ++o)
      if (us[a][o] < us[ba][bo]) { ba = a; bo = o; }
  int th = shapes[ba];
  double best = us[ba][bo];
  if (us_rows > 0 && us_rows < best) {
    th = SIM_TILE_ROWS;
    bo = 0;
    best = us_rows;
  }
  if (!(best < kMargin * us[0][0])) { th = 16; bo = 0; }
  double us16 = us[0][0], us8 = us[1][0];
  for (int o = 1; o < norders; ++o) {
    us16 = std::min(us16, us[0][o]);
    us8 = std::min(us8, us[1][o]);
  }
  {
    std::lock_guard<std::mutex> g(g_tune_mu);
    g_table[key_of(c)] = Entry{th, bo, us16, us8, us_rows};
  }
  if (th_out) *th_out = th;
  if (us_out) {
    us_out[0] = us16;
    us_out[1] = us8;
    us_out[2] = us_rows;
  }
  return SIM_OK;
}

}  // namespace

bool evsim_rt::tuned_tile_height(const sim_config& c, int* th, int* order) {
  std::lock_guard<std::mutex> g(g_tune_mu);
  auto it = g_table.find(key_of(c));
  if (it == g_table.end()) return false;
  *th = it->second.th;
  *order = it->second.order;
  return true;
}

extern "C" {

int sim_autotune(const sim_config* cfg, int32_t frames, int32_t* tile_height_out,
                 double* us_out) {
  if (!cfg || frames < 2 || frames > 64) return SIM_ERR_ARG;
  const sim_config c = *cfg;
  if (valid_cfg(c)) return SIM_ERR_ARG;
  const int F = frames + 1;  // frame 0 starts the stream
  const long long P = (long long)c.width * c.height;
  unsigned char* d_frames = nullptr;
  float2* d_flows = nullptr;
  cudaError_t e = cudaMalloc(&d_frames, (size_t)P * c.pixel_format * F);
  if (e == cudaSuccess) e = cudaMalloc(&d_flows, (size_t)P * sizeof(float2) * F);
  if (e == cudaSuccess) {
    const long long total = P * F;
    const int grid = (int)std::min<long long>((total + 255) / 256, 8192);
    k_probe<<<grid, 256>>>(d_frames, d_flows, c.width, c.height, c.pixel_format, F);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
  }
  int rc = e == cudaSuccess ? SIM_OK : (e == cudaErrorMemoryAllocation ? SIM_ERR_OOM : rc_of(e));
  if (!rc) {
    std::vector<const void*> fr(F);
    std::vector<const float*> fl(F);
    std::vector<int64_t> t(F);
    for (int j = 0; j < F; ++j) {
      fr[j] = d_frames + (size_t)j * P * c.pixel_format;
      fl[j] = (const float*)(d_flows + (size_t)j * P);
      t[j] = 16667LL * j;
    }
    rc = tune(c, F, fr.data(), (int64_t)c.width * c.pixel_format, fl.data(), t.data(),
              SIM_DEVICE, tile_height_out, us_out);
  }
  cudaFree(d_frames);
  cudaFree(d_flows);
  return rc;
}

int sim_autotune_sample(const sim_config* cfg, int32_t count, const void* const* frames,
                        int64_t pitch_bytes, const float* const* flows, const int64_t* t_us,
                        int32_t mem, int32_t* tile_height_out, double* us_out) {
  if (!cfg || count < 3 || count > SIM_MAX_BATCH || !frames || !flows || !t_us) return SIM_ERR_ARG;
  if (mem != SIM_HOST && mem != SIM_DEVICE) return SIM_ERR_ARG;
  if (valid_cfg(*cfg)) return SIM_ERR_ARG;
  return tune(*cfg, count, frames, pitch_bytes, flows, t_us, mem, tile_height_out, us_out);
}

int sim_autotune_save(const char* path) {
  if (!path) return SIM_ERR_ARG;
  FILE* f = std::fopen(path, "w");
  if (!f) return SIM_ERR_ARG;
  std::lock_guard<std::mutex> g(g_tune_mu);
  for (const auto& kv : g_table) {
    const Key& k = kv.first;
    std::fprintf(f, "%d %d %d %d %d %d %d %d %d %d %d %.3f %.3f %.3f\n", std::get<0>(k),
                 std::get<1>(k), std::get<2>(k), std::get<3>(k), std::get<4>(k), std::get<5>(k),
                 std::get<6>(k), std::get<7>(k), std::get<8>(k), kv.second.th, kv.second.order,
                 kv.second.us16, kv.second.us8, kv.second.us_rows);
  }
  const bool ok = std::fclose(f) == 0;
  return ok ? SIM_OK : SIM_ERR_ARG;
}

int sim_autotune_load(const char* path) {
  if (!path) return SIM_ERR_ARG;
  FILE* f = std::fopen(path, "r");
  if (!f) return SIM_ERR_ARG;
  std::map<Key, Entry> add;
  char line[512];
  bool bad = false;
  while (std::fgets(line, sizeof(line), f)) {
    int v[11];
    double a = 0, b = 0, r = 0;
    if (std::sscanf(line, "%d %d %d %d %d %d %d %d %d %d %d %lf %lf %lf", &v[0], &v[1], &v[2],
                    &v[3], &v[4], &v[5], &v[6], &v[7], &v[8], &v[9], &v[10], &a, &b, &r) != 14 ||
        (v[9] != 8 && v[9] != 16 && v[9] != SIM_TILE_ROWS) || v[10] < 0 || v[10] > 2) {
      bad = true;
      break;
    }
    add[Key{v[0], v[1], v[2], v[3], v[4], v[5], v[6], v[7], v[8]}] = Entry{v[9], v[10], a, b, r};
  }
  std::fclose(f);
  if (bad) return SIM_ERR_ARG;
  std::lock_guard<std::mutex> g(g_tune_mu);
  for (const auto& kv : add) g_table[kv.first] = kv.second;
  return SIM_OK;
}

}  // extern "C"
