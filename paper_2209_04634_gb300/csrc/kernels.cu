// CUDA kernels of the evsim library (sm_103a).
//
// Frames are simulated in batches (a single push is a batch of one).  One
// batch runs, on the handle's stream:
//   dense : [flowmax, adaptive N] -> [predict, plan: balanced order] -> dense
//           -> [units: rows flagged] -> order
//   sparse: [sparse_pre, adaptive N] -> [predict, plan] -> sparse -> [units] -> order
// The method (Ziegler et al., arXiv 2209.04634, Sec. III-A / III-B) and its
// integer arithmetic are described in include/evsim.h.  Every kernel checks
// the stream's sticky error word first and does nothing once it is set.
//
// The simulating kernels are persistent over the batch: each block owns one
// tile (dense) or one raster chunk (sparse) and carries it through every frame
// of the batch, keeping the reference in registers / shared memory.  Blocks
// never wait for each other, so the grid may exceed the resident capacity.
//
// Event order.  Within a frame, events are ordered by (substep, row, column,
// repeat); frames follow each other.  The simulating kernel works
// pixel-major and publishes one "segment" per (frame, substep, row of a
// 64 x 16 tile): the row's event and polarity bit masks, or - when a pixel
// of the row crossed more than one threshold in the substep - the row's
// events written to a staging area.  The order kernel scans the batch's
// segment counts in output order (a single-pass scan with decoupled
// look-back), writes the events into the stream's event buffer (expanding
// the masks, copying the staged rows), and the block that finishes the last
// chunk commits the whole batch.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "../../include/evsim.h"
#include "internal.h"

#include "tile.cuh"

namespace evsim {

namespace {

// ---------------------------------------------------------------------------
// frame 0 of a stream: fill the frame ring and the reference

__global__ void k_init(SimParams p, FrameDesc f) {
  const long long P = (long long)p.W * p.H;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < P;
       i += (long long)gridDim.x * blockDim.x) {
    const int y = (int)(i / p.W), x = (int)(i - (long long)y * p.W);
    const int v = load_luma(f.frame, f.pitch, p.ch, y, x);
    p.ring0[i] = (unsigned char)v;
    if (p.ref_mode == SIM_REF_ACCUM) p.R0[i] = p.lut[v];
  }
}

// ---------------------------------------------------------------------------
// adaptive N (dense): max over all pixels of the squared Q16 flow, per frame
// of the batch (blockIdx.y = frame)

__device__ __forceinline__ void flowmax_run(const SimParams& p, const BatchArg& b, int i, int bx,
                                            int nbx) {
  if (block_error(&p.ctl->err)) return;
  const FrameDesc f = b.frames[i];
  __shared__ unsigned long long s_m[NWARP];
  constexpr int U = 8;  // independent loads in flight per thread
  const long long P = (long long)p.W * p.H;
  unsigned long long m = 0;
  int dummy = 0;
  for (long long i0 = bx * (long long)NT * U + threadIdx.x; i0 < P; i0 += (long long)nbx * NT * U) {
    float2 fl[U];
#pragma unroll
    for (int q = 0; q < U; ++q) {
      const long long j = i0 + (long long)q * NT;
      fl[q] = j < P ? f.flow[j] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int q = 0; q < U; ++q) {
      const long long fx = flow_q16(fl[q].x, dummy), fy = flow_q16(fl[q].y, dummy);
      const unsigned long long f2 = (unsigned long long)(fx * fx + fy * fy);
      m = f2 > m ? f2 : m;
    }
  }
  m = warp_max_u64(m);
  if ((threadIdx.x & 31) == 0) s_m[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long bm = 0;
    for (int w = 0; w < NWARP; ++w) bm = s_m[w] > bm ? s_m[w] : bm;
    if (bm) atomicMax(&p.maxf2[i], bm);
  }
}

__global__ void __launch_bounds__(NT) k_flowmax(SimParams p, BatchArg b) {
  flowmax_run(p, b, blockIdx.y, blockIdx.x, gridDim.x);
}

// ---------------------------------------------------------------------------
// Difference-frame interpolation (Sec. III-C).  The difference frames of
// three consecutive frames, D_{i-1} = L_{i-1} - L_{i-2} and D_i = L_i - L_{i-1},
// are sampled and blended along the flow between them exactly as the dense
// method samples frames; each interpolated difference frame is thresholded
// with the strict two-case equations (no reference state).  Nothing carries
// from frame to frame, so every (tile, frame) of a batch is its own block.

// Bilinear tap of a difference plane (frame b minus frame a, LUT'd) in global
// memory at an absolute Q16 position, clamped to the image.
template <bool WIDE>
__device__ __forceinline__ int tap_global_diff(const FrameRef& fa, const FrameRef& fb, int W,
                                               int H, const int* slut, int px, int py) {
  px = min(max(px, 0), (W - 1) << 16);
  py = min(max(py, 0), (H - 1) << 16);
  const int ix = px >> 16, iy = py >> 16;
  const int fx = (px >> 4) & 0xFFF, fy = (py >> 4) & 0xFFF;
  const int x1 = min(ix + 1, W - 1), y1 = min(iy + 1, H - 1);
  auto d = [&](int y, int x) {
    return slut[load_luma(fb.ptr, fb.pitch, fb.ch, y, x)] -
           slut[load_luma(fa.ptr, fa.pitch, fa.ch, y, x)];
  };
  const int top = lerp12<WIDE>(d(iy, ix), d(iy, x1), fx);
  const int bot = lerp12<WIDE>(d(y1, ix), d(y1, x1), fx);
  return lerp12<WIDE>(top, bot, fy);
}

// Replicate-padded halo of the difference plane (frame b minus frame a) with
// reach (hx, hy) around the tile (same layout as fill_halo).
__device__ __forceinline__ void fill_halo_diff(int* dst, const int* slut, const FrameRef& fa,
                                               const FrameRef& fb, int W, int H, int tx0,
                                               int ty0, int hx, int hy) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ncols = TW + 2 * hx, nrows = TH + 2 * hy;
  for (int sr = warp; sr < nrows; sr += NTD / 32) {
    const int gy = min(max(ty0 - hy + sr, 0), H - 1);
    int* d = dst + (HMAX - hy + sr) * SW + (HMAX - hx);
    for (int sc = lane; sc < ncols; sc += 32) {
      const int gx = min(max(tx0 - hx + sc, 0), W - 1);
      d[sc] = slut[load_luma(fb.ptr, fb.pitch, fb.ch, gy, gx)] -
              slut[load_luma(fa.ptr, fa.pitch, fa.ch, gy, gx)];
    }
  }
}

// The substeps of this thread's two pixels (columns lane and lane + 32 of tile
// row `warp`) on the difference planes: FAST samples the shared halos (b0:
// D_{i-1}, b1: D_i), otherwise global memory (frames f2, f1, f0 = i-2, i-1, i).
template <bool WIDE, bool FAST>
__device__ __forceinline__ void diff_substeps(const SimParams& p, const int* swk,
                                              const unsigned* stk, int N, unsigned mN, int tx0,
                                              int ty0, unsigned b0, unsigned b1,
                                              const FrameRef& f2, const FrameRef& f1,
                                              const FrameRef& f0, const int* slut, Seg* segr,
                                              WarpStage* ws, const bool (&act)[2],
                                              const int (&Fx)[2], const int (&Fy)[2],
                                              const int (&Cp)[2], const int (&Cn)[2]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int px[2], py[2], ax[2], ay[2], qx[2], rx[2], qy[2], ry[2];
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    px[j] = FAST ? (lane + 32 * j + HMAX) << 16 : (tx0 + lane + 32 * j) << 16;
    py[j] = FAST ? (warp + HMAX) << 16 : (ty0 + warp) << 16;
    divmod_n(Fx[j], N, mN, qx[j], rx[j]);
    divmod_n(Fy[j], N, mN, qy[j], ry[j]);
    ax[j] = 0;
    ay[j] = 0;
  }
  for (int k = 0; k < N; ++k) {
    const int w = swk[k];
    int n[2];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      px[j] -= qx[j];
      ax[j] += rx[j];
      if (ax[j] >= N) { ax[j] -= N; px[j] -= 1; }
      py[j] -= qy[j];
      ay[j] += ry[j];
      if (ay[j] >= N) { ay[j] -= N; py[j] -= 1; }
      int s0, s1;
      if (FAST) {
        s0 = tap_shared<WIDE>(b0, px[j], py[j]);
        s1 = tap_shared<WIDE>(b1, px[j] + Fx[j], py[j] + Fy[j]);
      } else {
        s0 = tap_global_diff<WIDE>(f2, f1, p.W, p.H, slut, px[j], py[j]);
        s1 = tap_global_diff<WIDE>(f1, f0, p.W, p.H, slut, px[j] + Fx[j], py[j] + Fy[j]);
      }
      const int I = lerp12<WIDE>(s0, s1, w);
      n[j] = act[j] ? (I > Cp[j] ? 1 : (I < -Cn[j] ? -1 : 0)) : 0;
    }
    publish_row_dense(p, segr + (long long)k * p.segs_per_k, n[0], n[1], stk[k], tx0,
                      ty0 + warp, ws);
  }
}

template <bool MAPS, bool WIDE>
__global__ void __launch_bounds__(NTD, 2) k_diff(SimParams p, BatchArg b) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_fx, s_fy;
  __shared__ unsigned s_mN;
  __shared__ WarpStage s_stage[NTD / 32];
  Ctl* ctl = p.ctl;
  if (block_error(&ctl->err)) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int tile = blockIdx.x, fi = blockIdx.y;
  const int tcx = tile % p.tiles_x, tcy = tile / p.tiles_x;
  const int tx0 = tcx * TW, ty0 = tcy * TH;
  const int W = p.W, H = p.H, nmax = p.n_max;
  int* pb = (int*)smem_raw;  // D_{i-1} halo
  int* cb = pb + SH * SW;    // D_i halo
  int* slut = cb + SH * SW;
  int* swk = slut + 256;
  unsigned* stk = (unsigned*)(swk + nmax);
  if (tid < 256) slut[tid] = p.lut[tid];
  if ((tid & 31) == 0) s_stage[tid >> 5] = WarpStage{0, 0, 0};
  if (tid == 0) { s_fx = 0; s_fy = 0; }

  const int sel = ctl->sel;
  const unsigned char* r1p = (sel & 2) ? p.ring1 : p.ring0;  // frame before the batch
  unsigned char* r1n = (sel & 2) ? p.ring0 : p.ring1;
  const unsigned char* r2p = (sel & 2) ? p.ring2_1 : p.ring2_0;  // the frame before that
  unsigned char* r2n = (sel & 2) ? p.ring2_0 : p.ring2_1;
  const long long stream_i = ctl->committed + fi;  // frames of the stream before this one
  const FrameRef ring1{r1p, (long long)W, 1}, ring2{r2p, (long long)W, 1};
  const FrameDesc cd = b.frames[fi];
  const FrameRef f0{cd.frame, cd.pitch, p.ch};
  FrameRef f1 = ring1, f2 = ring2;
  if (fi >= 1) f1 = FrameRef{b.frames[fi - 1].frame, b.frames[fi - 1].pitch, p.ch};
  if (fi >= 2) f2 = FrameRef{b.frames[fi - 2].frame, b.frames[fi - 2].pitch, p.ch};
  else if (fi == 1) f2 = ring1;
  const int N = p.n_fixed > 0 ? p.n_fixed : adaptive_n(p.maxf2[fi], nmax);
  const long long tprev = fi == 0 ? ctl->t_prev : b.frames[fi - 1].t_rel;
  if (tid < N) {
    const int k = tid + 1;
    swk[tid] = (k * 8192 + N) / (2 * N);
    stk[tid] = (unsigned)(tprev + (k * (cd.t_rel - tprev)) / N);
  }
  if (tid == 0) s_mN = N > 1 ? (unsigned)(0x100000000ull / (unsigned)N) + 1u : 0u;

  // this block's pixels, their flow and thresholds; the next batch's frame ring
  bool act[2];
  int Fx[2], Fy[2], Cp[2], Cn[2];
  int clamps = 0;
  unsigned mfx = 0, mfy = 0;
  const int y = ty0 + warp;
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int x = tx0 + lane + 32 * q;
    act[q] = x < W && y < H;
    Fx[q] = 0; Fy[q] = 0; Cp[q] = p.cp; Cn[q] = p.cn;
    if (act[q]) {
      const long long i = (long long)y * W + x;
      const float2 fl = cd.flow[i];
      Fx[q] = flow_q16(fl.x, clamps);
      Fy[q] = flow_q16(fl.y, clamps);
      if (MAPS) { Cp[q] = p.cpmap[i]; Cn[q] = p.cnmap[i]; }
      mfx = max(mfx, (unsigned)abs(Fx[q]));
      mfy = max(mfy, (unsigned)abs(Fy[q]));
      if (fi == b.count - 1) r1n[i] = (unsigned char)load_luma(f0.ptr, f0.pitch, f0.ch, y, x);
      if (fi == b.count - 2) r2n[i] = (unsigned char)load_luma(f0.ptr, f0.pitch, f0.ch, y, x);
      if (b.count == 1) r2n[i] = r1p[i];
    }
  }
  // frames 0 and 1 of the stream only build the first difference frame
  const bool emits = stream_i >= 2;
  mfx = __reduce_max_sync(FULL, mfx);
  mfy = __reduce_max_sync(FULL, mfy);
  if (lane == 0) {
    atomicMax(&s_fx, (int)mfx);
    atomicMax(&s_fy, (int)mfy);
  }
  __syncthreads();
  const int hx = (s_fx >> 16) + 1, hy = (s_fy >> 16) + 1;
  const bool fast = hx <= HMAX && hy <= HMAX;
  if (emits && fast) {
    fill_halo_diff(pb, slut, f2, f1, W, H, tx0, ty0, hx, hy);
    fill_halo_diff(cb, slut, f1, f0, W, H, tx0, ty0, hx, hy);
  }
  __syncthreads();
  Seg* segr = p.seg + (long long)fi * nmax * p.segs_per_k + (long long)y * p.tiles_x + tcx;
  if (y < H) {  // warp-uniform
    if (!emits) {
      for (int k = lane; k < N; k += 32) segr[(long long)k * p.segs_per_k] = Seg{0ull, 0ull, 0, -1};
    } else if (fast) {
      diff_substeps<WIDE, true>(p, swk, stk, N, s_mN, tx0, ty0, (unsigned)__cvta_generic_to_shared(pb),
                                (unsigned)__cvta_generic_to_shared(cb), f2, f1, f0, slut, segr,
                                &s_stage[warp], act, Fx, Fy, Cp, Cn);
    } else {
      diff_substeps<WIDE, false>(p, swk, stk, N, s_mN, tx0, ty0, 0u, 0u, f2, f1, f0, slut, segr,
                                 &s_stage[warp], act, Fx, Fy, Cp, Cn);
    }
  }
  clamps = __reduce_add_sync(FULL, clamps);
  if (lane == 0 && clamps) atomicAdd(&ctl->clamped, (unsigned long long)clamps);
}

// Accumulated event frame (Fig. 1 caption: the output is either the events or
// a frame with the accumulated events): every event with t_begin <= t < t_end
// adds its polarity (+1 / -1) to its pixel.  Integer atomics: the result does
// not depend on the order the events are visited in.
__global__ void k_accumulate(const Ev* ev, long long n, int W, int H, long long t_begin,
                             long long t_end, int* frame) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const Ev e = ev[i];
    const long long t = e.t;
    if (t < t_begin || t >= t_end) continue;
    const int x = (int)(e.xyp & 0xFFFFu), yp = (int)(e.xyp >> 16);
    const int y = yp >> 1;
    if (x >= W || y >= H) continue;
    atomicAdd(frame + (long long)y * W + x, (yp & 1) ? 1 : -1);
  }
}

// Cost estimate of every tile over the batch about to run, for the balanced
// block order: a frame counts as busy for a tile when one of 16 flow samples
// spread over the tile (an 8 x 2 grid) is non-zero, and a busy frame costs
// about four quiet ones (measured on moving content: 20 against 8 us per
// 1280x720 frame with about half the tiles busy), so a tile's cost is
// count + 3 x its busy frames.  The samples only steer the schedule, never
// the events.  One block per tile: the batch's flow pointers are read into
// shared memory once, then every thread loads its (frame, sample) pairs -
// independent loads, four in flight - and marks the frames found moving.
constexpr int PRED_UNROLL = 4;
__global__ void __launch_bounds__(NT) k_predict(SimParams p, BatchArg b) {
  __shared__ const float2* s_flow[SIM_MAX_BATCH];
  __shared__ unsigned char s_busy[SIM_MAX_BATCH];
  __shared__ int s_n;
  const int tile = blockIdx.x, count = b.count;
  const int th = p.tile_h == 8 ? 8 : 16;
  const int x0 = (tile % p.tiles_x) * TW, y0 = (tile / p.tiles_x) * th;
  for (int f = threadIdx.x; f < count; f += NT) {
    s_flow[f] = b.frames[f].flow;
    s_busy[f] = 0;
  }
  if (threadIdx.x == 0) s_n = 0;
  __syncthreads();
  const int total = count * 16;
  for (int e0 = threadIdx.x; e0 < total; e0 += NT * PRED_UNROLL) {
    float2 v[PRED_UNROLL];
    bool ok[PRED_UNROLL];
#pragma unroll
    for (int u = 0; u < PRED_UNROLL; ++u) {
      const int e = e0 + u * NT, f = e >> 4, sm = e & 15;
      const int sx = x0 + 4 + 8 * (sm & 7), sy = y0 + (th >> 2) + (th >> 1) * (sm >> 3);
      ok[u] = e < total && sx < p.W && sy < p.H;
      v[u] = ok[u] ? s_flow[f][(long long)sy * p.W + sx] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < PRED_UNROLL; ++u)
      if (ok[u] && ((__float_as_uint(v[u].x) | __float_as_uint(v[u].y)) << 1) != 0u)
        s_busy[(e0 + u * NT) >> 4] = 1;
  }
  __syncthreads();
  int n = 0;
  for (int f = threadIdx.x; f < count; f += NT) n += s_busy[f];
  n = __reduce_add_sync(FULL, n);
  if ((threadIdx.x & 31) == 0 && n) atomicAdd(&s_n, n);
  __syncthreads();
  if (threadIdx.x == 0) p.tile_cost[tile] = (unsigned)(count + 3 * s_n);
}

// Balanced block order: tiles ranked by their estimated cost (heaviest
// first, ties by tile index), laid out in serpentine order over the ranks -
// the first wave of one block per SM takes the heaviest tiles, the second
// wave the lightest in reverse - so the heaviest tile shares its SM with the
// lightest.  An order of the tiles like any other: it changes only the
// schedule.  Every block ranks NT tiles against all T (costs in shared
// memory) and writes each tile to the block that takes its rank:
// serpentine_tile maps a block to a rank and is its own inverse (it reverses
// odd rounds only).
__global__ void __launch_bounds__(NT) k_plan(int T, int S, const unsigned* cost, int* order) {
  __shared__ unsigned sc[PLAN_MAX_TILES];
  for (int t = threadIdx.x; t < T; t += NT) sc[t] = cost[t];
  __syncthreads();
  const int t = blockIdx.x * NT + threadIdx.x;
  if (t >= T) return;
  const unsigned c = sc[t];
  int rank = 0;
  for (int u = 0; u < T; ++u) rank += (sc[u] > c) | ((sc[u] == c) & (u < t));
  order[serpentine_tile(rank, T, S)] = t;
}

// Adaptive N for the sparse method: max squared flow over the active pixels
// of each frame.  Warp w of block bx (of nbx) takes rows bx * NWARP + w,
// + nbx * NWARP, ...; each lane four columns of the row at a time, their
// loads issued together.
__device__ __forceinline__ void sparse_pre_run(const SimParams& p, const BatchArg& b, int fi,
                                               int bx, int nbx) {
  __shared__ int slut[256];
  __shared__ unsigned long long s_m[NWARP];
  Ctl* ctl = p.ctl;
  if (block_error(&ctl->err)) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  slut[tid] = p.lut[tid];
  __syncthreads();
  const unsigned char* ringp = (ctl->sel & 2) ? p.ring1 : p.ring0;
  const FrameDesc cur = b.frames[fi];
  const FrameRef prv = prev_frame(p, b, fi, ringp);
  const int W = p.W;
  constexpr int U = 4;
  unsigned long long m = 0;
  int dummy = 0;
  for (int y = bx * NWARP + warp; y < p.H; y += nbx * NWARP) {
    const unsigned char* rp = prv.ptr + (long long)y * prv.pitch;
    const unsigned char* rc = cur.frame + (long long)y * cur.pitch;
    const long long row = (long long)y * W;
    for (int x0 = lane; x0 < W; x0 += 32 * U) {
      int d[U], c[U];
#pragma unroll
      for (int q = 0; q < U; ++q) {
        const int x = x0 + q * 32;
        d[q] = -1;
        c[q] = 0;
        if (x < W) {
          const int vp = prv.ch == 1 ? rp[x] : load_luma(rp, 0, prv.ch, 0, x);
          const int vc = p.ch == 1 ? rc[x] : load_luma(rc, 0, p.ch, 0, x);
          const int cp = p.cpmap ? p.cpmap[row + x] : p.cp;
          const int cn = p.cnmap ? p.cnmap[row + x] : p.cn;
          d[q] = abs(slut[vc] - slut[vp]);
          c[q] = activity_threshold(p, cp, cn);
        }
      }
#pragma unroll
      for (int q = 0; q < U; ++q) {
        if (d[q] >= c[q]) {
          const float2 fl = cur.flow[row + x0 + q * 32];
          const long long fx = flow_q16(fl.x, dummy), fy = flow_q16(fl.y, dummy);
          const unsigned long long f2 = (unsigned long long)(fx * fx + fy * fy);
          m = f2 > m ? f2 : m;
        }
      }
    }
  }
  m = warp_max_u64(m);
  if (lane == 0) s_m[warp] = m;
  __syncthreads();
  if (tid == 0) {
    unsigned long long bm = 0;
    for (int w = 0; w < NWARP; ++w) bm = s_m[w] > bm ? s_m[w] : bm;
    if (bm) atomicMax(&p.maxf2[fi], bm);
  }
}

__global__ void __launch_bounds__(NT) k_sparse_pre(SimParams p, BatchArg b) {
  sparse_pre_run(p, b, blockIdx.y, blockIdx.x, gridDim.x);
}

// ---------------------------------------------------------------------------
// order: scan the segment counts of the whole batch in output order (frame,
// substep, row, tile column), write the events into the event buffer (from
// the segments' bit masks, or copied from staging), and commit the batch
// (all of its frames, or none).

// Position of the m-th (0-based) set bit of a 64-bit mask that has more than
// m set bits.
__device__ __forceinline__ int nth_set_bit(unsigned long long mask, int m) {
  const unsigned lo = (unsigned)mask, hi = (unsigned)(mask >> 32);
  const int c = __popc(lo);
  if (m < c) return (int)__fns(lo, 0, m + 1);
  return 32 + (int)__fns(hi, 0, m - c + 1);
}

// Shared memory of an order block (the multi-stream order kernel adds a
// member's parameters: both stay within the 48 KB of static shared memory).
static_assert(SIM_MAX_SUBSTEPS <= 255, "substep counts are kept in bytes");
struct OrderSmem {
  int ex[OCHUNK];
  int src[OCHUNK];
  unsigned long long mask[OCHUNK];
  unsigned long long pol[OCHUNK];
  unsigned t[OCHUNK];
  unsigned xy[OCHUNK];  // x0 | (y << 16)
  unsigned char N[SIM_MAX_BATCH];  // substeps of each frame of the batch (<= 64)
  int B[SIM_MAX_BATCH];  // flagged units of each frame (p.units set)
  int FN[SIM_MAX_BATCH + 1];  // live segments of the frames before each frame, in
                              // substeps (p.units null: x segs_per_k) or segments
  int warp[NWARP + 1];
  short cblk[OCHUNK];    // segments of the chunk with per-pixel counts
  int ncblk;
  int last;
  long long prefix;
};

// Substep counts of the batch's frames into o.N and the exclusive prefix of
// their live segments into o.FN; returns the number of chunks of the
// batch's live segments.  Live: the segments of substeps k < N of their
// frame, and with unit lists (p.units) only those of the frame's flagged
// units (FN counts segments: N_f x units_f per frame; the table holds fewer
// than 2^31 segments); without, every unit's (FN counts substeps, a frame's
// segments being N_f x segs_per_k).  All threads; contains barriers.
__device__ __forceinline__ int order_fill_n(const SimParams& p, const BatchArg& b, OrderSmem& o) {
  for (int i = threadIdx.x; i < b.count; i += NT) {
    o.N[i] = (unsigned char)(p.n_fixed > 0 ? p.n_fixed : adaptive_n(p.maxf2[i], p.n_max));
    o.B[i] = p.units ? p.unit_count[i] : 0;
  }
  __syncthreads();
  int carry = 0;
  for (int base = 0; base < b.count; base += NT) {
    const int i = base + threadIdx.x;
    int tot;
    const int v = i < b.count ? (p.units ? o.N[i] * o.B[i] : o.N[i]) : 0;
    const int ex = block_excl_scan(v, o.warp, &tot);
    if (i < b.count) o.FN[i] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) o.FN[b.count] = carry;
  __syncthreads();
  const long long live = p.units ? (long long)carry : (long long)carry * p.segs_per_k;
  return (int)max(1LL, (live + OCHUNK - 1) / OCHUNK);
}

// Chunk c (of nchunks) of one stream's batch: OCHUNK segments in output
// order; the block that finishes the batch's last chunk commits the batch.
// cursor and t_first are the stream's committed event count and time.
__device__ __forceinline__ void order_chunk(const SimParams& p, const BatchArg& b, int c,
                                            int nchunks, long long cursor, long long t_first,
                                            OrderSmem& o) {
  Ctl* ctl = p.ctl;
  const int tid = threadIdx.x;
  const long long S = p.segs_per_k;
  // live segments only: (frame, substep k < N of the frame, row); a chunk
  // index beyond them (a ticket range sized for n_max substeps) is empty
  const long long nlive = p.units ? (long long)o.FN[b.count] : (long long)o.FN[b.count] * S;
  // chunk 0 always runs: a batch without a live segment (no flagged unit
  // in any frame) is still committed by it
  if (c > 0 && (long long)c * OCHUNK >= nlive) return;
  // OSEG segments per thread: loaded interleaved (segment u * NT + tid, so a
  // warp's loads are contiguous) into the chunk's arrays, then scanned with
  // each thread owning OSEG consecutive segments
  if (tid == 0) o.ncblk = 0;
  // the chunk's first segment: without unit lists, frame-substep q0 and
  // row-segment rs0 (a segment ls of the chunk lies (rs0 + ls) / S
  // frame-substeps further: 32-bit, S and OCHUNK are far below 2^31); with
  // them, segment si0 of the live list; in both, frame fi0 and a few frames
  // further at most
  const long long si0 = (long long)c * OCHUNK;
  const long long q0 = p.units ? 0 : si0 / S;
  const int rs0 = p.units ? 0 : (int)(si0 - q0 * S);
  const long long key0 = p.units ? si0 : q0;
  int fi0 = 0;
  {
    int hi = b.count;
    while (hi - fi0 > 1) {
      const int mid = (fi0 + hi) >> 1;
      if (o.FN[mid] <= key0) fi0 = mid; else hi = mid;
    }
  }
#pragma unroll
  for (int u = 0; u < OSEG; ++u) {
    const int ls = u * NT + tid;  // segment of the chunk
    const long long si = si0 + ls;
    // a segment's masks, row position and time are needed only when it has
    // events (the scan reads the counts and sources of all)
    int cnt = 0, src = -1;
    if (si < nlive) {
      int fi = fi0, k, rs;
      bool written;
      if (p.units) {
        // live segment rem of frame fi: substep rem / units_f of the frame's
        // flagged unit rem mod units_f (frames without one hold no segment)
        while (o.FN[fi + 1] <= si) ++fi;
        const int rem = (int)(si - o.FN[fi]);
        const int nu = o.B[fi];
        k = (int)((unsigned)rem / (unsigned)nu);
        const long long ui = (long long)fi * S + (rem - k * nu);
        rs = in_bounds(ctl, ui, (long long)p.bmax * S) ? p.units[ui] : 0;
        written = true;
      } else {
        const unsigned dq = (unsigned)(rs0 + ls) / (unsigned)S;
        const long long q = q0 + dq;  // frame-substep of the batch
        rs = rs0 + ls - (int)(dq * (unsigned)S);
        while (o.FN[fi + 1] <= q) ++fi;  // FN[count] exceeds every live q
        k = (int)(q - o.FN[fi]);
        // a unit-frame that emitted nothing wrote a flag instead of its
        // segments
        written = !p.segflag || p.segflag[(long long)fi * S + rs];
      }
      const int N = o.N[fi];
      if (written) {
        const long long si2 = ((long long)fi * p.n_max + k) * S + rs;
        Seg sg{0ull, 0ull, 0, -1};
        if (in_bounds(ctl, si2, p.seg_cap)) sg = p.seg[si2];
        cnt = sg.cnt;
        src = sg.src;
        if (cnt > 0) {
          const int y = rs / p.tiles_x, tc = rs - y * p.tiles_x;
          const long long tp = fi == 0 ? t_first : b.frames[fi - 1].t_rel;
          const long long dt = b.frames[fi].t_rel - tp;
          // (k + 1) dt / N (dt > 0): a 32-bit division when the product fits
          const unsigned long long kd = (unsigned long long)(k + 1) * (unsigned long long)dt;
          o.mask[ls] = sg.mask;
          o.pol[ls] = sg.pol;
          o.t[ls] = (unsigned)(tp + (long long)(kd < 0x100000000ull ? (unsigned)kd / (unsigned)N
                                                                      : kd / (unsigned)N));
          o.xy[ls] = (unsigned)(tc * TW) | ((unsigned)y << 16);
        }
      }
    }
    o.ex[ls] = cnt;
    o.src[ls] = src;
  }
  __syncthreads();
  int mine = 0;
  int cnts[OSEG];
#pragma unroll
  for (int u = 0; u < OSEG; ++u) {
    cnts[u] = o.ex[tid * OSEG + u];
    mine += cnts[u];
  }
  int total;
  int ex = block_excl_scan(mine, o.warp, &total);
#pragma unroll
  for (int u = 0; u < OSEG; ++u) {
    const int ls = tid * OSEG + u;
    o.ex[ls] = ex;
    if (o.src[ls] <= -2 && cnts[u] > 0) o.cblk[atomicAdd(&o.ncblk, 1)] = (short)ls;
    ex += cnts[u];
  }
  if (tid < 32) {
    const long long ex0 = lookback_warp(p.order_status, c, b.serial, total, &ctl->err,
                                        p.spin_limit > 0 ? p.spin_limit : SPIN_LIMIT);
    if (tid == 0) o.prefix = ex0;
  }
  __syncthreads();
  const long long base = cursor + o.prefix;
  int lo = 0;  // the thread's events only move forward: each search starts at the last hit
  for (int jj = tid; jj < total; jj += NT) {
    int hi = OCHUNK;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (o.ex[mid] <= jj) lo = mid; else hi = mid;
    }
    const long long dst = base + jj;
    if (dst >= p.event_cap) continue;
    if (o.src[lo] <= -2) continue;  // per-pixel counts: expanded below
    const int m = jj - o.ex[lo];
    Ev ev;
    if (o.src[lo] >= 0) {
      if (!in_bounds(ctl, (long long)o.src[lo] + m, p.stage_cap)) continue;
      ev = p.staging[(long long)o.src[lo] + m];
    } else {
      const int bit = nth_set_bit(o.mask[lo], m);
      const unsigned xy0 = o.xy[lo];
      ev = make_event(o.t[lo], (int)(xy0 & 0xFFFF) + bit, (int)(xy0 >> 16),
                      (o.pol[lo] >> bit) & 1ull);
    }
    p.events[dst] = ev;
  }
  // rows published as per-pixel counts: one warp per row, columns l and
  // l + 32 on lane l, in column order with repeats adjacent
  {
    const int lane = tid & 31;
    for (int q = tid >> 5; q < o.ncblk; q += NWARP) {
      const int sidx = o.cblk[q];
      const long long cb = -2LL - o.src[sidx];
      const unsigned wd = in_bounds(ctl, cb + 15, p.stage_cap)
                              ? ((const unsigned*)(p.staging + cb))[lane] : 0u;
      const int a_lo = (int)(wd & 0xFFFFu), a_hi = (int)(wd >> 16);
      const int i_lo = warp_incl_scan(a_lo);
      const int t_lo = __shfl_sync(FULL, i_lo, 31);
      const int i_hi = warp_incl_scan(a_hi);
      const long long d0 = base + o.ex[sidx];
      const unsigned xy0 = o.xy[sidx], tk = o.t[sidx];
      const unsigned long long pl = o.pol[sidx];
      const int x0 = (int)(xy0 & 0xFFFF), y = (int)(xy0 >> 16);
      const Ev e_lo = make_event(tk, x0 + lane, y, (pl >> lane) & 1ull);
      const Ev e_hi = make_event(tk, x0 + lane + 32, y, (pl >> (lane + 32)) & 1ull);
      for (int m = 0; m < a_lo; ++m) {
        const long long dst = d0 + i_lo - a_lo + m;
        if (dst < p.event_cap) p.events[dst] = e_lo;
      }
      for (int m = 0; m < a_hi; ++m) {
        const long long dst = d0 + t_lo + i_hi - a_hi + m;
        if (dst < p.event_cap) p.events[dst] = e_hi;
      }
    }
  }
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    const unsigned d = atomicAdd(&ctl->order_done, 1u);
    o.last = d == (unsigned)(nchunks - 1);
  }
  __syncthreads();
  if (o.last) {
    // This block finished the batch's last chunk: commit or fail the batch.
    if (tid == 0) {
      __threadfence();
      const unsigned long long w = ld_volatile(&p.order_status[nchunks - 1]);
      const long long tot = (long long)(w & LB_VALUE);
      const bool over = ctl->batch_fail != 0 || tot >= (long long)LB_VALUE ||
                        cursor + tot > p.event_cap;
      if (ld_volatile(&ctl->err) == 0) {
        if (over) {
          atomicCAS(&ctl->err, 0, SIM_ERR_EVENT_OVERFLOW);
        } else {
          const long long P = (long long)p.W * p.H;
          long long nsum = 0;
          for (int i = 0; i < b.count; ++i) nsum += o.N[i];
          ctl->cursor = cursor + tot;
          ctl->sel ^= p.ref_mode == SIM_REF_ACCUM ? 3 : 2;
          ctl->t_prev = b.frames[b.count - 1].t_rel;
          ctl->committed += b.count;
          ctl->batch_events = tot;
          ctl->last_n = o.N[b.count - 1];
          ctl->work_px += P * nsum;
          ctl->work_active += p.mode == SIM_SPARSE ? ctl->active_n : P * nsum;
          ctl->last_active = p.mode == SIM_SPARSE ? ctl->active : P * b.count;
          ctl->work_pixels += ctl->last_active;
        }
      }
      ctl->active = 0;
      ctl->active_n = 0;
      ctl->stage_top = 0;
      ctl->unit_ticket = 0;
      ctl->order_done = 0;
      ctl->batch_fail = 0;
    }
    for (int i = tid; i < b.count; i += NT) p.maxf2[i] = 0;
  }
  __syncthreads();
}

// The flagged units of each frame of the batch in raster order (their
// segments are the only ones written), one block per frame: the order pass
// then walks live segments only instead of every (substep, unit) slot.
constexpr int UNT = 1024;
__global__ void __launch_bounds__(UNT) k_units(SimParams p, int count) {
  __shared__ int s_warp[UNT / 32 + 1];
  const int fi = blockIdx.x;
  if (fi >= count || block_error(&p.ctl->err)) return;
  const long long S = p.segs_per_k;
  const unsigned char* f = p.segflag + (long long)fi * S;
  int* u = p.units + (long long)fi * S;
  int carry = 0;
  for (long long base = 0; base < S; base += UNT) {
    const long long i = base + threadIdx.x;
    const int flag = i < S && f[i] ? 1 : 0;
    int tot;
    const int ex = block_excl_scan<UNT>(flag, s_warp, &tot);
    if (flag) u[carry + ex] = (int)i;
    carry += tot;
  }
  if (threadIdx.x == 0) p.unit_count[fi] = carry;
}

__global__ void __launch_bounds__(NT) k_order(SimParams p, BatchArg b) {
  __shared__ OrderSmem o;
  __shared__ int s_c;
  Ctl* ctl = p.ctl;
  if (block_error(&ctl->err)) return;
  const int tid = threadIdx.x;
  const int nchunks = order_fill_n(p, b, o);
  const long long cursor = ctl->cursor;
  const long long t_first = ctl->t_prev;  // t of the frame before the batch
  __syncthreads();
  for (;;) {
    if (tid == 0) s_c = (int)atomicAdd(&ctl->order_ticket, 1u);
    __syncthreads();
    const int c = s_c;
    if (c >= nchunks) break;
    order_chunk(p, b, c, nchunks, cursor, t_first, o);
  }
  if (tid == 0) {
    __threadfence();  // this block's ticket increments precede its exit count
    const unsigned e = atomicAdd(&ctl->order_exit, 1u);
    if (e == gridDim.x - 1) {  // every block has left the ticket loop
      ctl->order_ticket = 0;
      ctl->order_exit = 0;
    }
  }
}

// ---------------------------------------------------------------------------
// Multi-stream step: the same work for every member stream of a group in one
// launch per kernel.  Per-stream parameters are copied into shared memory by
// each block; streams without frames in this step (count 0) are skipped.

__device__ __forceinline__ void load_stream(const GroupArg& g, int s, SimParams& sp,
                                            BatchArg& sb) {
  constexpr int WORDS = sizeof(SimParams) / 4;
  static_assert(sizeof(SimParams) % 4 == 0 && WORDS <= NT, "parameter copy");
  if (threadIdx.x < WORDS) ((int*)&sp)[threadIdx.x] = ((const int*)&g.gs[s].p)[threadIdx.x];
  if (threadIdx.x == 0) {
    sb.frames = g.gs[s].frames;
    sb.count = g.steps[s].count;
    sb.serial = g.steps[s].serial;
    sb.host_mapped = 1;  // group tiles stage with cp.async
  }
}

// Largest s with begin[s] <= v over n ascending entries (shared memory).
__device__ __forceinline__ int find_stream(const int* begin, int n, int v) {
  int lo = 0, hi = n;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (begin[mid] <= v) lo = mid; else hi = mid;
  }
  return lo;
}

// Adaptive N pre-pass of every adaptive member (dense: flow maximum; sparse:
// flow maximum over active pixels): work items (stream, frame, block) taken
// in a grid-stride loop.
__global__ void __launch_bounds__(NT) k_pre_multi(GroupArg g) {
  __shared__ SimParams sp;
  __shared__ BatchArg sb;
  __shared__ int s_begin[MAX_GROUP];
  const int n = g.n;
  for (int i = threadIdx.x; i < n; i += NT) s_begin[i] = g.steps[i].pre_begin;
  const int items = g.tot->pre_items;
  int cur = -1;
  __syncthreads();
  for (int it = blockIdx.x; it < items; it += gridDim.x) {
    const int s = find_stream(s_begin, n, it);
    if (s != cur) {
      __syncthreads();  // previous users of sp / sb are done
      load_stream(g, s, sp, sb);
      cur = s;
    }
    __syncthreads();
    const int nb = g.gs[s].pre_blocks;
    const int r = it - s_begin[s];
    const int fi = r / nb, bx = r - fi * nb;
    if (sp.mode == SIM_SPARSE)
      sparse_pre_run(sp, sb, fi, bx, nb);
    else
      flowmax_run(sp, sb, fi, bx, nb);
  }
}

// Work items (member, frame, tile) of the members of one kernel class that
// have frames in this step: a persistent grid takes the items of the class's
// work list (act: members in table order with their first item; frames in
// order within a member) by ticket, so members without frames cost nothing
// and items of unequal cost balance across the SMs.
template <bool RESET, bool MAPS, bool WIDE, bool SPARSE, int TH_>
__global__ void __launch_bounds__(32 * TH_, 32 / TH_) k_tile_multi(GroupArg g,
                                                                   const ActiveTile* act,
                                                                   int cls) {
  constexpr int NTD = 32 * TH_;
  __shared__ SimParams sp;
  __shared__ BatchArg sb;
  __shared__ int s_begin[MAX_GROUP];
  __shared__ int s_member[MAX_GROUP];
  __shared__ int s_t;
  const int na = g.tot->active[cls], nt = g.tot->tiles[cls];
  for (int i = threadIdx.x; i < na; i += NTD) {
    const ActiveTile a = act[i];
    s_begin[i] = a.tile_begin;
    s_member[i] = a.member;
  }
  int cur = -1;
  for (;;) {
    __syncthreads();  // the work list is loaded; the previous tile is done with shared memory
    if (threadIdx.x == 0) s_t = (int)atomicAdd(&g.gctl->tile_ticket, 1u);
    __syncthreads();
    const int t = s_t;
    if (t >= nt) break;
    const int k = find_stream(s_begin, na, t);
    const int s = s_member[k];
    if (s != cur) {
      load_stream(g, s, sp, sb);
      cur = s;
      __syncthreads();
    }
    const int T = sp.tiles_x * sp.tiles_y, r = t - s_begin[k], fi = r / T;
    tile_frames<RESET, MAPS, WIDE, SPARSE, true, TH_>(sp, sb, r - fi * T, fi, fi + 1);
  }
  if (threadIdx.x == 0) {
    __threadfence();  // this block's ticket increments precede its exit count
    const unsigned e = atomicAdd(&g.gctl->tile_exit, 1u);
    if (e == gridDim.x - 1) {  // every block has left the ticket loop
      g.gctl->tile_ticket = 0;
      g.gctl->tile_exit = 0;
    }
  }
}

// Order pass of every member: one ticket counter over the concatenated
// chunks of all members (in member order); each member keeps its own
// look-back chain and commits its own batch.
__global__ void __launch_bounds__(NT) k_order_multi(GroupArg g) {
  __shared__ OrderSmem o;
  __shared__ SimParams sp;
  __shared__ BatchArg sb;
  __shared__ int s_begin[MAX_GROUP];
  __shared__ int s_c, s_err;
  __shared__ long long s_cursor, s_tfirst;
  const int tid = threadIdx.x;
  const int n = g.n;
  for (int i = tid; i < n; i += NT) s_begin[i] = g.steps[i].chunk_begin;
  const int chunks = g.tot->chunks;
  int cur = -1, nchunks = 0;
  __syncthreads();
  for (;;) {
    if (tid == 0) s_c = (int)atomicAdd(&g.gctl->order_ticket, 1u);
    __syncthreads();
    const int t = s_c;
    if (t >= chunks) break;
    const int s = find_stream(s_begin, n, t);
    if (s != cur) {
      load_stream(g, s, sp, sb);
      __syncthreads();
      nchunks = order_fill_n(sp, sb, o);
      if (tid == 0) {
        s_cursor = sp.ctl->cursor;
        s_tfirst = sp.ctl->t_prev;
      }
      cur = s;
    }
    if (tid == 0) s_err = ld_volatile(&sp.ctl->err);
    __syncthreads();
    if (s_err == 0) order_chunk(sp, sb, t - s_begin[s], nchunks, s_cursor, s_tfirst, o);
    __syncthreads();
  }
  if (tid == 0) {
    __threadfence();  // this block's ticket increments precede its exit count
    const unsigned e = atomicAdd(&g.gctl->order_exit, 1u);
    if (e == gridDim.x - 1) {  // every block has left the ticket loop
      g.gctl->order_ticket = 0;
      g.gctl->order_exit = 0;
    }
  }
}

// Delivery of every member's committed, undelivered events to host memory
// (one array, members in table order, each member's events in output order),
// with a table of what each member received.  Every block computes the same
// member offsets; the blocks copy in a grid-stride loop; the last block to
// finish writes the table and advances the members' delivered positions.
// Members whose events do not fit get a prefix (the rest waits for the next
// delivery).
__global__ void __launch_bounds__(NT) k_drain(GroupArg g, DrainArg d) {
  __shared__ long long s_off[MAX_GROUP + 1];
  __shared__ long long s_warp64[NWARP];
  __shared__ int s_last;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int n = g.n;
  // available events of member i: [drained, cursor); a failed member delivers nothing
  constexpr int PER = (MAX_GROUP + NT - 1) / NT;
  long long av[PER];
  long long run = 0;
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int i = tid * PER + q;
    av[q] = 0;
    if (i < n) {
      const Ctl* c = g.gs[i].p.ctl;
      av[q] = ld_volatile(&c->err) ? 0 : c->cursor - c->drained;
    }
    run += av[q];
  }
  // exclusive scan of the per-thread sums
  long long inc = run;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const long long v = __shfl_up_sync(FULL, inc, o);
    if (lane >= o) inc += v;
  }
  if (lane == 31) s_warp64[warp] = inc;
  __syncthreads();
  long long base = 0;
  for (int w = 0; w < warp; ++w) base += s_warp64[w];
  long long off = base + inc - run;
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int i = tid * PER + q;
    if (i < n) s_off[i] = off;
    off += av[q];
  }
  if (tid == NT - 1) s_off[n] = off;
  __syncthreads();
  const long long total = s_off[n] < d.cap ? s_off[n] : d.cap;
  for (long long j = (long long)blockIdx.x * NT + tid; j < total; j += (long long)gridDim.x * NT) {
    int lo = 0, hi = n;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (s_off[mid] <= j) lo = mid; else hi = mid;
    }
    const SimParams& p = g.gs[lo].p;
    d.events[j] = p.events[p.ctl->drained + (j - s_off[lo])];
  }
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    s_last = atomicAdd(d.done, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  for (int i = tid; i < n; i += NT) {
    Ctl* c = g.gs[i].p.ctl;
    const long long first = s_off[i] < d.cap ? s_off[i] : d.cap;
    const long long end = s_off[i + 1] < d.cap ? s_off[i + 1] : d.cap;
    Delivery e;
    e.id = d.ids[i];
    e.status = ld_volatile(&c->err);
    e.first = first;
    e.count = end - first;
    e.committed = c->committed;
    e.work_px = c->work_px;
    d.table[i] = e;
    if (e.status == 0) {
      c->drained += e.count;
      if (c->drained == c->cursor) {
        c->drained = 0;
        c->cursor = 0;
      }
    }
  }
  if (tid == 0) {
    *d.total = total;
    *d.done = 0;
  }
}
template <bool RESET, bool MAPS, bool WIDE, bool SPARSE>
cudaError_t set_tile_multi_attr(size_t bytes) {
  const cudaError_t e = cudaFuncSetAttribute(k_tile_multi<RESET, MAPS, WIDE, SPARSE, 16>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)bytes);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_tile_multi<RESET, MAPS, WIDE, SPARSE, 8>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <bool SPARSE>
cudaError_t launch_tile_multi_mode(const GroupArg& g, int cls, const ActiveTile* act, int grid,
                                   size_t sm, cudaStream_t st) {
  const bool reset = cls & TILE_RESET, maps = cls & TILE_MAPS, wide = cls & TILE_WIDE;
#define EVSIM_TILE(R, M, Wd)                                                                 \
  if (cls & TILE_TH8) k_tile_multi<R, M, Wd, SPARSE, 8><<<grid, 256, sm, st>>>(g, act, cls);    \
  else k_tile_multi<R, M, Wd, SPARSE, 16><<<grid, 512, sm, st>>>(g, act, cls)
  if (!reset && !maps && !wide) EVSIM_TILE(false, false, false);
  else if (!reset && maps && !wide) EVSIM_TILE(false, true, false);
  else if (!reset && !maps && wide) EVSIM_TILE(false, false, true);
  else if (!reset && maps && wide) EVSIM_TILE(false, true, true);
  else if (reset && !maps && !wide) EVSIM_TILE(true, false, false);
  else if (reset && maps && !wide) EVSIM_TILE(true, true, false);
  else if (reset && !maps && wide) EVSIM_TILE(true, false, true);
  else EVSIM_TILE(true, true, true);
#undef EVSIM_TILE
  return cudaGetLastError();
}

}  // namespace


size_t tile_smem_bytes(int n_max, int th) {
  const int tp = TW * th, sh = th + 2 * HMAX;
  return (size_t)(2 * sh * SW + 256 + tp + 2 * n_max) * 4 + (size_t)(n_max * tp + 3 * tp) * 2;
}

int device_sm_count() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  return n;
}

// Returns the first failing cudaFuncSetAttribute's error (each call's return
// code is checked; an error left pending by the caller is neither reported
// nor cleared here).
cudaError_t configure_kernels(int n_max) {
  cudaError_t e = configure_dense_kernels(n_max);
  if (e == cudaSuccess) e = configure_sparse_kernels(n_max);
  if (e == cudaSuccess) e = configure_xtime_dense_kernels(n_max);
  if (e == cudaSuccess) e = configure_xtime_sparse_kernels(n_max);
  return e;
}

namespace {
constexpr int LIMIT_DEVICES = 256;
std::mutex g_limit_mu;
int g_limit_nmax[LIMIT_DEVICES] = {};  // substep cap the current device's kernels allow
}  // namespace

// The limits are process-wide per kernel, so they only ever grow: a handle
// with a small substep cap must not shrink what another caller set up.
cudaError_t raise_kernel_limits(int n_max, bool again) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= LIMIT_DEVICES) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> g(g_limit_mu);
  if (!again && n_max <= g_limit_nmax[dev]) return cudaSuccess;
  const int want = std::max(n_max, again ? 0 : g_limit_nmax[dev]);
  e = configure_kernels(want);
  if (e == cudaSuccess) g_limit_nmax[dev] = want;
  return e;
}

cudaError_t launch_init(const SimParams& p, const FrameDesc& f, cudaStream_t st) {
  const long long P = (long long)p.W * p.H;
  const int grid = (int)std::min<long long>((P + NT - 1) / NT, 4096);
  k_init<<<grid, NT, 0, st>>>(p, f);
  return cudaGetLastError();
}

cudaError_t launch_flowmax(const SimParams& p, const BatchArg& b, cudaStream_t st) {
  const long long P = (long long)p.W * p.H;
  const int sms = device_sm_count();
  const long long per_frame = std::max(1LL, (long long)sms * 4 / std::max(1, b.count));
  const int gx = (int)std::max(1LL, std::min<long long>((P + NT * 8 - 1) / (NT * 8), per_frame));
  k_flowmax<<<dim3(gx, b.count), NT, 0, st>>>(p, b);
  return cudaGetLastError();
}

cudaError_t launch_accumulate(const Ev* ev, long long n, int W, int H, long long t_begin,
                              long long t_end, int* frame, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int grid = (int)std::min<long long>((n + NT - 1) / NT, (long long)device_sm_count() * 8);
  k_accumulate<<<std::max(grid, 1), NT, 0, st>>>(ev, n, W, H, t_begin, t_end, frame);
  return cudaGetLastError();
}

cudaError_t launch_plan(const SimParams& p, const BatchArg& b, cudaStream_t st) {
  const int T = p.tiles_x * p.tiles_y;
  if (T > PLAN_MAX_TILES || !p.tile_cost || !p.tile_order || b.count < 1) return cudaSuccess;
  k_predict<<<T, NT, 0, st>>>(p, b);
  k_plan<<<(T + NT - 1) / NT, NT, 0, st>>>(T, p.sms, p.tile_cost, p.tile_order);
  return cudaGetLastError();
}

size_t diff_smem_bytes(int n_max) { return (size_t)(2 * SH * SW + 256 + 2 * n_max) * 4; }

cudaError_t launch_diff(const SimParams& p, const BatchArg& b, cudaStream_t st) {
  const dim3 grid(p.tiles_x * p.tiles_y, b.count);
  const size_t sm = diff_smem_bytes(p.n_max);
  const bool maps = p.cpmap != nullptr, wide = p.intensity == SIM_LINEAR;
  if (!maps && !wide) k_diff<false, false><<<grid, NTD, sm, st>>>(p, b);
  else if (maps && !wide) k_diff<true, false><<<grid, NTD, sm, st>>>(p, b);
  else if (!maps && wide) k_diff<false, true><<<grid, NTD, sm, st>>>(p, b);
  else k_diff<true, true><<<grid, NTD, sm, st>>>(p, b);
  return cudaGetLastError();
}

cudaError_t launch_sparse_pre(const SimParams& p, const BatchArg& b, cudaStream_t st) {
  // one warp per row
  const int gx = (p.H + NWARP - 1) / NWARP;
  k_sparse_pre<<<dim3(gx, b.count), NT, 0, st>>>(p, b);
  return cudaGetLastError();
}

cudaError_t launch_order(const SimParams& p, const BatchArg& b, cudaStream_t st, int grid) {
  if (p.units) {
    k_units<<<b.count, UNT, 0, st>>>(p, b.count);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  k_order<<<grid, NT, 0, st>>>(p, b);
  return cudaGetLastError();
}

int tile_class(const SimParams& p) {
  return (p.ref_mode == SIM_REF_RESET ? TILE_RESET : 0) | (p.cpmap ? TILE_MAPS : 0) |
         (p.intensity == SIM_LINEAR ? TILE_WIDE : 0) | (p.mode == SIM_SPARSE ? TILE_SPARSE : 0) |
         (p.tile_h == 8 ? TILE_TH8 : 0);
}

cudaError_t configure_group_kernels(size_t t) {
  const cudaError_t es[16] = {
      set_tile_multi_attr<false, false, false, false>(t),
      set_tile_multi_attr<false, true, false, false>(t),
      set_tile_multi_attr<false, false, true, false>(t),
      set_tile_multi_attr<false, true, true, false>(t),
      set_tile_multi_attr<true, false, false, false>(t),
      set_tile_multi_attr<true, true, false, false>(t),
      set_tile_multi_attr<true, false, true, false>(t),
      set_tile_multi_attr<true, true, true, false>(t),
      set_tile_multi_attr<false, false, false, true>(t),
      set_tile_multi_attr<false, true, false, true>(t),
      set_tile_multi_attr<false, false, true, true>(t),
      set_tile_multi_attr<false, true, true, true>(t),
      set_tile_multi_attr<true, false, false, true>(t),
      set_tile_multi_attr<true, true, false, true>(t),
      set_tile_multi_attr<true, false, true, true>(t),
      set_tile_multi_attr<true, true, true, true>(t)};
  for (cudaError_t e : es)
    if (e != cudaSuccess) return e;
  return cudaSuccess;
}

cudaError_t launch_pre_multi(const GroupArg& g, int grid, cudaStream_t st) {
  k_pre_multi<<<grid, NT, 0, st>>>(g);
  return cudaGetLastError();
}

cudaError_t launch_tile_multi(const GroupArg& g, int cls, const ActiveTile* act, int grid,
                              size_t smem, cudaStream_t st) {
  if (cls & TILE_SPARSE) return launch_tile_multi_mode<true>(g, cls, act, grid, smem, st);
  return launch_tile_multi_mode<false>(g, cls, act, grid, smem, st);
}

cudaError_t launch_order_multi(const GroupArg& g, int grid, cudaStream_t st) {
  k_order_multi<<<grid, NT, 0, st>>>(g);
  return cudaGetLastError();
}

cudaError_t launch_drain(const GroupArg& g, const DrainArg& d, int grid, cudaStream_t st) {
  k_drain<<<grid, NT, 0, st>>>(g, d);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Diagnostic of the bounded device waits (sim_selftest_bounded_wait): one
// warp runs the order kernel's look-back for chunk 1 (which = 0) or a group
// tile's wait for its earlier frames (which = 1) on words the host prepared;
// when the awaited word is never published the wait gives up after
// p.spin_limit polls and leaves SIM_ERR_DEVICE_TIMEOUT in the control block.

__global__ void k_selftest_wait(SimParams p, int which, unsigned epoch) {
  if (which == 0) {
    lookback_warp(p.order_status, 1, epoch, 5, &p.ctl->err, p.spin_limit);
  } else if (threadIdx.x == 0) {
    wait_tile(p, 0, ((unsigned long long)epoch << 32) | 1u);
  }
}

}  // namespace evsim

extern "C" int sim_selftest_bounded_wait(int32_t which, int32_t publish, int32_t spin_limit,
                                         int32_t* device_status) {
  using namespace evsim;
  if (!device_status || (which != 0 && which != 1) || (publish != 0 && publish != 1) ||
      spin_limit < 1 || spin_limit > SPIN_LIMIT)
    return SIM_ERR_ARG;
  *device_status = SIM_OK;
  struct Words {
    Ctl ctl;
    unsigned long long status[2];
    unsigned long long tdone[1];
  };
  Words h;
  std::memset(&h, 0, sizeof(h));
  const unsigned epoch = 3;
  if (publish) {
    h.status[0] = ((unsigned long long)epoch << 32) | LB_INC | 7ull;
    h.tdone[0] = ((unsigned long long)epoch << 32) | 1ull;
  }
  Words* d = nullptr;
  cudaError_t e = cudaMalloc(&d, sizeof(Words));
  if (e == cudaSuccess) e = cudaMemcpy(d, &h, sizeof(Words), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    SimParams p{};
    p.ctl = &d->ctl;
    p.order_status = d->status;
    p.tdone = d->tdone;
    p.spin_limit = spin_limit;
    k_selftest_wait<<<1, 32>>>(p, which, epoch);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(&h, d, sizeof(Words), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) {
    note_cuda_error(e);
    return e == cudaErrorNoDevice || e == cudaErrorInsufficientDriver ||
                   e == cudaErrorNoKernelImageForDevice
               ? SIM_ERR_NO_DEVICE
               : SIM_ERR_CUDA;
  }
  *device_status = h.ctl.err;
  return SIM_OK;
}
