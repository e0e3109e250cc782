// CUDA kernels of the evsim library (sm_103a).
//
// Frames are simulated in batches (a single push is a batch of one).  One
// batch runs, on the handle's stream:
//   dense : [flowmax, adaptive N only] -> dense -> order
//   sparse: [sparse_pre, adaptive N only] -> sparse -> order
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
// repeat); frames follow each other.  The simulating kernels work
// pixel-major, so they record each pixel's per-substep count in shared
// memory, write their events to a staging area in their own local order and
// publish one (count, staging offset) entry per "segment" (dense: one row of
// a 64 x 16 tile; sparse: the active pixels of one chunk of 1024 raster
// pixels) per substep and frame.  The order kernel scans the batch's segment
// counts in output order (a single-pass scan with decoupled look-back),
// gathers the events into the stream's event buffer, and the block that
// finishes the last chunk commits the whole batch.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "../../include/evsim.h"
#include "internal.h"

namespace evsim {

namespace {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ int ld_volatile(const int* p) { return *(const volatile int*)p; }
__device__ __forceinline__ unsigned long long ld_volatile(const unsigned long long* p) {
  return *(const volatile unsigned long long*)p;
}
__device__ __forceinline__ void st_volatile(unsigned long long* p, unsigned long long v) {
  *(volatile unsigned long long*)p = v;
}

// Block-uniform read of the stream's sticky error word (one read per block,
// so that every thread of a block takes the same early exit).
__device__ __forceinline__ bool block_error(const int* err) {
  __shared__ int s_err;
  if (threadIdx.x == 0) s_err = ld_volatile(err);
  __syncthreads();
  return s_err != 0;
}

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Flow component (px, float) -> Q16: NaN -> 0, clamp to +-1024 px, nearest
// with ties to even.  The scaling by 2^16 is exact in float.
__device__ __forceinline__ int flow_q16(float f, int& clamped) {
  if (!(f == f)) return 0;
  if (f > 1024.f) { f = 1024.f; ++clamped; }
  if (f < -1024.f) { f = -1024.f; ++clamped; }
  return __float2int_rn(f * 65536.0f);
}

// Smallest N >= 1 with N^2 2^32 >= m (= ceil of the largest flow in px), capped.
__device__ __forceinline__ int adaptive_n(unsigned long long m, int nmax) {
  int n = 1;
  while (n < nmax && (unsigned long long)n * n * 4294967296ull < m) ++n;
  return n;
}

// a + floor(((b - a) f + 2048) / 4096): Q12-weighted blend, round half up,
// evaluated as (a (4096 - f) + b f + 2048) >> 12 (the same integer).  LOG
// values span 19 bits, so the 32-bit products cannot overflow; LINEAR values
// span 24 bits and take 64-bit products.
template <bool WIDE>
__device__ __forceinline__ int lerp12(int a, int b, int f) {
  if (WIDE) return a + (int)(((long long)(b - a) * f + 2048) >> 12);
  return (a * (4096 - f) + b * f + 2048) >> 12;
}

__device__ __forceinline__ int load_luma(const unsigned char* f, long long pitch, int ch,
                                         int y, int x) {
  const unsigned char* q = f + (long long)y * pitch + (long long)x * ch;
  if (ch == 1) return q[0];
  return (77 * q[0] + 150 * q[1] + 29 * q[2] + 128) >> 8;
}

// Bilinear tap from a replicate-padded shared tile at a tile-relative Q16
// position (always inside the filled region).  `base` is the tile's 32-bit
// shared-window address; the four taps are read with immediate offsets.
static_assert(SW * 4 == 384, "tap offsets below assume a 96-int shared stride");
template <bool WIDE>
__device__ __forceinline__ int tap_shared(unsigned base, int px, int py) {
  const int ix = px >> 16, iy = py >> 16;
  const int fx = (px >> 4) & 0xFFF, fy = (py >> 4) & 0xFFF;
  const unsigned a = base + (unsigned)(iy * SW + ix) * 4u;
  int l00, l01, l10, l11;
  asm volatile(
      "ld.shared.s32 %0, [%4];\n\t"
      "ld.shared.s32 %1, [%4+4];\n\t"
      "ld.shared.s32 %2, [%4+384];\n\t"
      "ld.shared.s32 %3, [%4+388];"
      : "=r"(l00), "=r"(l01), "=r"(l10), "=r"(l11)
      : "r"(a));
  const int top = lerp12<WIDE>(l00, l01, fx);
  const int bot = lerp12<WIDE>(l10, l11, fx);
  return lerp12<WIDE>(top, bot, fy);
}

// Bilinear tap from an 8-bit image in global memory at an absolute Q16
// position, clamped to the image (clamp-to-edge).
template <bool WIDE>
__device__ __forceinline__ int tap_global(const unsigned char* img, long long pitch, int ch,
                                          int W, int H, const int* slut, int px, int py) {
  px = min(max(px, 0), (W - 1) << 16);
  py = min(max(py, 0), (H - 1) << 16);
  const int ix = px >> 16, iy = py >> 16;
  const int fx = (px >> 4) & 0xFFF, fy = (py >> 4) & 0xFFF;
  const int x1 = min(ix + 1, W - 1), y1 = min(iy + 1, H - 1);
  const int l00 = slut[load_luma(img, pitch, ch, iy, ix)];
  const int l01 = slut[load_luma(img, pitch, ch, iy, x1)];
  const int l10 = slut[load_luma(img, pitch, ch, y1, ix)];
  const int l11 = slut[load_luma(img, pitch, ch, y1, x1)];
  const int top = lerp12<WIDE>(l00, l01, fx);
  const int bot = lerp12<WIDE>(l10, l11, fx);
  return lerp12<WIDE>(top, bot, fy);
}

// Threshold test of one interpolated value against the reference.
// ACCUM: every whole threshold crossed is one event and moves R by it.
// RESET: the paper's consecutive difference, strict comparisons.
// Must be called by all 32 lanes: a pixel that crosses two or more
// thresholds in one substep is rare, and the division it needs runs on a
// warp-uniform branch.
template <bool RESET>
__device__ __forceinline__ int threshold_step(int I, int& R, int cp, int cn) {
  const int D = I - R;
  if (RESET) {
    R = I;
    return D > cp ? 1 : (D < -cn ? -1 : 0);
  }
  int n = D >= cp ? 1 : (D <= -cn ? -1 : 0);
  if (__any_sync(FULL, D >= 2 * cp || D <= -2 * cn)) {
    if (D >= cp) n = D / cp;
    else if (D <= -cn) n = -((-D) / cn);
  }
  R += n * (n > 0 ? cp : cn);
  return n;
}

__device__ __forceinline__ int warp_incl_scan(int v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int u = __shfl_up_sync(FULL, v, o);
    if (lane >= o) v += u;
  }
  return v;
}

// Exclusive scan of one int per thread over a block of NTH threads; *total
// gets the sum.  s_warp needs NTH / 32 + 1 ints.  Contains barriers: call
// from all threads.
template <int NTH = NT>
__device__ __forceinline__ int block_excl_scan(int v, int* s_warp, int* total) {
  constexpr int NW = NTH / 32;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int incl = warp_incl_scan(v);
  if (lane == 31) s_warp[w] = incl;
  __syncthreads();
  if (w == 0) {
    const int s = lane < NW ? s_warp[lane] : 0;
    const int si = warp_incl_scan(s);
    if (lane < NW) s_warp[lane] = si - s;
    if (lane == NW - 1) s_warp[NW] = si;
  }
  __syncthreads();
  *total = s_warp[NW];
  const int r = incl - v + s_warp[w];
  __syncthreads();
  return r;
}

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long u = __shfl_xor_sync(FULL, v, o);
    v = u > v ? u : v;
  }
  return v;
}

// Single-pass scan across chunks with decoupled look-back, run by one full
// warp.  Publishes chunk c's aggregate, then inspects 32 predecessors per
// step (nearest first): their values are summed up to the nearest inclusive
// prefix, or the window slides back by 32 when all of them hold aggregates.
// The spin on predecessors that have not published is bounded.  Publishes
// chunk c's inclusive prefix and returns its exclusive prefix (all lanes).
// Values saturate at LB_VALUE, which callers treat as an overflow.
__device__ long long lookback_warp(unsigned long long* status, int c, unsigned epoch,
                                   long long agg, int* err) {
  const int lane = threadIdx.x & 31;
  const unsigned long long hi = (unsigned long long)epoch << 32;
  if (agg > (long long)LB_VALUE) agg = LB_VALUE;
  if (lane == 0) {
    __threadfence();
    st_volatile(&status[c], hi | (c == 0 ? LB_INC : LB_AGG) | (unsigned long long)agg);
  }
  if (c == 0) return 0;
  long long excl = 0;
  int j = c - 1;
  int spins = 0;
  for (;;) {
    const int idx = j - lane;
    bool valid = true, inc = true;
    long long v = 0;
    if (idx >= 0) {
      const unsigned long long w = ld_volatile(&status[idx]);
      valid = (unsigned)(w >> 32) == epoch && (w & (LB_AGG | LB_INC));
      inc = valid && (w & LB_INC);
      v = valid ? (long long)(w & LB_VALUE) : 0;
    }
    const unsigned vm = __ballot_sync(FULL, valid), im = __ballot_sync(FULL, inc);
    bool done = false, slide = false;
    unsigned take = 0;
    if (im) {
      const int f = __ffs(im) - 1;  // nearest inclusive prefix
      const unsigned need = f == 31 ? FULL : ((1u << (f + 1)) - 1);
      if ((vm & need) == need) { done = true; take = need; }
    } else if (vm == FULL) {
      slide = true;
      take = FULL;
    }
    if (done || slide) {
      long long t = (take >> lane) & 1 ? v : 0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(FULL, t, o);
      excl += t;
      if (done) break;
      j -= 32;
      continue;
    }
    if (++spins > SPIN_LIMIT) {
      if (lane == 0) atomicCAS(err, 0, SIM_ERR_DEVICE_TIMEOUT);
      break;
    }
    __nanosleep(32);
  }
  long long inc_v = excl + agg;
  if (inc_v > (long long)LB_VALUE) inc_v = LB_VALUE;
  if (lane == 0) {
    __threadfence();
    st_volatile(&status[c], hi | LB_INC | (unsigned long long)inc_v);
  }
  return excl;
}

__device__ __forceinline__ Ev make_event(unsigned t, int x, int y, bool pos) {
  Ev e;
  e.t = t;
  e.xyp = (unsigned)x | ((unsigned)((y << 1) | (pos ? 1 : 0)) << 16);
  return e;
}

// The previous frame of batch frame i: the frame ring for i = 0 (the last
// frame of the previous batch, luma), else the batch's own frame i - 1.
struct FrameRef {
  const unsigned char* ptr;
  long long pitch;
  int ch;
};

__device__ __forceinline__ FrameRef prev_frame(const SimParams& p, const BatchArg& b, int i,
                                               const unsigned char* ringp) {
  FrameRef r;
  if (i == 0) {
    r.ptr = ringp;
    r.pitch = p.W;
    r.ch = 1;
  } else {
    const FrameDesc d = b.frames[i - 1];
    r.ptr = d.frame;
    r.pitch = d.pitch;
    r.ch = p.ch;
  }
  return r;
}

// Tile-local offsets of `E` segment counts (substep-major), staging allocation.
// Returns the staging base, or -1 when the staging area is exhausted (the
// batch then fails and emits nothing more).
template <int NTH = NT>
__device__ __forceinline__ long long stage_segments(const SimParams& p, const int* cnt, int* off,
                                                    int E, int* s_warp, long long* s_base,
                                                    int* total_out) {
  const int tid = threadIdx.x;
  constexpr int PER = 2048 / NTH;  // entries per thread (E <= 2048)
  int v[PER], sum = 0;
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int e = PER * tid + q;
    v[q] = e < E ? cnt[e] : 0;
    sum += v[q];
  }
  int total;
  int ex = block_excl_scan<NTH>(sum, s_warp, &total);
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int e = PER * tid + q;
    if (e < E) off[e] = ex;
    ex += v[q];
  }
  if (tid == 0) {
    long long base = 0;
    if (total > 0) {
      const unsigned long long bb = atomicAdd(&p.ctl->stage_top, (unsigned long long)total);
      if (bb + (unsigned long long)total > (unsigned long long)p.stage_cap) {
        base = -1;
        atomicExch(&p.ctl->batch_fail, 1);
      } else {
        base = (long long)bb;
      }
    }
    *s_base = base;
  }
  __syncthreads();
  *total_out = total;
  return *s_base;
}

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

__global__ void __launch_bounds__(NT) k_flowmax(SimParams p, BatchArg b) {
  if (block_error(&p.ctl->err)) return;
  const int i = blockIdx.y;
  const FrameDesc f = b.frames[i];
  __shared__ unsigned long long s_m[NWARP];
  constexpr int U = 8;  // independent loads in flight per thread
  const long long P = (long long)p.W * p.H;
  unsigned long long m = 0;
  int dummy = 0;
  for (long long i0 = blockIdx.x * (long long)NT * U + threadIdx.x; i0 < P;
       i0 += (long long)gridDim.x * NT * U) {
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

// ---------------------------------------------------------------------------
// Tile simulation, dense (Sec. III-A) and sparse (Sec. III-B).  One block
// (NTD threads) per 64 x 16 tile carries the tile through every frame of the
// batch.  Per frame:
//   1. the pixels to simulate: dense - every pixel of the tile in the image,
//      warp w owning tile row w and lane l its columns l and l + 32, with the
//      reference and thresholds in the owner's registers for the whole batch;
//      sparse - the pixels whose log intensity changed by at least C_act from
//      frame i-1 to frame i, compacted in raster order ("slots") and spread
//      over the block, with the reference and thresholds in shared memory;
//   2. their flow is read and the tile's flow reach sizes a replicate-padded
//      halo of both log frames in shared memory.  Frame i's halo is kept as
//      the next frame's previous-frame halo whenever its extent suffices, so
//      usually one frame is loaded per frame;
//   3. every simulated pixel runs through the N substeps, recording each
//      pixel-substep's signed event count;
//   4. the tile's events are written to staging in (substep, row, column)
//      order and one segment entry per (substep, row) is published for the
//      order kernel.

__device__ __forceinline__ int activity_threshold(const SimParams& p, int cp, int cn) {
  return p.cact >= 0 ? p.cact : min(cp, cn);
}

constexpr int TP = TW * TH;  // pixels per tile (1024)

struct TileLayout {
  int* sLa;              // two halo buffers (SH x SW); roles swap between frames
  int* sLb;
  int* slut;
  int* sR;               // [TP] sparse: the tile's reference
  int* srow;             // [N][TH] events per (substep, tile row)
  int* soff;             // [N][TH] tile-local exclusive offsets
  unsigned* stk;
  int* swk;
  short* snk;            // [N][TP] signed event count per (substep, slot)
  short* sslot;          // [TP] sparse: tile pixel index (ty * TW + tx) of each slot
  unsigned short* sCp;   // [TP] sparse: per-pixel thresholds (maps)
  unsigned short* sCn;
};

__device__ __forceinline__ TileLayout tile_layout(unsigned char* raw, int nmax) {
  TileLayout L;
  L.sLa = (int*)raw;
  L.sLb = L.sLa + SH * SW;
  L.slut = L.sLb + SH * SW;
  L.sR = L.slut + 256;
  L.srow = L.sR + TP;
  L.soff = L.srow + nmax * TH;
  L.stk = (unsigned*)(L.soff + nmax * TH);
  L.swk = (int*)(L.stk + nmax);
  L.snk = (short*)(L.swk + nmax);
  L.sslot = L.snk + nmax * TP;
  L.sCp = (unsigned short*)(L.sslot + TP);
  L.sCn = L.sCp + TP;
  return L;
}

// Fill a replicate-padded halo buffer (LUT'd) of one frame with reach (hx, hy)
// around the tile.  The region is walked as a flat index (row = e / ncols by
// a multiply-high with ceil(2^32 / ncols), exact for e < 2^16).
__device__ __forceinline__ void fill_halo(int* dst, const int* slut, const FrameRef& f, int W,
                                          int H, int tx0, int ty0, int hx, int hy) {
  constexpr int FILL = 4;
  const int tid = threadIdx.x;
  const int c0 = HMAX - hx, ncols = TW + 2 * hx;
  const int r0 = HMAX - hy, nrows = TH + 2 * hy;
  const int total_fill = ncols * nrows;
  const unsigned mcols = 0xFFFFFFFFu / (unsigned)ncols + 1u;
  for (int e0 = 0; e0 < total_fill; e0 += NTD * FILL) {
    int v[FILL], at[FILL];
#pragma unroll
    for (int q = 0; q < FILL; ++q) {
      const int e = e0 + q * NTD + tid;
      at[q] = -1;
      if (e < total_fill) {
        const int sr = (int)__umulhi((unsigned)e, mcols);
        const int sc = e - sr * ncols;
        const int gy = min(max(ty0 - hy + sr, 0), H - 1);
        const int gx = min(max(tx0 - hx + sc, 0), W - 1);
        v[q] = load_luma(f.ptr, f.pitch, f.ch, gy, gx);
        at[q] = (r0 + sr) * SW + (c0 + sc);
      }
    }
#pragma unroll
    for (int q = 0; q < FILL; ++q)
      if (at[q] >= 0) dst[at[q]] = slut[v[q]];
  }
}

// The substeps of the (up to) two pixels of this thread.  `lx, ly` are the
// pixels' tile coordinates, `nk_at` their columns in the per-substep record.
// DENSE: the two pixels are columns lane, lane + 32 of tile row `warp`, and the
// row's event count is reduced over the warp in the loop.
template <bool RESET, bool WIDE, bool FAST, bool DENSE>
__device__ __forceinline__ void tile_substeps(const SimParams& p, const TileLayout& L, int N,
                                              int tx0, int ty0, unsigned b0, unsigned b1,
                                              const FrameRef& prv, const FrameDesc& cur,
                                              const int (&lx)[2], const int (&ly)[2],
                                              const int (&nk_at)[2], const bool (&act)[2],
                                              const int (&Fx)[2], const int (&Fy)[2],
                                              int (&R)[2], const int (&Cp)[2],
                                              const int (&Cn)[2]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int px[2], py[2], ax[2], ay[2], qx[2], rx[2], qy[2], ry[2];
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    // FAST: positions relative to the shared tile origin (tx0 - HMAX, ty0 - HMAX);
    // otherwise absolute image positions.
    px[j] = FAST ? (lx[j] + HMAX) << 16 : (tx0 + lx[j]) << 16;
    py[j] = FAST ? (ly[j] + HMAX) << 16 : (ty0 + ly[j]) << 16;
    // F = q N + r with 0 <= r < N: offset_k = q k + floor(r k / N)
    qx[j] = Fx[j] / N;
    rx[j] = Fx[j] - qx[j] * N;
    if (rx[j] < 0) { rx[j] += N; qx[j] -= 1; }
    qy[j] = Fy[j] / N;
    ry[j] = Fy[j] - qy[j] * N;
    if (ry[j] < 0) { ry[j] += N; qy[j] -= 1; }
    ax[j] = 0;
    ay[j] = 0;
  }
  for (int k = 0; k < N; ++k) {
    const int w = L.swk[k];
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
        s0 = tap_global<WIDE>(prv.ptr, prv.pitch, prv.ch, p.W, p.H, L.slut, px[j], py[j]);
        s1 = tap_global<WIDE>(cur.frame, cur.pitch, p.ch, p.W, p.H, L.slut, px[j] + Fx[j],
                              py[j] + Fy[j]);
      }
      const int I = lerp12<WIDE>(s0, s1, w);
      n[j] = threshold_step<RESET>(I, R[j], Cp[j], Cn[j]);
      if (!act[j]) n[j] = 0;
      L.snk[k * TP + nk_at[j]] = (short)n[j];
    }
    if (DENSE) {
      int c = abs(n[0]) + abs(n[1]);
      if (__any_sync(FULL, c != 0)) {
        c = __reduce_add_sync(FULL, c);
        if (lane == 0) L.srow[k * TH + warp] = c;
      }
    }
  }
}

template <bool RESET, bool MAPS, bool WIDE, bool SPARSE>
__global__ void __launch_bounds__(NTD, 2) k_tile(SimParams p, BatchArg b) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_warp[NTD / 32 + 1];
  __shared__ int s_fx, s_fy;
  __shared__ int s_rs[TH + 1];  // first slot of each tile row
  __shared__ long long s_base;
  Ctl* ctl = p.ctl;
  if (block_error(&ctl->err)) return;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nmax = p.n_max;
  const TileLayout L = tile_layout(smem_raw, nmax);
  const int tile = blockIdx.x;
  const int tcx = tile % p.tiles_x, tcy = tile / p.tiles_x;
  const int tx0 = tcx * TW, ty0 = tcy * TH;
  const int W = p.W, H = p.H;

  if (tid < 256) L.slut[tid] = p.lut[tid];
  const int sel = ctl->sel;
  const int* Rin = (sel & 1) ? p.R1 : p.R0;
  int* Rout = (sel & 1) ? p.R0 : p.R1;
  const unsigned char* ringp = (sel & 2) ? p.ring1 : p.ring0;
  unsigned char* ringn = (sel & 2) ? p.ring0 : p.ring1;
  long long tprev = ctl->t_prev;

  // Dense: thread (warp w, lane l) owns tile pixels (l, w) and (l + 32, w);
  // sparse: thread t owns tile pixels t and t + NTD for selection and the
  // reference store.
  int own[2];
  bool inimg[2];
  int Rd[2], Cpd[2], Cnd[2];  // dense: the owned pixels' reference and thresholds
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    own[q] = SPARSE ? tid + q * NTD : warp * TW + lane + 32 * q;
    const int x = tx0 + (own[q] & (TW - 1)), y = ty0 + own[q] / TW;
    inimg[q] = x < W && y < H;
    Rd[q] = 0; Cpd[q] = p.cp; Cnd[q] = p.cn;
    if (inimg[q]) {
      const long long i = (long long)y * W + x;
      if (SPARSE) {
        if (!RESET) L.sR[own[q]] = Rin[i];
        if (MAPS) { L.sCp[own[q]] = p.cpmap[i]; L.sCn[own[q]] = p.cnmap[i]; }
      } else {
        if (!RESET) Rd[q] = Rin[i];
        if (MAPS) { Cpd[q] = p.cpmap[i]; Cnd[q] = p.cnmap[i]; }
      }
    }
  }
  if (!SPARSE && tid == 0) {
    for (int r = 0; r <= TH; ++r) s_rs[r] = r * TW;
  }
  int clamps = 0;
  long long act_sum = 0, act_n = 0;
  bool failed = false;
  // halo buffers: `cb` will receive frame i; `pb` holds frame i-1 over the
  // extent (phx, phy), or nothing yet (-1)
  int* cb = L.sLb;
  int* pb = L.sLa;
  int phx = -1, phy = -1;
  int hfx = 1, hfy = 1;  // fill extents only grow within a batch
  __syncthreads();  // the table, reference and thresholds above are read by all threads

  for (int fi = 0; fi < b.count && !failed; ++fi) {
    const FrameDesc cur = b.frames[fi];
    const FrameRef prv = prev_frame(p, b, fi, ringp);
    FrameRef curf;
    curf.ptr = cur.frame;
    curf.pitch = cur.pitch;
    curf.ch = p.ch;
    const int N = p.n_fixed > 0 ? p.n_fixed : adaptive_n(p.maxf2[fi], nmax);
    if (tid == 0) { s_fx = 0; s_fy = 0; }
    if (tid < N) {
      const int k = tid + 1;
      L.swk[tid] = (k * 8192 + N) / (2 * N);
      const long long dt = cur.t_rel - tprev;
      L.stk[tid] = (unsigned)(tprev + (k * dt) / N);
    }
    for (int e = tid; e < N * TH; e += NTD) L.srow[e] = 0;

    // 1. the pixels to simulate
    int A = 0;
    int sel_flag[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int x = tx0 + (own[q] & (TW - 1)), y = ty0 + own[q] / TW;
      bool a = inimg[q];
      if (inimg[q] && (SPARSE || fi == b.count - 1)) {
        const int vc = load_luma(cur.frame, cur.pitch, p.ch, y, x);
        if (fi == b.count - 1) ringn[(long long)y * W + x] = (unsigned char)vc;
        if (SPARSE) {
          const int vp = load_luma(prv.ptr, prv.pitch, prv.ch, y, x);
          const int cp = MAPS ? (int)L.sCp[own[q]] : p.cp, cn = MAPS ? (int)L.sCn[own[q]] : p.cn;
          a = abs(L.slut[vc] - L.slut[vp]) >= activity_threshold(p, cp, cn);
        }
      }
      sel_flag[q] = a ? 1 : 0;
    }
    if (SPARSE) {
      // compaction in raster order: slots 0..NTD-1 (q = 0) come first
      const int packed = block_excl_scan<NTD>(sel_flag[0] | (sel_flag[1] << 16), s_warp, &A);
      const int A0 = A & 0xFFFF;
      A = A0 + (A >> 16);
      const int o0 = packed & 0xFFFF, o1 = A0 + (packed >> 16);
      if (sel_flag[0]) L.sslot[o0] = (short)tid;
      if (sel_flag[1]) L.sslot[o1] = (short)(tid + NTD);
      if ((tid & (TW - 1)) == 0) {
        const int r = tid / TW;
        s_rs[r] = o0;
        s_rs[r + NTD / TW] = o1;
      }
      if (tid == 0) s_rs[TH] = A;
      __syncthreads();
    } else {
      A = TP;
    }
    act_sum += A;
    act_n += (long long)A * N;

    // 2. the simulated pixels of this thread, their flow; the tile's reach
    int lx[2], ly[2], nk_at[2], Fx[2], Fy[2], R[2], Cp[2], Cn[2];
    bool act[2];
    unsigned mfx = 0, mfy = 0;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      int slot;
      if (SPARSE) {
        const int j = tid + q * NTD;
        act[q] = j < A;
        slot = act[q] ? L.sslot[j] : 0;
        nk_at[q] = j;
      } else {
        act[q] = inimg[q];
        slot = own[q];
        nk_at[q] = own[q];
      }
      lx[q] = slot & (TW - 1);
      ly[q] = slot / TW;
      Fx[q] = 0; Fy[q] = 0;
      R[q] = SPARSE ? 0 : Rd[q];
      Cp[q] = SPARSE ? p.cp : Cpd[q];
      Cn[q] = SPARSE ? p.cn : Cnd[q];
      if (act[q]) {
        const int x = tx0 + lx[q], y = ty0 + ly[q];
        const float2 fl = cur.flow[(long long)y * W + x];
        Fx[q] = flow_q16(fl.x, clamps);
        Fy[q] = flow_q16(fl.y, clamps);
        if (SPARSE) {
          if (MAPS) { Cp[q] = L.sCp[slot]; Cn[q] = L.sCn[slot]; }
          if (!RESET) R[q] = L.sR[slot];
        }
        if (RESET) R[q] = L.slut[load_luma(prv.ptr, prv.pitch, prv.ch, y, x)];
        mfx = max(mfx, (unsigned)abs(Fx[q]));
        mfy = max(mfy, (unsigned)abs(Fy[q]));
      }
    }
    mfx = __reduce_max_sync(FULL, mfx);
    mfy = __reduce_max_sync(FULL, mfy);
    if (lane == 0) {
      atomicMax(&s_fx, (int)mfx);
      atomicMax(&s_fy, (int)mfy);
    }
    __syncthreads();
    // Reach of every tap of the tile: floor(max |F|) + 1 pixels on each side.
    const int hx = (s_fx >> 16) + 1, hy = (s_fy >> 16) + 1;
    const bool fast = hx <= HMAX && hy <= HMAX;
    if (fast && A > 0) {
      hfx = max(hfx, hx);
      hfy = max(hfy, hy);
      if (phx < hx || phy < hy) {  // the kept halo of frame i-1 does not reach far enough
        fill_halo(pb, L.slut, prv, W, H, tx0, ty0, hfx, hfy);
        phx = hfx;
        phy = hfy;
      }
      fill_halo(cb, L.slut, curf, W, H, tx0, ty0, hfx, hfy);
    }
    __syncthreads();

    // 3. substeps (sparse: warps without a compacted pixel skip them)
    const unsigned b0 = (unsigned)__cvta_generic_to_shared(pb);
    const unsigned b1 = (unsigned)__cvta_generic_to_shared(cb);
    if (!SPARSE || warp * 32 < A || warp * 32 + NTD < A) {  // warp-uniform
      if (fast)
        tile_substeps<RESET, WIDE, true, !SPARSE>(p, L, N, tx0, ty0, b0, b1, prv, cur, lx, ly,
                                                  nk_at, act, Fx, Fy, R, Cp, Cn);
      else
        tile_substeps<RESET, WIDE, false, !SPARSE>(p, L, N, tx0, ty0, b0, b1, prv, cur, lx, ly,
                                                   nk_at, act, Fx, Fy, R, Cp, Cn);
    }
    if (!RESET) {
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        if (SPARSE) {
          if (act[q]) L.sR[lx[q] + ly[q] * TW] = R[q];
        } else {
          Rd[q] = R[q];
        }
      }
    }
    __syncthreads();

    // 4. sparse: events per (substep, row) from the records of the row's slots
    static_assert(NTD / 32 == TH, "one warp per tile row");
    if (SPARSE) {
      const int r = warp, s0 = s_rs[r], s1 = s_rs[r + 1];
      if (s1 > s0) {
        for (int k = 0; k < N; ++k) {
          int c = 0;
          for (int j = s0 + lane; j < s1; j += 32) c += abs((int)L.snk[k * TP + j]);
          if (__any_sync(FULL, c != 0)) {
            c = __reduce_add_sync(FULL, c);
            if (lane == 0) L.srow[k * TH + r] = c;
          }
        }
      }
      __syncthreads();
    }
    const int E = N * TH;
    int total;
    const long long base = stage_segments<NTD>(p, L.srow, L.soff, E, s_warp, &s_base, &total);
    const bool fail = base < 0;
    int2* segf = p.seg + (long long)fi * nmax * p.segs_per_k;
    for (int e = tid; e < E; e += NTD) {
      const int k = e / TH, ty = e % TH, yy = ty0 + ty;
      if (yy < H)
        segf[(long long)k * p.segs_per_k + (long long)yy * p.tiles_x + tcx] =
            make_int2(fail ? 0 : L.srow[e], (int)(fail ? 0 : base) + L.soff[e]);
    }
    if (!fail && total > 0) {
      // Emission: warp r writes its row's events, substep by substep, in
      // column order (the row's slots are contiguous and in raster order).
      const unsigned lt = lanemask_lt();
      const int r = warp, s0 = s_rs[r], s1 = s_rs[r + 1];
      const int y = ty0 + r;
      for (int k = 0; k < N; ++k) {
        const int e = k * TH + r;
        if (L.srow[e] == 0) continue;
        const unsigned tk = L.stk[k];
        long long o = base + L.soff[e];
        for (int j0 = s0; j0 < s1; j0 += 32) {
          const int j = j0 + lane;
          const int n = j < s1 ? L.snk[k * TP + j] : 0;
          const int a = abs(n);
          const int x = tx0 + (SPARSE ? (j < s1 ? (L.sslot[j] & (TW - 1)) : 0) : (j & (TW - 1)));
          const Ev ev = make_event(tk, x, y, n > 0);
          int seg_total;
          if (__all_sync(FULL, a <= 1)) {
            const unsigned bb = __ballot_sync(FULL, a != 0);
            if (a) p.staging[o + __popc(bb & lt)] = ev;
            seg_total = __popc(bb);
          } else {
            const int ia = warp_incl_scan(a);
            for (int m = 0; m < a; ++m) p.staging[o + ia - a + m] = ev;
            seg_total = __shfl_sync(FULL, ia, 31);
          }
          o += seg_total;
        }
      }
    }
    failed = fail;
    tprev = cur.t_rel;
    // frame i's halo becomes the previous-frame halo of frame i + 1
    if (fast && A > 0) {
      int* t = pb;
      pb = cb;
      cb = t;
      phx = hfx;
      phy = hfy;
    } else {
      phx = -1;
      phy = -1;
    }
    __syncthreads();
  }

  if (!RESET && !failed) {
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      if (!inimg[q]) continue;
      Rout[(long long)(ty0 + own[q] / TW) * W + tx0 + (own[q] & (TW - 1))] =
          SPARSE ? L.sR[own[q]] : Rd[q];
    }
  }
  clamps = __reduce_add_sync(FULL, clamps);
  if (lane == 0 && clamps) atomicAdd(&ctl->clamped, (unsigned long long)clamps);
  if (SPARSE && tid == 0 && act_sum) {
    atomicAdd((unsigned long long*)&ctl->active, (unsigned long long)act_sum);
    atomicAdd((unsigned long long*)&ctl->active_n, (unsigned long long)act_n);
  }
}

// Adaptive N for the sparse method: max squared flow over the active pixels
// of each frame (blockIdx.y = frame).
__global__ void __launch_bounds__(NT) k_sparse_pre(SimParams p, BatchArg b) {
  __shared__ int slut[256];
  __shared__ unsigned long long s_m[NWARP];
  Ctl* ctl = p.ctl;
  if (block_error(&ctl->err)) return;
  const int tid = threadIdx.x;
  const int fi = blockIdx.y;
  slut[tid] = p.lut[tid];
  __syncthreads();
  const unsigned char* ringp = (ctl->sel & 2) ? p.ring1 : p.ring0;
  const FrameDesc cur = b.frames[fi];
  const FrameRef prv = prev_frame(p, b, fi, ringp);
  const long long P = (long long)p.W * p.H;
  unsigned long long m = 0;
  int dummy = 0;
  for (long long i = blockIdx.x * (long long)NT + tid; i < P; i += (long long)gridDim.x * NT) {
    const int y = (int)(i / p.W), x = (int)(i - (long long)y * p.W);
    const int vp = load_luma(prv.ptr, prv.pitch, prv.ch, y, x);
    const int vc = load_luma(cur.frame, cur.pitch, p.ch, y, x);
    const int cp = p.cpmap ? p.cpmap[i] : p.cp;
    const int cn = p.cnmap ? p.cnmap[i] : p.cn;
    if (abs(slut[vc] - slut[vp]) >= activity_threshold(p, cp, cn)) {
      const float2 fl = cur.flow[i];
      const long long fx = flow_q16(fl.x, dummy), fy = flow_q16(fl.y, dummy);
      const unsigned long long f2 = (unsigned long long)(fx * fx + fy * fy);
      m = f2 > m ? f2 : m;
    }
  }
  m = warp_max_u64(m);
  if ((tid & 31) == 0) s_m[tid >> 5] = m;
  __syncthreads();
  if (tid == 0) {
    unsigned long long bm = 0;
    for (int w = 0; w < NWARP; ++w) bm = s_m[w] > bm ? s_m[w] : bm;
    if (bm) atomicMax(&p.maxf2[fi], bm);
  }
}

// ---------------------------------------------------------------------------
// order: scan the segment counts of the whole batch in output order (frame,
// substep, segment), gather the events from staging into the event buffer,
// and commit the batch (all of its frames, or none).

__global__ void __launch_bounds__(NT) k_order(SimParams p, BatchArg b) {
  __shared__ int s_ex[OCHUNK];
  __shared__ int s_src[OCHUNK];
  __shared__ int s_N[1024];
  __shared__ int s_warp[NWARP + 1];
  __shared__ int s_c, s_last, s_ok;
  __shared__ long long s_prefix;
  Ctl* ctl = p.ctl;
  if (block_error(&ctl->err)) return;
  const int tid = threadIdx.x;
  const int nmax = p.n_max;
  for (int i = tid; i < b.count; i += NT)
    s_N[i] = p.n_fixed > 0 ? p.n_fixed : adaptive_n(p.maxf2[i], nmax);
  const long long S = p.segs_per_k;
  const long long per_frame = (long long)nmax * S;
  const long long nseg = (long long)b.count * per_frame;
  const int nchunks = (int)max(1LL, (nseg + OCHUNK - 1) / OCHUNK);
  const long long cursor = ctl->cursor;
  __syncthreads();

  for (;;) {
    if (tid == 0) s_c = (int)atomicAdd(&ctl->order_ticket, 1u);
    __syncthreads();
    const int c = s_c;
    if (c >= nchunks) break;
    // four consecutive segments per thread; segments of substeps k >= N of
    // their frame were never written and count zero
    const long long s0 = (long long)c * OCHUNK + OPER * tid;
    long long fi = s0 / per_frame;
    long long rem = s0 - fi * per_frame;
    int cnt[OPER], src[OPER], sum = 0;
#pragma unroll
    for (int q = 0; q < OPER; ++q) {
      cnt[q] = 0;
      src[q] = 0;
      if (s0 + q < nseg && rem / S < s_N[fi]) {
        const int2 e = p.seg[s0 + q];
        cnt[q] = e.x;
        src[q] = e.y;
      }
      sum += cnt[q];
      if (++rem == per_frame) { rem = 0; ++fi; }
    }
    int total;
    int ex = block_excl_scan(sum, s_warp, &total);
#pragma unroll
    for (int q = 0; q < OPER; ++q) {
      s_ex[OPER * tid + q] = ex;
      s_src[OPER * tid + q] = src[q];
      ex += cnt[q];
    }
    if (tid < 32) {
      const long long ex0 = lookback_warp(p.order_status, c, b.serial, total, &ctl->err);
      if (tid == 0) s_prefix = ex0;
    }
    __syncthreads();
    const long long base = cursor + s_prefix;
    for (int jj = tid; jj < total; jj += NT) {
      int lo = 0, hi = OCHUNK;
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (s_ex[mid] <= jj) lo = mid; else hi = mid;
      }
      const long long dst = base + jj;
      if (dst < p.event_cap) p.events[dst] = p.staging[(long long)s_src[lo] + (jj - s_ex[lo])];
    }
    __syncthreads();
    if (tid == 0) {
      __threadfence();
      const unsigned d = atomicAdd(&ctl->order_done, 1u);
      s_last = d == (unsigned)(nchunks - 1);
    }
    __syncthreads();
    if (s_last) {
      // This block finished the batch's last chunk: commit or fail the batch.
      if (tid == 0) {
        __threadfence();
        const unsigned long long w = ld_volatile(&p.order_status[nchunks - 1]);
        const long long tot = (long long)(w & LB_VALUE);
        const bool over = ctl->batch_fail != 0 || tot >= (long long)LB_VALUE ||
                          cursor + tot > p.event_cap;
        int ok = 0;
        if (ld_volatile(&ctl->err) == 0) {
          if (over) {
            atomicCAS(&ctl->err, 0, SIM_ERR_EVENT_OVERFLOW);
          } else {
            const long long P = (long long)p.W * p.H;
            long long nsum = 0;
            for (int i = 0; i < b.count; ++i) nsum += s_N[i];
            ctl->cursor = cursor + tot;
            ctl->sel ^= p.ref_mode == SIM_REF_ACCUM ? 3 : 2;
            ctl->t_prev = b.frames[b.count - 1].t_rel;
            ctl->committed += b.count;
            ctl->batch_events = tot;
            ctl->last_n = s_N[b.count - 1];
            ctl->work_px += P * nsum;
            ctl->work_active += p.mode == SIM_SPARSE ? ctl->active_n : P * nsum;
            ctl->last_active = p.mode == SIM_SPARSE ? ctl->active : P * b.count;
            ok = 1;
          }
        }
        ctl->active = 0;
        ctl->active_n = 0;
        ctl->stage_top = 0;
        ctl->order_done = 0;
        ctl->batch_fail = 0;
        s_ok = ok;
      }
      for (int i = tid; i < b.count; i += NT) p.maxf2[i] = 0;
    }
    __syncthreads();
  }
  if (tid == 0) {
    const unsigned e = atomicAdd(&ctl->order_exit, 1u);
    if (e == gridDim.x - 1) {  // every block has left the ticket loop
      ctl->order_ticket = 0;
      ctl->order_exit = 0;
    }
  }
}

template <bool RESET, bool MAPS, bool WIDE, bool SPARSE>
void set_tile_attr(size_t bytes) {
  cudaFuncSetAttribute(k_tile<RESET, MAPS, WIDE, SPARSE>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <bool SPARSE>
cudaError_t launch_tile_mode(const SimParams& p, const BatchArg& b, cudaStream_t st) {
  const int grid = p.tiles_x * p.tiles_y;
  const size_t sm = tile_smem_bytes(p.n_max);
  const bool reset = p.ref_mode == SIM_REF_RESET;
  const bool maps = p.cpmap != nullptr;
  const bool wide = p.intensity == SIM_LINEAR;
#define EVSIM_TILE(R, M, Wd) k_tile<R, M, Wd, SPARSE><<<grid, NTD, sm, st>>>(p, b)
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

size_t tile_smem_bytes(int n_max) {
  return (size_t)(2 * SH * SW + 256 + TP + 2 * n_max * TH + 2 * n_max) * 4 +
         (size_t)(n_max * TP + 3 * TP) * 2;
}

int device_sm_count() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  return n;
}

cudaError_t configure_kernels(int n_max) {
  const size_t t = tile_smem_bytes(n_max);
  set_tile_attr<false, false, false, false>(t);
  set_tile_attr<false, true, false, false>(t);
  set_tile_attr<false, false, true, false>(t);
  set_tile_attr<false, true, true, false>(t);
  set_tile_attr<true, false, false, false>(t);
  set_tile_attr<true, true, false, false>(t);
  set_tile_attr<true, false, true, false>(t);
  set_tile_attr<true, true, true, false>(t);
  set_tile_attr<false, false, false, true>(t);
  set_tile_attr<false, true, false, true>(t);
  set_tile_attr<false, false, true, true>(t);
  set_tile_attr<false, true, true, true>(t);
  set_tile_attr<true, false, false, true>(t);
  set_tile_attr<true, true, false, true>(t);
  set_tile_attr<true, false, true, true>(t);
  set_tile_attr<true, true, true, true>(t);
  return cudaGetLastError();
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

cudaError_t launch_dense(const SimParams& p, const BatchArg& b, cudaStream_t st) {
  return launch_tile_mode<false>(p, b, st);
}

cudaError_t launch_sparse(const SimParams& p, const BatchArg& b, cudaStream_t st) {
  return launch_tile_mode<true>(p, b, st);
}

cudaError_t launch_sparse_pre(const SimParams& p, const BatchArg& b, cudaStream_t st) {
  const long long P = (long long)p.W * p.H;
  const int sms = device_sm_count();
  const long long per_frame = std::max(1LL, (long long)sms * 4 / std::max(1, b.count));
  const int gx = (int)std::max(1LL, std::min<long long>((P + NT - 1) / NT, per_frame));
  k_sparse_pre<<<dim3(gx, b.count), NT, 0, st>>>(p, b);
  return cudaGetLastError();
}

cudaError_t launch_order(const SimParams& p, const BatchArg& b, cudaStream_t st, int grid) {
  k_order<<<grid, NT, 0, st>>>(p, b);
  return cudaGetLastError();
}

}  // namespace evsim
