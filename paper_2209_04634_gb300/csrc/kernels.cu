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

// floor(F / N) and F - N floor(F / N) for |F| <= 2^26 (Q16 flows are
// clamped to 1024 px) and 1 <= N <= 64, with mN = floor(2^32 / N) + 1: the
// multiply-high of |F| by mN is floor(|F| / N) exactly, because
// |F| (mN - 2^32 / N) / 2^32 <= 2^-6 and the fraction (|F| mod N) / N is at most
// 1 - 1/N (and below 1 - 2^-6 whenever N = 64 and |F| = 2^26 is a multiple of N).
__device__ __forceinline__ void divmod_n(int F, int N, unsigned mN, int& q, int& r) {
  const unsigned a = (unsigned)abs(F);
  unsigned qa = N == 1 ? a : __umulhi(a, mN);
  int ra = (int)(a - qa * (unsigned)N);
  if (F < 0 && ra != 0) {
    qa += 1;
    ra = N - ra;
  }
  q = F < 0 ? -(int)qa : (int)qa;
  r = ra;
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
    // a failed stream publishes nothing more: stop waiting for it
    if ((spins & 1023) == 0 && __shfl_sync(FULL, ld_volatile(err), 0) != 0) break;
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
//   3. every simulated pixel runs through the N substeps;
//   4. for each (substep, tile row) one segment is published: the row's event
//      and polarity bit masks, or, when a pixel of the row crossed more than
//      one threshold, the row's events written to staging in column order.

__device__ __forceinline__ int activity_threshold(const SimParams& p, int cp, int cn) {
  return p.cact >= 0 ? p.cact : min(cp, cn);
}

constexpr int TP = TW * TH;  // pixels per tile (1024)

struct TileLayout {
  int* sLa;              // two halo buffers (SH x SW); roles swap between frames
  int* sLb;
  int* slut;
  int* sR;               // [TP] sparse: the tile's reference
  unsigned* stk;
  int* swk;
  short* snk;            // [N][TP] sparse: signed event count per (substep, slot)
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
  L.stk = (unsigned*)(L.sR + TP);
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

// Staging space of one warp: multi-crossing rows take their events' space
// from the warp's chunk of the stream's staging area, so that one global
// atomic serves many rows.  A row that does not fit the chunk either starts a
// new chunk (rows of at most STAGE_CHUNK / 4 events, wasting the old chunk's
// remainder: less than a third of what the chunk served) or takes exactly its
// own space.  Chunks are off (chunk == 0) where a block serves several
// streams.  Only lane 0 touches it.
struct WarpStage {
  long long base;
  int left;
  int chunk;
};

__device__ __forceinline__ long long stage_take(const SimParams& p, WarpStage& w, int total) {
  if (total <= w.left) {
    const long long b = w.base;
    w.base += total;
    w.left -= total;
    return b;
  }
  const bool refill = w.chunk > 0 && total <= w.chunk / 4;
  const long long size = refill ? w.chunk : total;
  const unsigned long long b = atomicAdd(&p.ctl->stage_top, (unsigned long long)size);
  if (b + (unsigned long long)size > (unsigned long long)p.stage_cap) {
    atomicExch(&p.ctl->batch_fail, 1);
    return -1;
  }
  if (refill) {
    w.base = (long long)b + total;
    w.left = (int)size - total;
  }
  return (long long)b;
}

// Stage the events of a row whose lanes hold a_lo events of e_lo (the lo
// half's column) and a_hi of e_hi, in column order with repeats adjacent, and
// publish the row's segment.  All 32 lanes must call this.
__device__ __forceinline__ void stage_row(const SimParams& p, WarpStage* ws, Seg* sg, int a_lo,
                                          int a_hi, Ev e_lo, Ev e_hi) {
  const int lane = threadIdx.x & 31;
  const int i_lo = warp_incl_scan(a_lo);
  const int t_lo = __shfl_sync(FULL, i_lo, 31);
  const int i_hi = warp_incl_scan(a_hi);
  const int total = t_lo + __shfl_sync(FULL, i_hi, 31);
  long long base = 0;
  if (lane == 0) base = stage_take(p, *ws, total);
  base = __shfl_sync(FULL, base, 0);
  if (base >= 0) {
    for (int m = 0; m < a_lo; ++m) p.staging[base + i_lo - a_lo + m] = e_lo;
    for (int m = 0; m < a_hi; ++m) p.staging[base + t_lo + i_hi - a_hi + m] = e_hi;
  }
  if (lane == 0) *sg = Seg{0ull, 0ull, base >= 0 ? total : 0, base >= 0 ? (int)base : -1};
}

// Publish the segment of one (substep, tile row) of a dense tile: lane l
// holds the event counts of columns l (n0) and l + 32 (n1).  All 32 lanes
// must call this.
__device__ __forceinline__ void publish_row_dense(const SimParams& p, Seg* sg, int n0, int n1,
                                                  unsigned tk, int tx0, int y, WarpStage* ws) {
  const int lane = threadIdx.x & 31;
  const unsigned e0 = __ballot_sync(FULL, n0 != 0), e1 = __ballot_sync(FULL, n1 != 0);
  if ((e0 | e1) == 0) {
    if (lane == 0) *sg = Seg{0ull, 0ull, 0, -1};
    return;
  }
  const unsigned multi = __ballot_sync(FULL, (unsigned)(n0 + 1) > 2u || (unsigned)(n1 + 1) > 2u);
  if (multi == 0) {
    const unsigned p0 = __ballot_sync(FULL, n0 > 0), p1 = __ballot_sync(FULL, n1 > 0);
    if (lane == 0)
      *sg = Seg{(unsigned long long)e0 | ((unsigned long long)e1 << 32),
                (unsigned long long)p0 | ((unsigned long long)p1 << 32), __popc(e0) + __popc(e1),
                -1};
    return;
  }
  // a pixel crossed two or more thresholds: rows of at least 16 events
  // publish their per-pixel counts (16 bits each, 128 bytes = 16 staging
  // slots, so staging never holds more slots than events), which the order
  // kernel expands; smaller rows stage their events
  const int a0 = abs(n0), a1 = abs(n1);
  const int total = __reduce_add_sync(FULL, a0 + a1);
  if (total < 16) {
    stage_row(p, ws, sg, a0, a1, make_event(tk, tx0 + lane, y, n0 > 0),
              make_event(tk, tx0 + lane + 32, y, n1 > 0));
    return;
  }
  const unsigned p0 = __ballot_sync(FULL, n0 > 0), p1 = __ballot_sync(FULL, n1 > 0);
  long long base = 0;
  if (lane == 0) base = stage_take(p, *ws, 16);
  base = __shfl_sync(FULL, base, 0);
  if (base >= 0) ((unsigned*)(p.staging + base))[lane] = (unsigned)a0 | ((unsigned)a1 << 16);
  if (lane == 0)
    *sg = base >= 0 ? Seg{(unsigned long long)e0 | ((unsigned long long)e1 << 32),
                          (unsigned long long)p0 | ((unsigned long long)p1 << 32), total,
                          -2 - (int)base}
                    : Seg{0ull, 0ull, 0, -1};
}

// Publish the segment of one (substep, tile row) from a warp that holds the
// row's pixels in two 32-lane halves: lanes' event counts n_lo (columns
// col_lo) and n_hi (columns col_hi); columns are the bit positions in the
// segment masks and must increase with the lane within each half, the lo
// half preceding the hi half.  A row with a multi-crossing pixel stages its
// events (column order, repeats adjacent).  All 32 lanes must call this.
__device__ __forceinline__ void publish_row(const SimParams& p, Seg* sg, int n_lo, int col_lo,
                                            bool v_lo, int n_hi, int col_hi, bool v_hi,
                                            unsigned tk, int tx0, int y, WarpStage* ws) {
  const int lane = threadIdx.x & 31;
  const unsigned b_lo = v_lo && n_lo ? 1u << (col_lo & 31) : 0u;
  const unsigned b_hi = v_hi && n_hi ? 1u << (col_hi & 31) : 0u;
  const bool lo_in_low = col_lo < 32, hi_in_low = col_hi < 32;
  const unsigned m_any = __ballot_sync(FULL, (v_lo && n_lo) || (v_hi && n_hi));
  if (m_any == 0) {
    if (lane == 0) *sg = Seg{0ull, 0ull, 0, -1};
    return;
  }
  const unsigned low = __reduce_or_sync(FULL, (lo_in_low ? b_lo : 0u) | (hi_in_low ? b_hi : 0u));
  const unsigned high = __reduce_or_sync(FULL, (lo_in_low ? 0u : b_lo) | (hi_in_low ? 0u : b_hi));
  const unsigned plow = __reduce_or_sync(FULL, (lo_in_low && n_lo > 0 ? b_lo : 0u) |
                                                   (hi_in_low && n_hi > 0 ? b_hi : 0u));
  const unsigned phigh = __reduce_or_sync(FULL, (!lo_in_low && n_lo > 0 ? b_lo : 0u) |
                                                    (!hi_in_low && n_hi > 0 ? b_hi : 0u));
  const int a_lo = v_lo ? abs(n_lo) : 0, a_hi = v_hi ? abs(n_hi) : 0;
  if (!__any_sync(FULL, a_lo > 1 || a_hi > 1)) {
    if (lane == 0)
      *sg = Seg{(unsigned long long)low | ((unsigned long long)high << 32),
                (unsigned long long)plow | ((unsigned long long)phigh << 32),
                __popc(low) + __popc(high), -1};
    return;
  }
  stage_row(p, ws, sg, a_lo, a_hi, make_event(tk, tx0 + col_lo, y, n_lo > 0),
            make_event(tk, tx0 + col_hi, y, n_hi > 0));
}

// The substeps of the (up to) two pixels of this thread.  `lx, ly` are the
// pixels' tile coordinates, `nk_at` their columns in the per-substep record.
// DENSE: the two pixels are columns lane, lane + 32 of tile row `warp`, and the
// row's segment is published from the loop.
template <bool RESET, bool WIDE, bool FAST, bool DENSE, int TH_ = 16>
__device__ __forceinline__ void tile_substeps(const SimParams& p, const TileLayout& L, int N,
                                              unsigned mN, int tx0, int ty0, unsigned b0, unsigned b1,
                                              const FrameRef& prv, const FrameDesc& cur,
                                              Seg* segf, const int (&lx)[2], const int (&ly)[2],
                                              const int (&nk_at)[2], const bool (&act)[2],
                                              const int (&Fx)[2], const int (&Fy)[2],
                                              int (&R)[2], const int (&Cp)[2],
                                              const int (&Cn)[2], WarpStage* ws) {
  constexpr int TH = TH_, NTD = 32 * TH_, TP = TW * TH_, SH = TH_ + 2 * HMAX;
  (void)TH; (void)NTD; (void)TP; (void)SH;
  const int warp = threadIdx.x >> 5;
  int px[2], py[2], ax[2], ay[2], qx[2], rx[2], qy[2], ry[2];
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    // FAST: positions relative to the shared tile origin (tx0 - HMAX, ty0 - HMAX);
    // otherwise absolute image positions.
    px[j] = FAST ? (lx[j] + HMAX) << 16 : (tx0 + lx[j]) << 16;
    py[j] = FAST ? (ly[j] + HMAX) << 16 : (ty0 + ly[j]) << 16;
    // F = q N + r with 0 <= r < N: offset_k = q k + floor(r k / N)
    divmod_n(Fx[j], N, mN, qx[j], rx[j]);
    divmod_n(Fy[j], N, mN, qy[j], ry[j]);
    ax[j] = 0;
    ay[j] = 0;
  }
  const int y = ty0 + warp;
  const bool row_in = !DENSE || y < p.H;
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
      if (!DENSE) L.snk[k * TP + nk_at[j]] = (short)n[j];
    }
    if (DENSE && row_in)  // warp-uniform
      publish_row(p, segf + (long long)k * p.segs_per_k + warp * p.tiles_x, n[0], lx[0], true,
                  n[1], lx[1], true, L.stk[k], tx0, y, ws);
  }
}

// floor(d / c) for d >= c > 0.  Narrow (log) values: d < 2^21, so the fast
// single-precision quotient is within one of the exact one, which an integer
// check corrects; wide (linear) values use integer division.
template <bool WIDE>
__device__ __forceinline__ int floordiv_pos(int d, int c) {
  if (WIDE) return d / c;
  int q = (int)__fdividef((float)d, (float)c);
  if (q * c > d) --q;
  else if ((q + 1) * c <= d) ++q;
  return q;
}

// Dense fast path: the substeps of this thread's two pixels (columns lane and
// lane + 32 of tile row `warp`, both in the image unless `act` says
// otherwise; FULLT: the whole tile row is in the image), sampling the shared
// halos; every substep's row segment is published from the loop.  The common
// case crosses at most one threshold per pixel and substep; a warp in which
// some pixel crossed two or more computes those pixels' counts exactly
// afterwards.  MASKS (N <= 32): the carries of the split offset floor(r k / N)
// come from the frame's carry table cmask[r] (bit 31 - (k - 1) set where the
// offset steps by one more at substep k), shifted out one bit per substep.
template <bool RESET, bool WIDE, bool FULLT, bool MASKS>
__device__ __forceinline__ void dense_substeps(const SimParams& p, const int* swk,
                                               const unsigned* stk, const unsigned* cmask,
                                               int N, unsigned mN, int tx0, int y, unsigned b0,
                                               unsigned b1, Seg* segr, WarpStage* ws,
                                               const bool (&act)[2], const int (&Fx)[2],
                                               const int (&Fy)[2], int (&R)[2],
                                               const int (&Cp)[2], const int (&Cn)[2]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int px[2], py[2], qx[2], qy[2];
  unsigned ax[2], ay[2], rx[2], ry[2];  // MASKS: carry bits; else Bresenham state
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    px[j] = (lane + 32 * j + HMAX) << 16;
    py[j] = (warp + HMAX) << 16;
    // F = q N + r with 0 <= r < N: offset_k = q k + floor(r k / N)
    int r_x, r_y;
    divmod_n(Fx[j], N, mN, qx[j], r_x);
    divmod_n(Fy[j], N, mN, qy[j], r_y);
    if (MASKS) {
      ax[j] = cmask[r_x];
      ay[j] = cmask[r_y];
      qx[j] = -qx[j];
      qy[j] = -qy[j];
    } else {
      rx[j] = (unsigned)r_x;
      ry[j] = (unsigned)r_y;
      ax[j] = 0;
      ay[j] = 0;
    }
  }
  for (int k = 0; k < N; ++k) {
    const int w = swk[k];
    int n[2], D[2];
    bool multi = false;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      if (MASKS) {
        px[j] += qx[j] + ((int)ax[j] >> 31);
        ax[j] <<= 1;
        py[j] += qy[j] + ((int)ay[j] >> 31);
        ay[j] <<= 1;
      } else {
        px[j] -= qx[j];
        ax[j] += rx[j];
        if (ax[j] >= (unsigned)N) { ax[j] -= N; px[j] -= 1; }
        py[j] -= qy[j];
        ay[j] += ry[j];
        if (ay[j] >= (unsigned)N) { ay[j] -= N; py[j] -= 1; }
      }
      const int s0 = tap_shared<WIDE>(b0, px[j], py[j]);
      const int s1 = tap_shared<WIDE>(b1, px[j] + Fx[j], py[j] + Fy[j]);
      const int I = lerp12<WIDE>(s0, s1, w);
      const int d = I - R[j];
      if (RESET) {
        R[j] = I;
        n[j] = d > Cp[j] ? 1 : (d < -Cn[j] ? -1 : 0);
      } else {
        n[j] = d >= Cp[j] ? 1 : (d <= -Cn[j] ? -1 : 0);
        R[j] += n[j] > 0 ? Cp[j] : (n[j] < 0 ? -Cn[j] : 0);
        // a second crossing remains exactly when the residual still crosses
        const int d2 = I - R[j];
        multi |= (FULLT || act[j]) && (d2 >= Cp[j] || d2 <= -Cn[j]);
        D[j] = d;
      }
      if (!FULLT && !act[j]) n[j] = 0;
    }
    if (!RESET && __any_sync(FULL, multi)) {
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        if ((FULLT || act[j]) && D[j] >= 2 * Cp[j]) {
          const int m = floordiv_pos<WIDE>(D[j], Cp[j]);
          R[j] += (m - 1) * Cp[j];
          n[j] = m;
        } else if ((FULLT || act[j]) && D[j] <= -2 * Cn[j]) {
          const int m = floordiv_pos<WIDE>(-D[j], Cn[j]);
          R[j] -= (m - 1) * Cn[j];
          n[j] = -m;
        }
      }
    }
    publish_row_dense(p, segr + (long long)k * p.segs_per_k, n[0], n[1], stk[k], tx0, y, ws);
  }
}

// Sparse fast path: the substeps of this thread's compacted pixels (slots
// tid and, NPX = 2, tid + NTD; `act` says which exist), sampling the shared
// halos.  Each pixel's count per substep goes to snk (slot order) and, when
// non-zero, into the tile's row masks: rowm[(k TH + row) 4 + {0,1}] event
// bits of columns 0-31 / 32-63, {2,3} polarity bits; rows in which a pixel
// crossed two or more thresholds are flagged in smulti[k] (bit = row).
template <bool RESET, bool WIDE, int NPX, int TH_>
__device__ __forceinline__ void sparse_substeps(const int* swk, int N, unsigned mN, unsigned b0,
                                                unsigned b1, short* snk, unsigned* rowm,
                                                unsigned* smulti, const int (&lx)[2],
                                                const int (&ly)[2], const bool (&act)[2],
                                                const int (&Fx)[2], const int (&Fy)[2],
                                                int (&R)[2], const int (&Cp)[2],
                                                const int (&Cn)[2]) {
  constexpr int TH = TH_, NTD = 32 * TH_, TP = TW * TH_, SH = TH_ + 2 * HMAX;
  (void)TH; (void)NTD; (void)TP; (void)SH;
  int px[NPX], py[NPX], ax[NPX], ay[NPX], qx[NPX], rx[NPX], qy[NPX], ry[NPX];
#pragma unroll
  for (int j = 0; j < NPX; ++j) {
    px[j] = (lx[j] + HMAX) << 16;
    py[j] = (ly[j] + HMAX) << 16;
    divmod_n(Fx[j], N, mN, qx[j], rx[j]);
    divmod_n(Fy[j], N, mN, qy[j], ry[j]);
    ax[j] = 0;
    ay[j] = 0;
  }
  for (int k = 0; k < N; ++k) {
    const int w = swk[k];
#pragma unroll
    for (int j = 0; j < NPX; ++j) {
      px[j] -= qx[j];
      ax[j] += rx[j];
      if (ax[j] >= N) { ax[j] -= N; px[j] -= 1; }
      py[j] -= qy[j];
      ay[j] += ry[j];
      if (ay[j] >= N) { ay[j] -= N; py[j] -= 1; }
      const int s0 = tap_shared<WIDE>(b0, px[j], py[j]);
      const int s1 = tap_shared<WIDE>(b1, px[j] + Fx[j], py[j] + Fy[j]);
      const int I = lerp12<WIDE>(s0, s1, w);
      const int d = I - R[j];
      int n;
      if (RESET) {
        R[j] = I;
        n = d > Cp[j] ? 1 : (d < -Cn[j] ? -1 : 0);
      } else {
        n = d >= Cp[j] ? 1 : (d <= -Cn[j] ? -1 : 0);
        if (d >= 2 * Cp[j]) n = floordiv_pos<WIDE>(d, Cp[j]);
        else if (d <= -2 * Cn[j]) n = -floordiv_pos<WIDE>(-d, Cn[j]);
        R[j] += n * (n > 0 ? Cp[j] : Cn[j]);
      }
      if (act[j]) {
        snk[k * TP + threadIdx.x + j * NTD] = (short)n;
        if (n != 0) {
          unsigned* m = rowm + (k * TH + ly[j]) * 4;
          const unsigned bit = 1u << (lx[j] & 31);
          const int h = lx[j] >> 5;
          atomicOr(m + h, bit);
          if (n > 0) atomicOr(m + 2 + h, bit);
          if (n > 1 || n < -1) atomicOr(smulti + k, 1u << ly[j]);
        }
      }
    }
  }
}

// Wait (thread 0, bounded) until the tile's progress word reaches `want`
// ([batch serial:32][frames done:32]); gives up when the stream has failed
// or after SPIN_LIMIT polls (then flags a timeout).
__device__ __forceinline__ void wait_tile(const SimParams& p, int tile, unsigned long long want) {
  int spins = 0;
  while (ld_volatile(&p.tdone[tile]) < want) {
    if (++spins > SPIN_LIMIT) {
      atomicCAS(&p.ctl->err, 0, SIM_ERR_DEVICE_TIMEOUT);
      break;
    }
    if ((spins & 1023) == 0 && ld_volatile(&p.ctl->err) != 0) break;
    __nanosleep(64);
  }
  __threadfence();
}

// Frames [f0, f1) of one tile, carried by one block: the tile's reference and
// thresholds stay in registers (dense) or shared memory (sparse) across the
// frames, and frame i's halo is kept as frame i+1's previous-frame halo.
// f0 > 0: the tile's earlier frames were simulated by another block; wait for
// them.  Publishes the tile's progress word at the end.  ONE: a single frame
// (f1 = f0 + 1), which needs no state carried from frame to frame.
template <bool RESET, bool MAPS, bool WIDE, bool SPARSE, bool ONE = false>
__device__ __forceinline__ void tile_frames(const SimParams& p, const BatchArg& b, int tile, int f0,
                                            int f1) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_warp[NTD / 32 + 1];
  __shared__ int s_fx, s_fy;
  __shared__ int s_rs[TH + 1];  // first slot of each tile row
  __shared__ WarpStage s_stage[NTD / 32];
  Ctl* ctl = p.ctl;
  if (block_error(&ctl->err)) return;
  // exact staging allocations: this block may serve several streams
  if ((threadIdx.x & 31) == 0) s_stage[threadIdx.x >> 5] = WarpStage{0, 0, 0};

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nmax = p.n_max;
  const TileLayout L = tile_layout(smem_raw, nmax);
  const int tcx = tile % p.tiles_x, tcy = tile / p.tiles_x;
  const int tx0 = tcx * TW, ty0 = tcy * TH;
  const int W = p.W, H = p.H;

  // frames before f0 were simulated by other blocks: wait for the last one
  if (f0 > 0) {
    if (tid == 0) wait_tile(p, tile, ((unsigned long long)b.serial << 32) | (unsigned)f0);
    if (block_error(&ctl->err)) return;
  }
  if (tid < 256) L.slut[tid] = p.lut[tid];
  const int sel = ctl->sel;
  const int* Rin = (sel & 1) ? p.R1 : p.R0;
  int* Rout = (sel & 1) ? p.R0 : p.R1;
  // frame 0 of the batch starts from the committed reference, a later first
  // frame from what the previous frame wrote (read through L2: another block
  // wrote it)
  const int* Rsrc = f0 == 0 ? Rin : Rout;
  const unsigned char* ringp = (sel & 2) ? p.ring1 : p.ring0;
  unsigned char* ringn = (sel & 2) ? p.ring0 : p.ring1;
  long long tprev = f0 == 0 ? ctl->t_prev : b.frames[f0 - 1].t_rel;

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
        if (!RESET) L.sR[own[q]] = __ldcg(Rsrc + i);
        if (MAPS) { L.sCp[own[q]] = p.cpmap[i]; L.sCn[own[q]] = p.cnmap[i]; }
      } else {
        if (!RESET) Rd[q] = __ldcg(Rsrc + i);
        if (MAPS) { Cpd[q] = p.cpmap[i]; Cnd[q] = p.cnmap[i]; }
      }
    }
  }
  int clamps = 0;
  long long act_sum = 0, act_n = 0;
  // halo buffers: `cb` will receive frame i; `pb` holds frame i-1 over the
  // extent (phx, phy), or nothing yet (-1)
  int* cb = L.sLb;
  int* pb = L.sLa;
  int phx = -1, phy = -1;
  int hfx = 1, hfy = 1;  // fill extents only grow within a batch
  // the tile's flow reach of the first frame; each frame resets it for the
  // next one once every thread has read it (a barrier always separates the
  // reset from the next frame's atomicMax)
  if (tid == 0) { s_fx = 0; s_fy = 0; }
  __syncthreads();  // the table, reference and thresholds above are read by all threads

  for (int fi = f0; fi < (ONE ? f0 + 1 : f1); ++fi) {
    const FrameDesc cur = b.frames[fi];
    const FrameRef prv = prev_frame(p, b, fi, ringp);
    FrameRef curf;
    curf.ptr = cur.frame;
    curf.pitch = cur.pitch;
    curf.ch = p.ch;
    const int N = p.n_fixed > 0 ? p.n_fixed : adaptive_n(p.maxf2[fi], nmax);
    const unsigned mN = N > 1 ? (unsigned)(0x100000000ull / (unsigned)N) + 1u : 0u;
    Seg* segf = p.seg + (long long)fi * nmax * p.segs_per_k + (long long)ty0 * p.tiles_x + tcx;
    if (tid < N) {
      const int k = tid + 1;
      L.swk[tid] = (k * 8192 + N) / (2 * N);
      const long long dt = cur.t_rel - tprev;
      L.stk[tid] = (unsigned)(tprev + (k * dt) / N);
    }

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
    if (tid == 0) { s_fx = 0; s_fy = 0; }  // hx, hy are read by now

    // 3. substeps (sparse: warps without a compacted pixel skip them); dense
    // rows publish their segments from the loop
    const unsigned b0 = (unsigned)__cvta_generic_to_shared(pb);
    const unsigned b1 = (unsigned)__cvta_generic_to_shared(cb);
    if (!SPARSE || warp * 32 < A || warp * 32 + NTD < A) {  // warp-uniform
      if (fast)
        tile_substeps<RESET, WIDE, true, !SPARSE>(p, L, N, mN, tx0, ty0, b0, b1, prv, cur, segf,
                                                  lx, ly, nk_at, act, Fx, Fy, R, Cp, Cn, &s_stage[warp]);
      else
        tile_substeps<RESET, WIDE, false, !SPARSE>(p, L, N, mN, tx0, ty0, b0, b1, prv, cur, segf,
                                                   lx, ly, nk_at, act, Fx, Fy, R, Cp, Cn, &s_stage[warp]);
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

    // 4. sparse: warp r publishes the segments of tile row r from the
    // records of the row's slots (contiguous, in column order)
    static_assert(NTD / 32 == TH, "one warp per tile row");
    if (SPARSE) {
      __syncthreads();
      const int r = warp, s0 = s_rs[r], s1 = s_rs[r + 1];
      const int y = ty0 + r;
      if (y < H) {
        if (s1 == s0) {
          for (int k = lane; k < N; k += 32) segf[(long long)k * p.segs_per_k + r * p.tiles_x] =
              Seg{0ull, 0ull, 0, -1};
        } else {
          const int j_lo = s0 + lane, j_hi = s0 + 32 + lane;
          const bool v_lo = j_lo < s1, v_hi = j_hi < s1;
          const int col_lo = v_lo ? (L.sslot[j_lo] & (TW - 1)) : 0;
          const int col_hi = v_hi ? (L.sslot[j_hi] & (TW - 1)) : 0;
          for (int k = 0; k < N; ++k) {
            const int n_lo = v_lo ? L.snk[k * TP + j_lo] : 0;
            const int n_hi = v_hi ? L.snk[k * TP + j_hi] : 0;
            publish_row(p, segf + (long long)k * p.segs_per_k + r * p.tiles_x, n_lo, col_lo, v_lo,
                        n_hi, col_hi, v_hi, L.stk[k], tx0, y, &s_stage[warp]);
          }
        }
      }
    }
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

  if (!RESET) {
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
  // frames [f0, f1) of the tile are done: their reference may be read
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    st_volatile(&p.tdone[tile], ((unsigned long long)b.serial << 32) | (unsigned)f1);
  }
}


// ---------------------------------------------------------------------------
// One stream's batch, software-pipelined over the frames.  One block per tile
// carries the tile through every frame of the batch (blocks never wait for
// one another), as tile_frames does, but the inputs of frame i+1 - its raw
// bytes over the tile's largest window, its flow at the tile's pixels, the
// descriptor of frame i+2 - are copied into shared memory asynchronously
// (cp.async) while frame i is simulated.  Per frame, the block then reads HBM
// only through copies already in flight; the halo of log values is built from
// the staged bytes.  Frames whose base or pitch is not a multiple of 4 bytes
// (flows: 8 bytes) are staged with plain loads instead.

__device__ __forceinline__ void cp_async4(unsigned dst, const void* src, int src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst), "l"(src), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async8(unsigned dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async16(unsigned dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

// Shared memory of the batch kernel.  `raw` holds two frames' bytes over the
// tile window (SH rows of SW pixels, stride SW * ch bytes): the previous and
// the current frame, the next frame being copied over the previous one
// during the substeps.  sflow holds the flows of two frames.  Dense tiles do
// not use the sparse arrays (sR, snk, sslot, sCp, sCn).
struct BatchLayout {
  float2* sflow;        // [2][TP]
  int* sLa;             // two halo buffers (SH x SW)
  int* sLb;
  int* slut;
  int* sR;              // [TP] sparse
  unsigned* stk;        // [2][nmax] substep times (frame parity)
  int* swk;             // [2][nmax] substep weights
  unsigned char* raw;   // [2][SH][SW * ch]
  short* snk;           // [nmax][TP] sparse
  short* sslot;         // [TP] sparse
  unsigned short* sCp;  // [TP] sparse maps
  unsigned short* sCn;
};

__host__ __device__ inline size_t batch_smem_bytes(int n_max, int ch, bool sparse, int th) {
  const int TP = TW * th, SH = th + 2 * HMAX;
  size_t b = (size_t)2 * TP * sizeof(float2);
  b += (size_t)(2 * SH * SW + 256 + (sparse ? TP : 0) + 4 * n_max) * 4;
  b += (size_t)2 * SH * SW * ch;
  if (sparse) b += (size_t)(n_max * TP + 3 * TP) * 2;
  return b;
}

template <bool SPARSE, int TH_>
__device__ __forceinline__ BatchLayout batch_layout(unsigned char* base, int nmax, int ch) {
  constexpr int TH = TH_, NTD = 32 * TH_, TP = TW * TH_, SH = TH_ + 2 * HMAX;
  (void)TH; (void)NTD; (void)TP; (void)SH;
  BatchLayout L;
  L.sflow = (float2*)base;
  L.sLa = (int*)(L.sflow + 2 * TP);
  L.sLb = L.sLa + SH * SW;
  L.slut = L.sLb + SH * SW;
  L.sR = L.slut + 256;
  L.stk = (unsigned*)(L.sR + (SPARSE ? TP : 0));
  L.swk = (int*)(L.stk + 2 * nmax);
  L.raw = (unsigned char*)(L.swk + 2 * nmax);
  L.snk = (short*)(L.raw + 2 * SH * SW * ch);
  L.sslot = L.snk + nmax * TP;
  L.sCp = (unsigned short*)(L.sslot + TP);
  L.sCn = L.sCp + TP;
  return L;
}

// Stage the bytes of frame f over the tile window (image rows ty0 - HMAX ..
// ty0 + TH + HMAX - 1 and columns tx0 - HMAX .. tx0 + TW + HMAX - 1, clipped
// to the image) into raw, row r of the window at raw + r * SW * ch.  Window
// rows and columns outside the image are never read.
template <int TH_>
__device__ __forceinline__ void stage_raw(unsigned char* raw, const FrameRef& f, int W, int H,
                                          int tx0, int ty0) {
  constexpr int TH = TH_, NTD = 32 * TH_, TP = TW * TH_, SH = TH_ + 2 * HMAX;
  (void)TH; (void)NTD; (void)TP; (void)SH;
  const int ch = f.ch, RW = SW * ch;
  const int r0 = max(0, HMAX - ty0), r1 = min(SH, H - ty0 + HMAX);
  const int cx0 = max(0, tx0 - HMAX), cx1 = min(W, tx0 + TW + HMAX);
  const int b0 = (cx0 - (tx0 - HMAX)) * ch;  // byte offset of column cx0 in a window row
  const int nb = (cx1 - cx0) * ch;            // bytes per row
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if ((((unsigned long long)f.ptr | (unsigned long long)f.pitch) & 3) == 0) {
    // cx0 * ch is a multiple of 16, so every word starts 4-byte aligned; the
    // last word of a row copies only the row's remaining bytes (zero fill
    // within the window row)
    const int nw = (nb + 3) >> 2;
    const unsigned dst0 = smem_addr(raw) + (unsigned)b0;
    for (int r = r0 + warp; r < r1; r += NTD / 32) {
      const unsigned char* src = f.ptr + (long long)(ty0 - HMAX + r) * f.pitch + (long long)cx0 * ch;
      for (int w = lane; w < nw; w += 32)
        cp_async4(dst0 + (unsigned)(r * RW + 4 * w), src + 4 * w, min(4, nb - 4 * w));
    }
  } else {
    for (int r = r0 + warp; r < r1; r += NTD / 32) {
      const unsigned char* src = f.ptr + (long long)(ty0 - HMAX + r) * f.pitch + (long long)cx0 * ch;
      for (int c = lane; c < nb; c += 32) raw[r * RW + b0 + c] = src[c];
    }
  }
}

// Stage the flow of the tile's pixels (tile pixel index ly * TW + lx) into sf;
// pixels outside the image are not written.
template <int TH_>
__device__ __forceinline__ void stage_flow(float2* sf, const float2* flow, int W, int H, int tx0,
                                           int ty0) {
  constexpr int TH = TH_, NTD = 32 * TH_, TP = TW * TH_, SH = TH_ + 2 * HMAX;
  (void)TH; (void)NTD; (void)TP; (void)SH;
  const bool al = ((unsigned long long)flow & 7) == 0;
  const unsigned d0 = smem_addr(sf);
#pragma unroll
  for (int q = 0; q < TP / NTD; ++q) {
    const int t = threadIdx.x + q * NTD;
    const int lx = t & (TW - 1), ly = t / TW;
    const int x = tx0 + lx, y = ty0 + ly;
    if (x < W && y < H) {
      const float2* src = flow + (long long)y * W + x;
      if (al) cp_async8(d0 + (unsigned)t * 8u, src);
      else sf[t] = *src;
    }
  }
}

// 8-bit luma of window pixel (row rr, column rc) of a staged frame.
__device__ __forceinline__ int raw_luma(const unsigned char* raw, int ch, int rr, int rc) {
  const unsigned char* q = raw + rr * (SW * ch) + rc * ch;
  if (ch == 1) return q[0];
  return (77 * q[0] + 150 * q[1] + 29 * q[2] + 128) >> 8;
}

// Replicate-padded halo of log values with reach (hx, hy) from a staged
// frame (same region and layout as fill_halo): one warp per halo row.
template <int TH_>
__device__ __forceinline__ void fill_halo_raw(int* dst, const int* slut, const unsigned char* raw,
                                              int ch, int W, int H, int tx0, int ty0, int hx,
                                              int hy) {
  constexpr int TH = TH_, NTD = 32 * TH_, TP = TW * TH_, SH = TH_ + 2 * HMAX;
  (void)TH; (void)NTD; (void)TP; (void)SH;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ncols = TW + 2 * hx, nrows = TH + 2 * hy;
  const int RW = SW * ch;
  for (int sr = warp; sr < nrows; sr += NTD / 32) {
    const int gy = min(max(ty0 - hy + sr, 0), H - 1);
    const unsigned char* src = raw + (gy - (ty0 - HMAX)) * RW;
    int* d = dst + (HMAX - hy + sr) * SW + (HMAX - hx);
    for (int sc = lane; sc < ncols; sc += 32) {
      const int gx = min(max(tx0 - hx + sc, 0), W - 1);
      const unsigned char* q = src + (gx - (tx0 - HMAX)) * ch;
      const int v = ch == 1 ? q[0] : (77 * q[0] + 150 * q[1] + 29 * q[2] + 128) >> 8;
      d[sc] = slut[v];
    }
  }
}

// Substep weights and times of one frame (threads k < N) into the parity's
// tables, and for N <= 32 its carry table (dense_substeps); thread 0
// publishes N and its division multiplier (divmod_n).  Called by threads
// 0..63 only.
__device__ __forceinline__ void substep_tables(const SimParams& p, unsigned long long maxf2,
                                               long long t_prev, long long t_cur, int* swk,
                                               unsigned* stk, int* sN, unsigned* smN,
                                               unsigned* cmask) {
  const int N = p.n_fixed > 0 ? p.n_fixed : adaptive_n(maxf2, p.n_max);
  if ((int)threadIdx.x < N) {
    const int k = threadIdx.x + 1;
    swk[threadIdx.x] = (k * 8192 + N) / (2 * N);
    stk[threadIdx.x] = (unsigned)(t_prev + (k * (t_cur - t_prev)) / N);
    if (N <= 32) {  // carry table of remainder r = threadIdx.x
      const int r = threadIdx.x;
      unsigned m = 0;
      for (int j = 1; j <= N; ++j)
        if ((r * j) / N != (r * (j - 1)) / N) m |= 1u << (32 - j);
      cmask[r] = m;
    }
  }
  if (threadIdx.x == 0) {
    *sN = N;
    *smN = N > 1 ? (unsigned)(0x100000000ull / (unsigned)N) + 1u : 0u;
  }
}

template <bool RESET, bool MAPS, bool WIDE, bool SPARSE, int TH_>
__device__ __forceinline__ void tile_batch(const SimParams& p, const BatchArg& b, int tile) {
  constexpr int TH = TH_, NTD = 32 * TH_, TP = TW * TH_, SH = TH_ + 2 * HMAX;
  (void)TH; (void)NTD; (void)TP; (void)SH;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_warp[NTD / 32 + 1];
  __shared__ int s_fx, s_fy;
  __shared__ int s_rs[TH + 1];
  __shared__ int s_N[2];
  __shared__ unsigned s_mN[2];
  __shared__ unsigned s_cmask[2][32];  // carry tables of the frame parities
  __shared__ unsigned s_multi[32];  // sparse: rows with multi-crossings, per substep
  __shared__ unsigned char s_act[TP];  // sparse: activity of each tile pixel
  __shared__ __align__(16) FrameDesc s_desc[4];     // frame fi at fi & 3
  __shared__ __align__(8) unsigned long long s_mf[4];  // its squared flow maximum
  __shared__ WarpStage s_stage[NTD / 32];
  Ctl* ctl = p.ctl;
  if (block_error(&ctl->err)) return;
  if ((threadIdx.x & 31) == 0) s_stage[threadIdx.x >> 5] = WarpStage{0, 0, p.stage_chunk};

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nmax = p.n_max, ch = p.ch, RW = SW * ch;
  const BatchLayout L = batch_layout<SPARSE, TH_>(smem_raw, nmax, ch);
  const int tcx = tile % p.tiles_x, tcy = tile / p.tiles_x;
  const int tx0 = tcx * TW, ty0 = tcy * TH;
  const int W = p.W, H = p.H, count = b.count;
  const bool adaptive = p.n_fixed <= 0;

  if (tid < 256) L.slut[tid] = p.lut[tid];
  const int sel = ctl->sel;
  const int* Rin = (sel & 1) ? p.R1 : p.R0;
  int* Rout = (sel & 1) ? p.R0 : p.R1;
  const unsigned char* ringp = (sel & 2) ? p.ring1 : p.ring0;
  unsigned char* ringn = (sel & 2) ? p.ring0 : p.ring1;
  const long long t_first = ctl->t_prev;

  // Dense: thread (warp w, lane l) owns tile pixels (l, w) and (l + 32, w);
  // sparse: thread t owns tile pixels t and t + NTD.
  int own[2];
  bool inimg[2];
  int Rd[2], Cpd[2], Cnd[2];
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

  // prologue: descriptors of frames 0 and 1, the previous frame (ring) and
  // frame 0 staged, frame 0's flow and substep tables
  if (tid < 2 && tid < count) {
    s_desc[tid] = b.frames[tid];
    s_mf[tid] = adaptive ? p.maxf2[tid] : 0ull;
  }
  if (tid == 0) { s_fx = 0; s_fy = 0; }
  __syncthreads();
  {
    const FrameRef ring{ringp, (long long)W, 1};
    const FrameDesc d0 = s_desc[0];
    stage_raw<TH_>(L.raw, ring, W, H, tx0, ty0);
    stage_raw<TH_>(L.raw + SH * RW, FrameRef{d0.frame, d0.pitch, ch}, W, H, tx0, ty0);
    stage_flow<TH_>(L.sflow, d0.flow, W, H, tx0, ty0);
    cp_async_commit();
    if (tid < 64)
      substep_tables(p, s_mf[0], t_first, d0.t_rel, L.swk, L.stk, &s_N[0], &s_mN[0], s_cmask[0]);
    cp_async_wait_all();
  }
  __syncthreads();

  int clamps = 0;
  long long act_sum = 0, act_n = 0;
  int rb = 1;  // raw buffer of the current frame; 1 - rb holds the previous frame
  int* cb = L.sLb;
  int* pb = L.sLa;
  int phx = -1, phy = -1;
  int hfx = 1, hfy = 1;  // halo extents only grow within a batch

  for (int fi = 0; fi < count; ++fi) {
    const int par = fi & 1;
    const FrameDesc cur = s_desc[fi & 3];
    FrameRef prv;
    if (fi == 0) {
      prv = FrameRef{ringp, (long long)W, 1};
    } else {
      const FrameDesc d = s_desc[(fi - 1) & 3];
      prv = FrameRef{d.frame, d.pitch, ch};
    }
    const FrameRef curf{cur.frame, cur.pitch, ch};
    const unsigned char* rawc = L.raw + rb * SH * RW;
    const unsigned char* rawp = L.raw + (1 - rb) * SH * RW;
    const int chp = fi == 0 ? 1 : ch;  // the ring holds luma
    const int N = s_N[par];
    const unsigned mN = s_mN[par];
    Seg* segf = p.seg + (long long)fi * nmax * p.segs_per_k + (long long)ty0 * p.tiles_x + tcx;

    // 1. the pixels to simulate (the previous and current bytes are staged)
    int A = 0;
    int sel_flag[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int lx = own[q] & (TW - 1), ly = own[q] / TW;
      bool a = inimg[q];
      if (inimg[q] && (SPARSE || fi == count - 1)) {
        const int vc = raw_luma(rawc, ch, ly + HMAX, lx + HMAX);
        if (fi == count - 1) ringn[(long long)(ty0 + ly) * W + tx0 + lx] = (unsigned char)vc;
        if (SPARSE) {
          const int vp = raw_luma(rawp, chp, ly + HMAX, lx + HMAX);
          const int cp = MAPS ? (int)L.sCp[own[q]] : p.cp, cn = MAPS ? (int)L.sCn[own[q]] : p.cn;
          a = abs(L.slut[vc] - L.slut[vp]) >= activity_threshold(p, cp, cn);
        }
      }
      sel_flag[q] = a ? 1 : 0;
      if (SPARSE) s_act[own[q]] = (unsigned char)sel_flag[q];
    }
    if (SPARSE) {
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
    // sparse tiles with at least 3/8 of their pixels active run the frame
    // through the dense loop (inactive pixels masked, their reference kept):
    // cheaper per pixel than compaction, per-slot records and mask atomics
    const bool dsw = SPARSE && 8 * A >= 3 * TP;

    // 2. the simulated pixels of this thread and their (staged) flow; the
    // tile's reach
    int lx[2], ly[2], nk_at[2], Fx[2], Fy[2], R[2], Cp[2], Cn[2];
    bool act[2];
    unsigned mfx = 0, mfy = 0;
    const float2* sfl = L.sflow + par * TP;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      int slot;
      if (dsw) {  // the dense mapping: columns lane, lane + 32 of row warp
        slot = warp * TW + lane + 32 * q;
        act[q] = s_act[slot] != 0;
        nk_at[q] = slot;
      } else if (SPARSE) {
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
        const float2 fl = sfl[slot];
        Fx[q] = flow_q16(fl.x, clamps);
        Fy[q] = flow_q16(fl.y, clamps);
        if (SPARSE) {
          if (MAPS) { Cp[q] = L.sCp[slot]; Cn[q] = L.sCn[slot]; }
          if (!RESET) R[q] = L.sR[slot];
        }
        if (RESET) R[q] = L.slut[raw_luma(rawp, chp, ly[q] + HMAX, lx[q] + HMAX)];
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
    const int hx = (s_fx >> 16) + 1, hy = (s_fy >> 16) + 1;
    const bool fast = hx <= HMAX && hy <= HMAX;
    // sparse fast path: row masks in the current flow buffer (its flows are
    // in registers by now), cleared here
    const bool maskpub = SPARSE && !dsw && fast && N <= 32;
    unsigned* rowm = (unsigned*)(L.sflow + par * TP);
    if (maskpub) {
      for (int i = tid; i < N * TH * 4; i += NTD) rowm[i] = 0u;
      if (tid < N) s_multi[tid] = 0u;
    }
    if (fast && A > 0) {
      hfx = max(hfx, hx);
      hfy = max(hfy, hy);
      if (phx < hx || phy < hy) {  // the kept halo of frame i-1 does not reach far enough
        fill_halo_raw<TH_>(pb, L.slut, rawp, chp, W, H, tx0, ty0, hfx, hfy);
        phx = hfx;
        phy = hfy;
      }
      fill_halo_raw<TH_>(cb, L.slut, rawc, ch, W, H, tx0, ty0, hfx, hfy);
    }
    __syncthreads();
    if (tid == 0) { s_fx = 0; s_fy = 0; }  // hx, hy are read by now

    // 3. the next frame's inputs: its bytes over the previous frame's raw
    // buffer (read by now), its flow, the descriptor two frames ahead; its
    // substep tables
    if (fi + 1 < count) {
      const FrameDesc nd = s_desc[(fi + 1) & 3];
      stage_raw<TH_>(L.raw + (1 - rb) * SH * RW, FrameRef{nd.frame, nd.pitch, ch}, W, H, tx0, ty0);
      stage_flow<TH_>(L.sflow + (par ^ 1) * TP, nd.flow, W, H, tx0, ty0);
      if (fi + 2 < count && tid < 2) {
        // descriptors are 32-byte, 16-byte aligned records
        cp_async16(smem_addr(&s_desc[(fi + 2) & 3]) + 16u * tid,
                   (const unsigned char*)&b.frames[fi + 2] + 16 * tid);
        if (tid == 0 && adaptive) cp_async8(smem_addr(&s_mf[(fi + 2) & 3]), &p.maxf2[fi + 2]);
      }
      cp_async_commit();
      if (tid < 64)
        substep_tables(p, s_mf[(fi + 1) & 3], cur.t_rel, nd.t_rel, L.swk + (par ^ 1) * nmax,
                       L.stk + (par ^ 1) * nmax, &s_N[par ^ 1], &s_mN[par ^ 1], s_cmask[par ^ 1]);
    }

    // 4. substeps (sparse: warps without a compacted pixel skip them); dense
    // rows publish their segments from the loop
    TileLayout V;
    V.slut = L.slut;
    V.stk = L.stk + par * nmax;
    V.swk = L.swk + par * nmax;
    V.snk = L.snk;
    const unsigned b0 = smem_addr(pb);
    const unsigned b1 = smem_addr(cb);
    if (SPARSE && dsw && !(fast && N <= 32)) {
      if (fast)
        tile_substeps<RESET, WIDE, true, true, TH_>(p, V, N, mN, tx0, ty0, b0, b1, prv, cur, segf,
                                                    lx, ly, nk_at, act, Fx, Fy, R, Cp, Cn,
                                                    &s_stage[warp]);
      else
        tile_substeps<RESET, WIDE, false, true, TH_>(p, V, N, mN, tx0, ty0, b0, b1, prv, cur,
                                                     segf, lx, ly, nk_at, act, Fx, Fy, R, Cp, Cn,
                                                     &s_stage[warp]);
    } else if ((!SPARSE || dsw) && fast) {
      if (ty0 + warp < H) {  // warp-uniform: rows below the image publish nothing
        // the row's 64 pixels are in the image (and, sparse, all simulated)
        const bool fullt = !SPARSE && tx0 + TW <= W;
#define EVSIM_DENSE(FT, MK)                                                                    \
  dense_substeps<RESET, WIDE, FT, MK>(p, V.swk, V.stk, s_cmask[par], N, mN, tx0, ty0 + warp, b0, \
                                      b1, segf + warp * p.tiles_x, &s_stage[warp], act, Fx, Fy,  \
                                      R, Cp, Cn)
        if (N <= 32) {
          if (fullt) EVSIM_DENSE(true, true);
          else EVSIM_DENSE(false, true);
        } else {
          if (fullt) EVSIM_DENSE(true, false);
          else EVSIM_DENSE(false, false);
        }
#undef EVSIM_DENSE
      }
    } else if (maskpub) {  // warp-uniform: one pixel per thread when A <= NTD
      if (A <= NTD) {
        if (warp * 32 < A)
          sparse_substeps<RESET, WIDE, 1, TH_>(V.swk, N, mN, b0, b1, L.snk, rowm, s_multi, lx, ly, act,
                                          Fx, Fy, R, Cp, Cn);
      } else {
        sparse_substeps<RESET, WIDE, 2, TH_>(V.swk, N, mN, b0, b1, L.snk, rowm, s_multi, lx, ly, act,
                                        Fx, Fy, R, Cp, Cn);
      }
    } else if (!SPARSE || warp * 32 < A || warp * 32 + NTD < A) {  // warp-uniform
      if (fast)
        tile_substeps<RESET, WIDE, true, !SPARSE, TH_>(p, V, N, mN, tx0, ty0, b0, b1, prv, cur, segf,
                                                  lx, ly, nk_at, act, Fx, Fy, R, Cp, Cn,
                                                  &s_stage[warp]);
      else
        tile_substeps<RESET, WIDE, false, !SPARSE, TH_>(p, V, N, mN, tx0, ty0, b0, b1, prv, cur, segf,
                                                   lx, ly, nk_at, act, Fx, Fy, R, Cp, Cn,
                                                   &s_stage[warp]);
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

    // 5. sparse, fast path: one thread per (substep, row) publishes the row's
    // masks; warp r stages the rows with multi-crossings from the records of
    // the row's slots (contiguous, in column order)
    if (maskpub) {
      __syncthreads();
      for (int t = tid; t < N * TH; t += NTD) {
        const int k = t / TH, r = t - k * TH;
        if (ty0 + r >= H || ((s_multi[k] >> r) & 1u)) continue;
        const unsigned* m = rowm + t * 4;
        const int cnt = __popc(m[0]) + __popc(m[1]);
        segf[(long long)k * p.segs_per_k + r * p.tiles_x] =
            cnt ? Seg{(unsigned long long)m[0] | ((unsigned long long)m[1] << 32),
                      (unsigned long long)m[2] | ((unsigned long long)m[3] << 32), cnt, -1}
                : Seg{0ull, 0ull, 0, -1};
      }
      const int r = warp, s0 = s_rs[r], s1 = s_rs[r + 1];
      const int y = ty0 + r;
      if (y < H) {
        const int j_lo = s0 + lane, j_hi = s0 + 32 + lane;
        const bool v_lo = j_lo < s1, v_hi = j_hi < s1;
        const int col_lo = v_lo ? (L.sslot[j_lo] & (TW - 1)) : 0;
        const int col_hi = v_hi ? (L.sslot[j_hi] & (TW - 1)) : 0;
        for (int k = 0; k < N; ++k) {
          if (!((s_multi[k] >> r) & 1u)) continue;  // warp-uniform
          const int n_lo = v_lo ? L.snk[k * TP + j_lo] : 0;
          const int n_hi = v_hi ? L.snk[k * TP + j_hi] : 0;
          publish_row(p, segf + (long long)k * p.segs_per_k + r * p.tiles_x, n_lo, col_lo, v_lo,
                      n_hi, col_hi, v_hi, V.stk[k], tx0, y, &s_stage[warp]);
        }
      }
    } else if (SPARSE && !dsw) {
      __syncthreads();
      const int r = warp, s0 = s_rs[r], s1 = s_rs[r + 1];
      const int y = ty0 + r;
      if (y < H) {
        if (s1 == s0) {
          for (int k = lane; k < N; k += 32) segf[(long long)k * p.segs_per_k + r * p.tiles_x] =
              Seg{0ull, 0ull, 0, -1};
        } else {
          const int j_lo = s0 + lane, j_hi = s0 + 32 + lane;
          const bool v_lo = j_lo < s1, v_hi = j_hi < s1;
          const int col_lo = v_lo ? (L.sslot[j_lo] & (TW - 1)) : 0;
          const int col_hi = v_hi ? (L.sslot[j_hi] & (TW - 1)) : 0;
          for (int k = 0; k < N; ++k) {
            const int n_lo = v_lo ? L.snk[k * TP + j_lo] : 0;
            const int n_hi = v_hi ? L.snk[k * TP + j_hi] : 0;
            publish_row(p, segf + (long long)k * p.segs_per_k + r * p.tiles_x, n_lo, col_lo, v_lo,
                        n_hi, col_hi, v_hi, V.stk[k], tx0, y, &s_stage[warp]);
          }
        }
      }
    }
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
    rb = 1 - rb;
    cp_async_wait_all();
    __syncthreads();
  }

  if (!RESET) {
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

// One stream's batch: one block per tile carries the tile through every
// frame of the batch, its inputs staged a frame ahead (blocks never wait for
// one another).
// Tile of block b in serpentine order (one of the autotuner's choices):
// blocks are placed on the SMs in rounds of one block per SM, and the blocks
// of consecutive rounds share SMs.  Odd rounds take their tiles in reverse
// order, so the blocks sharing an SM hold tiles from opposite ends of the
// image: where activity is concentrated in one region, its tiles do not pile
// up on the same SMs.  Tiles are independent, so the order changes only the
// schedule.
__device__ __forceinline__ int serpentine_tile(int b, int T, int S) {
  if (S < 1) return b;
  const int r = b / S, j = b - r * S;
  const int size = min(S, T - r * S);
  return r * S + ((r & 1) ? size - 1 - j : j);
}

template <bool RESET, bool MAPS, bool WIDE, bool SPARSE, int TH_>
__global__ void __launch_bounds__(32 * TH_, 32 / TH_) k_tile(SimParams p, BatchArg b) {
  const int bi = blockIdx.x;
  const int tile = p.block_order == 2 ? p.tile_order[bi]
                   : p.block_order == 1 ? serpentine_tile(bi, gridDim.x, p.sms)
                                        : bi;
  const long long c0 = clock64();
  tile_batch<RESET, MAPS, WIDE, SPARSE, TH_>(p, b, tile);
  if (p.tile_cost && threadIdx.x == 0) p.tile_cost[tile] = (unsigned)((clock64() - c0) >> 8);
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

// Balanced block order for the next batch (one block): tiles ranked by the
// cycles their blocks took in the last batch (heaviest first, ties by tile
// index), laid out in serpentine order over the ranks - round 0 of one block
// per SM takes the heaviest tiles, round 1 the lightest in reverse - so the
// heaviest tile shares its SM with the lightest.  An order of the tiles like
// any other: it changes only the schedule.
__global__ void k_plan(int T, int S, const unsigned* cost, int* order) {
  __shared__ unsigned sc[PLAN_MAX_TILES];
  __shared__ int sorted[PLAN_MAX_TILES];
  for (int t = threadIdx.x; t < T; t += blockDim.x) sc[t] = cost[t];
  __syncthreads();
  for (int t = threadIdx.x; t < T; t += blockDim.x) {
    const unsigned c = sc[t];
    int rank = 0;
    for (int u = 0; u < T; ++u) rank += sc[u] > c || (sc[u] == c && u < t);
    sorted[rank] = t;
  }
  __syncthreads();
  for (int b = threadIdx.x; b < T; b += blockDim.x) order[b] = sorted[serpentine_tile(b, T, S)];
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

// Shared memory of an order block.
struct OrderSmem {
  int ex[OCHUNK];
  int src[OCHUNK];
  unsigned long long mask[OCHUNK];
  unsigned long long pol[OCHUNK];
  unsigned t[OCHUNK];
  unsigned xy[OCHUNK];  // x0 | (y << 16)
  int N[SIM_MAX_BATCH];  // substeps of each frame of the batch
  int FN[SIM_MAX_BATCH + 1];  // substeps of the frames before each frame
  int warp[NWARP + 1];
  short cblk[OCHUNK];    // segments of the chunk with per-pixel counts
  int ncblk;
  int last;
  long long prefix;
};

// Substep counts of the batch's frames into o.N and their exclusive prefix
// into o.FN (FN[count] = all substeps of the batch); returns the number of
// chunks of the batch's live segments (those of substeps k < N of their
// frame).  All threads; contains barriers.
__device__ __forceinline__ int order_fill_n(const SimParams& p, const BatchArg& b, OrderSmem& o) {
  for (int i = threadIdx.x; i < b.count; i += NT)
    o.N[i] = p.n_fixed > 0 ? p.n_fixed : adaptive_n(p.maxf2[i], p.n_max);
  __syncthreads();
  int carry = 0;
  for (int base = 0; base < b.count; base += NT) {
    const int i = base + threadIdx.x;
    int tot;
    const int ex = block_excl_scan(i < b.count ? o.N[i] : 0, o.warp, &tot);
    if (i < b.count) o.FN[i] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) o.FN[b.count] = carry;
  __syncthreads();
  const long long live = (long long)carry * p.segs_per_k;
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
  const long long nlive = (long long)o.FN[b.count] * S;
  if ((long long)c * OCHUNK >= nlive) return;
  // OSEG segments per thread: loaded interleaved (segment u * NT + tid, so a
  // warp's loads are contiguous) into the chunk's arrays, then scanned with
  // each thread owning OSEG consecutive segments
  if (tid == 0) o.ncblk = 0;
#pragma unroll
  for (int u = 0; u < OSEG; ++u) {
    const int ls = u * NT + tid;  // segment of the chunk
    const long long si = (long long)c * OCHUNK + ls;
    int cnt = 0, src = -1;
    unsigned long long mask = 0, pol = 0;
    unsigned tk = 0, xy = 0;
    if (si < nlive) {
      const long long q = si / S;  // frame-substep of the batch
      const int rs = (int)(si - q * S);
      int fi = 0, hi = b.count;
      while (hi - fi > 1) {
        const int mid = (fi + hi) >> 1;
        if (o.FN[mid] <= q) fi = mid; else hi = mid;
      }
      const int k = (int)(q - o.FN[fi]);
      const int N = o.N[fi];
      const Seg sg = p.seg[((long long)fi * p.n_max + k) * S + rs];
      cnt = sg.cnt;
      src = sg.src;
      mask = sg.mask;
      pol = sg.pol;
      const int y = rs / p.tiles_x, tc = rs - y * p.tiles_x;
      xy = (unsigned)(tc * TW) | ((unsigned)y << 16);
      const long long tp = fi == 0 ? t_first : b.frames[fi - 1].t_rel;
      const long long dt = b.frames[fi].t_rel - tp;
      tk = (unsigned)(tp + ((long long)(k + 1) * dt) / N);
    }
    o.ex[ls] = cnt;
    o.src[ls] = src;
    o.mask[ls] = mask;
    o.pol[ls] = pol;
    o.t[ls] = tk;
    o.xy[ls] = xy;
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
    const long long ex0 = lookback_warp(p.order_status, c, b.serial, total, &ctl->err);
    if (tid == 0) o.prefix = ex0;
  }
  __syncthreads();
  const long long base = cursor + o.prefix;
  for (int jj = tid; jj < total; jj += NT) {
    int lo = 0, hi = OCHUNK;
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
      const unsigned wd = ((const unsigned*)(p.staging + (-2LL - o.src[sidx])))[lane];
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
        }
      }
      ctl->active = 0;
      ctl->active_n = 0;
      ctl->stage_top = 0;
      ctl->order_done = 0;
      ctl->batch_fail = 0;
    }
    for (int i = tid; i < b.count; i += NT) p.maxf2[i] = 0;
  }
  __syncthreads();
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
template <bool RESET, bool MAPS, bool WIDE, bool SPARSE>
__global__ void __launch_bounds__(NTD, 2) k_tile_multi(GroupArg g, const ActiveTile* act,
                                                       int cls) {
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
    tile_frames<RESET, MAPS, WIDE, SPARSE, true>(sp, sb, r - fi * T, fi, fi + 1);
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
void set_tile_attr(int n_max) {
  cudaFuncSetAttribute(k_tile<RESET, MAPS, WIDE, SPARSE, 16>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)batch_smem_bytes(n_max, 3, SPARSE, 16));
  cudaFuncSetAttribute(k_tile<RESET, MAPS, WIDE, SPARSE, 8>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)batch_smem_bytes(n_max, 3, SPARSE, 8));
}

template <bool RESET, bool MAPS, bool WIDE, bool SPARSE>
void set_tile_multi_attr(size_t bytes) {
  cudaFuncSetAttribute(k_tile_multi<RESET, MAPS, WIDE, SPARSE>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <bool SPARSE>
cudaError_t launch_tile_multi_mode(const GroupArg& g, int cls, const ActiveTile* act, int grid,
                                   size_t sm, cudaStream_t st) {
  const bool reset = cls & TILE_RESET, maps = cls & TILE_MAPS, wide = cls & TILE_WIDE;
#define EVSIM_TILE(R, M, Wd) k_tile_multi<R, M, Wd, SPARSE><<<grid, NTD, sm, st>>>(g, act, cls)
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

template <bool SPARSE, int TH_>
cudaError_t launch_tile_shape(const SimParams& p, const BatchArg& b, cudaStream_t st) {
  const int grid = p.tiles_x * p.tiles_y;
  const size_t sm = batch_smem_bytes(p.n_max, p.ch, SPARSE, TH_);
  const bool reset = p.ref_mode == SIM_REF_RESET;
  const bool maps = p.cpmap != nullptr;
  const bool wide = p.intensity == SIM_LINEAR;
#define EVSIM_TILE(R, M, Wd) k_tile<R, M, Wd, SPARSE, TH_><<<grid, 32 * TH_, sm, st>>>(p, b)
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

template <bool SPARSE>
cudaError_t launch_tile_mode(const SimParams& p, const BatchArg& b, cudaStream_t st) {
  if (p.tile_h == 8) return launch_tile_shape<SPARSE, 8>(p, b, st);
  return launch_tile_shape<SPARSE, 16>(p, b, st);
}

}  // namespace

size_t tile_smem_bytes(int n_max) {
  return (size_t)(2 * SH * SW + 256 + TP + 2 * n_max) * 4 + (size_t)(n_max * TP + 3 * TP) * 2;
}

int device_sm_count() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  return n;
}

cudaError_t configure_kernels(int n_max) {
  const int t = n_max;
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

cudaError_t launch_accumulate(const Ev* ev, long long n, int W, int H, long long t_begin,
                              long long t_end, int* frame, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int grid = (int)std::min<long long>((n + NT - 1) / NT, (long long)device_sm_count() * 8);
  k_accumulate<<<std::max(grid, 1), NT, 0, st>>>(ev, n, W, H, t_begin, t_end, frame);
  return cudaGetLastError();
}

cudaError_t launch_plan(const SimParams& p, cudaStream_t st) {
  const int T = p.tiles_x * p.tiles_y;
  if (T > PLAN_MAX_TILES || !p.tile_cost || !p.tile_order) return cudaSuccess;
  k_plan<<<1, 1024, 0, st>>>(T, p.sms, p.tile_cost, p.tile_order);
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
  k_order<<<grid, NT, 0, st>>>(p, b);
  return cudaGetLastError();
}

int tile_class(const SimParams& p) {
  return (p.ref_mode == SIM_REF_RESET ? TILE_RESET : 0) | (p.cpmap ? TILE_MAPS : 0) |
         (p.intensity == SIM_LINEAR ? TILE_WIDE : 0) | (p.mode == SIM_SPARSE ? TILE_SPARSE : 0);
}

cudaError_t configure_group_kernels(size_t t) {
  set_tile_multi_attr<false, false, false, false>(t);
  set_tile_multi_attr<false, true, false, false>(t);
  set_tile_multi_attr<false, false, true, false>(t);
  set_tile_multi_attr<false, true, true, false>(t);
  set_tile_multi_attr<true, false, false, false>(t);
  set_tile_multi_attr<true, true, false, false>(t);
  set_tile_multi_attr<true, false, true, false>(t);
  set_tile_multi_attr<true, true, true, false>(t);
  set_tile_multi_attr<false, false, false, true>(t);
  set_tile_multi_attr<false, true, false, true>(t);
  set_tile_multi_attr<false, false, true, true>(t);
  set_tile_multi_attr<false, true, true, true>(t);
  set_tile_multi_attr<true, false, false, true>(t);
  set_tile_multi_attr<true, true, false, true>(t);
  set_tile_multi_attr<true, false, true, true>(t);
  set_tile_multi_attr<true, true, true, true>(t);
  return cudaGetLastError();
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

}  // namespace evsim
