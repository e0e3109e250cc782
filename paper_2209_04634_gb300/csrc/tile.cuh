// Device code of the tile simulation (Sec. III-A dense, Sec. III-B sparse):
// the shared helpers of every kernel (bilinear taps, threshold step, scans,
// segment publishing, staging) and the batch-persistent tile kernel k_tile
// with its launch templates.  The translation units tile_dense.cu,
// tile_sparse.cu, tile_xtime_dense.cu and tile_xtime_sparse.cu instantiate
// k_tile for their mode, so the instances compile in parallel; kernels.cu
// holds the other kernels.
#pragma once
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

// Debug builds: whether index i lies in [0, n); a violation is recorded once
// as SIM_ERR_BOUNDS in the stream's error word and the caller skips the
// access.  Release builds: true, no code.
__device__ __forceinline__ bool in_bounds(Ctl* ctl, long long i, long long n) {
  if (!kBoundsCheck) return true;
  if (i >= 0 && i < n) return true;
  if (ctl) atomicCAS(&ctl->err, 0, SIM_ERR_BOUNDS);
  return false;
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
                                   long long agg, int* err, int limit = SPIN_LIMIT) {
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
    if (++spins > limit) {
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

template <int TH_ = TH>
__device__ __forceinline__ TileLayout tile_layout(unsigned char* raw, int nmax) {
  constexpr int TP = TW * TH_, SH = TH_ + 2 * HMAX;
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
template <int TH_ = TH>
__device__ __forceinline__ void fill_halo(int* dst, const int* slut, const FrameRef& f, int W,
                                          int H, int tx0, int ty0, int hx, int hy,
                                          Ctl* ctl = nullptr) {
  constexpr int TH = TH_, NTD = 32 * TH_, SH = TH_ + 2 * HMAX;
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
      if (at[q] >= 0 && in_bounds(ctl, at[q], SH * SW)) dst[at[q]] = slut[v[q]];
  }
}

// A segment write, checked in debug builds.
__device__ __forceinline__ void put_seg(const SimParams& p, Seg* sg, const Seg& v) {
  if (in_bounds(p.ctl, sg - p.seg, p.seg_cap)) *sg = v;
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
    for (int m = 0; m < a_lo; ++m) if (in_bounds(p.ctl, base + i_lo - a_lo + m, p.stage_cap)) p.staging[base + i_lo - a_lo + m] = e_lo;
    for (int m = 0; m < a_hi; ++m) if (in_bounds(p.ctl, base + t_lo + i_hi - a_hi + m, p.stage_cap)) p.staging[base + t_lo + i_hi - a_hi + m] = e_hi;
  }
  if (lane == 0) put_seg(p, sg, Seg{0ull, 0ull, base >= 0 ? total : 0, base >= 0 ? (int)base : -1});
}

// Publish the segment of one (substep, tile row) of a dense tile: lane l
// holds the event counts of columns l (n0) and l + 32 (n1).  All 32 lanes
// must call this.
__device__ __forceinline__ void publish_row_dense(const SimParams& p, Seg* sg, int n0, int n1,
                                                  unsigned tk, int tx0, int y, WarpStage* ws) {
  const int lane = threadIdx.x & 31;
  const unsigned e0 = __ballot_sync(FULL, n0 != 0), e1 = __ballot_sync(FULL, n1 != 0);
  if ((e0 | e1) == 0) {
    if (lane == 0) put_seg(p, sg, Seg{0ull, 0ull, 0, -1});
    return;
  }
  const unsigned multi = __ballot_sync(FULL, (unsigned)(n0 + 1) > 2u || (unsigned)(n1 + 1) > 2u);
  if (multi == 0) {
    const unsigned p0 = __ballot_sync(FULL, n0 > 0), p1 = __ballot_sync(FULL, n1 > 0);
    if (lane == 0)
      put_seg(p, sg, Seg{(unsigned long long)e0 | ((unsigned long long)e1 << 32),
                (unsigned long long)p0 | ((unsigned long long)p1 << 32), __popc(e0) + __popc(e1),
                -1});
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
  if (base >= 0 && in_bounds(p.ctl, base + 15, p.stage_cap))
    ((unsigned*)(p.staging + base))[lane] = (unsigned)a0 | ((unsigned)a1 << 16);
  if (lane == 0)
    put_seg(p, sg, base >= 0 ? Seg{(unsigned long long)e0 | ((unsigned long long)e1 << 32),
                          (unsigned long long)p0 | ((unsigned long long)p1 << 32), total,
                          -2 - (int)base}
                    : Seg{0ull, 0ull, 0, -1});
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
    if (lane == 0) put_seg(p, sg, Seg{0ull, 0ull, 0, -1});
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
      put_seg(p, sg, Seg{(unsigned long long)low | ((unsigned long long)high << 32),
                (unsigned long long)plow | ((unsigned long long)phigh << 32),
                __popc(low) + __popc(high), -1});
    return;
  }
  stage_row(p, ws, sg, a_lo, a_hi, make_event(tk, tx0 + col_lo, y, n_lo > 0),
            make_event(tk, tx0 + col_hi, y, n_hi > 0));
}

// Per-crossing event time (SIM_TIME_CROSSING).  Between two consecutive
// substeps a pixel's value is taken to move linearly in time, from ip (the
// previous substep's value; substep 0 is frame i-1 itself) at t0 to i at
// t0 + dt.  The m-th level the substep crosses, rb + m c rising or rb - m c
// falling (rb the reference before the substep), is reached at
// t0 + floor(dt (level - ip) / (i - ip)); a level at or behind ip (a sparse
// pixel whose reference stayed behind while it was inactive) gives t0.
struct Crossing {
  int ip, i, rb, c;
};

__device__ __forceinline__ unsigned crossing_time(unsigned t0, unsigned dt, const Crossing& x,
                                                  bool rising, int m) {
  const int num = rising ? x.rb + m * x.c - x.ip : x.ip - (x.rb - m * x.c);
  const int den = rising ? x.i - x.ip : x.ip - x.i;
  if (num <= 0 || den <= 0) return t0;
  // num <= den (the levels crossed lie at or before i) and den < 2^24 (the
  // range of the intensity tables), so both are exact floats and dt num < 2^56
  const unsigned long long want = (unsigned long long)dt * (unsigned)num;
  unsigned q;
  if (dt <= (1u << 20)) {
    // single-precision estimate of dt num / den: relative error below 2^-21,
    // so within 0.32 of the exact quotient and its truncation within one of
    // the floor; one exact integer comparison each way corrects it
    q = (unsigned)(__fdividef((float)num, (float)den) * (float)dt);
    const unsigned long long got = (unsigned long long)q * (unsigned)den;
    if (got > want) --q;
    else if (got + (unsigned)den <= want) ++q;
  } else {
    q = (unsigned)(want / (unsigned)den);
  }
  return t0 + q;
}

// Publish the segment of one (substep, tile row) with per-crossing times:
// every row with an event stages its events (column order, a pixel's
// crossings adjacent in crossing order), each with its own time; lanes hold
// the counts n_lo (column col_lo) and n_hi (col_hi) as in publish_row, t0 /
// t1 are the times of the previous and this substep.  All 32 lanes must call
// this.
__device__ __forceinline__ void publish_row_xt(const SimParams& p, Seg* sg, int n_lo, int col_lo,
                                               int n_hi, int col_hi, unsigned t0, unsigned t1,
                                               int tx0, int y, WarpStage* ws,
                                               const Crossing& x_lo, const Crossing& x_hi) {
  const int lane = threadIdx.x & 31;
  const int a_lo = abs(n_lo), a_hi = abs(n_hi);
  if (!__any_sync(FULL, (a_lo | a_hi) != 0)) {
    if (lane == 0) put_seg(p, sg, Seg{0ull, 0ull, 0, -1});
    return;
  }
  const int i_lo = warp_incl_scan(a_lo);
  const int t_lo = __shfl_sync(FULL, i_lo, 31);
  const int i_hi = warp_incl_scan(a_hi);
  const int total = t_lo + __shfl_sync(FULL, i_hi, 31);
  long long base = 0;
  if (lane == 0) base = stage_take(p, *ws, total);
  base = __shfl_sync(FULL, base, 0);
  if (base >= 0) {
    const unsigned dt = t1 - t0;
    for (int m = 0; m < a_lo; ++m)
      if (in_bounds(p.ctl, base + i_lo - a_lo + m, p.stage_cap)) p.staging[base + i_lo - a_lo + m] =
          make_event(crossing_time(t0, dt, x_lo, n_lo > 0, m + 1), tx0 + col_lo, y, n_lo > 0);
    for (int m = 0; m < a_hi; ++m)
      if (in_bounds(p.ctl, base + t_lo + i_hi - a_hi + m, p.stage_cap)) p.staging[base + t_lo + i_hi - a_hi + m] =
          make_event(crossing_time(t0, dt, x_hi, n_hi > 0, m + 1), tx0 + col_hi, y, n_hi > 0);
  }
  if (lane == 0) put_seg(p, sg, Seg{0ull, 0ull, base >= 0 ? total : 0, base >= 0 ? (int)base : -1});
}

// The substeps of the (up to) two pixels of this thread.  `lx, ly` are the
// pixels' tile coordinates, `nk_at` their columns in the per-substep record.
// DENSE: the two pixels are columns lane, lane + 32 of tile row `warp`, and the
// row's segment is published from the loop.  XT (DENSE only): per-crossing
// event times, t_frame the time of frame i-1.  MK (N <= 32): the offsets'
// carries come from the frame's carry table cmask, as in dense_substeps.
template <bool RESET, bool WIDE, bool FAST, bool DENSE, int TH_ = 16, bool XT = false,
          bool MK = false>
__device__ __forceinline__ void tile_substeps(const SimParams& p, const TileLayout& L, int N,
                                              unsigned mN, int tx0, int ty0, unsigned b0, unsigned b1,
                                              const FrameRef& prv, const FrameDesc& cur,
                                              Seg* segf, const int (&lx)[2], const int (&ly)[2],
                                              const int (&nk_at)[2], const bool (&act)[2],
                                              const int (&Fx)[2], const int (&Fy)[2],
                                              int (&R)[2], const int (&Cp)[2],
                                              const int (&Cn)[2], WarpStage* ws,
                                              unsigned t_frame = 0,
                                              const unsigned* cmask = nullptr) {
  constexpr int TH = TH_, NTD = 32 * TH_, TP = TW * TH_, SH = TH_ + 2 * HMAX;
  (void)TH; (void)NTD; (void)TP; (void)SH;
  static_assert(!XT || DENSE, "per-crossing times use the dense row mapping");
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
    ax[j] = MK ? (int)cmask[rx[j]] : 0;
    ay[j] = MK ? (int)cmask[ry[j]] : 0;
  }
  // XT: the value of the previous substep; substep 0 is frame i-1 at the
  // pixel (zero offset)
  int Ip[2] = {0, 0}, Iold[2] = {0, 0};
  Crossing cx[2];
  if (XT) {
#pragma unroll
    for (int j = 0; j < 2; ++j)
      Ip[j] = FAST ? tap_shared<WIDE>(b0, px[j], py[j])
                   : tap_global<WIDE>(prv.ptr, prv.pitch, prv.ch, p.W, p.H, L.slut, px[j], py[j]);
  }
  unsigned t_last = t_frame;
  const int y = ty0 + warp;
  const bool row_in = !DENSE || y < p.H;
  for (int k = 0; k < N; ++k) {
    const int w = L.swk[k];
    int n[2];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      if (MK) {  // the carry of substep k is the table's next bit, from bit 31 down
        px[j] -= qx[j] - (ax[j] >> 31);
        ax[j] = (int)((unsigned)ax[j] << 1);
        py[j] -= qy[j] - (ay[j] >> 31);
        ay[j] = (int)((unsigned)ay[j] << 1);
      } else {
        px[j] -= qx[j];
        ax[j] += rx[j];
        if (ax[j] >= N) { ax[j] -= N; px[j] -= 1; }
        py[j] -= qy[j];
        ay[j] += ry[j];
        if (ay[j] >= N) { ay[j] -= N; py[j] -= 1; }
      }
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
      if (XT) {
        Iold[j] = Ip[j];
        Ip[j] = I;
      }
      n[j] = threshold_step<RESET>(I, R[j], Cp[j], Cn[j]);
      if (!act[j]) n[j] = 0;
      if (!DENSE) L.snk[k * TP + nk_at[j]] = (short)n[j];
    }
    if (XT) {
      if (row_in) {  // warp-uniform
        // the reference before the substep: reset mode, the previous value;
        // else the reference after it less the levels crossed
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          const int c = n[j] > 0 ? Cp[j] : Cn[j];
          const int rb = RESET ? Iold[j] : R[j] - n[j] * c;
          cx[j] = Crossing{Iold[j], Ip[j], rb, c};
        }
        publish_row_xt(p, segf + (long long)k * p.segs_per_k + warp * p.tiles_x, n[0], lx[0],
                       n[1], lx[1], t_last, L.stk[k], tx0, y, ws, cx[0], cx[1]);
      }
      t_last = L.stk[k];
    } else if (DENSE && row_in) {  // warp-uniform
      publish_row(p, segf + (long long)k * p.segs_per_k + warp * p.tiles_x, n[0], lx[0], true,
                  n[1], lx[1], true, L.stk[k], tx0, y, ws);
    }
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

// Dense loop over a row whose pixels to simulate number at most 32 (sparse
// activity masks, or pixels that are quiet: both emit nothing and keep R),
// compacted one per lane: lane j runs column col (has: j holds a pixel),
// the row's column layout (lane l: columns l and l + 32) is restored for
// publishing by taking column l's count from lane s0 and column l + 32's from
// lane s1 (-1: not simulated, count 0).  Same arithmetic as dense_substeps,
// half the pixel work of its two-pixel lanes.
template <bool RESET, bool WIDE, bool MASKS>
__device__ __forceinline__ void dense_substeps1(const SimParams& p, const int* swk,
                                                const unsigned* stk, const unsigned* cmask,
                                                int N, unsigned mN, int tx0, int y, unsigned b0,
                                                unsigned b1, Seg* segr, WarpStage* ws, bool has,
                                                int col, int Fx, int Fy, int& R, int Cp, int Cn,
                                                int s0, int s1) {
  const int warp = threadIdx.x >> 5;
  int px = (col + HMAX) << 16, py = (warp + HMAX) << 16;
  int qx, qy, r_x, r_y;
  unsigned ax, ay, rx = 0, ry = 0;
  divmod_n(Fx, N, mN, qx, r_x);
  divmod_n(Fy, N, mN, qy, r_y);
  if (MASKS) {
    ax = cmask[r_x];
    ay = cmask[r_y];
    qx = -qx;
    qy = -qy;
  } else {
    rx = (unsigned)r_x;
    ry = (unsigned)r_y;
    ax = 0;
    ay = 0;
  }
  const int l0 = s0 & 31, l1 = s1 & 31;
  for (int k = 0; k < N; ++k) {
    const int w = swk[k];
    if (MASKS) {
      px += qx + ((int)ax >> 31);
      ax <<= 1;
      py += qy + ((int)ay >> 31);
      ay <<= 1;
    } else {
      px -= qx;
      ax += rx;
      if (ax >= (unsigned)N) { ax -= N; px -= 1; }
      py -= qy;
      ay += ry;
      if (ay >= (unsigned)N) { ay -= N; py -= 1; }
    }
    const int v0 = tap_shared<WIDE>(b0, px, py);
    const int v1 = tap_shared<WIDE>(b1, px + Fx, py + Fy);
    const int I = lerp12<WIDE>(v0, v1, w);
    const int d = I - R;
    int n;
    bool multi = false;
    if (RESET) {
      if (has) R = I;
      n = d > Cp ? 1 : (d < -Cn ? -1 : 0);
    } else {
      n = d >= Cp ? 1 : (d <= -Cn ? -1 : 0);
      if (has) R += n > 0 ? Cp : (n < 0 ? -Cn : 0);
      const int d2 = I - R;
      multi = has && (d2 >= Cp || d2 <= -Cn);
    }
    if (!has) n = 0;
    if (!RESET && __any_sync(FULL, multi)) {
      if (has && d >= 2 * Cp) {
        const int m = floordiv_pos<WIDE>(d, Cp);
        R += (m - 1) * Cp;
        n = m;
      } else if (has && d <= -2 * Cn) {
        const int m = floordiv_pos<WIDE>(-d, Cn);
        R -= (m - 1) * Cn;
        n = -m;
      }
    }
    int n0 = __shfl_sync(FULL, n, l0), n1 = __shfl_sync(FULL, n, l1);
    if (s0 < 0) n0 = 0;
    if (s1 < 0) n1 = 0;
    publish_row_dense(p, segr + (long long)k * p.segs_per_k, n0, n1, stk[k], tx0, y, ws);
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
  const int limit = p.spin_limit > 0 ? p.spin_limit : SPIN_LIMIT;
  while (ld_volatile(&p.tdone[tile]) < want) {
    if (++spins > limit) {
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
template <bool RESET, bool MAPS, bool WIDE, bool SPARSE, bool ONE = false, int TH_ = TH>
__device__ __forceinline__ void tile_frames(const SimParams& p, const BatchArg& b, int tile, int f0,
                                            int f1) {
  constexpr int TH = TH_, NTD = 32 * TH_, TP = TW * TH_, SH = TH_ + 2 * HMAX;
  (void)SH;
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
  const TileLayout L = tile_layout<TH_>(smem_raw, nmax);
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
        if (fi == b.count - 1) {
          const long long ri = (long long)y * W + x;
          if (in_bounds(p.ctl, ri, (long long)p.W * p.H)) ringn[ri] = (unsigned char)vc;
        }
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
        fill_halo<TH_>(pb, L.slut, prv, W, H, tx0, ty0, hfx, hfy, ctl);
        phx = hfx;
        phy = hfy;
      }
      fill_halo<TH_>(cb, L.slut, curf, W, H, tx0, ty0, hfx, hfy, ctl);
    }
    __syncthreads();
    if (tid == 0) { s_fx = 0; s_fy = 0; }  // hx, hy are read by now

    // 3. substeps (sparse: warps without a compacted pixel skip them); dense
    // rows publish their segments from the loop
    const unsigned b0 = (unsigned)__cvta_generic_to_shared(pb);
    const unsigned b1 = (unsigned)__cvta_generic_to_shared(cb);
    if (!SPARSE || warp * 32 < A || warp * 32 + NTD < A) {  // warp-uniform
      if (fast)
        tile_substeps<RESET, WIDE, true, !SPARSE, TH_>(p, L, N, mN, tx0, ty0, b0, b1, prv, cur,
                                                       segf, lx, ly, nk_at, act, Fx, Fy, R, Cp,
                                                       Cn, &s_stage[warp]);
      else
        tile_substeps<RESET, WIDE, false, !SPARSE, TH_>(p, L, N, mN, tx0, ty0, b0, b1, prv, cur,
                                                        segf, lx, ly, nk_at, act, Fx, Fy, R, Cp,
                                                        Cn, &s_stage[warp]);
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
          for (int k = lane; k < N; k += 32) put_seg(p, &segf[(long long)k * p.segs_per_k + r * p.tiles_x], Seg{0ull, 0ull, 0, -1});
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
      const long long ri = (long long)(ty0 + own[q] / TW) * W + tx0 + (own[q] & (TW - 1));
      if (in_bounds(p.ctl, ri, (long long)W * H)) Rout[ri] = SPARSE ? L.sR[own[q]] : Rd[q];
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
// 16-byte copy of which the first src_bytes (0..16) are read, the rest of
// the destination zero-filled.
__device__ __forceinline__ void cp_async16z(unsigned dst, const void* src, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

// The batch kernel's rarely taken substep loops, out of line: the general
// loop (frames whose flow reach exceeds the shared halo; sparse tiles
// without the fast path) and the dense loop for N > 32 (no carry tables).
// Inlined, their registers would weigh on the allocation of the whole
// kernel, and the spills that follow reach the per-frame path that every
// frame runs.  The per-pixel arrays travel in one record (local memory of
// the calling thread, on these paths only); R comes back through it.
struct PixArgs {
  int lx[2], ly[2], nk[2], Fx[2], Fy[2], R[2], Cp[2], Cn[2];
  bool act[2];
};

template <bool RESET, bool WIDE, bool FAST, bool DENSE, int TH_>
__device__ __noinline__ void tile_substeps_cold(const SimParams p, const TileLayout V, int N,
                                                unsigned mN, int tx0, int ty0, unsigned b0,
                                                unsigned b1, const FrameRef prv,
                                                const FrameDesc cur, Seg* segf, PixArgs& a,
                                                WarpStage* ws) {
  tile_substeps<RESET, WIDE, FAST, DENSE, TH_>(p, V, N, mN, tx0, ty0, b0, b1, prv, cur, segf, a.lx,
                                               a.ly, a.nk, a.act, a.Fx, a.Fy, a.R, a.Cp, a.Cn, ws);
}

template <bool RESET, bool WIDE, bool FULLT>
__device__ __noinline__ void dense_substeps_cold(const SimParams p, const int* swk,
                                                 const unsigned* stk, int N, unsigned mN, int tx0,
                                                 int y, unsigned b0, unsigned b1, Seg* segr,
                                                 WarpStage* ws, PixArgs& a) {
  dense_substeps<RESET, WIDE, FULLT, false>(p, swk, stk, nullptr, N, mN, tx0, y, b0, b1, segr, ws,
                                            a.act, a.Fx, a.Fy, a.R, a.Cp, a.Cn);
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
  unsigned char* raw;   // [2][SH][SW * ch]
  short* snk;           // [nmax][TP] sparse
  short* sslot;         // [TP] sparse
  unsigned short* sCp;  // [TP] sparse maps
  unsigned short* sCn;
};

__host__ __device__ inline size_t batch_smem_bytes(int n_max, int ch, bool sparse, int th) {
  const int TP = TW * th, SH = th + 2 * HMAX;
  size_t b = (size_t)2 * TP * sizeof(float2);
  b += (size_t)(2 * SH * SW + 256 + (sparse ? TP : 0)) * 4;
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
  L.raw = (unsigned char*)(L.sR + (SPARSE ? TP : 0));  // 16-byte aligned, at a fixed offset
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
  if ((((unsigned long long)f.ptr | (unsigned long long)f.pitch) & 15) == 0) {
    // cx0 * ch and every window row's start in raw are multiples of 16
    // bytes, so each 16-byte chunk is aligned on both sides; the last chunk
    // of a row reads only the row's remaining bytes and zero-fills the rest,
    // which stays inside the window row (its stride is a multiple of 16).
    // The window's chunks are dealt to the block's threads as one flat list
    // (at most SH x 18 < 1024 chunks: one or two per thread), the chunk's row
    // e / nw taken as (e * (floor(2^16 / nw) + 1)) >> 16, exact for e < 1024
    // and nw <= 18 (the error stays below 1024 / 2^16 < 1 / nw; checked
    // exhaustively).  A loop of a warp per row cost three times the
    // instructions (6 of 32 lanes busy on 8-bit frames).
    static_assert(SH * 18 < 1024 && SW * 3 <= 18 * 16, "flat chunk list of the staging window");
    const int nw = (nb + 15) >> 4;
    const unsigned mw = 65536u / (unsigned)nw + 1u;
    const unsigned dst0 = smem_addr(raw) + (unsigned)b0 + (unsigned)(r0 * RW);
    const unsigned char* src0 = f.ptr + (long long)(ty0 - HMAX + r0) * f.pitch + (long long)cx0 * ch;
    const int tot = (r1 - r0) * nw;
    for (int e = threadIdx.x; e < tot; e += NTD) {
      const int rr = (int)(((unsigned)e * mw) >> 16), w = e - rr * nw;
      const int left = nb - 16 * w;
      const unsigned d = dst0 + (unsigned)(rr * RW + 16 * w);
      const unsigned char* sp = src0 + (long long)rr * f.pitch + 16 * w;
      if (left >= 16) cp_async16(d, sp);
      else cp_async16z(d, sp, left);
    }
  } else if ((((unsigned long long)f.ptr | (unsigned long long)f.pitch) & 3) == 0) {
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
  if (((unsigned long long)flow & 15) == 0 && (W & 1) == 0) {
    // pixel pairs (2t, 2t + 1) of a tile row: both in the image or both
    // out (x even, W even), 16-byte aligned in the flow and in sf
    static_assert(TP / 2 == NTD, "one pixel pair per thread");
    const int t = threadIdx.x;
    const int lx = (2 * t) & (TW - 1), ly = (2 * t) / TW;
    const int x = tx0 + lx, y = ty0 + ly;
    if (x < W && y < H) cp_async16(d0 + (unsigned)t * 16u, flow + (long long)y * W + x);
    return;
  }
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
                                              int hy, Ctl* ctl = nullptr) {
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
      if (in_bounds(ctl, (HMAX - hy + sr) * SW + (HMAX - hx) + sc, SH * SW)) d[sc] = slut[v];
    }
  }
}

// Substep tables of one frame into a frame parity's buffers, by warp 0:
// the substep times (lanes t < N), and - only when N differs from the N
// these buffers last held, since they depend on N alone - the substep
// weights, for N <= 32 the carry table (dense_substeps), and N with its
// division multiplier (divmod_n).  *sN is read by the whole warp before
// lane 0 rewrites it.
__device__ __forceinline__ void substep_tables(const SimParams& p, unsigned long long maxf2,
                                               long long t_prev, long long t_cur, int* swk,
                                               unsigned* stk, int* sN, unsigned* smN,
                                               unsigned* cmask) {
  const int N = p.n_fixed > 0 ? p.n_fixed : adaptive_n(maxf2, p.n_max);
  const int lane = threadIdx.x & 31;
  const bool same = *sN == N;
  __syncwarp();
  const unsigned long long dt = (unsigned long long)(t_cur - t_prev);
  for (int t = lane; t < N; t += 32) {
    const int k = t + 1;
    // k dt / N (dt > 0): a 32-bit division when the product fits
    const unsigned long long kd = (unsigned long long)k * dt;
    const unsigned long long q = kd < 0x100000000ull ? (unsigned)kd / (unsigned)N : kd / (unsigned)N;
    stk[t] = (unsigned)(t_prev + (long long)q);
    if (!same) {
      swk[t] = (k * 8192 + N) / (2 * N);
      if (N <= 32) {  // carry table of remainder r = t: (r j) mod N stepped without divisions
        unsigned m = 0;
        int acc = 0;
        for (int j = 1; j <= N; ++j) {
          acc += t;
          if (acc >= N) {
            acc -= N;
            m |= 1u << (32 - j);
          }
        }
        cmask[t] = m;
      }
    }
  }
  if (lane == 0 && !same) {
    *sN = N;
    *smN = N > 1 ? (unsigned)(0x100000000ull / (unsigned)N) + 1u : 0u;
  }
}

template <bool RESET, bool MAPS, bool WIDE, bool SPARSE, int TH_, bool XT = false>
__device__ __forceinline__ void tile_batch(const SimParams& p, const BatchArg& b, int tile) {
  constexpr int TH = TH_, NTD = 32 * TH_, TP = TW * TH_, SH = TH_ + 2 * HMAX;
  (void)TH; (void)NTD; (void)TP; (void)SH;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_warp[NTD / 32 + 1];
  __shared__ int s_fx[2], s_fy[2];  // the tile's flow reach, per frame parity
  __shared__ int s_rs[TH + 1];
  __shared__ int s_N[2];
  __shared__ unsigned s_stk[2][MAXN];  // substep times and weights of the frame parities
  __shared__ int s_swk[2][MAXN];
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
  // a sparse stream with segment flags runs in this dense instance: its
  // pixels' activity masks the dense row loop, rows without a pixel to
  // simulate are skipped (no compaction, the reference stays in registers)
  const bool spm = !SPARSE && p.mode == SIM_SPARSE;

  if (tid < 256) L.slut[tid] = p.lut[tid];
  // the state buffers' double-buffer selector; the pointers are formed where
  // they are used (kept live across the frame loop they cost registers)
  const int sel = ctl->sel;
  const int* Rin = (sel & 1) ? p.R1 : p.R0;
  const unsigned char* ringp = (sel & 2) ? p.ring1 : p.ring0;
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
  if (tid < 2) { s_fx[tid] = 0; s_fy[tid] = 0; s_N[tid] = 0; }
  __syncthreads();
  {
    const FrameRef ring{ringp, (long long)W, 1};
    const FrameDesc d0 = s_desc[0];
    stage_raw<TH_>(L.raw, ring, W, H, tx0, ty0);
    stage_raw<TH_>(L.raw + SH * RW, FrameRef{d0.frame, d0.pitch, ch}, W, H, tx0, ty0);
    stage_flow<TH_>(L.sflow, d0.flow, W, H, tx0, ty0);
    cp_async_commit();
    if (warp == 0)
      substep_tables(p, s_mf[0], t_first, d0.t_rel, s_swk[0], s_stk[0], &s_N[0], &s_mN[0], s_cmask[0]);
    cp_async_wait_all();
  }
  __syncthreads();

  int clamps = 0;
  unsigned act_sum = 0, act_n = 0;  // < 2^26: at most 1024 pixels x 64 substeps x 1024 frames
  int rb = 1;  // raw buffer of the current frame; 1 - rb holds the previous frame
  int hsel = 0;  // halo of the current frame: sLb (0) or sLa (1); the other holds frame i-1
  int phx = -1, phy = -1;
  int hfx = 1, hfy = 1;  // halo extents only grow within a batch

  for (int fi = 0; fi < count; ++fi) {
    const int par = fi & 1;
    const FrameDesc cur = s_desc[fi & 3];
    FrameRef prv;
    if (fi == 0) {
      prv = FrameRef{(sel & 2) ? p.ring1 : p.ring0, (long long)W, 1};
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
    auto stage_next = [&]() {
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
        if (warp == 0)
          substep_tables(p, s_mf[(fi + 1) & 3], cur.t_rel, nd.t_rel, s_swk[par ^ 1], s_stk[par ^ 1],
                         &s_N[par ^ 1], &s_mN[par ^ 1], s_cmask[par ^ 1]);
      }
    };

    // 0. quiet frame (dense mapping, segment flags on): when every simulated
    // pixel of the tile has an exactly zero flow and both end values strictly
    // inside its threshold band (reset mode: a change within both
    // thresholds), the frame emits nothing and leaves every reference as it
    // was; the tile flags its rows empty, stages the next frame and moves
    // on.  A sufficient test: flows that round to zero in Q16 without being
    // zero take the full path below, which applies the exact test.
    // Dense mapping: each owned pixel's log end values and staged flow, read
    // once per frame for the quiet tests, the activity test and the flow
    // conversion below.
    int Lpo[2] = {0, 0}, Lco[2] = {0, 0};
    float2 flo[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    if (!SPARSE) {
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        if (!inimg[q]) continue;
        const int qx = lane + 32 * q + HMAX, qy = warp + HMAX;
        Lpo[q] = L.slut[raw_luma(rawp, chp, qy, qx)];
        Lco[q] = L.slut[raw_luma(rawc, ch, qy, qx)];
        flo[q] = L.sflow[par * TP + own[q]];
      }
    }
    if (!SPARSE && !XT && p.segflag) {
      bool calm = true;
      bool av[2];
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        av[q] = false;
        if (!inimg[q]) continue;
        const int Lp = Lpo[q], Lc = Lco[q];
        const int cp = MAPS ? Cpd[q] : p.cp, cn = MAPS ? Cnd[q] : p.cn;
        av[q] = !spm || abs(Lc - Lp) >= activity_threshold(p, cp, cn);
        if (!av[q]) continue;  // sparse: an inactive pixel keeps R and emits nothing
        const bool still = ((__float_as_uint(flo[q].x) | __float_as_uint(flo[q].y)) << 1) == 0u;
        const bool band = RESET ? (Lc - Lp <= cp && Lp - Lc <= cn)
                                : (max(Lp, Lc) - Rd[q] < cp && Rd[q] - min(Lp, Lc) < cn);
        calm = calm && still && band;
      }
      if (!__syncthreads_or(calm ? 0 : 1)) {
        if (fi == count - 1) {  // the last frame's luma into the ring
          unsigned char* ringn = (sel & 2) ? p.ring0 : p.ring1;
#pragma unroll
          for (int q = 0; q < 2; ++q) {
            if (!inimg[q]) continue;
            const long long ri = (long long)(ty0 + warp) * W + tx0 + lane + 32 * q;
            if (in_bounds(p.ctl, ri, (long long)p.W * p.H))
              ringn[ri] = (unsigned char)raw_luma(rawc, ch, warp + HMAX, lane + 32 * q + HMAX);
          }
        }
        if (spm) {
          const int na = __popc(__ballot_sync(FULL, av[0])) + __popc(__ballot_sync(FULL, av[1]));
          act_sum += na;
          act_n += na * N;
        }
        if (tid == 0) { s_fx[par ^ 1] = 0; s_fy[par ^ 1] = 0; }
        stage_next();
        if (ty0 + warp < H && lane == 0)
          if (in_bounds(p.ctl, (long long)fi * p.segs_per_k + (long long)(ty0 + warp) * p.tiles_x + tcx, p.seg_cap / p.n_max))
            p.segflag[(long long)fi * p.segs_per_k + (long long)(ty0 + warp) * p.tiles_x + tcx] = 0;
        phx = -1;
        phy = -1;
        rb = 1 - rb;
        cp_async_wait_all();
        __syncthreads();
        continue;
      }
    }

    // 1. the pixels to simulate (the previous and current bytes are staged);
    // spm: a sparse stream run by this dense instance - each pixel's
    // activity is tested in the dense mapping and masks its substeps
    int A = 0;
    int sel_flag[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int lx = own[q] & (TW - 1), ly = own[q] / TW;
      bool a = inimg[q];
      if (inimg[q] && (SPARSE || spm || fi == count - 1)) {
        if (fi == count - 1) {
          const long long ri = (long long)(ty0 + ly) * W + tx0 + lx;
          unsigned char* ringn = (sel & 2) ? p.ring0 : p.ring1;
          if (in_bounds(p.ctl, ri, (long long)p.W * p.H))
            ringn[ri] = (unsigned char)raw_luma(rawc, ch, ly + HMAX, lx + HMAX);
        }
        if (SPARSE || spm) {
          const int cp = MAPS ? (SPARSE ? (int)L.sCp[own[q]] : Cpd[q]) : p.cp;
          const int cn = MAPS ? (SPARSE ? (int)L.sCn[own[q]] : Cnd[q]) : p.cn;
          const int dl = SPARSE ? L.slut[raw_luma(rawc, ch, ly + HMAX, lx + HMAX)] -
                                      L.slut[raw_luma(rawp, chp, ly + HMAX, lx + HMAX)]
                                : Lco[q] - Lpo[q];
          a = abs(dl) >= activity_threshold(p, cp, cn);
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
    if (SPARSE) {
      act_sum += A;
      act_n += A * N;
    } else if (spm) {  // per warp; lane 0 adds the warp's count at the end
      const int na = __popc(__ballot_sync(FULL, sel_flag[0] != 0)) +
                     __popc(__ballot_sync(FULL, sel_flag[1] != 0));
      act_sum += na;
      act_n += na * N;
    }
    // sparse tiles with at least 3/8 of their pixels active run the frame
    // through the dense loop (inactive pixels masked, their reference kept):
    // cheaper per pixel than compaction, per-slot records and mask atomics
    // (per-crossing times: always, their rows are published by the dense loop)
    const bool dsw = SPARSE && (XT || 8 * A >= 3 * TP);

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
        act[q] = sel_flag[q] != 0;  // dense: in the image; spm: active
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
        const float2 fl = SPARSE ? sfl[slot] : flo[q];
        Fx[q] = flow_q16(fl.x, clamps);
        Fy[q] = flow_q16(fl.y, clamps);
        if (SPARSE) {
          if (MAPS) { Cp[q] = L.sCp[slot]; Cn[q] = L.sCn[slot]; }
          if (!RESET) R[q] = L.sR[slot];
        }
        if (RESET) R[q] = SPARSE ? L.slut[raw_luma(rawp, chp, ly[q] + HMAX, lx[q] + HMAX)] : Lpo[q];
        mfx = max(mfx, (unsigned)abs(Fx[q]));
        mfy = max(mfy, (unsigned)abs(Fy[q]));
      }
    }
    // substep times, segment flags on (dense, and sparse in the dense row
    // mapping): a simulated pixel is quiet when its flow is zero and both end
    // values lie strictly inside its threshold band
    // (reset mode: its change is within both thresholds).  With zero flow the
    // interpolated values lie between the end values (every Q12 blend stays
    // between its operands), so a quiet pixel emits nothing and keeps R; a
    // row of quiet pixels skips its substeps and writes a flag instead of its
    // segments, and a tile without a busy row builds no halo.
    bool quiet = false;
    bool qp[2] = {false, false};  // per pixel (dense mapping): nothing to simulate
    if (!XT && p.segflag) {  // sparse: inactive pixels count as quiet
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        qp[q] = true;
        if (!act[q]) continue;
        if ((Fx[q] | Fy[q]) != 0) {
          qp[q] = false;
          continue;
        }
        const int Lp = SPARSE ? L.slut[raw_luma(rawp, chp, ly[q] + HMAX, lx[q] + HMAX)] : Lpo[q];
        const int Lc = SPARSE ? L.slut[raw_luma(rawc, ch, ly[q] + HMAX, lx[q] + HMAX)] : Lco[q];
        if (RESET) qp[q] = Lc - Lp <= Cp[q] && Lp - Lc <= Cn[q];
        else qp[q] = max(Lp, Lc) - R[q] < Cp[q] && R[q] - min(Lp, Lc) < Cn[q];
      }
      quiet = qp[0] && qp[1];
    }
    mfx = __reduce_max_sync(FULL, mfx);
    mfy = __reduce_max_sync(FULL, mfy);
    if (lane == 0) {
      atomicMax(&s_fx[par], (int)mfx);
      atomicMax(&s_fy[par], (int)mfy);
    }
    const bool busy = __syncthreads_or(quiet ? 0 : 1) != 0;
    const int hx = (s_fx[par] >> 16) + 1, hy = (s_fy[par] >> 16) + 1;
    // the other parity's maxima (read during the previous frame, before its
    // closing barrier) start the next frame from zero
    if (tid == 0) { s_fx[par ^ 1] = 0; s_fy[par ^ 1] = 0; }
    const bool fast = hx <= HMAX && hy <= HMAX;
    // sparse fast path: row masks in the current flow buffer (its flows are
    // in registers by now), cleared here
    const bool maskpub = SPARSE && !dsw && fast && N <= 32;
    unsigned* rowm = (unsigned*)(L.sflow + par * TP);
    if (maskpub) {
      for (int i = tid; i < N * TH * 4; i += NTD) rowm[i] = 0u;
      if (tid < N) s_multi[tid] = 0u;
    }
    if (fast && A > 0 && busy) {
      hfx = max(hfx, hx);
      hfy = max(hfy, hy);
      if (phx < hx || phy < hy) {  // the kept halo of frame i-1 does not reach far enough
        fill_halo_raw<TH_>(hsel ? L.sLb : L.sLa, L.slut, rawp, chp, W, H, tx0, ty0, hfx, hfy, ctl);
        phx = hfx;
        phy = hfy;
      }
      fill_halo_raw<TH_>(hsel ? L.sLa : L.sLb, L.slut, rawc, ch, W, H, tx0, ty0, hfx, hfy, ctl);
    }
    // the halos (and, sparse, the cleared row masks) are complete before any
    // substep reads them; a dense tile that built no halo needs no barrier
    if (SPARSE || (fast && busy)) __syncthreads();

    // 3. the next frame's inputs: its bytes over the previous frame's raw
    // buffer (read by now), its flow, the descriptor two frames ahead; its
    // substep tables
    stage_next();

    // 4. substeps (sparse: warps without a compacted pixel skip them); dense
    // rows publish their segments from the loop
    TileLayout V;
    V.slut = L.slut;
    V.stk = s_stk[par];
    V.swk = s_swk[par];
    V.snk = L.snk;
    const unsigned b0 = smem_addr(hsel ? L.sLb : L.sLa);
    const unsigned b1 = smem_addr(hsel ? L.sLa : L.sLb);
    if (XT) {
      const unsigned t_frame = (unsigned)(fi == 0 ? t_first : s_desc[(fi - 1) & 3].t_rel);
      if (SPARSE && A == 0) {  // warp-uniform: nothing simulated, empty segments
        if (ty0 + warp < H)
          for (int k = lane; k < N; k += 32)
            put_seg(p, &segf[(long long)k * p.segs_per_k + warp * p.tiles_x], Seg{0ull, 0ull, 0, -1});
      } else {
#define EVSIM_XT(FA, MK)                                                                      \
  tile_substeps<RESET, WIDE, FA, true, TH_, true, MK>(p, V, N, mN, tx0, ty0, b0, b1, prv, cur, \
                                                      segf, lx, ly, nk_at, act, Fx, Fy, R, Cp, \
                                                      Cn, &s_stage[warp], t_frame, s_cmask[par])
        if (fast) {
          if (N <= 32) EVSIM_XT(true, true);
          else EVSIM_XT(true, false);
        } else {
          if (N <= 32) EVSIM_XT(false, true);
          else EVSIM_XT(false, false);
        }
#undef EVSIM_XT
      }
    } else if (SPARSE && dsw && !(fast && N <= 32)) {
      if (p.segflag && ty0 + warp < H && lane == 0)  // every row simulated
        if (in_bounds(p.ctl, (long long)fi * p.segs_per_k + (long long)(ty0 + warp) * p.tiles_x + tcx, p.seg_cap / p.n_max))
          p.segflag[(long long)fi * p.segs_per_k + (long long)(ty0 + warp) * p.tiles_x + tcx] = 1;
      if (fast)
        tile_substeps<RESET, WIDE, true, true, TH_>(p, V, N, mN, tx0, ty0, b0, b1, prv, cur, segf,
                                                    lx, ly, nk_at, act, Fx, Fy, R, Cp, Cn,
                                                    &s_stage[warp]);
      else
        tile_substeps<RESET, WIDE, false, true, TH_>(p, V, N, mN, tx0, ty0, b0, b1, prv, cur,
                                                     segf, lx, ly, nk_at, act, Fx, Fy, R, Cp, Cn,
                                                     &s_stage[warp]);
    } else if ((!SPARSE || dsw) && fast) {
      const bool skip = p.segflag && __all_sync(FULL, quiet);
      if (p.segflag && ty0 + warp < H && lane == 0)
        if (in_bounds(p.ctl, (long long)fi * p.segs_per_k + (long long)(ty0 + warp) * p.tiles_x + tcx, p.seg_cap / p.n_max))
          p.segflag[(long long)fi * p.segs_per_k + (long long)(ty0 + warp) * p.tiles_x + tcx] =
            skip ? 0 : 1;
      if (ty0 + warp < H && !skip) {  // warp-uniform: rows below the image publish nothing
        // the row's 64 pixels are in the image (and, sparse, all active)
        const bool fullt =
            !SPARSE && tx0 + TW <= W && (!spm || __all_sync(FULL, act[0] && act[1]));
        // the row's pixels to simulate: active and not quiet
        const bool sim0 = act[0] && !qp[0], sim1 = act[1] && !qp[1];
        const unsigned m0 = __ballot_sync(FULL, sim0), m1 = __ballot_sync(FULL, sim1);
        const int c0 = __popc(m0), nsim = c0 + __popc(m1);
#define EVSIM_DENSE(FT)                                                                        \
  dense_substeps<RESET, WIDE, FT, true>(p, V.swk, V.stk, s_cmask[par], N, mN, tx0, ty0 + warp, b0, \
                                        b1, segf + warp * p.tiles_x, &s_stage[warp], act, Fx, Fy,  \
                                        R, Cp, Cn)
        if (!SPARSE && N <= 32 && nsim <= 32) {  // warp-uniform: one pixel per lane
          const unsigned lt = lanemask_lt();
          const int s0 = sim0 ? __popc(m0 & lt) : -1, s1 = sim1 ? c0 + __popc(m1 & lt) : -1;
          const bool has = lane < nsim;
          const int col = !has ? 0
                          : lane < c0 ? (int)__fns(m0, 0, lane + 1)
                                      : 32 + (int)__fns(m1, 0, lane - c0 + 1);
          const int src = col & 31;
          const bool hi = col >= 32;
          auto take = [&](const int (&v)[2]) {
            const int a0 = __shfl_sync(FULL, v[0], src), a1 = __shfl_sync(FULL, v[1], src);
            return has ? (hi ? a1 : a0) : 0;
          };
          int Rj = take(R);
          dense_substeps1<RESET, WIDE, true>(p, V.swk, V.stk, s_cmask[par], N, mN, tx0, ty0 + warp,
                                             b0, b1, segf + warp * p.tiles_x, &s_stage[warp], has,
                                             col, take(Fx), take(Fy), Rj,
                                             MAPS ? take(Cp) : p.cp, MAPS ? take(Cn) : p.cn, s0, s1);
          const int r0 = __shfl_sync(FULL, Rj, s0 & 31), r1 = __shfl_sync(FULL, Rj, s1 & 31);
          if (s0 >= 0) R[0] = r0;
          if (s1 >= 0) R[1] = r1;
        } else if (N <= 32) {
          if (fullt) EVSIM_DENSE(true);
          else EVSIM_DENSE(false);
        } else {
          PixArgs a{{lx[0], lx[1]}, {ly[0], ly[1]}, {nk_at[0], nk_at[1]}, {Fx[0], Fx[1]},
                    {Fy[0], Fy[1]}, {R[0], R[1]}, {Cp[0], Cp[1]}, {Cn[0], Cn[1]}, {act[0], act[1]}};
          if (fullt)
            dense_substeps_cold<RESET, WIDE, true>(p, V.swk, V.stk, N, mN, tx0, ty0 + warp, b0, b1,
                                                   segf + warp * p.tiles_x, &s_stage[warp], a);
          else
            dense_substeps_cold<RESET, WIDE, false>(p, V.swk, V.stk, N, mN, tx0, ty0 + warp, b0, b1,
                                                    segf + warp * p.tiles_x, &s_stage[warp], a);
          R[0] = a.R[0];
          R[1] = a.R[1];
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
      if (!SPARSE && p.segflag && ty0 + warp < H && lane == 0)  // every row simulated
        if (in_bounds(p.ctl, (long long)fi * p.segs_per_k + (long long)(ty0 + warp) * p.tiles_x + tcx, p.seg_cap / p.n_max))
          p.segflag[(long long)fi * p.segs_per_k + (long long)(ty0 + warp) * p.tiles_x + tcx] = 1;
      PixArgs a{{lx[0], lx[1]}, {ly[0], ly[1]}, {nk_at[0], nk_at[1]}, {Fx[0], Fx[1]},
                {Fy[0], Fy[1]}, {R[0], R[1]}, {Cp[0], Cp[1]}, {Cn[0], Cn[1]}, {act[0], act[1]}};
      if (fast)
        tile_substeps_cold<RESET, WIDE, true, !SPARSE, TH_>(p, V, N, mN, tx0, ty0, b0, b1, prv, cur,
                                                            segf, a, &s_stage[warp]);
      else
        tile_substeps_cold<RESET, WIDE, false, !SPARSE, TH_>(p, V, N, mN, tx0, ty0, b0, b1, prv, cur,
                                                             segf, a, &s_stage[warp]);
      R[0] = a.R[0];
      R[1] = a.R[1];
    }
    if (!RESET) {
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        if (SPARSE) {
          if (act[q]) L.sR[lx[q] + ly[q] * TW] = R[q];
        } else if (act[q]) {  // spm: inactive pixels keep their reference
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
        put_seg(p, &segf[(long long)k * p.segs_per_k + r * p.tiles_x],
                cnt ? Seg{(unsigned long long)m[0] | ((unsigned long long)m[1] << 32),
                          (unsigned long long)m[2] | ((unsigned long long)m[3] << 32), cnt, -1}
                    : Seg{0ull, 0ull, 0, -1});
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
          for (int k = lane; k < N; k += 32) put_seg(p, &segf[(long long)k * p.segs_per_k + r * p.tiles_x], Seg{0ull, 0ull, 0, -1});
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
    if (fast && A > 0 && busy) {
      hsel ^= 1;
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
    int* Rout = (sel & 1) ? p.R0 : p.R1;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      if (!inimg[q]) continue;
      const long long ri = (long long)(ty0 + own[q] / TW) * W + tx0 + (own[q] & (TW - 1));
      if (in_bounds(p.ctl, ri, (long long)W * H)) Rout[ri] = SPARSE ? L.sR[own[q]] : Rd[q];
    }
  }
  clamps = __reduce_add_sync(FULL, clamps);
  if (lane == 0 && clamps) atomicAdd(&ctl->clamped, (unsigned long long)clamps);
  if (spm && lane == 0 && act_sum) {
    atomicAdd((unsigned long long*)&ctl->active, (unsigned long long)act_sum);
    atomicAdd((unsigned long long*)&ctl->active_n, (unsigned long long)act_n);
  }
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

template <bool RESET, bool MAPS, bool WIDE, bool SPARSE, int TH_, bool XT = false>
__global__ void __launch_bounds__(32 * TH_, 32 / TH_) k_tile(SimParams p, BatchArg b) {
  const int bi = blockIdx.x;
  const int tile = p.block_order == 2 ? p.tile_order[bi]
                   : p.block_order == 1 ? serpentine_tile(bi, gridDim.x, p.sms)
                                        : bi;
  tile_batch<RESET, MAPS, WIDE, SPARSE, TH_, XT>(p, b, tile);
}

// Dynamic shared-memory permission of one k_tile instance in both shapes;
// returns the first failing call's error.
template <bool RESET, bool MAPS, bool WIDE, bool SPARSE, bool XT = false>
cudaError_t set_tile_attr(int n_max) {
  cudaError_t e = cudaFuncSetAttribute(k_tile<RESET, MAPS, WIDE, SPARSE, 16, XT>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)batch_smem_bytes(n_max, 3, SPARSE, 16));
  if (e == cudaSuccess && !XT)  // per-crossing times run in 64 x 16 tiles only
    e = cudaFuncSetAttribute(k_tile<RESET, MAPS, WIDE, SPARSE, 8>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)batch_smem_bytes(n_max, 3, SPARSE, 8));
  return e;
}

// The eight (reset, maps, wide) instances of one mode.
template <bool SPARSE, bool XT = false>
cudaError_t set_mode_attrs(int n_max) {
  const cudaError_t es[8] = {
      set_tile_attr<false, false, false, SPARSE, XT>(n_max),
      set_tile_attr<false, true, false, SPARSE, XT>(n_max),
      set_tile_attr<false, false, true, SPARSE, XT>(n_max),
      set_tile_attr<false, true, true, SPARSE, XT>(n_max),
      set_tile_attr<true, false, false, SPARSE, XT>(n_max),
      set_tile_attr<true, true, false, SPARSE, XT>(n_max),
      set_tile_attr<true, false, true, SPARSE, XT>(n_max),
      set_tile_attr<true, true, true, SPARSE, XT>(n_max)};
  for (cudaError_t e : es)
    if (e != cudaSuccess) return e;
  return cudaSuccess;
}

template <bool SPARSE, int TH_, bool XT = false>
cudaError_t launch_tile_shape(const SimParams& p, const BatchArg& b, cudaStream_t st) {
  const int grid = p.tiles_x * p.tiles_y;
  const size_t sm = batch_smem_bytes(p.n_max, p.ch, SPARSE, TH_);
  const bool reset = p.ref_mode == SIM_REF_RESET;
  const bool maps = p.cpmap != nullptr;
  const bool wide = p.intensity == SIM_LINEAR;
#define EVSIM_TILE(R, M, Wd) k_tile<R, M, Wd, SPARSE, TH_, XT><<<grid, 32 * TH_, sm, st>>>(p, b)
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

}  // namespace evsim
