// CUDA kernels of the evsim library (sm_103a).
//
// One pushed frame runs, on the handle's stream:
//   dense : [flowmax, adaptive N only] -> dense -> order
//   sparse: [sparse_pre, adaptive N only] -> sparse -> order
// The method (Ziegler et al., arXiv 2209.04634, Sec. III-A / III-B) and its
// integer arithmetic are described in include/evsim.h.  Every kernel checks
// the stream's sticky error word first and does nothing once it is set.
// Per-frame arguments (input pointers, timestamp, push serial) come in a
// FrameArg, so that a batch of frames can be captured once as a CUDA graph
// whose kernels read their arguments from a device-resident table.
//
// Event order.  Within a frame, events are ordered by (substep, row, column,
// repeat).  The simulating kernels work pixel-major, so they record each
// pixel's per-substep count in shared memory, write their events to a
// staging area in their own local order and publish one (count, staging
// offset) entry per "segment" (dense: one row of a 64 x 16 tile; sparse: the
// active pixels of one chunk of 1024 raster pixels).  The order kernel scans
// the segment counts in output order (a single-pass scan with decoupled
// look-back) and gathers the events into the stream's event buffer; the
// block that finishes the last chunk commits the frame.
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

__device__ __forceinline__ FrameDesc frame_of(const FrameArg& f) { return f.ptr ? *f.ptr : f.val; }

// ---------------------------------------------------------------------------
// frame 0: fill the frame ring and the reference

__global__ void k_init(SimParams p, FrameArg fa) {
  const FrameDesc f = frame_of(fa);
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
// adaptive N (dense): max over all pixels of the squared Q16 flow

__global__ void __launch_bounds__(NT) k_flowmax(SimParams p, FrameArg fa) {
  if (block_error(&p.ctl->err)) return;
  const FrameDesc f = frame_of(fa);
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
      const long long i = i0 + (long long)q * NT;
      fl[q] = i < P ? f.flow[i] : make_float2(0.f, 0.f);
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
    unsigned long long b = 0;
    for (int w = 0; w < NWARP; ++w) b = s_m[w] > b ? s_m[w] : b;
    if (b) atomicMax(&p.ctl->maxf2, b);
  }
}

// ---------------------------------------------------------------------------
// dense simulation of one 64 x 16 tile: NTD threads, warp w owns tile row w,
// lane l owns columns l and l + 32 of it.

struct DenseLayout {
  int* sL0;
  int* sL1;
  int* slut;
  int* srow;   // [N][TH] events per (substep, tile row)
  int* soff;   // [N][TH] tile-local exclusive offsets
  unsigned* stk;
  int* swk;
  short* snk;  // [N][TH][TW] signed event count per pixel-substep
};

__device__ __forceinline__ DenseLayout dense_layout(unsigned char* raw, int nmax) {
  DenseLayout L;
  L.sL0 = (int*)raw;
  L.sL1 = L.sL0 + SH * SW;
  L.slut = L.sL1 + SH * SW;
  L.srow = L.slut + 256;
  L.soff = L.srow + nmax * TH;
  L.stk = (unsigned*)(L.soff + nmax * TH);
  L.swk = (int*)(L.stk + nmax);
  L.snk = (short*)(L.swk + nmax);
  return L;
}

template <bool RESET, bool WIDE, bool FAST>
__device__ __forceinline__ void dense_substeps(const SimParams& p, const FrameDesc& f,
                                               const DenseLayout& L, int N, int tx0, int ty0,
                                               const int (&Fx)[2], const int (&Fy)[2],
                                               int (&R)[2], const int (&Cp)[2],
                                               const int (&Cn)[2], const bool (&inb)[2],
                                               const unsigned char* ringp) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int px[2], py[2], ax[2], ay[2], qx[2], rx[2], qy[2], ry[2];
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const int lx = lane + 32 * j, ly = warp;
    // FAST: positions relative to the shared tile origin (tx0 - HMAX, ty0 - HMAX);
    // otherwise absolute image positions.
    px[j] = FAST ? (lx + HMAX) << 16 : (tx0 + lx) << 16;
    py[j] = FAST ? (ly + HMAX) << 16 : (ty0 + ly) << 16;
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
  short* nkrow = L.snk + warp * TW + lane;
  const unsigned b0 = (unsigned)__cvta_generic_to_shared(L.sL0);
  const unsigned b1 = (unsigned)__cvta_generic_to_shared(L.sL1);
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
        s0 = tap_global<WIDE>(ringp, p.W, 1, p.W, p.H, L.slut, px[j], py[j]);
        s1 = tap_global<WIDE>(f.frame, f.pitch, p.ch, p.W, p.H, L.slut, px[j] + Fx[j],
                              py[j] + Fy[j]);
      }
      const int I = lerp12<WIDE>(s0, s1, w);
      n[j] = threshold_step<RESET>(I, R[j], Cp[j], Cn[j]);
      if (!inb[j]) n[j] = 0;
    }
    short* q = nkrow + k * (TH * TW);
    q[0] = (short)n[0];
    q[32] = (short)n[1];
    int c0 = abs(n[0]) + abs(n[1]);
    if (__any_sync(FULL, c0 != 0)) {
      c0 = __reduce_add_sync(FULL, c0);
      if (lane == 0) L.srow[k * TH + warp] = c0;
    }
  }
}

// Tile-local offsets of `E` segment counts (substep-major), staging allocation
// and the segment table entries.  Returns the staging base, or -1 when the
// staging area is exhausted (the frame then fails and emits nothing).
template <int NTH = NT>
__device__ __forceinline__ int stage_segments(const SimParams& p, const int* cnt, int* off, int E,
                                              int* s_warp, int* s_base, int* total_out) {
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
    int base = 0;
    if (total > 0) {
      const unsigned long long b = atomicAdd(&p.ctl->stage_top, (unsigned long long)total);
      if (b + (unsigned long long)total > (unsigned long long)p.stage_cap) {
        base = -1;
        atomicExch(&p.ctl->frame_fail, 1);
      } else {
        base = (int)b;
      }
    }
    *s_base = base;
  }
  __syncthreads();
  *total_out = total;
  return *s_base;
}

template <bool RESET, bool MAPS, bool WIDE>
__global__ void __launch_bounds__(NTD, 2) k_dense(SimParams p, FrameArg fa) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_warp[NTD / 32 + 1];
  __shared__ int s_fx, s_fy, s_clamp, s_base;
  Ctl* ctl = p.ctl;
  if (block_error(&ctl->err)) return;
  const FrameDesc f = frame_of(fa);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nmax = p.n_max;
  const DenseLayout L = dense_layout(smem_raw, nmax);
  const int tile = blockIdx.x;
  const int tcx = tile % p.tiles_x, tcy = tile / p.tiles_x;
  const int tx0 = tcx * TW, ty0 = tcy * TH;
  const int W = p.W, H = p.H;

  if (tid < 256) L.slut[tid] = p.lut[tid];
  if (tid == 0) { s_fx = 0; s_fy = 0; s_clamp = 0; }
  const int N = p.n_fixed > 0 ? p.n_fixed : adaptive_n(ctl->maxf2, nmax);
  const int sel = ctl->sel;
  const int* Rin = (sel & 1) ? p.R1 : p.R0;
  int* Rout = (sel & 1) ? p.R0 : p.R1;
  const unsigned char* ringp = (sel & 2) ? p.ring1 : p.ring0;
  unsigned char* ringn = (sel & 2) ? p.ring0 : p.ring1;
  if (tile == 0 && tid == 0) ctl->n_frame = N;
  const long long tprev = ctl->t_prev;

  const int y = ty0 + warp;
  int Fx[2], Fy[2], R[2], Cp[2], Cn[2];
  bool inb[2];
  int clamps = 0;
  unsigned mfx = 0, mfy = 0;
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const int x = tx0 + lane + 32 * j;
    inb[j] = x < W && y < H;
    Fx[j] = 0; Fy[j] = 0; R[j] = 0; Cp[j] = p.cp; Cn[j] = p.cn;
    if (inb[j]) {
      const long long i = (long long)y * W + x;
      const float2 fl = f.flow[i];
      Fx[j] = flow_q16(fl.x, clamps);
      Fy[j] = flow_q16(fl.y, clamps);
      if (!RESET) R[j] = Rin[i];
      if (MAPS) { Cp[j] = p.cpmap[i]; Cn[j] = p.cnmap[i]; }
      mfx = max(mfx, (unsigned)abs(Fx[j]));
      mfy = max(mfy, (unsigned)abs(Fy[j]));
    }
  }
  mfx = __reduce_max_sync(FULL, mfx);
  mfy = __reduce_max_sync(FULL, mfy);
  clamps = __reduce_add_sync(FULL, clamps);
  if (tid < N) {
    const int k = tid + 1;
    L.swk[tid] = (k * 8192 + N) / (2 * N);
    const long long dt = f.t_rel - tprev;
    L.stk[tid] = (unsigned)(tprev + (k * dt) / N);
  }
  for (int e = tid; e < N * TH; e += NTD) L.srow[e] = 0;
  __syncthreads();
  if (lane == 0) {
    atomicMax(&s_fx, (int)mfx);
    atomicMax(&s_fy, (int)mfy);
    if (clamps) atomicAdd(&s_clamp, clamps);
  }
  __syncthreads();
  if (tid == 0 && s_clamp) atomicAdd(&ctl->clamped, (unsigned long long)s_clamp);
  // Reach of every tap of the tile: floor(max |F|) + 1 pixels on each side.
  const int hx = (s_fx >> 16) + 1, hy = (s_fy >> 16) + 1;
  const bool fast = hx <= HMAX && hy <= HMAX;

  if (fast) {
    // Replicate-padded halo tiles of both log frames; the tile interior of the
    // new frame also goes to the frame ring for the next push.  The region is
    // walked as a flat index (row = e / ncols by a multiply-high with
    // ceil(2^32 / ncols), exact for e < 2^16), FILL loads in flight per thread.
    constexpr int FILL = 2;
    const int c0 = HMAX - hx, ncols = TW + 2 * hx;
    const int r0 = HMAX - hy, nrows = TH + 2 * hy;
    const int total_fill = ncols * nrows;
    const unsigned mcols = 0xFFFFFFFFu / (unsigned)ncols + 1u;
    for (int e0 = 0; e0 < total_fill; e0 += NTD * FILL) {
      int vp[FILL], vc[FILL], at[FILL], ring_at[FILL];
#pragma unroll
      for (int q = 0; q < FILL; ++q) {
        const int e = e0 + q * NTD + tid;
        at[q] = -1;
        ring_at[q] = -1;
        if (e < total_fill) {
          const int sr = (int)__umulhi((unsigned)e, mcols);
          const int sc = e - sr * ncols;
          const int ry = ty0 - hy + sr, rxx = tx0 - hx + sc;
          const int gy = min(max(ry, 0), H - 1), gx = min(max(rxx, 0), W - 1);
          vp[q] = ringp[(long long)gy * W + gx];
          vc[q] = load_luma(f.frame, f.pitch, p.ch, gy, gx);
          at[q] = (r0 + sr) * SW + (c0 + sc);
          if (ry == gy && rxx == gx && sr >= hy && sr < hy + TH && sc >= hx && sc < hx + TW)
            ring_at[q] = gy * W + gx;
        }
      }
#pragma unroll
      for (int q = 0; q < FILL; ++q) {
        if (at[q] < 0) continue;
        L.sL0[at[q]] = L.slut[vp[q]];
        L.sL1[at[q]] = L.slut[vc[q]];
        if (ring_at[q] >= 0) ringn[ring_at[q]] = (unsigned char)vc[q];
      }
    }
  } else {
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      if (!inb[j]) continue;
      const int x = tx0 + lane + 32 * j;
      ringn[(long long)y * W + x] = (unsigned char)load_luma(f.frame, f.pitch, p.ch, y, x);
    }
  }
  __syncthreads();
  if (RESET) {
    // Consecutive differences start from frame i-1 itself.
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      if (!inb[j]) continue;
      const int x = tx0 + lane + 32 * j;
      R[j] = L.slut[ringp[(long long)y * W + x]];
    }
  }

  if (fast)
    dense_substeps<RESET, WIDE, true>(p, f, L, N, tx0, ty0, Fx, Fy, R, Cp, Cn, inb, ringp);
  else
    dense_substeps<RESET, WIDE, false>(p, f, L, N, tx0, ty0, Fx, Fy, R, Cp, Cn, inb, ringp);

  if (!RESET) {
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      if (!inb[j]) continue;
      const int x = tx0 + lane + 32 * j;
      Rout[(long long)y * W + x] = R[j];
    }
  }
  __syncthreads();

  // Tile-local offsets of the (substep, row) segments, substep-major.
  const int E = N * TH;
  int total;
  const int base = stage_segments<NTD>(p, L.srow, L.soff, E, s_warp, &s_base, &total);
  const bool fail = base < 0;
  for (int e = tid; e < E; e += NTD) {
    const int k = e / TH, ty = e % TH, yy = ty0 + ty;
    if (yy < H)
      p.seg[((long long)k * H + yy) * p.tiles_x + tcx] =
          make_int2(fail ? 0 : L.srow[e], (fail ? 0 : base) + L.soff[e]);
  }
  if (fail || total == 0) return;

  // Emission: each warp writes the events of its row, substep by substep.
  const unsigned lt = lanemask_lt();
  for (int k = 0; k < N; ++k) {
    const int e = k * TH + warp;
    if (L.srow[e] == 0) continue;
    const unsigned tk = L.stk[k];
    const unsigned o = (unsigned)base + (unsigned)L.soff[e];
    const int na = L.snk[e * TW + lane], nb = L.snk[e * TW + lane + 32];
    const int aa = abs(na), ab = abs(nb);
    const int xa = tx0 + lane, xb = tx0 + lane + 32;
    if (__all_sync(FULL, (aa | ab) <= 1)) {
      const unsigned ba = __ballot_sync(FULL, aa != 0), bb = __ballot_sync(FULL, ab != 0);
      if (aa) p.staging[o + __popc(ba & lt)] = make_event(tk, xa, y, na > 0);
      if (ab) p.staging[o + __popc(ba) + __popc(bb & lt)] = make_event(tk, xb, y, nb > 0);
    } else {
      const int ia = warp_incl_scan(aa);
      const int ta = __shfl_sync(FULL, ia, 31);
      const int ib = warp_incl_scan(ab);
      const Ev ea = make_event(tk, xa, y, na > 0), eb = make_event(tk, xb, y, nb > 0);
      const unsigned oa = o + ia - aa, ob = o + ta + ib - ab;
      for (int m = 0; m < aa; ++m) p.staging[oa + m] = ea;
      for (int m = 0; m < ab; ++m) p.staging[ob + m] = eb;
    }
  }
}

// ---------------------------------------------------------------------------
// sparse (Sec. III-B): per chunk of SCHUNK raster pixels, find the active
// pixels (|L_i - L_{i-1}| >= C_act), compact them in raster order and
// simulate only those.  Segments are (substep, chunk).

// Activity test of one pixel; also returns the two luma values.
__device__ __forceinline__ bool pixel_active(const SimParams& p, const FrameDesc& f,
                                             const int* slut, const unsigned char* ringp,
                                             long long i, int& vc) {
  const int y = (int)(i / p.W), x = (int)(i - (long long)y * p.W);
  const int vp = ringp[i];
  vc = load_luma(f.frame, f.pitch, p.ch, y, x);
  const int d = abs(slut[vc] - slut[vp]);
  int ca = p.cact;
  if (ca < 0) {
    const int a = p.cpmap ? p.cpmap[i] : p.cp;
    const int b = p.cnmap ? p.cnmap[i] : p.cn;
    ca = min(a, b);
  }
  return d >= ca;
}

// Adaptive N for the sparse method: max squared flow over active pixels.
__global__ void __launch_bounds__(NT) k_sparse_pre(SimParams p, FrameArg fa) {
  __shared__ int slut[256];
  __shared__ unsigned long long s_m[NWARP];
  Ctl* ctl = p.ctl;
  if (block_error(&ctl->err)) return;
  const FrameDesc f = frame_of(fa);
  const int tid = threadIdx.x;
  slut[tid] = p.lut[tid];
  __syncthreads();
  const unsigned char* ringp = (ctl->sel & 2) ? p.ring1 : p.ring0;
  const long long P = (long long)p.W * p.H;
  unsigned long long m = 0;
  int dummy = 0;
  for (long long i = blockIdx.x * (long long)NT + tid; i < P; i += (long long)gridDim.x * NT) {
    int vc;
    if (pixel_active(p, f, slut, ringp, i, vc)) {
      const float2 fl = f.flow[i];
      const long long fx = flow_q16(fl.x, dummy), fy = flow_q16(fl.y, dummy);
      const unsigned long long f2 = (unsigned long long)(fx * fx + fy * fy);
      m = f2 > m ? f2 : m;
    }
  }
  m = warp_max_u64(m);
  if ((tid & 31) == 0) s_m[tid >> 5] = m;
  __syncthreads();
  if (tid == 0) {
    unsigned long long b = 0;
    for (int w = 0; w < NWARP; ++w) b = s_m[w] > b ? s_m[w] : b;
    if (b) atomicMax(&ctl->maxf2, b);
  }
}

template <bool RESET, bool MAPS, bool WIDE>
__global__ void __launch_bounds__(NT) k_sparse(SimParams p, FrameArg fa) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_warp[NWARP + 1];
  __shared__ int s_base, s_clamp, s_active;
  __shared__ int sidx[SCHUNK];
  Ctl* ctl = p.ctl;
  if (block_error(&ctl->err)) return;
  const FrameDesc f = frame_of(fa);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nmax = p.n_max;
  int* slut = (int*)smem_raw;
  int* swk = slut + 256;
  unsigned* stk = (unsigned*)(swk + nmax);
  int* scnt = (int*)(stk + nmax);            // [N][SROUNDS][NWARP] counts
  int* soff = scnt + nmax * SROUNDS * NWARP; // [N][SROUNDS][NWARP] chunk-local offsets
  int* skt = soff + nmax * SROUNDS * NWARP;  // [N] events per substep in the chunk
  short* snk = (short*)(skt + nmax);         // [N][SCHUNK]

  slut[tid] = p.lut[tid];
  if (tid == 0) { s_clamp = 0; s_active = 0; }
  const long long P = (long long)p.W * p.H;
  const int S = (int)((P + SCHUNK - 1) / SCHUNK);
  const int N = p.n_fixed > 0 ? p.n_fixed : adaptive_n(ctl->maxf2, nmax);
  if (blockIdx.x == 0 && tid == 0) ctl->n_frame = N;
  const int sel = ctl->sel;
  const unsigned char* ringp = (sel & 2) ? p.ring1 : p.ring0;
  unsigned char* ringn = (sel & 2) ? p.ring0 : p.ring1;
  const long long tprev = ctl->t_prev;
  if (tid < N) {
    const int k = tid + 1;
    swk[tid] = (k * 8192 + N) / (2 * N);
    const long long dt = f.t_rel - tprev;
    stk[tid] = (unsigned)(tprev + (k * dt) / N);
  }
  const int W = p.W, H = p.H;
  const unsigned lt = lanemask_lt();
  const int ESEG = N * SROUNDS * NWARP;
  int clamps = 0, active_total = 0;
  __syncthreads();

  for (int c = blockIdx.x; c < S; c += gridDim.x) {
    // 1. activity of the chunk's pixels, compacted in raster order
    const long long i0 = (long long)c * SCHUNK + SROUNDS * tid;
    unsigned flags = 0;
    int cnt = 0;
#pragma unroll
    for (int q = 0; q < SROUNDS; ++q) {
      const long long i = i0 + q;
      if (i < P) {
        int vc;
        if (pixel_active(p, f, slut, ringp, i, vc)) { flags |= 1u << q; ++cnt; }
        ringn[i] = (unsigned char)vc;
      }
    }
    for (int e = tid; e < ESEG; e += NT) scnt[e] = 0;
    int A;
    int o = block_excl_scan(cnt, s_warp, &A);
#pragma unroll
    for (int q = 0; q < SROUNDS; ++q)
      if (flags & (1u << q)) sidx[o++] = (int)(i0 + q);
    if (tid == 0) p.chunk_active[c] = A;
    active_total += A;
    __syncthreads();

    // 2. simulate the active pixels, NT at a time (round r: pixels r NT + tid)
    const int rounds = (A + NT - 1) / NT;
    for (int r = 0; r < rounds; ++r) {
      const int j = r * NT + tid;
      const bool act = j < A;
      const int i = act ? sidx[j] : 0;
      const int y = i / W, x = i - y * W;
      int Fx = 0, Fy = 0, R = 0, cp = p.cp, cn = p.cn;
      if (act) {
        const float2 fl = f.flow[i];
        Fx = flow_q16(fl.x, clamps);
        Fy = flow_q16(fl.y, clamps);
        if (MAPS) { cp = p.cpmap[i]; cn = p.cnmap[i]; }
        if (RESET) {
          R = slut[ringp[i]];
        } else {
          R = p.R0[i];
          p.Rsave[(long long)c * SCHUNK + j] = R;
          p.idx[(long long)c * SCHUNK + j] = i;
        }
      }
      int qx = Fx / N, rx = Fx - qx * N;
      if (rx < 0) { rx += N; qx -= 1; }
      int qy = Fy / N, ry = Fy - qy * N;
      if (ry < 0) { ry += N; qy -= 1; }
      int px = x << 16, py = y << 16, ax = 0, ay = 0;
      for (int k = 0; k < N; ++k) {
        px -= qx;
        ax += rx;
        if (ax >= N) { ax -= N; px -= 1; }
        py -= qy;
        ay += ry;
        if (ay >= N) { ay -= N; py -= 1; }
        const int s0 = tap_global<WIDE>(ringp, W, 1, W, H, slut, px, py);
        const int s1 = tap_global<WIDE>(f.frame, f.pitch, p.ch, W, H, slut, px + Fx, py + Fy);
        const int I = lerp12<WIDE>(s0, s1, swk[k]);
        int n = threshold_step<RESET>(I, R, cp, cn);
        if (!act) n = 0;
        snk[k * SCHUNK + j] = (short)n;
        if (__any_sync(FULL, n != 0)) {
          const int cw = __reduce_add_sync(FULL, abs(n));
          if (lane == 0) scnt[(k * SROUNDS + r) * NWARP + warp] = cw;
        }
      }
      if (!RESET && act) p.R0[i] = R;
    }
    __syncthreads();

    // 3. chunk-local offsets in (substep, round, warp) order, staging, segments
    int total;
    const int base = stage_segments(p, scnt, soff, ESEG, s_warp, &s_base, &total);
    const bool fail = base < 0;
    if (tid < N) {
      const int e0 = tid * SROUNDS * NWARP;
      const int kt = soff[e0 + SROUNDS * NWARP - 1] + scnt[e0 + SROUNDS * NWARP - 1] - soff[e0];
      p.seg[(long long)tid * S + c] = make_int2(fail ? 0 : kt, (fail ? 0 : base) + soff[e0]);
    }
    if (!fail && total > 0) {
      for (int k = 0; k < N; ++k) {
        for (int r = 0; r < rounds; ++r) {
          const int e = (k * SROUNDS + r) * NWARP + warp;
          if (scnt[e] == 0) continue;
          const int j = r * NT + tid;
          const int n = j < A ? snk[k * SCHUNK + j] : 0;
          const int a = abs(n);
          const int i = j < A ? sidx[j] : 0;
          const int y = i / W, x = i - y * W;
          const unsigned oo = (unsigned)base + (unsigned)soff[e];
          const Ev ev = make_event(stk[k], x, y, n > 0);
          if (__all_sync(FULL, a <= 1)) {
            const unsigned b = __ballot_sync(FULL, a != 0);
            if (a) p.staging[oo + __popc(b & lt)] = ev;
          } else {
            const int ia = warp_incl_scan(a);
            for (int m = 0; m < a; ++m) p.staging[oo + ia - a + m] = ev;
          }
        }
      }
    }
    __syncthreads();
  }
  clamps = __reduce_add_sync(FULL, clamps);
  if (lane == 0 && clamps) atomicAdd(&s_clamp, clamps);
  if (tid == 0 && active_total) atomicAdd(&s_active, active_total);
  __syncthreads();
  if (tid == 0) {
    if (s_clamp) atomicAdd(&ctl->clamped, (unsigned long long)s_clamp);
    if (s_active) atomicAdd((unsigned long long*)&ctl->active, (unsigned long long)s_active);
  }
}

// ---------------------------------------------------------------------------
// order: scan segment counts in output order, gather events, commit the frame

__global__ void __launch_bounds__(NT) k_order(SimParams p, FrameArg fa) {
  __shared__ int s_ex[OCHUNK];
  __shared__ int s_src[OCHUNK];
  __shared__ int s_warp[NWARP + 1];
  __shared__ int s_c, s_last, s_ok;
  __shared__ long long s_prefix;
  Ctl* ctl = p.ctl;
  if (block_error(&ctl->err)) return;
  const FrameDesc f = frame_of(fa);
  const int tid = threadIdx.x;
  const int N = ctl->n_frame;
  const bool sparse = p.mode == SIM_SPARSE;
  const long long P = (long long)p.W * p.H;
  const long long S = sparse ? (P + SCHUNK - 1) / SCHUNK : (long long)p.H * p.tiles_x;
  const long long nseg = (long long)N * S;
  const int nchunks = (int)max(1LL, (nseg + OCHUNK - 1) / OCHUNK);
  const long long cursor = ctl->cursor;

  for (;;) {
    if (tid == 0) s_c = (int)atomicAdd(&ctl->order_ticket, 1u);
    __syncthreads();
    const int c = s_c;
    if (c >= nchunks) break;
    const long long si = (long long)c * OCHUNK + tid;
    int cnt = 0, src = 0;
    if (si < nseg) {
      const int2 e = p.seg[si];
      cnt = e.x;
      src = e.y;
    }
    int total;
    const int ex = block_excl_scan(cnt, s_warp, &total);
    s_ex[tid] = ex;
    s_src[tid] = src;
    if (tid < 32) {
      const long long ex0 = lookback_warp(p.order_status, c, f.serial, total, &ctl->err);
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
      if (dst < p.event_cap) p.events[dst] = p.staging[s_src[lo] + (jj - s_ex[lo])];
    }
    __syncthreads();
    if (tid == 0) {
      __threadfence();
      const unsigned d = atomicAdd(&ctl->order_done, 1u);
      s_last = d == (unsigned)(nchunks - 1);
    }
    __syncthreads();
    if (s_last) {
      // This block finished the frame's last chunk: commit or fail the frame.
      if (tid == 0) {
        __threadfence();
        const unsigned long long w = ld_volatile(&p.order_status[nchunks - 1]);
        const long long tot = (long long)(w & LB_VALUE);
        const bool over = ctl->frame_fail != 0 || tot >= (long long)LB_VALUE ||
                          cursor + tot > p.event_cap;
        int ok = 0;
        if (ld_volatile(&ctl->err) == 0) {
          if (over) {
            atomicCAS(&ctl->err, 0, SIM_ERR_EVENT_OVERFLOW);
          } else {
            int flip = 2;
            if (!sparse && p.ref_mode == SIM_REF_ACCUM) flip |= 1;
            ctl->cursor = cursor + tot;
            ctl->sel ^= flip;
            ctl->t_prev = f.t_rel;
            ctl->committed += 1;
            ctl->frame_events = tot;
            ctl->work_px += P * N;
            ctl->work_active += (sparse ? ctl->active : P) * N;
            ok = 1;
          }
        }
        ctl->last_active = ctl->active;
        ctl->active = 0;
        ctl->stage_top = 0;
        ctl->order_done = 0;
        ctl->maxf2 = 0;
        ctl->frame_fail = 0;
        s_ok = ok;
      }
      __syncthreads();
      if (!s_ok && sparse && p.ref_mode == SIM_REF_ACCUM) {
        // Roll back the in-place reference of the active pixels.
        for (int c2 = 0; c2 < (int)S; ++c2) {
          const int A = p.chunk_active[c2];
          for (int j = tid; j < A; j += NT) {
            const long long slot = (long long)c2 * SCHUNK + j;
            p.R0[p.idx[slot]] = p.Rsave[slot];
          }
        }
      }
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

template <bool RESET, bool MAPS, bool WIDE>
void set_dense_attr(size_t bytes) {
  cudaFuncSetAttribute(k_dense<RESET, MAPS, WIDE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)bytes);
}

template <bool RESET, bool MAPS, bool WIDE>
void set_sparse_attr(size_t bytes) {
  cudaFuncSetAttribute(k_sparse<RESET, MAPS, WIDE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)bytes);
}

}  // namespace

size_t dense_smem_bytes(int n_max) {
  return (size_t)(2 * SH * SW + 256 + 2 * n_max * TH + 2 * n_max) * 4 +
         (size_t)n_max * TH * TW * 2;
}

size_t sparse_smem_bytes(int n_max) {
  return (size_t)(256 + 2 * n_max + 2 * n_max * SROUNDS * NWARP + n_max) * 4 +
         (size_t)n_max * SCHUNK * 2;
}

int device_sm_count() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  return n;
}

cudaError_t configure_kernels(int n_max) {
  const size_t d = dense_smem_bytes(n_max), s = sparse_smem_bytes(n_max);
  set_dense_attr<false, false, false>(d);
  set_dense_attr<false, true, false>(d);
  set_dense_attr<false, false, true>(d);
  set_dense_attr<false, true, true>(d);
  set_dense_attr<true, false, false>(d);
  set_dense_attr<true, true, false>(d);
  set_dense_attr<true, false, true>(d);
  set_dense_attr<true, true, true>(d);
  set_sparse_attr<false, false, false>(s);
  set_sparse_attr<false, true, false>(s);
  set_sparse_attr<false, false, true>(s);
  set_sparse_attr<false, true, true>(s);
  set_sparse_attr<true, false, false>(s);
  set_sparse_attr<true, true, false>(s);
  set_sparse_attr<true, false, true>(s);
  set_sparse_attr<true, true, true>(s);
  return cudaGetLastError();
}

cudaError_t launch_init(const SimParams& p, const FrameArg& f, cudaStream_t st) {
  const long long P = (long long)p.W * p.H;
  const int grid = (int)std::min<long long>((P + NT - 1) / NT, 4096);
  k_init<<<grid, NT, 0, st>>>(p, f);
  return cudaGetLastError();
}

cudaError_t launch_flowmax(const SimParams& p, const FrameArg& f, cudaStream_t st) {
  const long long P = (long long)p.W * p.H;
  const int sms = device_sm_count();
  const int grid = (int)std::max(1LL, std::min<long long>((P + NT * 8 - 1) / (NT * 8), (long long)sms * 4));
  k_flowmax<<<grid, NT, 0, st>>>(p, f);
  return cudaGetLastError();
}

cudaError_t launch_dense(const SimParams& p, const FrameArg& f, cudaStream_t st) {
  const int grid = p.tiles_x * p.tiles_y;
  const size_t sm = dense_smem_bytes(p.n_max);
  const bool reset = p.ref_mode == SIM_REF_RESET;
  const bool maps = p.cpmap != nullptr;
  const bool wide = p.intensity == SIM_LINEAR;
#define EVSIM_DENSE(R, M, Wd) k_dense<R, M, Wd><<<grid, NTD, sm, st>>>(p, f)
  if (!reset && !maps && !wide) EVSIM_DENSE(false, false, false);
  else if (!reset && maps && !wide) EVSIM_DENSE(false, true, false);
  else if (!reset && !maps && wide) EVSIM_DENSE(false, false, true);
  else if (!reset && maps && wide) EVSIM_DENSE(false, true, true);
  else if (reset && !maps && !wide) EVSIM_DENSE(true, false, false);
  else if (reset && maps && !wide) EVSIM_DENSE(true, true, false);
  else if (reset && !maps && wide) EVSIM_DENSE(true, false, true);
  else EVSIM_DENSE(true, true, true);
#undef EVSIM_DENSE
  return cudaGetLastError();
}

cudaError_t launch_sparse_pre(const SimParams& p, const FrameArg& f, cudaStream_t st, int grid) {
  k_sparse_pre<<<grid, NT, 0, st>>>(p, f);
  return cudaGetLastError();
}

cudaError_t launch_sparse(const SimParams& p, const FrameArg& f, cudaStream_t st, int grid) {
  const size_t sm = sparse_smem_bytes(p.n_max);
  const bool reset = p.ref_mode == SIM_REF_RESET;
  const bool maps = p.cpmap != nullptr;
  const bool wide = p.intensity == SIM_LINEAR;
#define EVSIM_SPARSE(R, M, Wd) k_sparse<R, M, Wd><<<grid, NT, sm, st>>>(p, f)
  if (!reset && !maps && !wide) EVSIM_SPARSE(false, false, false);
  else if (!reset && maps && !wide) EVSIM_SPARSE(false, true, false);
  else if (!reset && !maps && wide) EVSIM_SPARSE(false, false, true);
  else if (!reset && maps && wide) EVSIM_SPARSE(false, true, true);
  else if (reset && !maps && !wide) EVSIM_SPARSE(true, false, false);
  else if (reset && maps && !wide) EVSIM_SPARSE(true, true, false);
  else if (reset && !maps && wide) EVSIM_SPARSE(true, false, true);
  else EVSIM_SPARSE(true, true, true);
#undef EVSIM_SPARSE
  return cudaGetLastError();
}

cudaError_t launch_order(const SimParams& p, const FrameArg& f, cudaStream_t st, int grid) {
  k_order<<<grid, NT, 0, st>>>(p, f);
  return cudaGetLastError();
}

}  // namespace evsim
