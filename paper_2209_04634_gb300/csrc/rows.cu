// Row kernel of the frame-interpolation simulators (Sec. III-A dense,
// Sec. III-B sparse): the batch kernel for streams whose work is uneven over
// the image.
//
// The work unit is one 64-pixel row segment (image row y, columns
// 64 c .. 64 c + 63), carried through every frame of the batch by one warp:
// lane l owns columns 64 c + l and 64 c + l + 32, their reference and
// thresholds stay in its registers for the whole batch, and no warp ever
// waits for another (no block barrier after the prologue).  Warps take units
// from a ticket counter in the stream's control block, so a busy region of
// the image spreads over every SM instead of over the few blocks that hold
// its tiles.  Bilinear taps read the frames' bytes directly (through L1; the
// log table is in shared memory), the flow is read only at the pixels that
// are simulated.
//
// Per (unit, frame):
//   1. each lane tests its two pixels: sparse (Sec. III-B) - active when the
//      log intensity changed by at least C_act from frame i-1 to frame i;
//      dense - every pixel of the image.  An active pixel with zero flow
//      whose two end values, L_{i-1}(x) and L_i(x), both lie strictly inside
//      the band (R - C_neg, R + C_pos) (reset mode: whose change is within
//      both thresholds) is quiet: with zero flow the N interpolated values
//      lie between the end values (every blend of the Q12 arithmetic stays
//      between its two operands), so none can cross a threshold and R does
//      not move.  Quiet pixels skip the substeps exactly.
//   2. a unit-frame with no pixel left to simulate writes one flag byte
//      (empty) instead of its N segments; the order kernel reads no segment
//      of it;
//   3. otherwise the N substeps run as in the dense tile kernel (one
//      segment per substep, published by ballot; multi-crossing rows staged)
//      and the flag byte says that the unit-frame's segments are written.
#include "tile.cuh"

namespace evsim {

namespace {

constexpr int RT = 256;  // threads per block of the row kernel (8 warps)
constexpr int RWARPS = RT / 32;

// One frame's substep tables, held by the lanes of a warp: N and its
// division multiplier (every lane), the Q12 weight and the time of substeps
// k = lane + 1 (w0, t0) and k = lane + 33 (w1, t1, N > 32 only), and, for
// N <= 32, the carry table entry of remainder r = lane (bit 31 - (k - 1) set
// where floor(r k / N) steps by one at substep k).
struct RowTab {
  int N;
  unsigned mN;
  int w0, w1;
  unsigned t0, t1;
  unsigned cm;
};

__device__ __forceinline__ int substep_count(const SimParams& p, unsigned long long maxf2) {
  return p.n_fixed > 0 ? p.n_fixed : adaptive_n(maxf2, p.n_max);
}

__device__ __forceinline__ RowTab row_tables(int N, long long tprev, long long tcur) {
  const int lane = threadIdx.x & 31;
  RowTab T;
  T.N = N;
  T.mN = N > 1 ? (unsigned)(0x100000000ull / (unsigned)N) + 1u : 0u;
  const long long dt = tcur - tprev;
  int k = lane + 1;
  T.w0 = (k * 8192 + N) / (2 * N);
  T.t0 = (unsigned)(tprev + ((long long)k * dt) / N);
  T.w1 = 0;
  T.t1 = 0;
  if (N > 32) {
    k = lane + 33;
    T.w1 = (k * 8192 + N) / (2 * N);
    T.t1 = (unsigned)(tprev + ((long long)k * dt) / N);
  }
  unsigned m = 0;
  if (N <= 32 && lane < N) {
    int acc = 0;  // (lane j) mod N, stepping j = 1 .. N
    for (int j = 1; j <= N; ++j) {
      acc += lane;
      if (acc >= N) {
        acc -= N;
        m |= 1u << (32 - j);
      }
    }
  }
  T.cm = m;
  return T;
}

// The substeps of this lane's two pixels (columns x0 + lane, x0 + lane + 32
// of row y), sampling the frames in global memory (clamp-to-edge bilinear
// taps through the shared log table).  Pixels with sim[j] false take no
// samples and emit nothing; their reference is left as it is.  Every
// substep's row segment is published from the loop.  MASKS (N <= 32): the
// offsets' carries come from the carry table, as in dense_substeps.
template <bool RESET, bool WIDE, bool MASKS>
__device__ __forceinline__ void row_substeps(const SimParams& p, const int* slut,
                                             const FrameRef& prv, const FrameRef& cur,
                                             const RowTab& T, int x0, int y, Seg* segr,
                                             WarpStage* ws, const bool (&sim)[2],
                                             const int (&Fx)[2], const int (&Fy)[2], int (&R)[2],
                                             const int (&Cp)[2], const int (&Cn)[2]) {
  const int lane = threadIdx.x & 31;
  const int N = T.N;
  int px[2], py[2], qx[2], qy[2];
  unsigned ax[2], ay[2], rx[2], ry[2];
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    px[j] = (x0 + lane + 32 * j) << 16;
    py[j] = y << 16;
    int r_x, r_y;
    divmod_n(Fx[j], N, T.mN, qx[j], r_x);
    divmod_n(Fy[j], N, T.mN, qy[j], r_y);
    if (MASKS) {
      // all lanes take part in the shuffles (r < N <= 32)
      ax[j] = __shfl_sync(FULL, T.cm, r_x);
      ay[j] = __shfl_sync(FULL, T.cm, r_y);
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
    const int w = k < 32 ? __shfl_sync(FULL, T.w0, k) : __shfl_sync(FULL, T.w1, k - 32);
    const unsigned tk = k < 32 ? __shfl_sync(FULL, T.t0, k) : __shfl_sync(FULL, T.t1, k - 32);
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
      n[j] = 0;
      D[j] = 0;
      if (sim[j]) {
        const int s0 = tap_global<WIDE>(prv.ptr, prv.pitch, prv.ch, p.W, p.H, slut, px[j], py[j]);
        const int s1 = tap_global<WIDE>(cur.ptr, cur.pitch, cur.ch, p.W, p.H, slut,
                                        px[j] + Fx[j], py[j] + Fy[j]);
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
          multi |= d2 >= Cp[j] || d2 <= -Cn[j];
          D[j] = d;
        }
      }
    }
    if (!RESET && __any_sync(FULL, multi)) {
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        if (sim[j] && D[j] >= 2 * Cp[j]) {
          const int m = floordiv_pos<WIDE>(D[j], Cp[j]);
          R[j] += (m - 1) * Cp[j];
          n[j] = m;
        } else if (sim[j] && D[j] <= -2 * Cn[j]) {
          const int m = floordiv_pos<WIDE>(-D[j], Cn[j]);
          R[j] -= (m - 1) * Cn[j];
          n[j] = -m;
        }
      }
    }
    publish_row_dense(p, segr + (long long)k * p.segs_per_k, n[0], n[1], tk, x0, y, ws);
  }
}

template <bool RESET, bool MAPS, bool WIDE, bool SPARSE>
__global__ void __launch_bounds__(RT, 4) k_rows(SimParams p, BatchArg b) {
  __shared__ int slut[256];
  __shared__ WarpStage s_stage[RWARPS];
  Ctl* ctl = p.ctl;
  if (block_error(&ctl->err)) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int i = tid; i < 256; i += RT) slut[i] = p.lut[i];
  if (lane == 0) s_stage[warp] = WarpStage{0, 0, p.stage_chunk};
  __syncthreads();

  const int W = p.W, H = p.H, count = b.count;
  const int sel = ctl->sel;
  const int* Rin = (sel & 1) ? p.R1 : p.R0;
  int* Rout = (sel & 1) ? p.R0 : p.R1;
  const unsigned char* ringp = (sel & 2) ? p.ring1 : p.ring0;
  unsigned char* ringn = (sel & 2) ? p.ring0 : p.ring1;
  const long long t_first = ctl->t_prev;
  const long long S = p.segs_per_k;
  const int units = H * p.tiles_x;
  WarpStage* ws = &s_stage[warp];

  int clamps = 0;
  long long act_sum = 0, act_n = 0;
  for (;;) {
    int u = 0;
    if (lane == 0) u = (int)atomicAdd(&ctl->unit_ticket, 1u);
    u = __shfl_sync(FULL, u, 0);
    if (u >= units) break;
    const int y = u / p.tiles_x, tc = u - y * p.tiles_x;
    const int x0 = tc * TW;
    bool inimg[2];
    int R[2], Cp[2], Cn[2];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int x = x0 + lane + 32 * j;
      inimg[j] = x < W;
      R[j] = 0;
      Cp[j] = p.cp;
      Cn[j] = p.cn;
      if (inimg[j]) {
        const long long i = (long long)y * W + x;
        if (!RESET) R[j] = Rin[i];
        if (MAPS) { Cp[j] = p.cpmap[i]; Cn[j] = p.cnmap[i]; }
      }
    }
    const int cact[2] = {activity_threshold(p, Cp[0], Cn[0]), activity_threshold(p, Cp[1], Cn[1])};
    long long tprev = t_first;
    for (int fi = 0; fi < count; ++fi) {
      const FrameDesc cd = b.frames[fi];
      FrameRef prv;
      if (fi == 0) {
        prv = FrameRef{ringp, (long long)W, 1};
      } else {
        const FrameDesc d = b.frames[fi - 1];
        prv = FrameRef{d.frame, d.pitch, p.ch};
      }
      const FrameRef cur{cd.frame, cd.pitch, p.ch};
      const int N = substep_count(p, p.n_fixed > 0 ? 0ull : p.maxf2[fi]);
      // 1. the pixels to simulate
      bool act[2], sim[2];
      int Fx[2] = {0, 0}, Fy[2] = {0, 0};
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        act[j] = false;
        sim[j] = false;
        if (!inimg[j]) continue;
        const int x = x0 + lane + 32 * j;
        const int vc = load_luma(cur.ptr, cur.pitch, cur.ch, y, x);
        const int vp = load_luma(prv.ptr, prv.pitch, prv.ch, y, x);
        if (fi == count - 1 && in_bounds(ctl, (long long)y * W + x, (long long)W * H))
          ringn[(long long)y * W + x] = (unsigned char)vc;
        const int Lc = slut[vc], Lp = slut[vp];
        act[j] = !SPARSE || abs(Lc - Lp) >= cact[j];
        if (RESET) R[j] = Lp;
        if (!act[j]) continue;
        const float2 fl = cd.flow[(long long)y * W + x];
        Fx[j] = flow_q16(fl.x, clamps);
        Fy[j] = flow_q16(fl.y, clamps);
        bool quiet = (Fx[j] | Fy[j]) == 0;
        if (RESET) quiet = quiet && Lc - Lp <= Cp[j] && Lp - Lc <= Cn[j];
        else quiet = quiet && max(Lp, Lc) - R[j] < Cp[j] && R[j] - min(Lp, Lc) < Cn[j];
        sim[j] = !quiet;
      }
      if (SPARSE) {
        const int na = __popc(__ballot_sync(FULL, act[0])) + __popc(__ballot_sync(FULL, act[1]));
        act_sum += na;
        act_n += (long long)na * N;
      }
      Seg* segr = p.seg + (long long)fi * p.n_max * S + u;
      const bool any = __any_sync(FULL, sim[0] || sim[1]);
      if (lane == 0 && in_bounds(ctl, (long long)fi * S + u, p.seg_cap / p.n_max))
        p.segflag[(long long)fi * S + u] = any ? 1 : 0;
      if (any) {
        // 2. substeps; the unit-frame's segments are written
        const RowTab T = row_tables(N, tprev, cd.t_rel);
        if (N <= 32)
          row_substeps<RESET, WIDE, true>(p, slut, prv, cur, T, x0, y, segr, ws, sim, Fx, Fy, R,
                                          Cp, Cn);
        else
          row_substeps<RESET, WIDE, false>(p, slut, prv, cur, T, x0, y, segr, ws, sim, Fx, Fy, R,
                                           Cp, Cn);
      }
      tprev = cd.t_rel;
    }
    if (!RESET) {
#pragma unroll
      for (int j = 0; j < 2; ++j)
        if (inimg[j] && in_bounds(ctl, (long long)y * W + x0 + lane + 32 * j, (long long)W * H))
          Rout[(long long)y * W + x0 + lane + 32 * j] = R[j];
    }
  }
  clamps = __reduce_add_sync(FULL, clamps);
  if (lane == 0 && clamps) atomicAdd(&ctl->clamped, (unsigned long long)clamps);
  if (SPARSE && lane == 0 && act_sum) {
    atomicAdd((unsigned long long*)&ctl->active, (unsigned long long)act_sum);
    atomicAdd((unsigned long long*)&ctl->active_n, (unsigned long long)act_n);
  }
}

template <bool RESET, bool MAPS, bool WIDE, bool SPARSE>
void launch_rows_inst(const SimParams& p, const BatchArg& b, int grid, cudaStream_t st) {
  k_rows<RESET, MAPS, WIDE, SPARSE><<<grid, RT, 0, st>>>(p, b);
}

template <bool SPARSE>
cudaError_t launch_rows_mode(const SimParams& p, const BatchArg& b, cudaStream_t st) {
  const long long units = (long long)p.H * p.tiles_x;
  const int sms = p.sms > 0 ? p.sms : 1;
  const int grid = (int)std::max(1LL, std::min<long long>((long long)sms * 4,
                                                          (units + RWARPS - 1) / RWARPS));
  const bool reset = p.ref_mode == SIM_REF_RESET;
  const bool maps = p.cpmap != nullptr;
  const bool wide = p.intensity == SIM_LINEAR;
  if (!reset && !maps && !wide) launch_rows_inst<false, false, false, SPARSE>(p, b, grid, st);
  else if (!reset && maps && !wide) launch_rows_inst<false, true, false, SPARSE>(p, b, grid, st);
  else if (!reset && !maps && wide) launch_rows_inst<false, false, true, SPARSE>(p, b, grid, st);
  else if (!reset && maps && wide) launch_rows_inst<false, true, true, SPARSE>(p, b, grid, st);
  else if (reset && !maps && !wide) launch_rows_inst<true, false, false, SPARSE>(p, b, grid, st);
  else if (reset && maps && !wide) launch_rows_inst<true, true, false, SPARSE>(p, b, grid, st);
  else if (reset && !maps && wide) launch_rows_inst<true, false, true, SPARSE>(p, b, grid, st);
  else launch_rows_inst<true, true, true, SPARSE>(p, b, grid, st);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_rows(const SimParams& p, const BatchArg& b, cudaStream_t st) {
  if (!p.segflag) return cudaErrorInvalidValue;
  return p.mode == SIM_SPARSE ? launch_rows_mode<true>(p, b, st)
                              : launch_rows_mode<false>(p, b, st);
}

}  // namespace evsim
