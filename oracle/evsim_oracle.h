/*
 * Plain CPU oracle for the flow-interpolation event simulator.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library
 * and its Python binding) may include, link, load or call this code; only
 * the tests, the smoke check and the CPU-baseline leg of the benchmark do.
 * It shares no code, header, table or constant generator with the CUDA path.
 *
 * What it computes (paper: Ziegler et al., "Real-time event simulation with
 * frame-based cameras", arXiv 2209.04634):
 *   - Sec. III: frames are differenced and thresholded after Kaiser et al.;
 *     optical flow plus linear interpolation raises the temporal rate.
 *   - Sec. III-A (dense frame interpolation): N frames are interpolated along
 *     the flow between frames i-1 and i, consecutive results are differenced
 *     and thresholded with C_pos / C_neg (the two-case equations of III-A),
 *     and events <x, y, t, p> are emitted.
 *   - Sec. III-B (sparse frame interpolation): only pixels whose change from
 *     frame i-1 to frame i reaches a threshold are interpolated.
 *   - Sec. III-C (difference frame interpolation): difference frames of three
 *     consecutive frames are interpolated along the flow between them and
 *     each interpolated difference frame is thresholded (orc_run_diff).
 * The fixed-point readings (Q16 log LUT, Q12 weights, clamp-to-edge bilinear
 * sampling, reference-accumulating threshold test) are stated beside each
 * function in evsim_oracle.c.
 *
 * All arithmetic is integer (int64 intermediates); loops run substep-major in
 * raster order, exactly in the order the events are defined to appear.
 */
#ifndef EVSIM_ORACLE_H
#define EVSIM_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_DENSE = 0, ORC_SPARSE = 1 };
enum { ORC_LOG = 0, ORC_LINEAR = 1 };
enum { ORC_ACCUM = 0, ORC_RESET = 1 };
enum { ORC_T_SUBSTEP = 0, ORC_T_CROSSING = 1 };

typedef struct {
  int32_t width, height;
  int32_t channels;      /* 1: 8-bit luma; 3: 8-bit RGB, interleaved (BT.601 luma) */
  int32_t mode;          /* ORC_DENSE | ORC_SPARSE */
  int32_t substeps;      /* > 0: fixed N; 0: adaptive N from the flow */
  int32_t max_substeps;  /* cap on adaptive N */
  int32_t intensity;     /* ORC_LOG | ORC_LINEAR */
  int32_t ref_mode;      /* ORC_ACCUM | ORC_RESET */
  int32_t c_pos_q16;     /* uniform C_pos (Q16) when no per-pixel map is given */
  int32_t c_neg_q16;     /* uniform |C_neg| (Q16) */
  int32_t c_act_q16;     /* sparse activity threshold (Q16); < 0: min(Cp(x), Cn(x)) */
  int32_t event_time;    /* ORC_T_SUBSTEP: every crossing of substep k at t_k;
                            ORC_T_CROSSING: each crossing at its own time between
                            t_{k-1} and t_k (see orc_crossing_time) */
  int32_t row_begin;     /* orc_run simulates rows [row_begin, row_end) only (the other */
  int32_t row_end;       /* rows' events are not produced, their R is not meaningful);
                            row_end <= 0: through the last row.  Frames, flows and the
                            adaptive N are still read / computed over the whole image,
                            so the events of consecutive row bands, merged per
                            (frame, substep) in band order, are those of one run. */
} orc_config;

typedef struct {
  uint32_t t;   /* microseconds since the first frame */
  uint16_t x;
  uint16_t yp;  /* (y << 1) | (polarity > 0) */
} orc_event;

/* Log / linear intensity table (256 entries, Q16). */
void orc_lut(int32_t intensity, int32_t lut[256]);
/* BT.601 integer luma of one RGB triple. */
int32_t orc_luma(int32_t r, int32_t g, int32_t b);
/* float flow component -> Q16 (NaN -> 0, clamped to +-1024 px); *clamped += 1 on a clamp. */
int32_t orc_flow_q16(float f, int32_t* clamped);
/* Clamp-to-edge bilinear sample of a Q16 image at a Q16 position. */
int32_t orc_bilinear(const int32_t* L, int32_t W, int32_t H, int64_t px, int64_t py);
/* Time of one threshold crossing inside substep k (ORC_T_CROSSING): the
 * pixel's value is taken to move linearly in time from i_prev (substep k-1,
 * at t_prev) to i_cur (substep k, at t_cur); the crossing happens where it
 * reaches `level`.  rising: the level is above i_prev (positive event).
 * Levels at or behind i_prev give t_prev. */
int64_t orc_crossing_time(int64_t t_prev, int64_t t_cur, int64_t i_prev, int64_t i_cur,
                          int64_t level, int32_t rising);
/* Adaptive substep count for a maximum squared Q16 flow magnitude. */
int32_t orc_adaptive_substeps(int64_t max_f2, int32_t max_substeps);

/*
 * Run one stream over n_frames frames.
 *   frames     : n_frames x H x W x channels bytes, contiguous.
 *   flows      : n_frames x H x W x 2 floats (dx, dy in px, frame i-1 -> i,
 *                stored at index i); flows for frame 0 are ignored.
 *   t_us       : n_frames timestamps, strictly increasing.
 *   cpos_map, cneg_map : optional W*H Q16 thresholds (NULL: uniform).
 *   out        : receives up to cap events in output order.
 *   R_final    : optional W*H int32, the reference state after the last frame
 *                (ACCUM mode) or the last frame's log image (RESET mode).
 *   n_per_frame: optional n_frames ints, the N used per frame (0 for frame 0).
 *   ev_per_frame: optional n_frames int64, events emitted per frame.
 * Returns the total event count (which may exceed cap; only cap are
 * written), or a negative value on a bad argument (-1), a non-increasing
 * timestamp (-2), a timestamp beyond 2^32-1 us after the first frame (-3),
 * or an allocation failure (-4).
 */
int64_t orc_run(const orc_config* cfg, int32_t n_frames, const uint8_t* frames,
                const float* flows, const int64_t* t_us,
                const uint16_t* cpos_map, const uint16_t* cneg_map,
                orc_event* out, int64_t cap, int32_t* R_final,
                int32_t* n_per_frame, int64_t* ev_per_frame,
                int64_t* active_per_frame, int64_t* clamped_total);

/*
 * Difference-frame interpolation (Sec. III-C) over n_frames frames: the same
 * arguments as orc_run (mode, ref_mode and c_act_q16 are not used; flows[i]
 * is the flow between difference frames i-1 and i).  Frames 0 and 1 emit
 * nothing.  Returns the event count or a negative error as orc_run.
 */
int64_t orc_run_diff(const orc_config* cfg, int32_t n_frames, const uint8_t* frames,
                     const float* flows, const int64_t* t_us,
                     const uint16_t* cpos_map, const uint16_t* cneg_map,
                     orc_event* out, int64_t cap, int32_t* n_per_frame,
                     int64_t* ev_per_frame, int64_t* clamped_total);

/* Accumulated event frame (Fig. 1 caption): frame[y * W + x] += +1 / -1 for
 * every positive / negative event with t_begin <= t < t_end (frame not
 * cleared first; events outside the frame skipped). */
void orc_accumulate(const orc_event* ev, int64_t n, int32_t W, int32_t H, int64_t t_begin,
                    int64_t t_end, int32_t* frame);

/* Pyramidal Lucas-Kanade optical flow (the flow the paper's sparse and
 * difference simulators use, Sec. III-B, Sec. IV-A); the reading O17 is
 * stated in evsim_oracle.c.  levels 1..8, radius 1..7 (window 2r+1 square),
 * iterations 1..16 per level, min_eig: the smallest eigenvalue of the
 * window's gradient matrix per window pixel below which a pixel keeps its
 * guess (gradients in Q4 units, twice the derivative). */
typedef struct {
  int32_t levels;
  int32_t radius;
  int32_t iterations;
  int32_t pad;
  double min_eig;
} orc_lk_config;

/* Flow from frame f0 to frame f1 (W x H, 1 or 3 channels, rows packed):
 * flow[2 (y W + x) + {0, 1}] = (dx, dy) in Q16 px.  Returns 0, -1 on bad
 * arguments, -4 when out of memory. */
int orc_flow_lk(const orc_lk_config* c, int32_t W, int32_t H, int32_t channels,
                const uint8_t* f0, const uint8_t* f1, int32_t* flow);

#ifdef __cplusplus
}
#endif
#endif
