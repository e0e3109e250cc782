/*
 * evsim: GB300-native frame-to-event simulator (C ABI).
 *
 * Implements the data-parallel core of the dense and sparse frame
 * interpolation methods of Ziegler et al., "Real-time event simulation with
 * frame-based cameras" (arXiv 2209.04634):
 *   - Sec. III:   consecutive frames are differenced and thresholded; optical
 *                 flow plus linear interpolation raises the temporal rate.
 *   - Sec. III-A: dense frame interpolation.  N frames are interpolated along
 *                 the flow between camera frames i-1 and i; each interpolated
 *                 frame is compared with a reference and thresholded with
 *                 C_pos / C_neg (the two-case equations of III-A); the output
 *                 is a stream of events <x, y, t, p> (Fig. 1 caption).
 *   - Sec. III-B: sparse frame interpolation.  Only pixels whose change from
 *                 frame i-1 to frame i reaches an activity threshold are
 *                 interpolated; the others emit nothing.
 *   - Sec. III-C: difference-frame interpolation (SIM_DIFF).  From frames
 *                 i-2, i-1, i the difference frames D_{i-1} = L_{i-1} - L_{i-2}
 *                 and D_i = L_i - L_{i-1} are formed; the pushed flow of frame
 *                 i is the flow between the two difference frames; N difference
 *                 frames are interpolated between them with the sampling and
 *                 blend below (D in place of L) and each is thresholded with
 *                 the strict two-case equations (> Cp positive, < -Cn
 *                 negative, at most one event per substep, no reference:
 *                 ref_mode is ignored).  Frames 0 and 1 of a stream emit
 *                 nothing.  SIM_DIFF streams are single handles (not group
 *                 members, not sim_step_pair_static).
 * The flow itself is an input (the paper computes it with OpenCV; it is not
 * part of this library).
 *
 * Arithmetic (all integer, bit-exact across runs and devices):
 *   - intensity: Q16 log table LUT[v] = round(65536 ln(v + 1)) (SIM_LOG), or
 *     LUT[v] = 65536 v (SIM_LINEAR, the paper's linear differences of Sec. III
 *     with thresholds in 8-bit units as in Table I);
 *   - flow: float px -> Q16 (NaN -> 0, clamped to +-1024 px, ties to even);
 *   - substep k of N: offset floor(F k / N); samples at x - offset in frame
 *     i-1 and x + F - offset in frame i (flow read at the target pixel),
 *     clamp-to-edge bilinear with 12-bit fractions, blended with the Q12
 *     weight round-half-up(4096 k / N); substep time t_{i-1} + floor(k dt / N);
 *   - SIM_REF_ACCUM: per-pixel reference R; D = I - R; D >= Cp emits floor(D/Cp)
 *     positive events and moves R by that many Cp (likewise for -D >= Cn);
 *     SIM_REF_RESET: the paper's consecutive difference, strict > Cp / < -Cn,
 *     at most one event per substep;
 *   - output order: frame, substep, row, column, repeated crossings adjacent.
 *
 * Threading and streams: one handle must not be used from two host threads
 * at once.  All device work of a handle is ordered on its CUDA stream.
 *
 * Errors: functions return SIM_OK (0), SIM_MORE (1, informational) or a
 * negative SIM_ERR_* code.  Nothing aborts or throws across this boundary.
 */
#ifndef EVSIM_H
#define EVSIM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ------------------------------------------------------- */
#define SIM_OK 0
#define SIM_MORE 1                 /* pop: more events remain */
#define SIM_ERR_ARG (-1)           /* invalid argument or configuration */
#define SIM_ERR_CUDA (-2)          /* a CUDA runtime call failed */
#define SIM_ERR_OOM (-3)           /* device or host allocation failed */
#define SIM_ERR_TIME (-4)          /* timestamp not strictly increasing */
#define SIM_ERR_TIME_RANGE (-5)    /* more than 2^32-1 us after the first frame */
#define SIM_ERR_EVENT_OVERFLOW (-6)/* a frame's events did not fit; not committed */
#define SIM_ERR_DEVICE_TIMEOUT (-7)/* a bounded device-side wait gave up */
#define SIM_ERR_STATE (-8)         /* call not valid in the handle's state */
#define SIM_ERR_ADMIT (-9)         /* batch: admission refused (memory budget / slots) */
#define SIM_ERR_NO_DEVICE (-10)    /* no usable CUDA device / kernel image */
#define SIM_ERR_TOO_LARGE (-11)    /* sim_step_pair_static: problem exceeds its scratch */
#define SIM_ERR_BOUNDS (-12)       /* debug builds only: a kernel index left its buffer */

/* ---- enumerations ------------------------------------------------------- */
enum { SIM_LUMA8 = 1, SIM_RGB8 = 3 };          /* bytes per input pixel */
enum { SIM_DENSE = 0, SIM_SPARSE = 1, SIM_DIFF = 2 };
enum { SIM_LOG = 0, SIM_LINEAR = 1 };
enum { SIM_REF_ACCUM = 0, SIM_REF_RESET = 1 };
enum { SIM_HOST = 0, SIM_DEVICE = 1 };         /* where a buffer lives */

#define SIM_MAX_DIM 8192
#define SIM_MAX_SUBSTEPS 64
#define SIM_MAX_BATCH 1024          /* frames per device batch of sim_push_frames */

typedef struct sim_s sim_t;   /* opaque, owned by the library */

/* One event, 8 bytes: t = microseconds since the stream's first frame;
 * yp = (y << 1) | (polarity > 0). */
typedef struct {
  uint32_t t_us;
  uint16_t x;
  uint16_t yp;
} sim_event;

typedef struct {
  int32_t width, height;     /* 1..SIM_MAX_DIM */
  int32_t pixel_format;      /* SIM_LUMA8 | SIM_RGB8 (BT.601 luma on device) */
  int32_t mode;              /* SIM_DENSE | SIM_SPARSE | SIM_DIFF (see below) */
  int32_t substeps;          /* > 0: fixed N; 0: N = ceil(max |flow|) per frame */
  int32_t max_substeps;      /* cap, 1..SIM_MAX_SUBSTEPS */
  int32_t intensity;         /* SIM_LOG | SIM_LINEAR */
  int32_t ref_mode;          /* SIM_REF_ACCUM | SIM_REF_RESET */
  int32_t c_pos_q16;         /* uniform C_pos, Q16 (0.2 log units = 13107) */
  int32_t c_neg_q16;         /* uniform |C_neg|, Q16 */
  int32_t c_act_q16;         /* sparse activity threshold, Q16; < 0: min(Cp(x), Cn(x)) */
  int32_t max_batch;         /* frames per device batch (<= SIM_MAX_BATCH); 0: what a
                                512 MB segment table holds */
  const uint16_t* c_pos_map; /* optional host W*H Q16 per-pixel C_pos (copied at create) */
  const uint16_t* c_neg_map; /* optional host W*H Q16 per-pixel |C_neg| */
  int64_t event_capacity;    /* device event buffer (events); 0: default max(2^20, 8 W H) */
  void* cuda_stream;         /* cudaStream_t to order work on; NULL: library-owned stream;
                                cudaStreamLegacy for the legacy default stream */
  int32_t tile_height;       /* batch kernel: SIM_TILE_AUTO, SIM_TILE_TUNE, 8 or 16 (64 x 8
                                tiles of 256 threads / 64 x 16 of 512), or SIM_TILE_ROWS (the
                                row kernel, below); see sim_autotune.  Group members always
                                use 16. */
  int32_t event_time;        /* SIM_TIME_SUBSTEP | SIM_TIME_CROSSING (see below) */
  int32_t host_inputs;       /* SIM_HOST_STAGE (default): host batches are copied into
                                device staging chunk by chunk, the copies overlapping the
                                kernels; SIM_HOST_MAPPED: host frames and flows in pinned
                                (page-locked, device-mapped) memory are read in place by the
                                kernels through their device mapping, over the host link,
                                with no staging copy (pageable ones are still staged).
                                Measured on 1280 x 720 RGB: staging is twice as fast (the
                                tile kernels read overlapping windows) */
  int32_t reserved;
} sim_config;

enum { SIM_HOST_STAGE = 0, SIM_HOST_MAPPED = 1 };

/* Event times (sim_config.event_time).  The paper's events carry a time t
 * (Sec. III) without fixing where inside an interpolation step a crossing
 * falls.
 *   SIM_TIME_SUBSTEP : every crossing of substep k gets t_k = t_{i-1} +
 *                      floor(k (t_i - t_{i-1}) / N) (the default).
 *   SIM_TIME_CROSSING: between substeps k-1 and k (substep 0 = frame i-1) a
 *                      pixel's value is taken to move linearly in time; the
 *                      j-th level crossed, R + j C_pos (rising) or
 *                      R - j C_neg (falling), R the reference before the
 *                      substep (in reset mode the value of substep k-1), is
 *                      reached at t_{k-1} + floor((t_k - t_{k-1})
 *                      (level - I_{k-1}) / (I_k - I_{k-1})); a level at or
 *                      behind I_{k-1} (a sparse pixel whose reference stayed
 *                      behind while it was inactive) gets t_{k-1}.  Events keep
 *                      their (frame, substep, row, column) order, so times are
 *                      non-decreasing from substep to substep but not inside
 *                      one.  Dense and sparse only (SIM_ERR_ARG for SIM_DIFF);
 *                      single handles only (simb_admit and
 *                      sim_step_pair_static refuse it); the batch kernel runs
 *                      in 64 x 16 tiles, every row with an event staging its
 *                      events. */
enum { SIM_TIME_SUBSTEP = 0, SIM_TIME_CROSSING = 1 };

/* Tile shape choices of sim_config.tile_height. */
enum {
  SIM_TILE_AUTO = 0,    /* the shape the autotuner table holds for this configuration, else 16 */
  SIM_TILE_TUNE = -1,   /* as SIM_TILE_AUTO, but run sim_autotune first on a table miss */
  SIM_TILE_ROWS = 1     /* the row kernel: warps take 64 x 1 row units by ticket and carry
                           each through the batch; frames are sampled in global memory,
                           unit-frames with nothing to simulate (sparse: no active pixel;
                           both modes: every pixel quiet, i.e. zero flow and both end values
                           strictly inside the threshold band) cost one flag byte.  Dense and
                           sparse substep-time streams (SIM_DIFF and SIM_TIME_CROSSING use 16) */
};

typedef struct {
  int64_t frames_pushed;     /* frames accepted by sim_push_frame */
  int64_t frames_committed;  /* frames whose events and state are committed */
  int64_t events_pending;    /* committed events not yet popped */
  int64_t events_popped;     /* events returned by sim_pop_events so far */
  int64_t last_active;       /* pixels simulated in the last committed batch (sparse:
                                active pixels summed over its frames) */
  int64_t last_batch_events; /* events of the last committed batch (a single push is a
                                batch of one frame) */
  int64_t flow_clamped;      /* flow components clamped to +-1024 px so far */
  int32_t last_substeps;     /* N of the last committed frame */
  int32_t max_batch;         /* frames per device batch */
  int64_t pixel_substeps;    /* sum over committed frames of width * height * N */
  int64_t active_substeps;   /* sum over committed frames of (pixels simulated) * N */
  int32_t tile_height;       /* the batch kernel: tile height 8 or 16, or SIM_TILE_ROWS */
  int32_t block_order;       /* its tile order: 0 linear, 1 serpentine, 2 balanced
                                (see sim_autotune) */
  int64_t active_pixels;     /* sum over committed frames of the pixels simulated (dense:
                                width * height per frame; sparse: the active pixels) */
} sim_stats;

/* Kernel kinds for sim_kernel_time. */
enum { SIM_K_INIT = 0, SIM_K_FLOWMAX = 1, SIM_K_DENSE = 2, SIM_K_MASK = 3,
       SIM_K_SPARSE = 4, SIM_K_ORDER = 5, SIM_K_COPY = 6, SIM_K_COUNT = 7 };

/* A threshold in log units (SIM_LOG) or 8-bit intensity units (SIM_LINEAR,
 * Table I's C = 2 / 10 / 20) as the Q16 integer that sim_config carries:
 * round-half-even(|c| 65536).  The sign is dropped (Table I lists C_neg as a
 * negative number; the library takes magnitudes).  Returns SIM_ERR_ARG for a
 * value that is not finite or whose Q16 form is 2^30 or more.  Thresholds
 * cross this boundary as Q16 integers so that the library and any checker
 * compare them exactly. */
int32_t sim_threshold_q16(double c);

/* Fill *cfg with defaults for a width x height luma stream: dense, N = 8,
 * log intensity, accumulate mode, C = 0.2, substep event times, autotuned
 * tile shape, library-owned stream. */
int sim_config_default(sim_config* cfg, int32_t width, int32_t height);

/* Create a simulator (the per-stream state of the methods of Sec. III-A /
 * III-B: the reference each pixel's interpolated log intensity is compared
 * with, the previous frame, the thresholds C_pos / C_neg of the two-case
 * equations of Sec. III-A).  Allocates all device state (frame ring, reference,
 * staging and event buffers) and copies the optional threshold maps.
 * Thresholds must be >= 1; in accumulate mode they must also be at least
 * (LUT[255] - LUT[0]) / 32766 (12 for SIM_LOG, 511 for SIM_LINEAR) so that one
 * substep emits at most 32767 events per pixel.  *out is set on SIM_OK only. */
int sim_create(const sim_config* cfg, sim_t** out);

/* Push camera frame i with the flow from frame i-1 to frame i: the
 * interpolation of N frames along the flow between frames i-1 and i and the
 * threshold test of each against the reference (Sec. III, Sec. III-A; Sec.
 * III-B for SIM_SPARSE).
 *   frame : height rows of pitch_bytes bytes, width * pixel_format bytes used.
 *   flow  : height * width * 2 floats (dx, dy) in px per frame interval,
 *           row-major, 8-byte aligned; ignored (may be NULL) on the first push.
 *   t_us  : timestamp; strictly increasing; < 2^32 us after the first frame.
 *   mem   : SIM_HOST or SIM_DEVICE.  Either way the buffers are read by work
 *           enqueued on the handle's stream: they must stay valid and
 *           unchanged until the stream has passed this push (sim_sync or the
 *           next sim_pop_events).
 * Asynchronous: returns once the work is enqueued.  The first push sets the
 * reference from frame 0 and emits no events.  A device-side failure (event
 * overflow) is reported by the next sim_sync / sim_pop_events; the failing
 * frame and any frame pushed after it are then not committed.  Same as
 * sim_push_frames with count = 1. */
int sim_push_frame(sim_t* s, const void* frame, int64_t pitch_bytes, const float* flow,
                   int64_t t_us, int32_t mem);

/* Push count frames in one call: frames[i], flows[i], t_us[i] (host arrays of
 * pointers; the pointers point to host or device memory per mem).  The
 * frames are simulated as device batches of up to sim_stats.max_batch frames,
 * three kernel launches per batch: each tile (or raster chunk) is carried
 * through every frame of the batch by one block.  A batch commits as a whole:
 * if its events do not fit, none of its frames commit (SIM_ERR_EVENT_OVERFLOW
 * at the next sim_sync / sim_pop_events).  Host-memory frames are copied
 * into a device staging area (two slots, grown to fit) in chunks of
 * max(4, ceil(count / 8)) frames (at most max_batch), each chunk a device
 * batch of its own: the next chunk is copied on a library-owned copy stream
 * while the previous one is simulated (pinned host memory lets the copies
 * run asynchronously; pageable memory is still correct).  Timestamps are
 * validated for the whole call before anything is enqueued.  The event
 * stream equals that of count sim_push_frame calls. */
int sim_push_frames(sim_t* s, int32_t count, const void* const* frames, int64_t pitch_bytes,
                    const float* const* flows, const int64_t* t_us, int32_t mem);

/* The output of the method: events <x, y, t, p> (Fig. 1 caption), here
 * sim_event records.  Copy up to cap committed events, in output order, into out (host or device
 * memory per mem) and set *n_out.  Returns SIM_MORE if events remain (the next
 * call continues where this one stopped).  Waits for the handle's stream.
 * If a pushed frame failed on the device, returns that error code and
 * delivers nothing (*n_out = 0); the events of the frames committed before
 * the failure stay for the next call, and the handle continues from the last
 * committed frame (see sim_stats.frames_committed). */
int sim_pop_events(sim_t* s, sim_event* out, int64_t cap, int64_t* n_out, int32_t mem);

/* Wait for all work of the handle; returns (and clears) a pending device error. */
int sim_sync(sim_t* s);

/* Statistics (waits for the handle's stream). */
int sim_get_stats(sim_t* s, sim_stats* st);

/* Copy the committed per-pixel reference R (Q16, W*H int32, row-major) to
 * host memory.  In reset mode the library keeps no reference: SIM_ERR_STATE. */
int sim_get_reference(sim_t* s, int32_t* out_host);

/* Enable (1) or disable (0) per-kernel device timing with CUDA events. */
int sim_set_profiling(sim_t* s, int32_t enable);

/* Accumulated device time (ms) and launch count of one kernel kind since
 * profiling was enabled or last reset (reset = 1 clears after reading). */
int sim_kernel_time(sim_t* s, int32_t kind, double* ms, int64_t* launches, int32_t reset);

/* Restart the stream: drop all committed state, pending events and any
 * pending error, keep the allocations.  The next push is a first frame.
 * Waits for the handle's stream. */
int sim_reset(sim_t* s);

/* End of a stream (the paper's simulators run over a finite frame sequence,
 * Sec. IV-A).  Release every resource of the handle (waits for its stream). */
int sim_destroy(sim_t* s);

/* Static English description of a return code. */
const char* sim_strerror(int code);

/* Description of the last CUDA runtime error that made a call of this host
 * thread return SIM_ERR_CUDA / SIM_ERR_OOM / SIM_ERR_NO_DEVICE. */
const char* sim_last_cuda_error(void);

/* Accumulated event frame, the paper's second output form (Fig. 1 caption:
 * "a frame with the accumulated events"): frame[y * width + x] += +1 for
 * every positive and -1 for every negative event of events[0..n) with
 * t_begin <= t_us < t_end.  events (n sim_event) and frame (width * height
 * int32, caller-owned, not cleared first, so windows add up) are device
 * memory; events outside the frame are skipped.  The work is enqueued on
 * cuda_stream (NULL: the legacy default stream) and not waited for.  The
 * sum is exact and independent of the event order (integer atomics).
 * SIM_ERR_ARG for a negative n, a NULL buffer or a bad size; SIM_ERR_CUDA
 * if the launch fails. */
int sim_accumulate(const sim_event* events, int64_t n, int32_t width, int32_t height,
                   int64_t t_begin, int64_t t_end, int32_t* frame, void* cuda_stream);

/* ---- checkpoint / restore ---------------------------------------------
 * The paper has no counterpart (it runs recorded sequences end to end).  A
 * stream's simulation state - committed frame count, the first frame's and
 * the last committed frame's times, the last frame's luma (SIM_DIFF: and the
 * frame before it), the reference (SIM_REF_ACCUM) and the statistics - can
 * be saved to host memory and restored into another handle, so a stream can
 * move between handles, devices or processes and continue bit-exactly.
 * Events not yet popped are output, not state: they stay with the source
 * handle.
 *
 * sim_state_size: bytes of a checkpoint of s (a function of its
 * configuration: a header plus W*H, plus W*H in SIM_DIFF, plus 4*W*H in
 * SIM_REF_ACCUM).
 * sim_get_state: waits for s's stream and writes the checkpoint into the
 * caller's host buffer of exactly that size.  SIM_ERR_STATE if a batch failed
 * and has not been reported yet (call sim_sync first); SIM_ERR_ARG for a NULL
 * or wrongly sized buffer.
 * sim_set_state: replaces s's state (and drops its pending events) with a
 * checkpoint taken from a handle of the same configuration (size, pixel
 * format, mode, intensity, reference mode, substeps, thresholds, threshold
 * maps present; the map contents are the caller's to match).  SIM_ERR_ARG
 * for a mismatching or malformed checkpoint (nothing changed). */
int sim_state_size(const sim_t* s, int64_t* bytes);
int sim_get_state(sim_t* s, void* buf, int64_t bytes);
int sim_set_state(sim_t* s, const void* buf, int64_t bytes);

/* Library version, "major.minor.patch". */
const char* sim_version(void);

/* ---- autotuner -------------------------------------------------------------
 * The paper has no counterpart (it runs one configuration on one machine).
 * The batch kernel comes in two tile shapes: 64 x 16 pixels per 512-thread
 * block (two blocks per SM) and 64 x 8 per 256-thread block (four per SM),
 * and takes its tiles in one of three block orders: linear; serpentine (odd
 * rounds of one block per SM reversed, so that the blocks sharing an SM hold
 * tiles from opposite ends of the image); or balanced (before each batch a
 * pre-pass estimates every tile's cost from samples of the batch's flows -
 * frames in which the tile moves cost more - and the tiles are placed in
 * serpentine order over that ranking, so that the heaviest tile shares its
 * SM with the lightest; frames up to 4096 tiles).
 * The smaller shape has twice the blocks for a frame of a given size - more
 * parallelism for small frames, finer balance across SMs - at the price of
 * a larger halo per pixel.  Which one is faster depends on the frame size,
 * the mode and the substep count, so it is measured.
 *
 * sim_autotune runs the simulation kernel of a stream configured as *cfg in
 * both shapes on `frames` (2..64) synthetic frames (after a first frame)
 * generated on the device
 * (a moving sinusoidal texture with a constant flow of (3.0, -2.0) px per
 * frame; frame and flow content do not depend on the shape), times each
 * kernel launch with CUDA events, and records the fastest shape and order
 * (another choice than 64 x 16 in linear order only when it is at least 5 %
 * faster: a sample's timings scatter by a few percent) in a process-wide
 * table keyed by (width, height, pixel_format, mode, substeps,
 * max_substeps, intensity, ref_mode, threshold maps present).  sim_create
 * consults the table when cfg->tile_height is SIM_TILE_AUTO or SIM_TILE_TUNE.
 * The row kernel (SIM_TILE_ROWS) is timed too (dense and sparse modes) and
 * is chosen on the same 5 % rule.
 * *tile_height_out (if not NULL) receives 16, 8 or SIM_TILE_ROWS; us_out (if
 * not NULL, 3 doubles) the kernel time per frame in microseconds of shapes 16
 * and 8 (each in its faster order) and of the row kernel (0 when not timed).  sim_get_stats reports a handle's shape and
 * order.  The table serves substep-time handles (cfg->event_time is not
 * part of its key and is not timed); SIM_TIME_CROSSING handles run 64 x 16
 * tiles in block order.
 * Allocates two temporary simulators and the probe's frames on the current
 * device and frees them before returning; blocks until done.  Errors:
 * SIM_ERR_ARG (bad configuration or frames), SIM_ERR_OOM, SIM_ERR_CUDA. */
int sim_autotune(const sim_config* cfg, int32_t frames, int32_t* tile_height_out,
                 double* us_out);

/* As sim_autotune, but on the caller's frames: frames[0..count) (count 3..
 * SIM_MAX_BATCH) with flows and timestamps as for sim_push_frames (frame 0
 * starts the stream, flows[0] is not read; mem = SIM_HOST | SIM_DEVICE for
 * all of them, pitch_bytes per row), pushed as one batch through a
 * temporary simulator of each shape - twice, the second pass timed.  A
 * sample of the stream that will run gives the choice for its content (flow
 * reach, event density, active fraction), which a synthetic probe does not
 * know.  The caller's buffers are only read.  Errors as sim_autotune, plus
 * those of sim_push_frames for the sample (SIM_ERR_TIME ...). */
int sim_autotune_sample(const sim_config* cfg, int32_t count, const void* const* frames,
                        int64_t pitch_bytes, const float* const* flows, const int64_t* t_us,
                        int32_t mem, int32_t* tile_height_out, double* us_out);

/* Write the autotuner table to a text file (one line per configuration:
 * the key's nine fields, the chosen tile height and block order, the three
 * per-frame times),
 * or merge such a file into the table (later lines win).  Return SIM_OK or
 * SIM_ERR_ARG (NULL path, unreadable or malformed file: nothing merged). */
int sim_autotune_save(const char* path);
int sim_autotune_load(const char* path);

/* ---- multi-stream group ---------------------------------------------------
 * Many independent camera streams of mixed sizes and settings advanced
 * together (a serving-side batching pattern; the paper itself runs one
 * stream).  Each member is a full stream with the semantics, arithmetic
 * and event stream of a sim_t handle fed the same frames: the group only
 * changes how the work is launched.  simb_step advances every member that has
 * queued frames with one launch per kernel for all of them: an adaptive-N
 * pre-pass over (member, frame, block) work items, one tile launch per tile
 * class present (dense/sparse x accumulate/reset x log/linear x maps), and one
 * order launch whose tickets run over the chunks of all members (each member
 * keeps its own look-back chain and commits its own frames).  With graphs on,
 * that launch sequence is captured once per member set and replayed; the
 * per-step data (frame counts, batch serials, frame descriptors) are read
 * from a device table that the step uploads in one copy.
 *
 * All work of the group is ordered on one CUDA stream.  Not thread-safe: one
 * host thread drives a group. */
#define SIM_MAX_GROUP 1024

typedef struct simb_s simb_t;  /* opaque, owned by the library */

typedef struct {
  int32_t max_streams;       /* members at most, 1..SIM_MAX_GROUP */
  int32_t frames_per_step;   /* frames a member may queue between steps, 1..64 */
  int64_t hbm_budget_bytes;  /* admission bound on the members' device state; 0: 8 GiB */
  int32_t use_graphs;        /* 1: replay one CUDA graph per member set; 0: plain launches */
  int32_t reserved;
  void* cuda_stream;         /* cudaStream_t; NULL: group-owned stream */
  int64_t delivery_events;   /* simb_step_deliver: events per delivery area; 0: 2^23 */
} simb_config;

typedef struct {
  int32_t members;           /* admitted streams */
  int32_t tile_classes;      /* tile launches per step for the current members */
  int64_t bytes_used;        /* device state of the members (admission accounting) */
  int64_t budget;            /* hbm_budget_bytes */
  int64_t steps;             /* simb_step calls that launched work */
  int64_t frames_stepped;    /* member frames advanced by those steps */
  int64_t graph_captures;    /* graphs captured (one per member set) */
  int64_t graph_launches;    /* steps run as a graph replay */
  int64_t kernel_launches;   /* kernels launched by steps (a replay counts its kernels) */
  int64_t admit_refused;     /* simb_admit calls refused with SIM_ERR_ADMIT */
} simb_stats;

/* Defaults: 64 streams, 4 frames per step, 8 GiB budget, graphs on. */
int simb_config_default(simb_config* cfg);

/* Create an empty group (allocates its tables: about 1 KB per possible member
 * plus 32 bytes per member frame slot). */
int simb_create(const simb_config* cfg, simb_t** out);

/* Device bytes a stream of this configuration holds as a member (what
 * admission charges against the budget). */
int simb_state_bytes(const simb_t* g, const sim_config* cfg, int64_t* bytes);

/* Admit a stream: allocates its device state (as sim_create, with max_batch
 * = frames_per_step and the group's stream; cfg->cuda_stream and
 * cfg->max_batch are ignored).  *id is a small integer naming the member
 * until it is evicted (ids of evicted members are reused).  Returns
 * SIM_ERR_ADMIT, allocating nothing, when the group is full or the state
 * would exceed the budget.  Waits for the group's stream. */
int simb_admit(simb_t* g, const sim_config* cfg, int32_t* id);

/* Queue frame i of member id, as sim_push_frame (same buffer rules: device
 * buffers must stay valid until the step that consumes them has finished,
 * e.g. until the next simb_pop / simb_sync).  A member's first frame sets its
 * reference at once (one small launch) and is never queued.  Host frames are
 * copied into the member's staging slots.  SIM_ERR_STATE when the member
 * already has frames_per_step frames queued (call simb_step). */
int simb_push(simb_t* g, int32_t id, const void* frame, int64_t pitch_bytes, const float* flow,
              int64_t t_us, int32_t mem);

/* Advance every member with queued frames by all of its queued frames
 * (asynchronous; *frames, if not NULL, receives the number of member frames
 * launched, 0 when nothing was queued).  Device-side failures of a member
 * (event overflow) are reported by that member's next simb_pop and roll only
 * that member back, as for a sim_t. */
int simb_step(simb_t* g, int64_t* frames);

/* One member's share of a delivered step. */
typedef struct {
  int32_t id;                /* member id */
  int32_t status;            /* SIM_OK, or the member's device error (its frames of this
                                step and later queued frames are dropped, as for a sim_t;
                                see sim_pop_events) */
  int64_t first;             /* index of its first event in the delivered array */
  int64_t count;             /* events delivered (in the member's output order) */
  int64_t frames_committed;  /* the member's committed frames after this step */
  int64_t pixel_substeps;    /* the member's sum over committed frames of W H N */
} simb_delivery;

/* Serving form of a step: simb_step, then one more kernel that copies every
 * member's committed, undelivered events into a library-owned pinned host
 * area (delivery_events events; members in table order, each member's events
 * contiguous) and fills one simb_delivery per member.  Asynchronous: two
 * deliveries may be in flight (the areas alternate), so the next step can be
 * launched before the host reads this one.  Events that do not fit the area
 * stay on the device for the next delivery.  May be called with no frames
 * queued (delivers only).  A group that delivers must not use simb_pop
 * (SIM_ERR_STATE); SIM_ERR_STATE as well when two deliveries are already
 * uncollected. */
int simb_step_deliver(simb_t* g, int64_t* frames);

/* Wait for the oldest uncollected delivery and return its table (*n entries,
 * one per member at the time of the step) and its events (*n_events).  The
 * pointers stay valid until the second simb_step_deliver after this call.
 * Members that reported a device error are rolled back here (this waits for
 * the group's stream).  SIM_ERR_STATE when no delivery is in flight. */
int simb_collect(simb_t* g, const simb_delivery** table, int32_t* n, const sim_event** events,
                 int64_t* n_events);

/* 1 if the oldest uncollected delivery has finished on the device (so that
 * simb_collect will not wait), 0 if not; SIM_ERR_STATE when none is in
 * flight. */
int simb_delivery_ready(simb_t* g);

/* Committed events of member id, as sim_pop_events (waits for the group's
 * stream). */
int simb_pop(simb_t* g, int32_t id, sim_event* out, int64_t cap, int64_t* n_out, int32_t mem);

/* Statistics of member id, as sim_get_stats. */
int simb_stream_stats(simb_t* g, int32_t id, sim_stats* st);

/* Remove member id and free its state (waits for the group's stream);
 * its undelivered events are dropped.  SIM_ERR_STATE while deliveries are
 * uncollected. */
int simb_evict(simb_t* g, int32_t id);

/* Wait for the group's stream. */
int simb_sync(simb_t* g);

int simb_get_stats(simb_t* g, simb_stats* st);

/* Evict every member and free the group. */
int simb_destroy(simb_t* g);

/* ---- serving loop -----------------------------------------------------------
 * A request loop over the library (host code, one thread): camera streams
 * arrive as a Poisson process, are admitted while their device state fits a
 * memory budget (first come, first served; a stream that does not fit waits),
 * release frames on a wall-clock timeline at their own frame rate, and leave
 * when their duration ends.  Two policies serve the same arrival trace:
 *   SIM_SERVE_GROUP      continuous batching: every iteration queues the
 *                        frames that have arrived and launches one group step
 *                        for all streams (simb_step_deliver); the host
 *                        collects a step's events while the next one runs.
 *   SIM_SERVE_PER_STREAM one sim_t and one CUDA stream per camera: each frame
 *                        is pushed as it arrives, and each stream with frames
 *                        in flight is popped every iteration.
 * Latency of a frame = time its events are in host memory - its release time.
 * Frames are device-resident content pools (a camera feeding device memory,
 * e.g. a hardware decoder); frame j of a stream is pool frame
 * pingpong(j + phase). */
enum { SIM_SERVE_GROUP = 0, SIM_SERVE_PER_STREAM = 1 };

typedef struct {
  int32_t width, height;             /* luma frames, pitch = width */
  int32_t frames;                    /* U >= 2 pool frames, replayed forward and backward */
  int32_t substeps, max_substeps;    /* as sim_config */
  int32_t c_pos_q16, c_neg_q16;
  int32_t reserved;
  const void* const* frame;          /* U device pointers */
  const float* const* flow;          /* U device pointers: flow from pool frame u-1 to u */
  const float* const* flow_back;     /* U device pointers: flow from pool frame u to u-1 */
  const uint16_t* c_pos_map;         /* optional host W*H maps, as sim_config */
  const uint16_t* c_neg_map;
} sim_serve_pool;

typedef struct {
  int32_t sid;                       /* index in the arrival trace */
  int32_t width, height, fps;
  int32_t pool, phase;
  int32_t frames;                    /* frames whose events were delivered (frame 0 included) */
  int32_t status;                    /* SIM_OK or the stream's first device error */
  int64_t events;
  uint64_t digest;                   /* sum of e_i M^(n-1-i) mod 2^64 over the delivered
                                        events e_0..e_{n-1} as 64-bit little-endian words,
                                        M = 0x9E3779B97F4A7C15 */
} sim_serve_stream;

typedef struct {
  int32_t policy;                    /* SIM_SERVE_GROUP | SIM_SERVE_PER_STREAM */
  int32_t mode;                      /* SIM_DENSE | SIM_SPARSE */
  double horizon_s;                  /* frames are released for this long */
  double warmup_s;                   /* frames released earlier are not in the latency stats */
  double rate_per_s;                 /* stream arrivals per second */
  double dur_min_s, dur_max_s;       /* stream duration, uniform */
  int32_t warm_start;                /* 1: streams that arrived in the dur_max_s before t = 0
                                        and are still running are present at t = 0 */
  int32_t n_pools;                   /* stream size: one of the pools, uniform */
  const sim_serve_pool* pools;
  int32_t n_fps;                     /* stream frame rate: uniform over fps[] */
  int32_t reserved;
  const int32_t* fps;
  uint64_t seed;                     /* arrival trace */
  int32_t max_streams;               /* streams at once */
  int32_t frames_per_step;           /* frames a stream may have in flight */
  int64_t hbm_budget_bytes;          /* admission bound on the streams' device state */
  int64_t events_per_pixel;          /* event buffer of a stream: this x W x H events */
  double* latency_ms;                /* optional: latencies of the counted frames */
  int64_t latency_cap;
  sim_serve_stream* streams;         /* optional: one record per admitted stream */
  int32_t streams_cap;
  int32_t reserved2;
} sim_serve_config;

typedef struct {
  int64_t arrived, admitted, never_admitted, peak_streams;
  int64_t frames_released, frames_completed, frames_failed;
  int64_t events, pixel_substeps, steps, kernel_launches;
  double wall_s;                     /* from t = 0 until the last event was delivered */
  double gpix_substeps_per_s, events_per_s;
  double lat_p50_ms, lat_p90_ms, lat_p99_ms, lat_max_ms, lat_mean_ms;
  double admit_wait_p50_ms, admit_wait_p99_ms;
  int64_t latencies;                 /* frames in the latency statistics */
  int32_t streams_written;
  int32_t reserved;
} sim_serve_result;

/* Run the loop to the horizon and until every released frame is delivered.
 * Uses the current device; allocates and frees all state itself. */
int sim_serve_run(const sim_serve_config* cfg, sim_serve_result* res);

/* Diagnostic of failure detection (the paper has no counterpart): runs one
 * of the library's bounded device-side waits on the current device with a
 * poll limit of spin_limit (1 .. 2^22; the kernels use 2^22):
 *   which = 0: the order kernel's single-pass scan waiting for its
 *              predecessor chunk's prefix (look-back);
 *   which = 1: a group tile waiting for the tile's earlier frames.
 * publish = 1 prepares the awaited word as published (the wait ends at
 * once), 0 leaves it unpublished: the wait must give up after spin_limit
 * polls and return, leaving SIM_ERR_DEVICE_TIMEOUT in the stream's error
 * word instead of hanging the GPU.  *device_status receives that word
 * (SIM_OK or SIM_ERR_DEVICE_TIMEOUT).  Allocates and frees a few bytes of
 * device memory; synchronises the device.  Returns SIM_OK, SIM_ERR_ARG,
 * SIM_ERR_CUDA or SIM_ERR_NO_DEVICE. */
int sim_selftest_bounded_wait(int32_t which, int32_t publish, int32_t spin_limit,
                              int32_t* device_status);

/* ---- optical flow on the device -------------------------------------------
 * Pyramidal Lucas-Kanade flow between two consecutive frames: the flow the
 * paper's sparse and difference simulators use (Sec. III-B: the selected
 * pixels' flow from "any sparse optical flow algorithm"; Sec. IV-A, Figs. 3
 * and 4: "Sparse int. w. LK", "Difference int. w. LK"; the paper runs
 * OpenCV's).  Computed on the device, its output is a flow buffer that
 * sim_push_frame(s) takes as it is.
 *
 * Arithmetic (bit-exact across runs and devices): level 0 is the 8-bit luma
 * (BT.601 for RGB) times 16; level l+1 the 2 x 2 box average of level l,
 * rounded half up, of size ((W+1)/2, (H+1)/2); gradients of the first
 * frame are twice the central differences (reads clamped); the window of a
 * pixel is the (2r+1)^2 pixels around it, coordinates clamped; a pixel is
 * tracked when the smaller eigenvalue of its window's gradient matrix, per
 * window pixel, is at least min_eig (gradient units: twice the derivative
 * in 1/16 intensity levels); each of `iterations` updates resamples the
 * second frame with the simulator's clamped Q16 bilinear at the current
 * estimate and adds -2 G^-1 b (G the gradient matrix, b the sums of
 * gradient times temporal difference), solved in IEEE double with every
 * operation rounded in a fixed order, rounded to Q16; the guess of a pixel
 * is twice its parent's flow one level up; flows are clamped to +-1024 px.
 * Untracked pixels keep their guess (zero at the top level). */
typedef struct sim_flow_s sim_flow_t;  /* opaque, owned by the library */

typedef struct {
  int32_t width, height;   /* 1..SIM_MAX_DIM */
  int32_t pixel_format;    /* SIM_LUMA8 | SIM_RGB8 */
  int32_t levels;          /* pyramid levels, 1..8 (default 3) */
  int32_t radius;          /* window radius r, 1..7: (2r+1)^2 pixels (default 3) */
  int32_t iterations;      /* updates per level, 1..16 (default 3) */
  double min_eig;          /* tracking threshold >= 0 (default 64) */
  void* cuda_stream;       /* cudaStream_t to order work on; NULL: library-owned stream */
} sim_flow_config;

/* Defaults for a width x height luma stream (see the field comments). */
int sim_flow_config_default(sim_flow_config* cfg, int32_t width, int32_t height);

/* Allocate the pyramids of both frames and the per-level flows on the
 * current device.  *out is set on SIM_OK only.  Errors: SIM_ERR_ARG,
 * SIM_ERR_OOM, SIM_ERR_NO_DEVICE, SIM_ERR_CUDA. */
int sim_flow_create(const sim_flow_config* cfg, sim_flow_t** out);

/* Flow from frame prev (i-1) to frame cur (i), both device memory (rows of
 * the given pitch, width * pixel_format bytes used), into flow (device,
 * height * width * 2 floats (dx, dy) in px, 8-byte aligned) - the layout
 * sim_push_frame reads.  Asynchronous on the handle's stream; the buffers
 * must stay valid until the stream passes the call.  One handle must not
 * be used from two host threads at once, and its calls are ordered on its
 * stream. */
int sim_flow_compute(sim_flow_t* f, const void* prev, int64_t prev_pitch, const void* cur,
                     int64_t cur_pitch, float* flow);

/* Release the handle (waits for its stream). */
int sim_flow_destroy(sim_flow_t* f);

/* ---- allocation-free frame pair ------------------------------------------
 * The paper has no counterpart: this is a library service for callers that
 * must not allocate device memory while they run, such as code whose device
 * memory belongs to another framework's caching allocator (a raw cudaMalloc
 * bypasses and fragments that pool, and cudaFree synchronises the whole
 * device), frame-rate pipelines with a no-allocation rule after start-up
 * (cudaMalloc / cudaFree have unbounded latency), or plug-ins that are handed
 * device buffers by their host application and may not allocate their own.
 *
 * One step of the simulation from camera frame i-1 to frame i, with the same
 * arithmetic and event order as a sim_t handle that was given frame i-1 and
 * then frame i.  All inputs and outputs are the caller's device memory; every
 * scratch buffer the kernels use (control block, log table, luma frames,
 * segment table, staging, look-back words) is carved out of one file-scope
 * device array of SIM_STATIC_SCRATCH_BYTES per device.  The call makes no
 * cudaMalloc, cudaFree or other allocating call.
 *
 *   cfg        : width, height, pixel_format, mode, substeps, max_substeps,
 *                intensity, ref_mode, c_pos_q16, c_neg_q16, c_act_q16 as for
 *                sim_create (same limits); c_pos_map / c_neg_map must be NULL;
 *                max_batch and event_capacity are ignored; cuda_stream orders
 *                the work (NULL: the legacy default stream).
 *   prev_frame, prev_pitch : frame i-1 (device, rows of prev_pitch bytes).
 *   frame, pitch           : frame i (device).
 *   flow       : device, H * W * 2 floats (dx, dy), flow from frame i-1 to
 *                frame i, 8-byte aligned.
 *   t_prev_us, t_us : times of frames i-1 and i; 0 <= t_prev_us < t_us <
 *                2^32; event times are t_prev_us + floor(k (t_us - t_prev_us) / N).
 *   ref_in, ref_out : accumulate mode: the per-pixel reference R (Q16, W*H
 *                int32, device, 4-byte aligned) before and after the step.
 *                ref_in = NULL starts a stream: R = LUT[luma of frame i-1].
 *                ref_in may equal ref_out (updated in place).  Reset mode:
 *                both ignored (may be NULL).
 *   events, event_capacity : device output, 8-byte aligned; the step's
 *                events in output order.
 *   n_events   : host; events written (0 on any error).
 * Returns SIM_OK, or: SIM_ERR_ARG (invalid argument), SIM_ERR_TIME /
 * SIM_ERR_TIME_RANGE, SIM_ERR_TOO_LARGE when the problem does not fit the
 * scratch array (checked before any device work), SIM_ERR_EVENT_OVERFLOW
 * when the events exceed event_capacity or the 8-byte staging that remains
 * after the other parts, SIM_ERR_DEVICE_TIMEOUT, SIM_ERR_CUDA /
 * SIM_ERR_NO_DEVICE.
 * A failed step changes no reference the caller can still need: ref_in is
 * never written; ref_out is written only by a step that returns SIM_OK when
 * it equals ref_in or ref_in is NULL (the new reference is built in the
 * scratch array and copied to ref_out once the step has been checked), so
 * the same call can be repeated, e.g. with a larger event buffer.  With
 * distinct ref_in and ref_out, ref_out is undefined after an error.  The
 * events buffer holds no usable result after an error.
 *
 * Scratch: the array needs about 2 W H + 24.3 N_max H ceil(W / 64) bytes
 * (N_max = substeps, or max_substeps when adaptive), plus 4 W H more for an
 * in-place or stream-starting accumulate step (ref_in == ref_out or NULL),
 * plus 2 KB, plus at least 1 MiB of staging; larger problems get
 * SIM_ERR_TOO_LARGE.  The 32 MiB array admits 1280 x 720 at any N_max and
 * 1920 x 1080 up to N_max = 36 (in place: 25); 3840 x 2160 up to N_max = 5
 * (in place: does not fit).
 * Set-up: on the first call on a device (and again after the device's
 * context changes, e.g. after cudaDeviceReset) the call looks the array's
 * address up in the current context (cudaGetSymbolAddress) and sets the
 * kernels' shared-memory limits; make that first call before any stream
 * capture begins.  Each call clears the parts of the array
 * that must start at zero.  Every call on a device shares the one array:
 * calls whose device work overlaps (two streams, or two host threads) race
 * and corrupt each other's results; order them on one stream or serialise
 * them.  The call is synchronous: it waits for its stream before returning
 * (it reads the step's status and event count back into host memory). */
#define SIM_STATIC_SCRATCH_BYTES (32LL << 20)
int sim_step_pair_static(const sim_config* cfg, const void* prev_frame, int64_t prev_pitch,
                         const void* frame, int64_t pitch, const float* flow, int64_t t_prev_us,
                         int64_t t_us, const int32_t* ref_in, int32_t* ref_out,
                         sim_event* events, int64_t event_capacity, int64_t* n_events);

#ifdef __cplusplus
}
#endif
#endif /* EVSIM_H */
