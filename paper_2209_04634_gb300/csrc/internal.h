// Internal structures shared by the kernels (kernels.cu) and the host
// runtime (runtime.cu) of the evsim library.  Not part of the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace evsim {

// Tile of the simulation kernel (dense and sparse): TW x TH pixels, NTD
// threads, up to two simulated pixels per thread.  The batch kernel also
// comes in a TW x 8 shape (256 threads), chosen per stream by the
// autotuner; multi-stream group launches use TW x TH.
constexpr int TW = 64;
constexpr int TH = 16;
constexpr int NTD = 512;
// Block size of the other kernels.
constexpr int NT = 256;
constexpr int NWARP = NT / 32;
// Largest per-tile flow reach (pixels) served from the shared-memory halo;
// tiles whose flow reaches further sample global memory instead.
constexpr int HMAX = 16;
constexpr int SW = TW + 2 * HMAX;  // shared tile stride (int32 elements)
constexpr int SH = TH + 2 * HMAX;
constexpr int MAXN = 64;           // largest substep count
// Order kernel: segments per chunk (OSEG per thread).
constexpr int OSEG = 4;
constexpr int OCHUNK = NT * OSEG;
// Staging chunk of one warp of the batch tile kernel (events).  A stream's
// staging area holds 4/3 of its event capacity plus one chunk per warp of its
// tiles, so chunking never turns a batch that fits into an overflow.
constexpr int STAGE_CHUNK = 64;

// Look-back status word: [epoch:32][flag:2][value:30].
constexpr unsigned long long LB_AGG = 1ull << 30;
constexpr unsigned long long LB_INC = 2ull << 30;
constexpr unsigned long long LB_VALUE = (1ull << 30) - 1;
constexpr int MAX_EVENTS = (1 << 30) - 2;  // per batch (and event buffer capacity)
// Debug builds (compiled with EVSIM_BOUNDS_CHECK): the kernels check the
// indices of their global writes, of the order kernel's segment and staging
// reads and of the shared-memory halo writes, record the first violation as
// SIM_ERR_BOUNDS in the stream's error word and skip the access.  Release
// builds compile the checks away.
#ifdef EVSIM_BOUNDS_CHECK
constexpr bool kBoundsCheck = true;
#else
constexpr bool kBoundsCheck = false;
#endif
// Bounded spin: polls before a look-back (or a tile's wait for its earlier
// frames) gives up and flags a timeout; SimParams.spin_limit overrides it
// (0: this default).
constexpr int SPIN_LIMIT = 1 << 22;

// Device-resident control block of one stream.  Fields marked "committed"
// change only when a batch of frames commits; the others are per-batch
// scratch that the order kernel resets when it finishes a batch.
struct Ctl {
  int err;                       // sticky error (0 or a SIM_ERR_* code)
  int sel;                       // committed: bit0 reference ping-pong, bit1 frame ring
  int last_n;                    // committed: substeps of the last frame
  int batch_fail;                // staging overflow seen while simulating this batch
  long long t_prev;              // committed: t of the last frame - t_0 (us)
  long long cursor;              // committed: events held in the event buffer
  long long committed;           // committed: frames
  long long batch_events;        // committed: events of the last committed batch
  long long active;              // sparse: active pixels of the batch in flight
  long long last_active;         // sparse: active pixels of the last committed batch
  long long work_px;             // committed: sum over frames of W H N
  long long work_active;         // committed: sum over frames of (pixels simulated) N
  long long active_n;            // sparse: sum over the batch in flight of active pixels x N
  unsigned long long clamped;    // flow components clamped so far
  unsigned long long stage_top;  // staging bump allocator (events)
  unsigned int order_ticket;     // order kernel: chunk tickets
  unsigned int order_done;       // order kernel: chunks finished
  unsigned int order_exit;       // order kernel: blocks that left the ticket loop
  unsigned int unit_ticket;      // row kernel: next unit (reset when the batch finishes)
  long long drained;             // group delivery: events of the buffer already delivered
  long long work_pixels;         // committed: sum over frames of the pixels simulated
};

// Per-frame arguments of a batch (device-resident table).
struct FrameDesc {
  const unsigned char* frame;   // input frame (device)
  long long pitch;              // bytes per input row
  const float2* flow;           // H*W (dx, dy); unused for a stream's first frame
  long long t_rel;              // t_i - t_0 (us)
};

struct BatchArg {
  const FrameDesc* frames;      // count descriptors (device)
  int count;
  unsigned int serial;          // batch serial: epoch of the look-back words
  int host_mapped;              // 1: the frames are pinned host memory read in place
  int pad;
};

struct Ev {  // same layout as sim_event
  unsigned int t;
  unsigned int xyp;  // x | (yp << 16)
};

// The events of one segment: one (frame, substep, tile row).  When no pixel
// of the row crossed more than one threshold in the substep (src == -1), the
// events are bit b of `mask` (pixel tx0 + b has an event) with polarity bit b
// of `pol`; the order kernel materialises them.  Otherwise either the tile
// kernel wrote the row's `cnt` events to staging at `src` (src >= 0), or -
// dense tiles - the row's per-pixel event counts are in staging at
// -2 - src (src <= -2): 32 words, word l holding the counts of columns l (low
// 16 bits) and l + 32 (high 16 bits), with `mask` and `pol` marking the
// pixels with events and their polarity as for a one-crossing row.
struct Seg {
  unsigned long long mask;
  unsigned long long pol;
  int cnt;
  int src;
};

// Everything the kernels need about one stream (fixed for its lifetime).
struct SimParams {
  int W, H, ch;
  int tiles_x, tiles_y;          // tiles of TW x tile_h pixels
  int mode, ref_mode, intensity;
  int n_fixed, n_max;
  int cp, cn, cact;
  int bmax;                     // frames per batch the segment table holds
  int stage_chunk;              // staging chunk per warp of the batch kernel (0: exact)
  int tile_h;                   // batch kernel tile height: 16 (512 threads) or 8 (256)
  int sms;                      // SMs of the device (block placement of the batch kernel)
  int block_order;              // batch kernel: 0 tiles in block order, 1 serpentine,
                                // 2 balanced by the batch's estimated tile costs
  int xtime;                    // 1: per-crossing event times (64 x 16 tiles, every row
                                // with an event staged)
  unsigned int* tile_cost;      // balanced order: [tiles] each tile's estimated cost (k_predict)
  int* tile_order;              // balanced order: [tiles] tile of each block
  const unsigned short* cpmap;
  const unsigned short* cnmap;
  const int* lut;               // 256 Q16 entries (device)
  unsigned char* ring0;         // luma frame ring (last frame of the previous batch)
  unsigned char* ring1;
  unsigned char* ring2_0;       // difference mode: the frame before that (ping-pong as ring)
  unsigned char* ring2_1;
  int* R0;                      // reference ping-pong pair
  int* R1;
  Ctl* ctl;
  unsigned long long* maxf2;    // [bmax] adaptive: max squared Q16 flow per frame
  Ev* staging;
  long long stage_cap;
  unsigned long long* tdone;    // per tile: [batch serial:32][frames of the batch done:32]
  Seg* seg;                     // per (frame, substep, tile row)
  long long segs_per_k;         // segments per substep of one frame
  long long seg_cap;            // segments the table holds (debug bounds checks)
  unsigned long long* order_status;
  Ev* events;
  long long event_cap;
  int spin_limit;               // polls of a bounded device wait (0: SPIN_LIMIT)
  unsigned char* segflag;       // row kernel: per (frame, row, 64-column unit) 1 when the
                                // unit-frame's segments are written, 0 when it emitted
                                // nothing and wrote none; null: every segment is written
  int* units;                   // with segflag (null: none): per frame, the indices of its
                                // flagged units in raster order (segs_per_k slots a frame)
  int* unit_count;              // [bmax] flagged units of each frame
};

// ---- multi-stream step (one launch per kernel for every member of a group)
constexpr int MAX_GROUP = 1024;  // members of one group
// Tile kernel classes (template flags); members of one class share a launch.
// TILE_TH8: the member's tiles are 64 x 8 (256-thread blocks), else 64 x 16.
enum { TILE_RESET = 1, TILE_MAPS = 2, TILE_WIDE = 4, TILE_SPARSE = 8, TILE_TH8 = 16,
       TILE_CLASSES = 32 };

struct GroupStream {            // per member; changes only when members change
  SimParams p;
  const FrameDesc* frames;      // the member's descriptor slots (device)
  int pre_blocks;               // pre-pass blocks per frame (adaptive members)
  int pad;
};

struct StreamStep {             // per member and step
  int count;                    // frames in this step (0: idle)
  unsigned int serial;          // batch serial (look-back epoch)
  int chunk_begin;              // first order ticket of the member
  int pre_begin;                // first pre-pass work item of the member
};

struct GroupTotals {            // per step
  int chunks;                   // order tickets over all members
  int pre_items;                // pre-pass work items over all members
  int tiles[TILE_CLASSES];      // tiles of the members with frames, per class
  int active[TILE_CLASSES];     // members with frames, per class
};

// A member with frames in this step, in its class's work list: tiles
// [tile_begin, tile_begin + its tile count) of the class's step are its.
struct ActiveTile {
  int member;
  int tile_begin;
};

struct GroupCtl {
  unsigned int order_ticket;
  unsigned int order_exit;
  unsigned int drain_done;
  unsigned int tile_ticket;     // tile launches: next item of the class's work list
  unsigned int tile_exit;       // tile launches: blocks done
  unsigned int pad[3];
};

// One member's share of a delivered step (same layout as simb_delivery).
struct Delivery {
  int id;
  int status;
  long long first;
  long long count;
  long long committed;
  long long work_px;
};

// Destination of a delivery: host memory the device writes through its
// mapping.
struct DrainArg {
  Ev* events;                   // cap events
  long long cap;
  Delivery* table;              // one entry per member
  long long* total;             // events delivered
  const int* ids;               // member ids in table order (device)
  unsigned int* done;           // blocks finished (device, reset by the last block)
};

struct GroupArg {
  const GroupStream* gs;        // n members (device)
  const StreamStep* steps;      // n members (device)
  const GroupTotals* tot;       // device
  GroupCtl* gctl;               // device
  int n;
};

// Shared-memory bytes of the multi-stream tile kernel (dense and sparse) for a
// substep cap and a tile height (8 or 16).
size_t tile_smem_bytes(int n_max, int th);

// Launchers (kernels.cu; launch_dense in tile_dense.cu, launch_sparse in
// tile_sparse.cu).  Each returns the cudaError_t of the launch.
cudaError_t launch_init(const SimParams& p, const FrameDesc& f, cudaStream_t st);
cudaError_t launch_flowmax(const SimParams& p, const BatchArg& b, cudaStream_t st);
cudaError_t launch_dense(const SimParams& p, const BatchArg& b, cudaStream_t st);
cudaError_t launch_sparse_pre(const SimParams& p, const BatchArg& b, cudaStream_t st);
cudaError_t launch_sparse(const SimParams& p, const BatchArg& b, cudaStream_t st);
cudaError_t launch_diff(const SimParams& p, const BatchArg& b, cudaStream_t st);
// Row kernel (rows.cu): dense or sparse batch in 64-pixel row units taken by
// ticket (p.tile_h == 1; needs p.segflag).
cudaError_t launch_rows(const SimParams& p, const BatchArg& b, cudaStream_t st);
cudaError_t launch_accumulate(const Ev* ev, long long n, int W, int H, long long t_begin,
                              long long t_end, int* frame, cudaStream_t st);
// Balanced block order for the batch about to run: estimate every tile's
// cost from samples of the batch's flows (one block per tile), rank the
// tiles and lay them out (one block).
cudaError_t launch_plan(const SimParams& p, const BatchArg& b, cudaStream_t st);
constexpr int PLAN_MAX_TILES = 4096;  // tiles a balanced plan covers
cudaError_t launch_order(const SimParams& p, const BatchArg& b, cudaStream_t st, int grid);
cudaError_t configure_kernels(int n_max);
// Raise the tile kernels' shared-memory limits on the current device to what
// n_max substeps need, never lowering them (the limits are shared by every
// handle and entry point); again = true sets them even if recorded as done
// (a new CUDA context on the device).
cudaError_t raise_kernel_limits(int n_max, bool again);
// Per-mode tile kernels (tile_dense.cu, tile_sparse.cu): dynamic shared-memory
// limits of their k_tile instances for batches of up to n_max substeps.
cudaError_t configure_dense_kernels(int n_max);
cudaError_t configure_sparse_kernels(int n_max);
// Per-crossing event times (tile_xtime_dense.cu, tile_xtime_sparse.cu): the
// tile kernel instances of each mode; launch_dense / launch_sparse route to
// them when p.xtime.
cudaError_t configure_xtime_dense_kernels(int n_max);
cudaError_t configure_xtime_sparse_kernels(int n_max);
cudaError_t launch_xtime_dense(const SimParams& p, const BatchArg& b, cudaStream_t st);
cudaError_t launch_xtime_sparse(const SimParams& p, const BatchArg& b, cudaStream_t st);
int tile_class(const SimParams& p);
cudaError_t launch_pre_multi(const GroupArg& g, int grid, cudaStream_t st);
cudaError_t launch_tile_multi(const GroupArg& g, int cls, const ActiveTile* act, int grid,
                              size_t smem, cudaStream_t st);
cudaError_t launch_order_multi(const GroupArg& g, int grid, cudaStream_t st);
cudaError_t launch_drain(const GroupArg& g, const DrainArg& d, int grid, cudaStream_t st);
// Shared-memory permission of the multi-stream tile kernels.
cudaError_t configure_group_kernels(size_t smem);

// Record a CUDA error for sim_last_cuda_error (runtime.cu).
void note_cuda_error(cudaError_t e);
int device_sm_count();

}  // namespace evsim
