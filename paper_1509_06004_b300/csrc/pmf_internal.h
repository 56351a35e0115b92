// Internal layout shared by the C ABI (pmf_api.cpp) and the kernels
// (pmf_kernels.cu).  Not part of the public interface.
#pragma once
#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include "pmf.h"

namespace pmf {

constexpr int TILE_W = 32;                 // row pitch alignment (one warp = 32 lanes)
constexpr int TILE_IN = 30;                // interior columns of a tile: lanes 1..30; lanes 0
                                           // and 31 mirror the neighbouring tiles' columns
constexpr int ROW_ALIGN = 16;              // rows padded so tile heights 4/8/16 divide them
constexpr int32_t HINF = 0x3fffffff;       // label of a pixel that cannot reach t
constexpr int BFS_ROWS = 32;               // rows of a relabel strip (a column of tiles)
// per relabel strip, 32 lanes each: 6 arc masks, 3 border residuals, 32 label
// rows (used by the forward pass), and the member tiles' active counts (lane
// j: tile j) as last written
constexpr int RW_CNT = 9 + BFS_ROWS;
constexpr int STRIP_REC_WORDS = (RW_CNT + 1) * 32;
constexpr int N_INST_PLANES = 8;           // e, h, rt, fR, fD, src0, slope, ct
constexpr int N_IMG_PLANES = 2;            // w_h, w_v
enum Plane { P_E = 0, P_H = 1, P_RT = 2, P_FR = 3, P_FD = 4, P_SRC0 = 5, P_SLOPE = 6, P_CT = 7 };
// Tensor-memory-access staging of a relabel strip's first visit: one box of the
// instance's planes e, h, rt, fR, fD (consecutive, so one 3-D copy) and one of
// the image's w_h, w_v, each 32 rows x STAGE_BOX_W columns starting at the
// strip's first column rounded down to a multiple of 4 (a copy's innermost
// coordinate must be 16-byte aligned)
constexpr int STAGE_BOX_W = 36;
constexpr int STAGE_INST_PLANES = 5;
constexpr int STAGE_WORDS = (STAGE_INST_PLANES + N_IMG_PLANES) * BFS_ROWS * STAGE_BOX_W;
constexpr int STAGE_BYTES = STAGE_WORDS * 4;
constexpr int TMAP_BYTES = 128;            // one CUtensorMap

// instance phases
// PH_FWD: after a certified step of an instance whose caller swapped s and t,
// the pass that finds the pixels reachable from excess (its cut)
// PH_WARM: at the start of each later lambda step, the strip pass that raises
// the source capacities (GGT warm start) and counts the tiles left active
// PH_COPY: after the certified step an instance forks at, the strip pass that
// copies its state into the forked instance (pmf_set_fork)
// PH_WAIT: a forked instance before its parent's copy pass has run
// PH_SETUP: server mode, a newly admitted instance's strip pass: it checks its
// capacities, zeroes the padding, sets up the lambda_0 preflow and resets its
// tiles; then the first global relabel
enum Phase { PH_BFS = 0, PH_PR = 1, PH_DONE = 2, PH_FWD = 3, PH_WARM = 4, PH_COPY = 5, PH_WAIT = 6,
             PH_SETUP = 7 };
// tile queue states
enum TState { T_IDLE = 0, T_QUEUED = 1, T_RUNNING = 2, T_DIRTY = 3 };
// global error flags; GE_INTERNAL_MASK marks a broken scheduler invariant, after
// which no instance's result is trusted
enum GErr { GE_STALL = 1, GE_RING = 2, GE_SLOT = 4, GE_TIMEOUT = 8, GE_PHASE = 16, GE_STAGE = 32 };
constexpr int GE_INTERNAL_MASK = GE_RING | GE_PHASE | GE_STAGE;
// per-instance validation flags (set by the pad/init kernels)
enum VFlag { VF_NEG = 1, VF_OVERFLOW = 2, VF_SLOPE = 4, VF_BADCAP = 8 };

struct DevInst {                 // read-only during a solve
    int32_t H, W, pitch, rows;
    int32_t image;
    int32_t tiles_x, tiles_y, n_tiles;
    int32_t tile_base;
    int32_t n_lambda;
    int32_t hcap;                // labels >= hcap become HINF (= H*W)
    int32_t lead_base;           // index of this instance's first relabel strip in the leader list
    int64_t plane_off;           // int32 elements from the instance-plane base
    int64_t img_off;             // int32 elements from the image-plane base
    int64_t mask_off;            // bytes from the mask base
    int32_t n_leads;             // relabel strips (tiles_x * ceil(tiles_y / strip_span))
    int16_t cut_rule;            // 0: maximal source set; 1: s and t swapped by the caller (pmf_set_cut_rule)
    int16_t slope_side;          // 0: cs = src0 + slope*lambda, ct = sink; 1: cs = src0, ct = sink - slope*lambda
    int32_t fork_parent;         // -1, or the instance whose state this one starts from (pmf_set_fork)
    int32_t fork_child;          // -1, or the instance forked from this one
    int32_t fork_k;              // the step of this instance after which its child is forked
};
static_assert(sizeof(DevInst) % 16 == 0, "DevInst is loaded as int4s");

// 16-byte aligned: the worker reads the first four fields with one 16-byte
// vector load, which faults on a misaligned address
struct alignas(128) InstState {  // mutable during a solve
    // written only by the warp that runs a phase change (nothing of the
    // instance is queued or running then); read by the workers
    int32_t phase, k, epoch, status;
    int32_t vflags;                  // validation flags of the inputs
    int32_t pr_budget;               // push/relabel visits allowed before the next global relabel
    int32_t want_bfs;                // set once by the visit that spends the budget
    int32_t lab_cap;                 // labels at or above this are treated as "cannot reach t"
    unsigned long long pr_mark;      // pr_visits when the current push/relabel phase began
    unsigned long long step_mark;    // pr_visits + bfs_visits when the current lambda step began
    unsigned long long epochs;       // global relabels so far
    int32_t lam_prev;                // lambda the state was certified at (the warm start raises from it)
    int32_t pad_c_;
    // updated atomically by the workers, on their own cache line
    alignas(128) int32_t outstanding, active, dmax, pad3_;
    unsigned long long flow;         // int64 two's complement: total flow into t
    unsigned long long pr_visits, bfs_visits;
    unsigned long long warm_visits;  // strip visits of the warm-start phases
};

static_assert(sizeof(InstState) % 16 == 0, "InstState array elements must stay 16-byte aligned");
static_assert(offsetof(InstState, phase) == 0 && offsetof(InstState, k) == 4 &&
              offsetof(InstState, epoch) == 8 && offsetof(InstState, status) == 12,
              "the worker loads phase, k, epoch, status as one int4");

// trace record of an instance phase change
struct TraceEvent {
    unsigned long long t_ns;
    int32_t inst, event, k, epoch;
    long long pr_visits, bfs_visits;
    long long flow;              // flow into t so far (current lambda step)
    int32_t active, pad_;        // pixels with excess that reach t, as of the last relabel
};
enum TraceKind { TR_BFS_START = 0, TR_STEP_DONE = 1, TR_PR_START = 2, TR_DONE = 3, TR_NOT_CONVERGED = 4 };
constexpr int TRACE_CAP = 1 << 16;

struct TileState {
    int32_t state, epoch, pad_, active;   // pad_: unused
};

// the queue counters sit on separate 128-byte lines: head is hit by every pop,
// tail by every push
struct Globals {
    alignas(128) unsigned long long head;
    alignas(128) unsigned long long tail;
    alignas(128) int32_t inst_done;  // instances that reached PH_DONE (the launch ends at n_inst)
    alignas(128) int32_t err, round_mode;
    unsigned long long round_end;
    unsigned long long t_start;      // %globaltimer at the start of the launch
    unsigned long long progress;     // bumped by warps running kept items (no queue traffic)
    alignas(128) unsigned long long trace_n;
    // server mode: mailbox entries taken, instances started, next mailbox check
    alignas(128) int32_t cmd_head, admitted;
    unsigned long long mb_next_ns;
    // warp-time breakdown (ns summed over warps), recorded with the trace:
    // [0] waiting for work, [1] push/relabel visits, [2] relabel (BFS) visits,
    // [3] retiring items (wake-ups, requeue, phase changes), [4] sweeps run,
    // [5..7] SM cycles in the load, sweep and write-back stages of push/relabel visits,
    // [8..10] the same for relabel-strip visits (load, relaxation, write-back),
    // [11] relaxation rounds of relabel-strip visits
    unsigned long long prof[PMF_PROFILE_COUNTERS];
};

// Server mode: the host posts instance slots whose inputs it has copied in
// to a mailbox in mapped host memory; idle workers take them from there.
constexpr int MB_CAP = 4096;
struct Mailbox {
    int32_t tail;                // entries posted so far (written by the host after the entry)
    int32_t stop;                // 1: the kernel ends once every posted instance is finished
    int32_t pad_[30];
    int32_t ring[MB_CAP];        // slot of entry t at ring[t % MB_CAP]
};

struct Params {
    TraceEvent *trace;           // phase-change trace (TRACE_CAP records) or nullptr
    Mailbox *mailbox;            // server mode (device address of mapped host memory), else nullptr
    int32_t *planes;             // instance planes base
    const int32_t *img;          // image planes base
    uint8_t *masks;
    const DevInst *inst;
    InstState *ist;
    TileState *tiles;
    const int32_t *tile_inst;
    int32_t *ring;
    int32_t *strip_cache;        // [relabel strips][STRIP_REC_WORDS]
    const int32_t *lambdas;      // [n_inst][max_lambdas]
    long long *flows;            // [n_inst][max_lambdas]
    Globals *g;
    const int32_t *img_flags;    // [n_images] validation flags of set_capacities
    int32_t *inst_flags;         // [n_inst] validation flags of set_terminals
    int32_t *done_flags;         // [n_inst] host-mapped: 1 + status once an instance is finished (or nullptr)
    unsigned long long ring_mask;
    int32_t n_inst, n_tiles_total, max_lambdas, sweeps;
    int32_t n_leads_total, chain_push;   // chain_push: push order of the sweeps (pmf_tuning.push_order)
    int32_t n_leads_queued;      // relabel strips queued at the start (forked instances' strips come last
                                 // and wait for their parent)
    int32_t relabel_pct, tile_h;
    int32_t relabel_extra;       // visits added to every phase's budget
    int32_t relabel_reach;       // a phase's budget is at least relabel_reach% of the last relabel's largest distance
    int32_t any_sink_side;       // some instance's sink capacities fall with lambda (slope_side 1)
    int32_t wide_regs;           // tile height 4 on 1-3 blocks per SM: the build with more registers
    int32_t poll_ns, label_slack;
    // tensor maps for staged relabel-strip loads: [n_inst] instance planes, then
    // [n_images] image planes (TMAP_BYTES each, device memory), or nullptr
    const unsigned char *tmaps;
    int32_t strip_stage;         // 1: first relabel visits load through tmaps (dynamic shared memory)
    long long max_visits_per_tile;
    long long stall_ns;          // a worker gives up after this long without progress
    long long max_ns;            // ... or after this long in one launch
};

// launch wrappers (pmf_kernels.cu)
cudaError_t launch_pad_image(const Params &P, int image, const DevInst &d, const int32_t *w_h,
                             const int32_t *w_v, int32_t *flags, cudaStream_t s);
cudaError_t launch_pad_terminals(const Params &P, int inst, const DevInst &d, const int32_t *src0,
                                 const int32_t *slope, const int32_t *sink, cudaStream_t s);
cudaError_t launch_reset(const Params &P, cudaStream_t s);
cudaError_t launch_init(const Params &P, int max_pixels, cudaStream_t s);
cudaError_t launch_worker(const Params &P, int grid, cudaStream_t s);
// server mode: clear the slots' tiles, queue and instance states (slot = tile / max_tiles)
cudaError_t launch_server_reset(const Params &P, int max_tiles, cudaStream_t s);
cudaError_t launch_server_worker(const Params &P, int grid, cudaStream_t s);
cudaError_t server_occupancy(int *blocks_per_sm);
cudaError_t launch_begin_round(const Params &P, cudaStream_t s);
// flags: 3 int32 of device scratch for the sweeps' termination test
cudaError_t launch_return_excess(const Params &P, const DevInst &d, int lambda, int max_sweeps,
                                 int32_t *f_h, int32_t *f_v, int32_t *f_s, int32_t *f_t, int32_t *status,
                                 int32_t *flags, cudaStream_t s);
int worker_warps_per_block();
// records "where: <CUDA error text>" for pmf_last_error (this thread) and
// returns PMF_ERR_CUDA; PMF_OK for cudaSuccess
pmf_status cuda_err_at(cudaError_t e, const char *where);
cudaError_t worker_occupancy(int tile_h, int *blocks_per_sm, bool staged = false);
// lets the batch kernels take the staging buffer's shared memory (once per process)
cudaError_t prepare_stage_kernels();
// device tensor maps of a batch's planes for staged strip loads (host side);
// false when the driver offers no tensor-map encoder
bool encode_plane_maps(unsigned char *host_out, const int32_t *inst_base, const int32_t *img_base,
                       int n_inst, const int64_t *plane_off, const int *inst_image, int n_images,
                       const int64_t *img_off, const int *rows, const int *pitch);

}  // namespace pmf
