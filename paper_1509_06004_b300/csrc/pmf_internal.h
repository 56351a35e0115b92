// Internal layout shared by the C ABI (pmf_api.cpp) and the kernels
// (pmf_kernels.cu).  Not part of the public interface.
#pragma once
#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

namespace pmf {

constexpr int TILE_W = 32;                 // tile width = one warp, lane = column
constexpr int ROW_ALIGN = 16;              // rows padded so tile heights 4/8/16 divide them
constexpr int32_t HINF = 0x3fffffff;       // label of a pixel that cannot reach t
constexpr int N_INST_PLANES = 8;           // e, h, rt, fR, fD, src0, slope, ct
constexpr int N_IMG_PLANES = 2;            // w_h, w_v
enum Plane { P_E = 0, P_H = 1, P_RT = 2, P_FR = 3, P_FD = 4, P_SRC0 = 5, P_SLOPE = 6, P_CT = 7 };

// instance phases
enum Phase { PH_BFS = 0, PH_PR = 1, PH_DONE = 2 };
// tile queue states
enum TState { T_IDLE = 0, T_QUEUED = 1, T_RUNNING = 2, T_DIRTY = 3 };
// global error flags
enum GErr { GE_STALL = 1, GE_RING = 2, GE_SLOT = 4, GE_TIMEOUT = 8 };
// per-instance validation flags (set by the pad/init kernels)
enum VFlag { VF_NEG = 1, VF_OVERFLOW = 2, VF_SLOPE = 4, VF_BADCAP = 8 };

struct DevInst {                 // read-only during a solve
    int32_t H, W, pitch, rows;
    int32_t image;
    int32_t tiles_x, tiles_y, n_tiles;
    int32_t tile_base;
    int32_t n_lambda;
    int32_t hcap;                // labels >= hcap become HINF (= H*W)
    int32_t pad_;
    int64_t plane_off;           // int32 elements from the instance-plane base
    int64_t img_off;             // int32 elements from the image-plane base
    int64_t mask_off;            // bytes from the mask base
};

struct InstState {               // mutable during a solve
    int32_t phase, k, epoch, outstanding;
    int32_t active, want_bfs, status, vflags;
    unsigned long long flow;     // int64 two's complement
    int32_t pr_since, pad_;
    unsigned long long pr_visits, bfs_visits, epochs, visits_step;
};

struct TileState {
    int32_t state, epoch, lam, active;
};

struct Globals {
    unsigned long long head, tail;
    unsigned long long round_end;
    long long pending;
    unsigned long long completed;
    int32_t err, round_mode;
    unsigned long long items;    // total items processed (stat)
    unsigned long long t_start;  // %globaltimer at the start of the launch
};

struct Params {
    int32_t *planes;             // instance planes base
    const int32_t *img;          // image planes base
    uint8_t *masks;
    const DevInst *inst;
    InstState *ist;
    TileState *tiles;
    const int32_t *tile_inst;
    int32_t *ring;
    const int32_t *lambdas;      // [n_inst][max_lambdas]
    long long *flows;            // [n_inst][max_lambdas]
    Globals *g;
    const int32_t *img_flags;    // [n_images] validation flags of set_capacities
    int32_t *inst_flags;         // [n_inst] validation flags of set_terminals
    unsigned long long ring_mask;
    int32_t n_inst, n_tiles_total, max_lambdas, sweeps;
    int32_t relabel_pct, tile_h;
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
cudaError_t launch_begin_round(const Params &P, cudaStream_t s);
int worker_warps_per_block();
cudaError_t worker_occupancy(int tile_h, int *blocks_per_sm);

}  // namespace pmf
