// Device code: tiled push-relabel with a global-relabel wavefront BFS, GGT
// lambda warm start and exact residual-reachability cut extraction, driven by
// a persistent kernel that pops (instance, tile) work items from a device
// queue.
//
// Method (Sections 2-3 of the paper): maximum flow / minimum cut of the
// 4-connected grid graph of each instance; the paper solves it with a GPU
// push-relabel (Goldberg-Tarjan) and batches many (seed, lambda) problems into
// one "supergraph" (Section 3.1) so that one launch fills the GPU.  The
// parametric lambda schedule (Section 2.1) reuses the previous flow when the
// source capacities grow (Gallo-Grigoriadis-Tarjan, cited in Sections 2.1, 3).
//
// State of one instance (int32 planes, row pitch a multiple of 32):
//   e   excess of each pixel (source arcs are kept saturated: cs(p, lambda)
//       is pushed into e when lambda is applied)
//   h   height label (HINF = cannot reach t; set exactly by the BFS)
//   rt  residual capacity of p->t
//   fR  net flow on the edge p -> right neighbour, in [-w_h, w_h]
//   fD  net flow on the edge p -> down neighbour,  in [-w_v, w_v]
// so residual(p->right) = w_h - fR, residual(right->p) = w_h + fR, etc.
//
// A work item is one tile of 32 x TH pixels handled by ONE warp: lane = column,
// each lane keeps its TH pixels in registers.  Horizontal neighbours are
// reached with warp shuffles, vertical ones are in the same thread; nothing in
// a tile visit needs a block barrier, so every warp of the GPU is an
// independent worker.
//
// Concurrency argument.  Two tiles may be visited at the same time.  A tile
// only ever changes its own pixels' h and rt, pushes flow OUT across its
// border (which only raises the neighbour's excess and only moves the shared
// edge flow in the outward direction) and writes the pixels and edges on its
// border back as atomic deltas.  Adding the deltas of both sides keeps every
// edge flow inside [-w, w] and every excess >= 0, so the global state is
// always a valid preflow; stale halo heights can only cost extra work.  The
// result is certified independently of the labels: a lambda step ends only
// when an exact BFS from t (the global relabel) finds no pixel with positive
// excess that can reach t.  At that point the flow into t is a maximum flow
// value and the pixels the BFS cannot reach form the maximal source set.
#include <cstdint>

#include <cooperative_groups.h>
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstring>
#include <mutex>

#include "pmf.h"
#include "pmf_internal.h"

namespace cg = cooperative_groups;

namespace pmf {

#define FULL_MASK 0xffffffffu

__device__ __forceinline__ unsigned long long gtime_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ int ldv(const int *p) { return *(const volatile int *)p; }
// load with acquire semantics at device scope: every later load of this thread
// sees what the writer wrote before its release (a fence, then this word)
__device__ __forceinline__ int ld_acquire(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long ldv64(const unsigned long long *p) {
    return *(const volatile unsigned long long *)p;
}
__device__ __forceinline__ long long ldv64s(const long long *p) { return *(const volatile long long *)p; }
// a load of data that stays fixed while a batch solves (descriptors, lambda
// table, capacity planes): through the non-coherent read-only path in batch
// kernels; through L2 in the server kernel (SV), where the host rewrites a
// slot's data between the requests that occupy it
template <bool SV, typename T>
__device__ __forceinline__ T ldro(const T *p) {
    if constexpr (SV) return __ldcg(p);
    else return __ldg(p);
}

// per-warp scratch: values of the two border columns at load (their updates
// are written back as deltas)
template <int TH>
struct WarpSmem {
    int e0[2][TH];          // excess of lanes 1 and 30 at load
    int f0[2][TH];          // fR of lane 0 (left border edge) and lane 30 (right border edge)
    int dl0[2][BFS_ROWS];   // relabel: labels of lanes 1 and 30 at load (a strip's side columns)
    int d[BFS_ROWS][33];    // relabel: the strip's labels, row i / column l (one pad column, so
                            // a lane walking a row and a lane walking a column both hit 32 banks)
};

// --------------------------------------------------------------------------
// staged strip loads (batch kernels): a relabel strip's first visit of an
// epoch reads seven planes over its 32 rows.  Instead of per-lane loads in
// batches of a few rows (one memory round trip each), one elected lane starts
// two tensor copies (the instance's e, h, rt, fR, fD box and the image's w_h,
// w_v box) into a shared-memory buffer of the block, and the warp waits once on
// an mbarrier for all of it.  One buffer per block: a warp that finds it taken
// loads per lane as before.
// --------------------------------------------------------------------------
struct StripStage {
    int32_t *buf;                   // [5 + 2 planes][BFS_ROWS][STAGE_BOX_W]
    unsigned long long *bar;        // completion of the copies into buf
    int *lock;                      // 0 free, 1 held by a warp of the block, 2 out of use
    int *uses;                      // completed uses of buf (parity of the barrier's phase)
};
constexpr unsigned long long STAGE_WAIT_NS = 1000000000ULL;   // a copy not done by then is an error

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// block start (thread 0): the barrier expects one arrival per phase, plus the
// copies' bytes
__device__ __forceinline__ void stage_init(const StripStage &SS) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(SS.bar)) : "memory");
    *SS.lock = 0;
    *SS.uses = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void stage_copy(uint32_t dst, const unsigned char *tmap, int x, int y, int z,
                                           uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
        "l"(tmap), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}

// lane 0: takes the buffer if it is free and starts the copies of the box whose
// first column is x0 (a multiple of 4; may be negative: the copy fills zeros
// outside the plane) and first row y0.  Returns the barrier parity to wait
// for, or -1 when the buffer is taken.
__device__ int stage_begin(const Params &P, const StripStage &SS, int inst, int image, int x0, int y0) {
    if (atomicCAS(SS.lock, 0, 1) != 0) return -1;
    __threadfence_block();
    const int parity = *(volatile int *)SS.uses & 1;
    const uint32_t bar = smem_addr(SS.bar);
    // the planes were written through the generic proxy (by other warps, seen
    // through this lane's acquires); the copies read through the async proxy
    asm volatile("fence.proxy.async.global;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(STAGE_BYTES) : "memory");
    stage_copy(smem_addr(SS.buf), P.tmaps + (size_t)inst * TMAP_BYTES, x0, y0, P_E, bar);
    stage_copy(smem_addr(SS.buf + STAGE_INST_PLANES * BFS_ROWS * STAGE_BOX_W),
               P.tmaps + (size_t)(P.n_inst + image) * TMAP_BYTES, x0, y0, 0, bar);
    return parity;
}

// whole warp: wait until every lane sees the copies done (the barrier's phase
// of this parity complete); false after STAGE_WAIT_NS
__device__ bool stage_wait(const StripStage &SS, int parity) {
    const uint32_t bar = smem_addr(SS.bar);
    unsigned long long t0 = 0;
    for (int spin = 0;; ++spin) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (__all_sync(FULL_MASK, ok != 0)) return true;
        unsigned long long now = gtime_ns();
        now = __shfl_sync(FULL_MASK, now, 0);
        if (t0 == 0) t0 = now;
        else if (now - t0 > STAGE_WAIT_NS) return false;
    }
}

// whole warp, after every lane has read the buffer: hand it back
__device__ __forceinline__ void stage_end(const StripStage &SS) {
    __syncwarp();
    if ((threadIdx.x & 31) == 0) {
        *(volatile int *)SS.uses = *(volatile int *)SS.uses + 1;
        __threadfence_block();
        atomicExch(SS.lock, 0);
    }
    __syncwarp();
}

// --------------------------------------------------------------------------
// device work queue: ring of tile ids, ticket counters head/tail
// --------------------------------------------------------------------------
__device__ __forceinline__ bool slot_wait(const Params &P, volatile int *slot, bool want_empty,
                                          int *out) {
    unsigned long long t0 = 0;
    int spins = 0;
    for (;;) {
        int v = *slot;
        if (want_empty ? (v == -1) : (v != -1)) { *out = v; return true; }
        if (++spins > 32) {
            __nanosleep(64);
            unsigned long long now = gtime_ns();
            if (t0 == 0) t0 = now;
            else if (now - t0 > (unsigned long long)P.stall_ns) {
                atomicOr(&P.g->err, GE_SLOT);
                return false;
            }
        }
    }
}

__device__ void push1(const Params &P, int v) {   // one lane
    unsigned long long t = atomicAdd(&P.g->tail, 1ULL);
    volatile int *slot = (volatile int *)(P.ring + (t & P.ring_mask));
    int dummy;
    if (!slot_wait(P, slot, true, &dummy)) return;
    *slot = v;
}

// persistent mode: every pop takes a ticket with one atomicAdd and then waits
// on its own ring slot, so idle warps poll distinct addresses.  The ring has
// room for every tile plus every resident warp's ticket, so a slot is never
// shared by two outstanding tickets.
__device__ int ring_pop_ticket(const Params &P) {   // one lane; -1 = stop
    Globals *G = P.g;
    const unsigned long long h = atomicAdd(&G->head, 1ULL);
    volatile int *slot = (volatile int *)(P.ring + (h & P.ring_mask));
    unsigned ns = 32;
    unsigned long long last_tail = ~0ULL, last_prog = ~0ULL, t_since = 0;
    int last_pend = -1;
    for (unsigned polls = 1;; ++polls) {
        const int v = *slot;
        if (v != -1) {
            *slot = -1;
            __threadfence();
            return v;
        }
        if ((polls & 3) == 0) {
            if (ldv(&G->err)) return -1;
            const int ndone = ldv(&G->inst_done);
            if (ndone >= P.n_inst) return -1;
            const unsigned long long now = gtime_ns();
            if (now - ldv64(&G->t_start) > (unsigned long long)P.max_ns) {
                atomicOr(&G->err, GE_TIMEOUT);
                return -1;
            }
            const unsigned long long tl = ldv64(&G->tail), pg = ldv64(&G->progress);
            if (tl != last_tail || ndone != last_pend || pg != last_prog) {
                last_tail = tl;
                last_pend = ndone;
                last_prog = pg;
                t_since = now;
            } else if (now - t_since > (unsigned long long)P.stall_ns) {
                atomicOr(&G->err, GE_STALL);
                return -1;
            }
        }
        __nanosleep(ns);
        if (ns < (unsigned)P.poll_ns) ns <<= 1;
    }
}

// round mode (host-polled): claim only tickets below the round's end
__device__ int ring_pop_round(const Params &P) {   // one lane; -1 = round over
    Globals *G = P.g;
    for (int it = 0; it < (1 << 20); ++it) {
        if (ldv(&G->err)) return -1;
        const unsigned long long h = ldv64(&G->head);
        const unsigned long long re = ldv64(&G->round_end);
        if (h >= re) return -1;
        if (atomicCAS(&G->head, h, h + 1) == h) {
            volatile int *slot = (volatile int *)(P.ring + (h & P.ring_mask));
            int v;
            if (!slot_wait(P, slot, false, &v)) return -1;
            *slot = -1;
            __threadfence();
            return v;
        }
    }
    atomicOr(&G->err, GE_RING);
    return -1;
}

// read-only instance descriptor through the non-coherent (texture) path; the
// table is written before the worker launch and never during it
template <bool SV>
__device__ __forceinline__ DevInst load_inst(const Params &P, int inst) {
    static_assert(sizeof(DevInst) % 16 == 0, "DevInst is loaded as int4s");
    DevInst d;
    const int4 *src = reinterpret_cast<const int4 *>(P.inst + inst);
    int4 *dst = reinterpret_cast<int4 *>(&d);
#pragma unroll
    for (int j = 0; j < (int)(sizeof(DevInst) / 16); ++j) dst[j] = ldro<SV>(src + j);
    return d;
}

// --------------------------------------------------------------------------
// instance phase changes, run by the warp that finished the instance's last
// outstanding item (so nothing of this instance is queued or running)
// --------------------------------------------------------------------------
// Queue tiles of an instance for its new phase.  Each tile is claimed with a
// CAS from IDLE: tiles released from earlier chunks start running at once and
// may already have woken a neighbour that this loop has not reached yet; that
// neighbour is queued (or running) and must not be queued twice.
constexpr int SCAN_U = 8;   // tile records each lane reads per step (loads in flight)

__device__ int count_active_tiles(const Params &P, const DevInst &D) {
    const int lane = threadIdx.x & 31;
    int total = 0;
    for (int c0 = 0; c0 < D.n_tiles; c0 += 32 * SCAN_U) {
        int a[SCAN_U];
#pragma unroll
        for (int u = 0; u < SCAN_U; ++u) {
            const int j = c0 + u * 32 + lane;
            a[u] = j < D.n_tiles ? ldv(&P.tiles[D.tile_base + j].active) : 0;
        }
#pragma unroll
        for (int u = 0; u < SCAN_U; ++u) total += __popc(__ballot_sync(FULL_MASK, a[u] > 0));
    }
    return total;
}

// claim the selected tiles (one per lane) and append them to the ring
__device__ __forceinline__ void enqueue_chunk(const Params &P, int inst, int t, bool sel) {
    const int lane = threadIdx.x & 31;
    if (sel) sel = atomicCAS(&P.tiles[t].state, T_IDLE, T_QUEUED) == T_IDLE;
    const unsigned m = __ballot_sync(FULL_MASK, sel);
    const int cnt = __popc(m);
    if (cnt == 0) return;
    unsigned long long base = 0;
    if (lane == 0) {
        atomicAdd(&P.ist[inst].outstanding, cnt);
        __threadfence();
        base = atomicAdd(&P.g->tail, (unsigned long long)cnt);
    }
    base = __shfl_sync(FULL_MASK, base, 0);
    __syncwarp();
    if (sel) {
        __threadfence();
        const unsigned long long tk = base + __popc(m & ((1u << lane) - 1u));
        volatile int *slot = (volatile int *)(P.ring + (tk & P.ring_mask));
        int dummy;
        if (slot_wait(P, slot, true, &dummy)) *slot = t;
    }
}

__device__ void enqueue_tiles(const Params &P, int inst, const DevInst &D, bool only_active, bool leaders_only) {
    const int lane = threadIdx.x & 31;
    if (leaders_only) {
        // leader j of the relabel strips: strip row j / tiles_x, tile column j % tiles_x
        const int span = BFS_ROWS / P.tile_h;
        for (int c0 = 0; c0 < D.n_leads; c0 += 32) {
            const int j = c0 + lane;
            const int r = j / D.tiles_x;
            const int t = D.tile_base + (r * span) * D.tiles_x + (j - r * D.tiles_x);
            enqueue_chunk(P, inst, t, j < D.n_leads);
        }
        return;
    }
    for (int c0 = 0; c0 < D.n_tiles; c0 += 32 * SCAN_U) {
        bool sel[SCAN_U];
#pragma unroll
        for (int u = 0; u < SCAN_U; ++u) {
            const int j = c0 + u * 32 + lane;
            sel[u] = j < D.n_tiles && (!only_active || ldv(&P.tiles[D.tile_base + j].active) > 0);
        }
#pragma unroll 1
        for (int u = 0; u < SCAN_U; ++u) enqueue_chunk(P, inst, D.tile_base + c0 + u * 32 + lane, sel[u]);
    }
}

__device__ void trace(const Params &P, int inst, int event, volatile InstState *S) {
    if (!P.trace) return;
    const unsigned long long i = atomicAdd(&P.g->trace_n, 1ULL);
    if (i >= (unsigned long long)TRACE_CAP) return;
    TraceEvent e;
    e.t_ns = gtime_ns();
    e.inst = inst;
    e.event = event;
    e.k = S->k;
    e.epoch = S->epoch;
    e.pr_visits = (long long)S->pr_visits;
    e.bfs_visits = (long long)S->bfs_visits;
    e.flow = (long long)S->flow;
    e.active = S->active;
    e.pad_ = 0;
    P.trace[i] = e;
}

// An instance has reached PH_DONE: tell the host (a word in mapped host
// memory), after everything the instance wrote (its masks and flow values,
// made visible at device scope by the visits' fences) is ordered before it.
__device__ void mark_done(const Params &P, int inst, int status) {
    __threadfence_system();
    if (P.done_flags) *(volatile int32_t *)(P.done_flags + inst) = 1 + status;
}

// A forked instance whose parent stopped before forking it never starts:
// it and every instance forked from it finish with the parent's status.
template <bool SV>
__device__ __noinline__ void cancel_forks(const Params &P, int child, int status) {
    for (int c = child, it = 0; c >= 0 && it < P.n_inst; ++it) {
        volatile InstState *C = P.ist + c;
        if (C->phase != PH_WAIT) break;
        C->status = status;
        C->phase = PH_DONE;
        atomicAdd(&P.g->inst_done, 1);
        mark_done(P, c, status);
        c = ldro<SV>(&P.inst[c].fork_child);
    }
}

// Start a forked instance once its parent's copy pass has written the
// parent's state into its planes: it continues from the parent's lambda
// (flow value, largest distance and labels as the parent certified them) with
// the warm-start pass of its own first lambda.  Returns true when the child's
// strips all finished before the guard was released: the caller must then run
// the child's next phase change.
template <bool SV>
__device__ __noinline__ bool start_fork(const Params &P, int child, volatile InstState *parent) {
    const int lane = threadIdx.x & 31;
    volatile InstState *C = P.ist + child;
    const DevInst DC = load_inst<SV>(P, child);
    int go = 0;
    if (lane == 0) {
        if (C->status != PMF_OK) {
            const int st = C->status;
            C->phase = PH_WAIT;             // cancel_forks finishes it with its own status
            cancel_forks<SV>(P, child, st);
        } else {
            C->flow = parent->flow;
            C->dmax = parent->dmax;
            C->lam_prev = parent->lam_prev;
            C->k = 0;
            C->want_bfs = 0;
            C->step_mark = 0;
            C->phase = PH_WARM;
            go = 1;
            atomicAdd(&P.ist[child].outstanding, 1);   // guard while its strips are queued
        }
        __threadfence();
    }
    go = __shfl_sync(FULL_MASK, go, 0);
    if (!go) return false;
    __syncwarp();
    enqueue_tiles(P, child, DC, false, true);
    int last = 0;
    if (lane == 0) {
        __threadfence();
        last = atomicAdd(&P.ist[child].outstanding, -1) == 1;
    }
    return __shfl_sync(FULL_MASK, last, 0) != 0;
}

// One phase change.  Returns true when the items it queued had all finished
// before it let go of its guard: the caller is then the instance's last
// finisher again and must run the next phase change itself.  *other is set to
// an instance (a child it forked) whose own phase change the caller must run.
template <bool SV>
__device__ bool transition_once(const Params &P, int inst, int *other) {
    const int lane = threadIdx.x & 31;
    volatile InstState *S = P.ist + inst;
    const DevInst D = load_inst<SV>(P, inst);
    __threadfence();
    int mode = 0;   // 0 nothing, 1 all tiles, 2 tiles with active pixels
    int fork_now = 0;
    if (lane == 0) {
        const int phase = S->phase;
        if (S->status != PMF_OK) {
            S->phase = PH_DONE;
            atomicAdd(&P.g->inst_done, 1);
            mark_done(P, inst, S->status);
            cancel_forks<SV>(P, D.fork_child, S->status);
        } else if (phase == PH_SETUP) {        // server: set up, start the first global relabel
            S->dmax = 0;
            S->phase = PH_BFS;
            mode = 1;
        } else if (phase == PH_WARM) {         // the step's first push/relabel phase
            S->phase = PH_PR;
            S->pr_mark = S->pr_visits;
            S->want_bfs = 0;
            mode = 2;
            trace(P, inst, TR_PR_START, S);
        } else if (phase == PH_PR) {           // start a global relabel
            S->dmax = 0;
            S->epoch = S->epoch + 1;
            S->epochs = S->epochs + 1;
            S->phase = PH_BFS;
            S->want_bfs = 0;
            mode = 1;
            trace(P, inst, TR_BFS_START, S);
        } else if (phase == PH_BFS && S->active == 0 && D.cut_rule == 1) {
            // certified, and the caller swapped s and t: the flow value is
            // final; the cut comes from a forward pass over the strips
            P.flows[(size_t)inst * P.max_lambdas + S->k] = (long long)S->flow;
            S->epoch = S->epoch + 1;
            S->phase = PH_FWD;
            mode = 1;
        } else if (phase == PH_COPY) {
            // the copy pass is over: start the child, then go on
            fork_now = 1;
            if (S->k >= D.n_lambda) {
                S->phase = PH_DONE;
                atomicAdd(&P.g->inst_done, 1);
                mark_done(P, inst, PMF_OK);
                trace(P, inst, TR_DONE, S);
            } else {
                S->phase = PH_WARM;
                mode = 1;
            }
        } else if (phase == PH_BFS || phase == PH_FWD) {
            const unsigned long long visits = S->pr_visits + S->bfs_visits;
            if (phase == PH_FWD || S->active == 0) {   // lambda step certified: record, advance
                const int k = S->k;
                if (phase == PH_BFS) P.flows[(size_t)inst * P.max_lambdas + k] = (long long)S->flow;
                S->k = k + 1;
                S->lam_prev = ldro<SV>(P.lambdas + (size_t)inst * P.max_lambdas + k);
                S->step_mark = visits;
                trace(P, inst, TR_STEP_DONE, S);
                if (D.fork_child >= 0 && k == D.fork_k) {
                    // copy this state into the forked instance, strip by strip
                    S->phase = PH_COPY;
                    mode = 1;
                } else if (k + 1 >= D.n_lambda) {
                    S->phase = PH_DONE;
                    atomicAdd(&P.g->inst_done, 1);
                    mark_done(P, inst, PMF_OK);
                    trace(P, inst, TR_DONE, S);
                } else {
                    // raise the source capacities to the next lambda, strip by strip
                    S->phase = PH_WARM;
                    mode = 1;
                }
            } else if ((long long)(visits - S->step_mark) > P.max_visits_per_tile * (long long)D.n_tiles) {
                S->status = PMF_ERR_NOT_CONVERGED;
                S->phase = PH_DONE;
                atomicAdd(&P.g->inst_done, 1);
                mark_done(P, inst, PMF_ERR_NOT_CONVERGED);
                trace(P, inst, TR_NOT_CONVERGED, S);
                cancel_forks<SV>(P, D.fork_child, PMF_ERR_NOT_CONVERGED);
            } else {
                S->phase = PH_PR;
                S->pr_mark = S->pr_visits;
                S->want_bfs = 0;
                mode = 2;
                trace(P, inst, TR_PR_START, S);
            }
        }
        __threadfence();
    }
    mode = __shfl_sync(FULL_MASK, mode, 0);
    fork_now = __shfl_sync(FULL_MASK, fork_now, 0);
    if (fork_now && start_fork<SV>(P, D.fork_child, S)) *other = D.fork_child;
    if (!mode) return false;
    // the phase's parameters are published before any of its tiles can run
    const int n = (mode == 2) ? count_active_tiles(P, D) : D.n_tiles;
    if (lane == 0 && S->phase == PH_PR) {
        // a push/relabel phase may spend relabel_pct% of the tiles it starts
        // with (at least 4 visits) before the next global relabel: when only
        // a few tiles hold active pixels, stranded excess is otherwise pushed
        // back and forth between them long before a relabel removes it.  With
        // relabel_reach set, the budget is at least that percentage of the
        // largest exact distance of the last relabel: the excess left in the
        // long tail of a hard step then gets visits enough to travel that far
        // instead of a global relabel every few hundred visits
        long long bud = (long long)P.relabel_pct * n / 100 + P.relabel_extra;
        bud = max(bud, (long long)P.relabel_reach * S->dmax / 100);
        S->pr_budget = (int)(bud < 4 ? 4 : (bud > (1LL << 30) ? (1LL << 30) : bud));
        // labels far above every exact distance of the last relabel belong
        // to excess that keeps climbing without reaching t: park it until
        // the next relabel (which re-activates whatever can still reach t)
        const long long cap = (long long)S->dmax + P.label_slack;
        S->lab_cap = (P.label_slack <= 0 || cap >= D.hcap) ? D.hcap : (int)cap;
    }
    // a guard item keeps the phase open while its tiles are queued: tiles of
    // the first chunks may run and retire before later chunks are counted,
    // and without it the instance's count could reach zero in between and a
    // second phase change would start while this one is still queueing
    if (lane == 0) atomicAdd(&P.ist[inst].outstanding, 1);
    __threadfence();
    __syncwarp();
    // a relabel, forward, warm-start or copy pass works on strips (their
    // leader tiles are queued); push/relabel on tiles
    const int ph = S->phase;
    enqueue_tiles(P, inst, D, mode == 2,
                  ph == PH_BFS || ph == PH_FWD || ph == PH_WARM || ph == PH_COPY || ph == PH_SETUP);
    int last = 0;
    if (lane == 0) {
        __threadfence();
        last = atomicAdd(&P.ist[inst].outstanding, -1) == 1;
    }
    return __shfl_sync(FULL_MASK, last, 0) != 0;
}

// Phase changes of an instance, run by the warp that retired its last
// outstanding item.  Repeats while a phase ends before its own queueing did
// (a phase with no tiles to queue, or tiles that all finished meanwhile);
// every repetition is a phase change that the visit watchdog counts, and a
// hard cap flags the launch if it is ever reached.  A forked child whose
// strips all finished before its start was complete is run the same way.
template <bool SV>
__device__ void transition(const Params &P, int inst) {
    int cur = inst, pending = -1;
    for (int it = 0; it < (1 << 16); ++it) {
        int other = -1;
        const bool again = transition_once<SV>(P, cur, &other);
        if (other >= 0) pending = other;
        if (again) continue;
        if (pending < 0) return;
        cur = pending;
        pending = -1;
    }
    if ((threadIdx.x & 31) == 0) atomicOr(&P.g->err, GE_RING);
}

// finish an item: wake neighbours, requeue or retire the tile, maybe change
// the instance's phase.  Lanes 0-3 wake the four neighbours in parallel, lane 4
// settles this tile; the instance's outstanding count changes once by the net
// number of items (pushed - 1), BEFORE the new items become visible.
// With keep set, one new item (this tile if it runs again, else the first
// woken neighbour) is returned to the caller, which runs it next on the same
// warp instead of queueing it: chains of dependent visits then stay on an SM
// whose caches hold the code and the neighbourhood (the queue otherwise hands
// an item to the warp that has been idle longest).  Returns -1 otherwise.
// OOL: the phase change is called out of line (see worker_kernel).
template <bool SV>
__device__ __noinline__ void transition_ool(const Params &P, int inst) {
    transition<SV>(P, inst);
}

template <bool SV, bool OOL = false>
__device__ int finish(const Params &P, int g, int inst, int phase, bool requeue, unsigned nb,
                      const DevInst &D, bool keep) {
    const int lane = threadIdx.x & 31;
    volatile InstState *IS = P.ist + inst;
    bool allow = false;
    if (IS->status == PMF_OK) {
        if (phase == PH_BFS || phase == PH_FWD) allow = true;
        else if (phase == PH_PR) allow = (IS->want_bfs == 0);
    }
    int item = -1;
    if (allow && lane < 4 && ((nb >> lane) & 1u)) {
        const int lt = g - D.tile_base;
        const int ty = lt / D.tiles_x, tx = lt - ty * D.tiles_x;
        int t = -1;
        const int vs = (phase == PH_BFS || phase == PH_FWD) ? BFS_ROWS / P.tile_h : 1;   // strips
        if (lane == 0 && ty >= vs) t = g - vs * D.tiles_x;
        if (lane == 1 && ty + vs < D.tiles_y) t = g + vs * D.tiles_x;
        if (lane == 2 && tx > 0) t = g - 1;
        if (lane == 3 && tx < D.tiles_x - 1) t = g + 1;
        if (t >= 0) {
            int *st = &P.tiles[t].state;
            for (int it = 0; it < 1024; ++it) {
                const int old = atomicCAS(st, T_IDLE, T_QUEUED);
                if (old == T_IDLE) { item = t; break; }
                if (old == T_QUEUED || old == T_DIRTY) break;
                const int o2 = atomicCAS(st, T_RUNNING, T_DIRTY);   // its visitor will run it again
                if (o2 != T_IDLE) break;
                if (it == 1023) atomicOr(&P.g->err, GE_RING);
            }
        }
    }
    if (lane == 4) {
        int *st = &P.tiles[g].state;
        if (requeue && allow) {
            atomicExch(st, T_QUEUED);
            item = g;
        } else {
            const int old = atomicCAS(st, T_RUNNING, T_IDLE);
            if (old == T_DIRTY) {
                if (allow) { atomicExch(st, T_QUEUED); item = g; }
                else atomicExch(st, T_IDLE);
            }
        }
    }
    const unsigned pm_all = __ballot_sync(FULL_MASK, item >= 0);
    const int k = __popc(pm_all);
    // the kept item: lane 4 (this tile) if set, else the lowest lane's
    const int kl = !keep || pm_all == 0 ? -1 : ((pm_all >> 4) & 1u) ? 4 : __ffs(pm_all) - 1;
    const int kept = kl >= 0 ? __shfl_sync(FULL_MASK, item, kl) : -1;
    const unsigned pm = kl >= 0 ? pm_all & ~(1u << kl) : pm_all;
    const int kq = __popc(pm);           // items for the ring
    int trans = 0;
    unsigned long long base = 0;
    if (lane == 0) {
        const int delta = k - 1;
        if (delta < 0) {                 // the count can only reach zero when it falls
            const int old = atomicAdd(&P.ist[inst].outstanding, delta);
            trans = (old + delta == 0);
        } else if (delta > 0) {          // no result needed: a reduction, no round trip
            atomicAdd(&P.ist[inst].outstanding, delta);
        }
        if (kq) {
            __threadfence();
            base = atomicAdd(&P.g->tail, (unsigned long long)kq);
        }
    }
    base = __shfl_sync(FULL_MASK, base, 0);
    trans = __shfl_sync(FULL_MASK, trans, 0);
    __syncwarp();
    if ((pm >> lane) & 1u) {
        const unsigned long long tk = base + __popc(pm & ((1u << lane) - 1u));
        volatile int *slot = (volatile int *)(P.ring + (tk & P.ring_mask));
        int dummy;
        if (slot_wait(P, slot, true, &dummy)) *slot = item;
    }
    if (trans) {                         // only when k == 0, so nothing is kept
        if constexpr (OOL) transition_ool<SV>(P, inst);
        else transition<SV>(P, inst);
    }
    return kept;
}

// --------------------------------------------------------------------------
// push/relabel visit of one tile (Goldberg-Tarjan push and relabel operations,
// the solver the paper runs through NPPI, Section 3)
// --------------------------------------------------------------------------
// Tile geometry.  A tile is TH rows x 30 interior columns.  Lane l of the warp
// holds column X = 30*tx - 1 + l in registers (TH pixels); lanes 0 and 31 are
// "ghost" lanes holding the neighbouring tiles' border columns: their labels
// are read-only for the visit, flow pushed into them accumulates in their
// registers and is added to the neighbour's state at write-back.  Every lane
// runs the same straight-line code, so the independent rows of a sweep
// overlap.
struct TileGeo {
    int ty, tx, y0, X, lane;
    bool ghost, inb;
};

__device__ __forceinline__ TileGeo tile_geo(int g, const DevInst &D, int TH) {
    TileGeo t;
    t.lane = threadIdx.x & 31;
    const int lt = g - D.tile_base;
    t.ty = lt / D.tiles_x;
    t.tx = lt - t.ty * D.tiles_x;
    t.y0 = t.ty * TH;
    t.X = t.tx * TILE_IN - 1 + t.lane;
    t.ghost = (t.lane == 0) || (t.lane == 31);
    t.inb = (t.X >= 0) && (t.X < D.pitch);
    return t;
}

// --------------------------------------------------------------------------
// push/relabel visit of one tile (Goldberg-Tarjan push and relabel operations,
// the solver the paper runs through NPPI, Section 3)
// --------------------------------------------------------------------------
template <int TH, int PO, bool SV>
__device__ void pr_visit(const Params &P, WarpSmem<TH> &S, int g, int inst, const DevInst &D,
                         int kcur, bool &self_active, unsigned &nbmask) {
    const TileGeo T = tile_geo(g, D, TH);
    const int lane = T.lane;
    const bool own = T.inb && !T.ghost;     // a pixel this tile updates
    const int pitch = D.pitch;
    const size_t PS = (size_t)D.rows * pitch;
    int *base = P.planes + D.plane_off;
    int *E = base + P_E * PS, *Hh = base + P_H * PS, *RT = base + P_RT * PS;
    int *FR = base + P_FR * PS, *FD = base + P_FD * PS;
    const int *WH = P.img + D.img_off;
    const int *WV = WH + PS;
    const long long c_start = P.trace ? clock64() : 0;

    int e[TH], h[TH], rt[TH], fr[TH], fd[TH], wh[TH], wv[TH];
    long long srt0 = 0;
#pragma unroll
    for (int i = 0; i < TH; ++i) {
        const size_t idx = (size_t)(T.y0 + i) * pitch + T.X;
        e[i] = own ? __ldcg(E + idx) : 0;
        h[i] = T.inb ? __ldcg(Hh + idx) : HINF;
        rt[i] = own ? __ldcg(RT + idx) : 0;
        fr[i] = (T.inb && lane != 31) ? __ldcg(FR + idx) : 0;
        fd[i] = own ? __ldcg(FD + idx) : 0;
        wh[i] = (T.inb && lane != 31) ? ldro<SV>(WH + idx) : 0;
        wv[i] = own ? ldro<SV>(WV + idx) : 0;
        srt0 += rt[i];
    }
    const int e0top = e[0], e0bot = e[TH - 1], fd0b = fd[TH - 1];
    if (lane == 1 || lane == 30) {
        const int c = lane == 1 ? 0 : 1;
#pragma unroll
        for (int i = 0; i < TH; ++i) S.e0[c][i] = e[i];
    }
    if (lane == 0 || lane == 30) {
        const int c = lane == 0 ? 0 : 1;
#pragma unroll
        for (int i = 0; i < TH; ++i) S.f0[c][i] = fr[i];
    }

    // rows above and below the tile
    int hT = HINF, wvT = 0, fdT = 0, hB = HINF;
    if (own && T.y0 > 0) {
        const size_t j = (size_t)(T.y0 - 1) * pitch + T.X;
        hT = __ldcg(Hh + j);
        wvT = ldro<SV>(WV + j);
        fdT = __ldcg(FD + j);
    }
    const int fdT0 = fdT;
    if (own && T.y0 + TH < D.rows) hB = __ldcg(Hh + (size_t)(T.y0 + TH) * pitch + T.X);
    __syncwarp();

    int outU = 0, outD = 0;
    const int hcap = min(D.hcap, *(volatile int *)&P.ist[inst].lab_cap);
    unsigned nsw = 0;
    bool any_act;
    {
        bool a = false;
#pragma unroll
        for (int i = 0; i < TH; ++i) a |= (e[i] > 0 && h[i] < HINF);
        any_act = __any_sync(FULL_MASK, a);
    }
    const long long c_loaded = P.trace ? clock64() + (e[0] & 0) : 0;
    for (int sw = 0; sw < P.sweeps && any_act; ++sw) {
        ++nsw;
        // Every row of a sweep works from the state at the start of the sweep
        // (Jacobi order), so the rows are independent.  Heights do not change
        // during the push phase, so the two ends of an edge never push
        // against each other.  Push phase: an active pixel sends excess to t
        // first, then to lower neighbours along residual arcs.
        if constexpr (PO == 1) {
            // Chain order: excess may move on in the same sweep after it
            // arrives.  Every push is still along a residual arc to a lower
            // neighbour from a pixel holding the excess it sends, so this is
            // the same push operation in a different order.
#pragma unroll
            for (int i = 0; i < TH; ++i) {             // to t
                const bool a = own && e[i] > 0 && h[i] < HINF;
                const int dT = a ? min(e[i], rt[i]) : 0;
                e[i] -= dT;
                rt[i] -= dT;
            }
            // the sweeps alternate: even ones push down the columns and
            // rightwards along the rows, odd ones up and leftwards.  A sweep
            // is a chain of dependent steps (its rows are the only
            // independent work), so half the steps make each sweep about
            // half as long, and over two sweeps excess still moves every way.
            // The last sweep of a visit with an odd number of sweeps goes
            // every way, so that each visit offers every admissible arc a push
            // (a pixel whose only admissible arcs lead up or left must not
            // wait for a sweep that never comes).
            const bool even = (sw & 1) == 0;
            const bool full = (P.sweeps & 1) && sw == P.sweeps - 1;
            if (even || full) {
#pragma unroll
            for (int i = 0; i < TH; ++i) {             // down the column, top to bottom
                const int hD = (i < TH - 1) ? h[i + 1] : hB;
                const int rD = wv[i] - fd[i];
                const bool a = own && e[i] > 0 && h[i] < HINF;
                const int d = (a && rD > 0 && hD < h[i]) ? min(e[i], rD) : 0;
                e[i] -= d;
                fd[i] += d;
                if (i < TH - 1) e[i + 1] += d; else outD += d;
            }
            }
            if (!even || full) {
#pragma unroll
            for (int i = TH - 1; i >= 0; --i) {        // up the column, bottom to top
                const int hU = (i > 0) ? h[i - 1] : hT;
                const int rU = (i > 0) ? (wv[i - 1] + fd[i - 1]) : (wvT + fdT);
                const bool a = own && e[i] > 0 && h[i] < HINF;
                const int d = (a && rU > 0 && hU < h[i]) ? min(e[i], rU) : 0;
                e[i] -= d;
                if (i > 0) { e[i - 1] += d; fd[i - 1] -= d; } else { outU += d; fdT -= d; }
            }
            }
            // along the row: a pixel forwards min(its excess + what arrives
            // from the previous pixel of the run, residual of its arc) when
            // the arc leads to a lower neighbour.  Such maps x -> min(a + x, b)
            // compose into the same form, (a1, b1) then (a2, b2) giving
            // (a1 + a2, min(a2 + b1, b2)), so one warp scan yields every
            // pixel's outflow.  a is clamped at 2^29: residuals are below
            // 2^29, so a larger a never changes the result.
            constexpr int ACL = 1 << 29;
            // all rows scan in step (independent shuffles overlap); a direction
            // is skipped when no pixel of the tile can send anything along it
            if (even || full) {                        // rightwards
                int A[TH], B[TH];
                bool go = false;
#pragma unroll
                for (int i = 0; i < TH; ++i) {
                    const int hR = __shfl_down_sync(FULL_MASK, h[i], 1);
                    const int rR = wh[i] - fr[i];
                    const bool live = own && h[i] < HINF;
                    A[i] = live ? min(e[i], ACL) : 0;
                    B[i] = (live && rR > 0 && hR < h[i]) ? rR : 0;
                    go |= A[i] > 0 && B[i] > 0;
                }
                if (__any_sync(FULL_MASK, go)) {
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
                        for (int i = 0; i < TH; ++i) {
                            const int A2 = __shfl_up_sync(FULL_MASK, A[i], o);
                            const int B2 = __shfl_up_sync(FULL_MASK, B[i], o);
                            if (lane >= o) {
                                B[i] = min(A[i] + B2, B[i]);
                                A[i] = min(A2 + A[i], ACL);
                            }
                        }
                    }
#pragma unroll
                    for (int i = 0; i < TH; ++i) {
                        const int out = min(A[i], B[i]);
                        const int in = __shfl_up_sync(FULL_MASK, out, 1);
                        e[i] += (lane > 0 ? in : 0) - out;
                        fr[i] += out;
                    }
                }
            }
            if (!even || full) {                       // leftwards
                int A[TH], B[TH];
                bool go = false;
#pragma unroll
                for (int i = 0; i < TH; ++i) {
                    const int hL = __shfl_up_sync(FULL_MASK, h[i], 1);
                    const int rL = __shfl_up_sync(FULL_MASK, wh[i] + fr[i], 1);
                    const bool live = own && h[i] < HINF;
                    A[i] = live ? min(e[i], ACL) : 0;
                    B[i] = (live && rL > 0 && hL < h[i]) ? rL : 0;
                    go |= A[i] > 0 && B[i] > 0;
                }
                if (__any_sync(FULL_MASK, go)) {
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
                        for (int i = 0; i < TH; ++i) {
                            const int A2 = __shfl_down_sync(FULL_MASK, A[i], o);
                            const int B2 = __shfl_down_sync(FULL_MASK, B[i], o);
                            if (lane + o < 32) {
                                B[i] = min(A[i] + B2, B[i]);
                                A[i] = min(A2 + A[i], ACL);
                            }
                        }
                    }
#pragma unroll
                    for (int i = 0; i < TH; ++i) {
                        const int out = min(A[i], B[i]);
                        const int in = __shfl_down_sync(FULL_MASK, out, 1);
                        e[i] += (lane < 31 ? in : 0) - out;
                        fr[i] -= (lane < 31 ? in : 0);
                    }
                }
            }
        } else {
            int dDa[TH], dUa[TH];
    #pragma unroll
            for (int i = 0; i < TH; ++i) {
                const int hp = h[i];
                const int hL = __shfl_up_sync(FULL_MASK, hp, 1);
                const int hR = __shfl_down_sync(FULL_MASK, hp, 1);
                const int rL = __shfl_up_sync(FULL_MASK, wh[i] + fr[i], 1);
                const int hU = (i > 0) ? h[i - 1] : hT;
                const int hD = (i < TH - 1) ? h[i + 1] : hB;
                const int rR = wh[i] - fr[i];
                const int rD = wv[i] - fd[i];
                const int rU = (i > 0) ? (wv[i - 1] + fd[i - 1]) : (wvT + fdT);
                const bool a = own && e[i] > 0 && hp < HINF;
                int ex = a ? e[i] : 0;
                const int dT = min(ex, rt[i]);
                ex -= dT;
                const int dD = (rD > 0 && hD < hp) ? min(ex, rD) : 0;
                ex -= dD;
                const int dR = (rR > 0 && hR < hp) ? min(ex, rR) : 0;
                ex -= dR;
                const int dU = (rU > 0 && hU < hp) ? min(ex, rU) : 0;
                ex -= dU;
                const int dL = (rL > 0 && hL < hp) ? min(ex, rL) : 0;
                e[i] -= dT + dD + dR + dU + dL;
                rt[i] -= dT;
                dDa[i] = dD;
                dUa[i] = dU;
                // horizontal transfers stay inside the row (ghost lanes collect
                // what crosses the tile's left and right borders)
                fr[i] += dR;
                const int inR = __shfl_up_sync(FULL_MASK, dR, 1);
                const int inL = __shfl_down_sync(FULL_MASK, dL, 1);
                e[i] += (lane > 0 ? inR : 0) + (lane < 31 ? inL : 0);
                fr[i] -= (lane < 31 ? inL : 0);
            }
            // vertical transfers, after every row has decided
    #pragma unroll
            for (int i = 0; i < TH; ++i) {
                fd[i] += dDa[i];
                if (i < TH - 1) e[i + 1] += dDa[i]; else outD += dDa[i];
                if (i > 0) { e[i - 1] += dUa[i]; fd[i - 1] -= dUa[i]; } else { outU += dUa[i]; fdT -= dUa[i]; }
            }
        }
        // relabel phase: an active pixel without an admissible arc moves to
        // one above its lowest residual neighbour (t has label 0); all rows
        // read the heights of the start of the sweep
        int hn[TH];
        bool act = false;
#pragma unroll
        for (int i = 0; i < TH; ++i) {
            const int hp = h[i];
            const int hL = __shfl_up_sync(FULL_MASK, hp, 1);
            const int hR = __shfl_down_sync(FULL_MASK, hp, 1);
            const int rL = __shfl_up_sync(FULL_MASK, wh[i] + fr[i], 1);
            const int hU = (i > 0) ? h[i - 1] : hT;
            const int hD = (i < TH - 1) ? h[i + 1] : hB;
            const int rU = (i > 0) ? (wv[i - 1] + fd[i - 1]) : (wvT + fdT);
            int hmin = rt[i] > 0 ? 0 : HINF;
            hmin = (wv[i] - fd[i] > 0) ? min(hmin, hD) : hmin;
            hmin = (wh[i] - fr[i] > 0) ? min(hmin, hR) : hmin;
            hmin = (rU > 0) ? min(hmin, hU) : hmin;
            hmin = (rL > 0) ? min(hmin, hL) : hmin;
            const bool a = own && e[i] > 0 && hp < HINF;
            const int nh = (hmin >= HINF - 1 || hmin + 1 >= hcap) ? HINF : hmin + 1;
            hn[i] = (a && hmin >= hp) ? nh : hp;
            act |= a && hn[i] < HINF;
        }
#pragma unroll
        for (int i = 0; i < TH; ++i) h[i] = hn[i];
        any_act = __any_sync(FULL_MASK, act);
    }

    // write back; pixels and edges on the tile border as atomic deltas
    const long long c_swept = P.trace ? clock64() : 0;
    long long srt1 = 0;
    bool act = false, got_l = false, got_r = false;
#pragma unroll
    for (int i = 0; i < TH; ++i) {
        const size_t idx = (size_t)(T.y0 + i) * pitch + T.X;
        srt1 += rt[i];
        act |= own && (e[i] > 0 && h[i] < HINF);
        if (own) {
            int e0 = e[i];
            bool perim = true;
            if (lane == 1) e0 = S.e0[0][i];
            else if (lane == 30) e0 = S.e0[1][i];
            else if (i == 0) e0 = e0top;
            else if (i == TH - 1) e0 = e0bot;
            else perim = false;
            if (perim) {
                if (e[i] != e0) atomicAdd(E + idx, e[i] - e0);
            } else {
                __stcg(E + idx, e[i]);
            }
            __stcg(Hh + idx, h[i]);
            __stcg(RT + idx, rt[i]);
            if (lane == 30) {
                if (fr[i] != S.f0[1][i]) atomicAdd(FR + idx, fr[i] - S.f0[1][i]);
            } else {
                __stcg(FR + idx, fr[i]);
            }
            if (i == TH - 1) {
                if (fd[i] != fd0b) atomicAdd(FD + idx, fd[i] - fd0b);
            } else {
                __stcg(FD + idx, fd[i]);
            }
        } else if (T.inb) {
            // ghost lane: excess pushed across the border, and (left) the
            // flow on the left border edge, owned by the neighbour's pixel
            if (e[i]) {
                atomicAdd(E + idx, e[i]);
                if (lane == 0) got_l = true; else got_r = true;
            }
            if (lane == 0 && fr[i] != S.f0[0][i]) atomicAdd(FR + idx, fr[i] - S.f0[0][i]);
        }
    }
    if (own && T.y0 > 0) {
        const size_t j = (size_t)(T.y0 - 1) * pitch + T.X;
        if (outU) atomicAdd(E + j, outU);
        if (fdT != fdT0) atomicAdd(FD + j, fdT - fdT0);
    }
    if (own && outD && T.y0 + TH < D.rows) atomicAdd(E + (size_t)(T.y0 + TH) * pitch + T.X, outD);
    unsigned nb = 0;
    if (__any_sync(FULL_MASK, outU > 0)) nb |= 1;
    if (__any_sync(FULL_MASK, outD > 0)) nb |= 2;
    if (__any_sync(FULL_MASK, got_l)) nb |= 4;
    if (__any_sync(FULL_MASK, got_r)) nb |= 8;
    nbmask = nb;
    self_active = __any_sync(FULL_MASK, act);

    long long df = srt0 - srt1;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) df += __shfl_down_sync(FULL_MASK, df, o);
    if (P.trace) {
        __threadfence();
        const long long c_end = clock64();
        if (lane == 0) {
            atomicAdd(&P.g->prof[5], (unsigned long long)(c_loaded - c_start));
            atomicAdd(&P.g->prof[6], (unsigned long long)(c_swept - c_loaded));
            atomicAdd(&P.g->prof[7], (unsigned long long)(c_end - c_swept));
        }
    }
    if (lane == 0) {
        if (P.trace) atomicAdd(&P.g->prof[4], (unsigned long long)nsw);
        if (df) atomicAdd(&P.ist[inst].flow, (unsigned long long)df);
        const unsigned long long v = atomicAdd(&P.ist[inst].pr_visits, 1ULL) + 1;
        const long long since = (long long)(v - *(volatile unsigned long long *)&P.ist[inst].pr_mark);
        if (since >= (long long)*(volatile int *)&P.ist[inst].pr_budget) P.ist[inst].want_bfs = 1;
    }
}

// --------------------------------------------------------------------------
// warm-start visit: GGT's change of the terminal capacities from lambda_{k-1}
// to lambda_k (Section 2.1's monotone case keeps the labels valid) for one
// strip.  Rising source capacities: the new capacity becomes excess, and the
// part the sink arc can take goes to t.  Falling sink capacities: the sink
// arc's residual shrinks, and where the arc carried more than its new capacity
// the surplus flow is taken back from t and becomes excess.  Either way each
// member tile's count of active pixels (excess and a finite label) is set for
// the step's first push/relabel phase.  Nothing else of the instance runs in
// this phase, so every value is written directly.
// --------------------------------------------------------------------------
template <int TH, bool SINK, bool SV>
__device__ void warm_visit(const Params &P, int g, int inst, const DevInst &D, int kcur) {
    constexpr int BR = BFS_ROWS;
    constexpr int SPAN = BR / TH;
    const TileGeo T = tile_geo(g, D, TH);
    const int lane = T.lane;
    const bool own = T.inb && !T.ghost;
    const int pitch = D.pitch;
    const size_t PS = (size_t)D.rows * pitch;
    int *base = P.planes + D.plane_off;
    int *E = base + P_E * PS, *RT = base + P_RT * PS;
    const int *Hh = base + P_H * PS, *SLOPE = base + P_SLOPE * PS;
    const int *L = P.lambdas + (size_t)inst * P.max_lambdas;
    // from the lambda the state was certified at: the previous step's, or for
    // a forked instance's first step its parent's
    const int dl = ldro<SV>(L + kcur) - ldv(&P.ist[inst].lam_prev);
    // which terminal arcs follow lambda (only kernels built for batches with
    // falling sink capacities look)
    const bool sink_side = SINK && ldro<SV>(&P.inst[inst].slope_side) != 0;
    // the member tiles' counts as last written, kept in the strip record
    int32_t *cnt_rec = P.strip_cache + (size_t)(D.lead_base + (T.ty / SPAN) * D.tiles_x + T.tx) * STRIP_REC_WORDS
                       + RW_CNT * 32;
    const int cnt_old = lane < SPAN ? ldv(cnt_rec + lane) : 0;
    long long sent = 0;
    unsigned live = 0;   // bit i: row i's pixel is active after the raise
    constexpr int LB = 8;
#pragma unroll 1
    for (int c0 = 0; c0 < BR; c0 += LB) {
        int e[LB], rt[LB], h[LB], sl[LB];
#pragma unroll
        for (int j = 0; j < LB; ++j) {
            const int y = T.y0 + c0 + j;
            const bool ok = own && y < D.rows;
            const size_t idx = (size_t)y * pitch + T.X;
            e[j] = ok ? __ldcg(E + idx) : 0;
            rt[j] = ok ? __ldcg(RT + idx) : 0;
            h[j] = ok ? __ldcg(Hh + idx) : HINF;
            sl[j] = ok ? ldro<SV>(SLOPE + idx) : 0;
        }
#pragma unroll
        for (int j = 0; j < LB; ++j) {
            const int y = T.y0 + c0 + j;
            const bool ok = own && y < D.rows;
            const int d = sl[j] * dl;
            if constexpr (SINK) {
                // the source capacity rises by up or the sink capacity falls
                // by dn; a sink arc left carrying more than its capacity gives
                // the surplus back to its pixel; then the part of the excess
                // the sink arc can take goes to t
                const int up = sink_side ? 0 : d, dn = sink_side ? d : 0;
                const int back = max(dn - rt[j], 0);
                const int rt1 = max(rt[j] - dn, 0);
                const int e1 = e[j] + up + back;
                const int m = min(e1, rt1);
                const int en = e1 - m, rtn = rt1 - m;
                if (ok && d) {
                    const size_t idx = (size_t)y * pitch + T.X;
                    if (en != e[j]) __stcg(E + idx, en);
                    if (rtn != rt[j]) __stcg(RT + idx, rtn);
                }
                sent += ok ? m - back : 0;
                live |= (ok && en > 0 && h[j] < HINF) ? (1u << (c0 + j)) : 0u;
            } else {
                // the raise becomes excess; the part the sink arc can take goes to t
                const int m = min(e[j] + d, rt[j]);
                const int en = e[j] + d - m;
                if (ok && d) {
                    const size_t idx = (size_t)y * pitch + T.X;
                    __stcg(E + idx, en);
                    if (m) __stcg(RT + idx, rt[j] - m);
                }
                sent += ok ? m : 0;
                live |= (ok && en > 0 && h[j] < HINF) ? (1u << (c0 + j)) : 0u;
            }
        }
    }
    int cnt[SPAN];
    constexpr unsigned TMASK = (TH == 32) ? 0xffffffffu : ((1u << TH) - 1u);
#pragma unroll
    for (int j = 0; j < SPAN; ++j)
        cnt[j] = (int)__reduce_add_sync(FULL_MASK, (unsigned)__popc(live & (TMASK << (j * TH))));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sent += __shfl_down_sync(FULL_MASK, sent, o);
    __threadfence();
    __syncwarp();
    int delta = 0;
    if (lane < SPAN && T.ty + lane < D.tiles_y) {
        int mine = 0;
#pragma unroll
        for (int j = 0; j < SPAN; ++j) mine = (j == lane) ? cnt[j] : mine;
        *(volatile int *)&P.tiles[g + lane * D.tiles_x].active = mine;
        __stcg(cnt_rec + lane, mine);
        delta = mine - cnt_old;
    }
#pragma unroll
    for (int o = SPAN / 2; o > 0; o >>= 1) delta += __shfl_down_sync(FULL_MASK, delta, o);
    if (lane == 0) {
        if (delta) atomicAdd(&P.ist[inst].active, delta);
        if (sent) atomicAdd(&P.ist[inst].flow, (unsigned long long)sent);
        atomicAdd(&P.ist[inst].warm_visits, 1ULL);
    }
}

template <int TH, bool SINK, bool SV>
__device__ __noinline__ void warm_visit_ool(const Params &P, int g, int inst, const DevInst &D, int kcur) {
    warm_visit<TH, SINK, SV>(P, g, inst, D, kcur);
}

// --------------------------------------------------------------------------
// copy visit: one strip of a parent's state (e, h, rt, fR, fD and the terminal
// planes src0, slope, ct) into the instance forked from it.  Both instances
// have the same image, so the same layout; nothing of either runs meanwhile
// (the parent is in its copy pass, the child waits for it).
// --------------------------------------------------------------------------
template <int TH, bool SV>
__device__ __noinline__ void copy_visit(const Params &P, int g, int inst, const DevInst &D) {
    constexpr int BR = BFS_ROWS;
    const TileGeo T = tile_geo(g, D, TH);
    const bool own = T.inb && !T.ghost;
    const int pitch = D.pitch;
    const size_t PS = (size_t)D.rows * pitch;
    const int *src = P.planes + D.plane_off;
    int *dst = P.planes + ldro<SV>(&P.inst[D.fork_child].plane_off);
    constexpr int LB = 4;
#pragma unroll 1
    for (int c0 = 0; c0 < BR; c0 += LB) {
        int v[LB][N_INST_PLANES];
#pragma unroll
        for (int j = 0; j < LB; ++j) {
            const int y = T.y0 + c0 + j;
            const bool ok = own && y < D.rows;
            const size_t idx = (size_t)y * pitch + T.X;
#pragma unroll
            for (int q = 0; q < N_INST_PLANES; ++q) v[j][q] = ok ? __ldcg(src + q * PS + idx) : 0;
        }
#pragma unroll
        for (int j = 0; j < LB; ++j) {
            const int y = T.y0 + c0 + j;
            if (own && y < D.rows) {
                const size_t idx = (size_t)y * pitch + T.X;
#pragma unroll
                for (int q = 0; q < N_INST_PLANES; ++q) __stcg(dst + q * PS + idx, v[j][q]);
            }
        }
    }
}

// --------------------------------------------------------------------------
// global-relabel visit: one strip's share of the BFS from t over reverse
// residual arcs (exact distances by label-correcting relaxation to a fixpoint;
// unreachable pixels keep HINF).  A strip is a column of BFS_ROWS / TH tiles
// (30 x 32 pixels), queued through its top ("leader") tile; each lane keeps the
// strip column's 32 labels in registers and the residual arcs as bit masks, so
// one visit carries distances across 32 rows.  It also writes the cut mask of
// the current lambda (1 = cannot reach t = source side) and each member tile's
// count of active pixels for the push/relabel phase that may follow.
// --------------------------------------------------------------------------
template <int TH, bool FWD, bool SV>
__device__ void bfs_visit(const Params &P, WarpSmem<TH> &S, const StripStage &SS, int g, int inst,
                          const DevInst &D, int epoch, int kcur, bool &self_again, unsigned &nbmask) {
    constexpr int BR = BFS_ROWS;
    constexpr int SPAN = BR / TH;
    const TileGeo T = tile_geo(g, D, TH);
    const int lane = T.lane;
    const bool own = T.inb && !T.ghost;
    const int pitch = D.pitch;
    const size_t PS = (size_t)D.rows * pitch;
    int *base = P.planes + D.plane_off;
    const int *E = base + P_E * PS, *RT = base + P_RT * PS;
    const int *FR = base + P_FR * PS, *FD = base + P_FD * PS;
    int *Hh = base + P_H * PS;
    const int *WH = P.img + D.img_off;
    const int *WV = WH + PS;
    TileState *TS = P.tiles + g;
    const int vstride = SPAN * D.tiles_x;
    const long long c_start = P.trace ? clock64() : 0;

    // labels of a neighbouring strip count only once it has been visited in
    // this relabel epoch (otherwise they are left over from push/relabel).  A
    // visit stores its labels and record, fences, then stores its epoch; the
    // epochs are read with acquire loads, so the reads of those labels and of
    // this strip's own record that follow see them (each lane acquires the
    // epochs whose data it reads)
    const bool own_valid = ld_acquire(&TS->epoch) == epoch;
    const bool vT = T.ty >= SPAN && ld_acquire(&P.tiles[g - vstride].epoch) == epoch;
    const bool vB = T.ty + SPAN < D.tiles_y && ld_acquire(&P.tiles[g + vstride].epoch) == epoch;
    bool vX = own_valid;
    if (lane == 0) vX = T.tx > 0 && ld_acquire(&P.tiles[g - 1].epoch) == epoch;
    if (lane == 31) vX = T.tx < D.tiles_x - 1 && ld_acquire(&P.tiles[g + 1].epoch) == epoch;
    // the member tiles' active counts as last written (lane j: tile j), kept in
    // the strip record so that replacing them needs no read after the relaxation;
    // the previous writer may be on another SM, so the read bypasses L1
    const int32_t *cnt_rec = P.strip_cache + (size_t)(D.lead_base + (T.ty / SPAN) * D.tiles_x + T.tx) * STRIP_REC_WORDS
                             + RW_CNT * 32;
    const int cnt_old = (!FWD && lane < SPAN) ? ldv(cnt_rec + lane) : 0;

    // This strip's record: the arc bit masks and border residuals its first
    // visit of the epoch found (arcs do not change during a relabel phase),
    // and, for the forward pass, its labels as its last visit left them (a
    // relabel keeps its labels in the label plane only).  Words [k][lane]:
    // k = 0..5 masks R, D, U, E, Q, V; 6..8 residuals up from row 0, down
    // into row 0, up into the last row; 9 + i the label of row i;
    // RW_CNT the member tiles' active counts.
    int32_t *REC = P.strip_cache + (size_t)(D.lead_base + (T.ty / SPAN) * D.tiles_x + T.tx) * STRIP_REC_WORDS;
    // the forward pass keeps its labels in the records only (the distances to
    // t in the label plane stay for push/relabel), so it reads neighbouring
    // strips' labels there: the left strip's column 30, the right strip's
    // column 1, the last row of the strip above, the first row of the one below
    const int32_t *REC_L = REC - STRIP_REC_WORDS, *REC_R = REC + STRIP_REC_WORDS;
    const int32_t *REC_T = REC - (size_t)D.tiles_x * STRIP_REC_WORDS;
    const int32_t *REC_B = REC + (size_t)D.tiles_x * STRIP_REC_WORDS;
    auto ghost_label = [&](int i) -> int {      // lanes 0 and 31, row i, neighbour visited
        if constexpr (FWD) return __ldcg(lane == 0 ? REC_L + (9 + i) * 32 + 30 : REC_R + (9 + i) * 32 + 1);
        else return __ldcg(Hh + (size_t)(T.y0 + i) * pitch + T.X);
    };
    int(*Dl)[33] = S.d;
    unsigned bR = 0, bD = 0, bU = 0, bE = 0, bQ = 0, bV = 0;
    int hT = HINF, res_up0 = 0, res_down_above = 0, res_up_last = 0, dold_top = HINF, dold_bot = HINF;
    const bool below = T.y0 + BR < D.rows;
    int hB = HINF;
    if (own && vB && below) {
        if constexpr (FWD) hB = __ldcg(REC_B + 9 * 32 + lane);
        else hB = __ldcg(Hh + (size_t)(T.y0 + BR) * pitch + T.X);
    }
    if (own_valid) {
        // a second visit in this epoch: masks and residuals from the record,
        // labels of this strip's own columns as its last visit left them (the
        // label plane; the forward pass: the record), the ghost columns' from
        // the neighbouring strips' labels
        bR = (unsigned)__ldcg(REC + 0 * 32 + lane);
        bD = (unsigned)__ldcg(REC + 1 * 32 + lane);
        bU = (unsigned)__ldcg(REC + 2 * 32 + lane);
        bE = (unsigned)__ldcg(REC + 3 * 32 + lane);
        bQ = (unsigned)__ldcg(REC + 4 * 32 + lane);
        bV = (unsigned)__ldcg(REC + 5 * 32 + lane);
        res_up0 = __ldcg(REC + 6 * 32 + lane);
        res_down_above = __ldcg(REC + 7 * 32 + lane);
        res_up_last = __ldcg(REC + 8 * 32 + lane);
        if (own && T.y0 > 0 && vT) {
            if constexpr (FWD) hT = __ldcg(REC_T + (9 + BR - 1) * 32 + lane);
            else hT = __ldcg(Hh + (size_t)(T.y0 - 1) * pitch + T.X);
        }
        constexpr int LH = 32;
#pragma unroll 1
        for (int c0 = 0; c0 < BR; c0 += LH) {
            int dv[LH];
#pragma unroll
            for (int j = 0; j < LH; ++j) {
                const int i = c0 + j;
                const bool rowok = T.y0 + i < D.rows;
                if constexpr (FWD) dv[j] = own ? __ldcg(REC + (9 + i) * 32 + lane) : (T.inb && rowok && vX) ? ghost_label(i) : HINF;
                else dv[j] = (T.inb && rowok && (own || vX)) ? __ldcg(Hh + (size_t)(T.y0 + i) * pitch + T.X) : HINF;
            }
#pragma unroll
            for (int j = 0; j < LH; ++j) {
                const int i = c0 + j;
                if (i == 0) dold_top = dv[j];
                if (i == BR - 1) dold_bot = dv[j];
                Dl[i][lane] = dv[j];
                if (lane == 1) S.dl0[0][i] = dv[j];
                if (lane == 30) S.dl0[1][i] = dv[j];
            }
        }
    } else {
    // staged loads: lane 0 starts the copies of the strip's box before the
    // loads of the row above, so that both are in flight together.  The box
    // starts at lane 0's column rounded down to a multiple of 4; lane l reads
    // box column sx + l.  Lane 0 first acquires the right neighbour's epoch as
    // well (lane 31 did, for the labels of its column that the copy brings in).
    int parity = -1;
    const int xl = T.tx * TILE_IN - 1;
    const int x0 = xl - (((xl % 4) + 4) % 4);
    const int sx = xl - x0;
    if constexpr (!SV) {
        if (P.strip_stage) {
            __syncwarp();
            if (lane == 0) {
                if (T.tx < D.tiles_x - 1) (void)ld_acquire(&P.tiles[g + 1].epoch);
                parity = stage_begin(P, SS, inst, D.image, x0, T.y0);
            }
            parity = __shfl_sync(FULL_MASK, parity, 0);
        }
    }
    // the row above the strip: residual of the arcs up and down across the border
    if (own && T.y0 > 0) {
        const size_t j = (size_t)(T.y0 - 1) * pitch + T.X;
        const int wvT = ldro<SV>(WV + j), fdT = __ldcg(FD + j);
        res_up0 = wvT + fdT;          // row 0 -> above
        res_down_above = wvT - fdT;   // above -> row 0
        if (vT) {
            if constexpr (FWD) hT = __ldcg(REC_T + (9 + BR - 1) * 32 + lane);
            else hT = __ldcg(Hh + j);
        }
    }

    // residual arcs as bit masks (bit i = row i): R/L/D/U = from the pixel to
    // that neighbour; E = positive excess; Q = arc from this column to the one
    // on its right (read by lane 1 from ghost lane 0); V = arc from the right
    // neighbour into this column (used by lane 30).  Labels live in this
    // lane's own column of the warp's shared memory.
    bool staged = parity >= 0;
    if (staged && !stage_wait(SS, parity)) {
        // the copies did not finish in time: an error for the launch; wait once
        // more for them, then either use the data or retire the buffer (a copy
        // might still land in it) and load per lane
        if (lane == 0) atomicOr(&P.g->err, GE_STAGE);
        staged = stage_wait(SS, parity);
        if (!staged && lane == 0) atomicExch(SS.lock, 2);
    }
    int prev_up = res_up0;
    // 4 rows at a time: every global load of a batch is issued before any of
    // its results is used or written to shared memory, so a batch costs one
    // memory round trip instead of one per row
    constexpr int LB = 4;
    constexpr int PW = BFS_ROWS * STAGE_BOX_W;     // words per staged plane
#pragma unroll 1
    for (int c0 = 0; c0 < BR; c0 += LB) {
        int fr[LB], wh[LB], fd[LB], wv[LB], rt[LB], ev[LB], dv[LB];
        if (staged) {
#pragma unroll
            for (int j = 0; j < LB; ++j) {
                const bool rowok = T.y0 + c0 + j < D.rows;
                const bool ldc = T.inb && rowok && lane != 31;
                const bool ldo = own && rowok;
                const int32_t *sb = SS.buf + (c0 + j) * STAGE_BOX_W + sx + lane;
                fr[j] = ldc ? sb[(P_FR - P_E) * PW] : 0;
                wh[j] = ldc ? sb[STAGE_INST_PLANES * PW] : 0;
                fd[j] = ldo ? sb[(P_FD - P_E) * PW] : 0;
                wv[j] = ldo ? sb[(STAGE_INST_PLANES + 1) * PW] : 0;
                rt[j] = ldo ? sb[(P_RT - P_E) * PW] : 0;
                ev[j] = ldo ? sb[0] : 0;
                if constexpr (FWD) dv[j] = (T.inb && rowok && vX) ? ghost_label(c0 + j) : HINF;
                else dv[j] = (T.inb && rowok && vX) ? sb[(P_H - P_E) * PW] : HINF;
            }
        } else {
#pragma unroll
            for (int j = 0; j < LB; ++j) {
                const int y = T.y0 + c0 + j;
                const bool rowok = y < D.rows;
                const size_t idx = (size_t)y * pitch + T.X;
                const bool ldc = T.inb && rowok && lane != 31;
                const bool ldo = own && rowok;
                fr[j] = ldc ? __ldcg(FR + idx) : 0;
                wh[j] = ldc ? ldro<SV>(WH + idx) : 0;
                fd[j] = ldo ? __ldcg(FD + idx) : 0;
                wv[j] = ldo ? ldro<SV>(WV + idx) : 0;
                rt[j] = ldo ? __ldcg(RT + idx) : 0;
                ev[j] = ldo ? __ldcg(E + idx) : 0;
                if constexpr (FWD) dv[j] = (T.inb && rowok && vX) ? ghost_label(c0 + j) : HINF;
                else dv[j] = (T.inb && rowok && vX) ? __ldcg(Hh + idx) : HINF;
            }
        }
#pragma unroll
        for (int j = 0; j < LB; ++j) {
            const int i = c0 + j;
            const bool rowok = T.y0 + i < D.rows;
            const bool ldc = T.inb && rowok && lane != 31;
            const bool ldo = own && rowok;
            const unsigned bit = 1u << i;
            bR |= (ldo && wh[j] - fr[j] > 0) ? bit : 0u;
            bD |= (ldo && wv[j] - fd[j] > 0) ? bit : 0u;
            bU |= (ldo && prev_up > 0) ? bit : 0u;
            bE |= (ldo && ev[j] > 0) ? bit : 0u;
            bQ |= (ldc && wh[j] - fr[j] > 0) ? bit : 0u;
            bV |= (ldc && wh[j] + fr[j] > 0) ? bit : 0u;
            prev_up = wv[j] + fd[j];
            if (i == BR - 1) res_up_last = wv[j] + fd[j];     // below -> last row
            if (i == 0) dold_top = dv[j];
            if (i == BR - 1) dold_bot = dv[j];
            // distances to t start at 1 where the arc to t is residual; the
            // forward pass starts at 0 on pixels holding excess
            if constexpr (FWD) Dl[i][lane] = (ldo && ev[j] > 0) ? 0 : dv[j];
            else Dl[i][lane] = (ldo && rt[j] > 0) ? min(dv[j], 1) : dv[j];
            if (lane == 1) S.dl0[0][i] = dv[j];
            if (lane == 30) S.dl0[1][i] = dv[j];
        }
    }
    if (staged) stage_end(SS);
    // the record's masks and residuals for the epoch's later visits
    __stcg(REC + 0 * 32 + lane, (int)bR);
    __stcg(REC + 1 * 32 + lane, (int)bD);
    __stcg(REC + 2 * 32 + lane, (int)bU);
    __stcg(REC + 3 * 32 + lane, (int)bE);
    __stcg(REC + 4 * 32 + lane, (int)bQ);
    __stcg(REC + 5 * 32 + lane, (int)bV);
    __stcg(REC + 6 * 32 + lane, res_up0);
    __stcg(REC + 7 * 32 + lane, res_down_above);
    __stcg(REC + 8 * 32 + lane, res_up_last);
    }
    // arcs from this column to the one on its left: the left column's
    // residual w + f towards it (bV of the lane on the left)
    unsigned bL = __shfl_up_sync(FULL_MASK, bV, 1);
    if (!own) bL = 0;
    // arcs the relaxation follows, as masks: for distances to t the arcs out
    // of the pixel (d(p) <= d(q) + 1 for p -> q); for the forward pass the arcs
    // into it (d(p) <= d(q) + 1 for q -> p): from above (row i-1 down to i), from
    // below (i+1 up to i), from the left column and from the right column
    unsigned aU = bU, aD = bD, aL = bL, aR = bR;
    if constexpr (FWD) {
        aU = (bD << 1) | (res_down_above > 0 ? 1u : 0u);
        aD = (bU >> 1) | (res_up_last > 0 ? 0x80000000u : 0u);
        aL = __shfl_up_sync(FULL_MASK, bQ, 1);
        aR = bV;
        if (!own) aU = aD = aL = aR = 0;
    }

    // d(p) <= d(q) + 1 for every residual arc p -> q, relaxed to the fixpoint
    // (ghost lanes only supply their neighbours' labels)
    // the same arcs by row for the transposed horizontal passes: lane i gets
    // row i's right and left arcs as bit masks over the columns
    unsigned rowR = 0, rowL = 0;
#pragma unroll 4
    for (int i = 0; i < BR; ++i) {
        const unsigned r = __ballot_sync(FULL_MASK, (aR >> i) & 1u);
        const unsigned l = __ballot_sync(FULL_MASK, (aL >> i) & 1u);
        if (lane == i) { rowR = r; rowL = l; }
    }
    const long long c_loaded = P.trace ? clock64() + (Dl[0][lane] & 0) : 0;
    bool capped = true;
    int rounds = 0;
    for (int it = 0; it < 4 * BR; ++it) {
        ++rounds;
        // A pass down and a pass up a column leave every vertical constraint
        // met (on a path, one sweep each way gives the exact distances), and
        // the two row passes do the same for the horizontal ones.  So a round
        // whose row passes change nothing ends at the fixpoint: only their
        // changes are tracked.
        bool ch = false;
        {   // vertical: a pass down and a pass up the column, 8 rows at a time
            constexpr int CH = 8;
            int up = hT;
#pragma unroll 1
            for (int c0 = 0; c0 < BR; c0 += CH) {       // from above along arcs p -> up
                int d[CH];
#pragma unroll
                for (int j = 0; j < CH; ++j) d[j] = Dl[c0 + j][lane];
#pragma unroll
                for (int j = 0; j < CH; ++j) {
                    const bool bb = ((aU >> (c0 + j)) & 1u) && up + 1 < d[j];
                    d[j] = bb ? up + 1 : d[j];
                    up = d[j];
                }
#pragma unroll
                for (int j = 0; j < CH; ++j) Dl[c0 + j][lane] = d[j];
            }
            int dn = hB;
#pragma unroll 1
            for (int c0 = BR - CH; c0 >= 0; c0 -= CH) { // from below along arcs p -> down
                int d[CH];
#pragma unroll
                for (int j = 0; j < CH; ++j) d[j] = Dl[c0 + j][lane];
#pragma unroll
                for (int j = CH - 1; j >= 0; --j) {
                    const bool bb = ((aD >> (c0 + j)) & 1u) && dn + 1 < d[j];
                    d[j] = bb ? dn + 1 : d[j];
                    dn = d[j];
                }
#pragma unroll
                for (int j = 0; j < CH; ++j) Dl[c0 + j][lane] = d[j];
            }
        }
        // horizontal, transposed: lane i walks row i left to right along arcs
        // p -> p-1 and back along arcs p -> p+1 (ghost columns 0 and 31 have
        // no arcs of their own, so they only pass their labels in)
        __syncwarp();
        if (lane < BR) {
            int prev = Dl[lane][0];
#pragma unroll 8
            for (int c = 1; c < 32; ++c) {
                int v = Dl[lane][c];
                if (((rowL >> c) & 1u) && prev + 1 < v) { v = prev + 1; Dl[lane][c] = v; ch = true; }
                prev = v;
            }
            prev = Dl[lane][31];
#pragma unroll 8
            for (int c = 30; c >= 0; --c) {
                int v = Dl[lane][c];
                if (((rowR >> c) & 1u) && prev + 1 < v) { v = prev + 1; Dl[lane][c] = v; ch = true; }
                prev = v;
            }
        }
        __syncwarp();
        if (!__any_sync(FULL_MASK, ch)) { capped = false; break; }
    }
    self_again = capped;
    const long long c_relaxed = P.trace ? clock64() : 0;

    // which neighbouring strips can now improve: a border pixel p got a smaller
    // label than the neighbour q could have read, q -> p is residual and q's
    // label is above d(p) + 1
    bool wT = false, wB = false, wL = false, wR = false;
    const int d_top = Dl[0][lane], d_bot = Dl[BR - 1][lane];
    // the arc across the border that the neighbour's label would follow
    const bool arcT = FWD ? res_up0 > 0 : res_down_above > 0;
    const bool arcB = FWD ? ((bD >> (BR - 1)) & 1u) != 0 : res_up_last > 0;
    if (own && T.y0 > 0) wT = d_top < dold_top && arcT && d_top + 1 < hT;
    if (own && below && T.ty + SPAN < D.tiles_y)
        wB = d_bot < dold_bot && arcB && d_bot + 1 < hB;
    const unsigned qbits = __shfl_up_sync(FULL_MASK, bQ, 1);     // lane 0's arcs into lane 1
    // lanes 1 and 30 compare their column with the ghost column beside it
    if ((lane == 1 && own && T.tx > 0) || (lane == 30 && own && T.tx < D.tiles_x - 1)) {
        const int side = lane == 1 ? 0 : 1, q = lane == 1 ? 0 : 31;
        const unsigned arcs = FWD ? (lane == 1 ? bL : bR) : (lane == 1 ? qbits : bV);
        bool w = false;
#pragma unroll 8
        for (int i = 0; i < BR; ++i) {
            const int di = Dl[i][lane];
            w |= di < S.dl0[side][i] && ((arcs >> i) & 1u) && di + 1 < Dl[i][q];
        }
        if (lane == 1) wL = w; else wR = w;
    }
    unsigned nb = 0;
    if (__any_sync(FULL_MASK, wT)) nb |= 1;
    if (__any_sync(FULL_MASK, wB)) nb |= 2;
    if (__any_sync(FULL_MASK, wL)) nb |= 4;
    if (__any_sync(FULL_MASK, wR)) nb |= 8;
    nbmask = nb;

    // labels, mask of lambda_k, active counts of the member tiles
    uint8_t *M = P.masks + D.mask_off + (size_t)kcur * PS;
    unsigned live = 0;      // bit i: row i's label is finite
    int dm = 0;
#pragma unroll 8
    for (int i = 0; i < BR; ++i) {
        const int y = T.y0 + i;
        const size_t idx = (size_t)y * pitch + T.X;
        const int di = Dl[i][lane];
        if (own && y < D.rows) {
            if constexpr (!FWD) __stcg(Hh + idx, di);
            M[idx] = di >= HINF ? 1 : 0;
            dm = di < HINF ? max(dm, di) : dm;
        }
        if (FWD && own) __stcg(REC + (9 + i) * 32 + lane, di);
        live |= di < HINF ? (1u << i) : 0u;
    }
    // active pixels (positive excess, finite label) of each member tile
    int cnt[SPAN];
    constexpr unsigned TMASK = (TH == 32) ? 0xffffffffu : ((1u << TH) - 1u);
#pragma unroll
    for (int j = 0; j < SPAN; ++j)
        cnt[j] = (int)__reduce_add_sync(FULL_MASK, (unsigned)__popc(bE & live & (TMASK << (j * TH))));
    dm = (int)__reduce_max_sync(FULL_MASK, (unsigned)dm);
    __threadfence();
    __syncwarp();
    // member tile j's active count, lane j (the counts are warp-uniform); the
    // forward pass changes neither counts nor the largest distance
    int delta = 0;
    if (!FWD && lane < SPAN && T.ty + lane < D.tiles_y) {
        int mine = 0;
#pragma unroll
        for (int j = 0; j < SPAN; ++j) mine = (j == lane) ? cnt[j] : mine;
        *(volatile int *)&P.tiles[g + lane * D.tiles_x].active = mine;
        __stcg(REC + RW_CNT * 32 + lane, mine);
        delta = mine - cnt_old;
    }
#pragma unroll
    for (int o = SPAN / 2; o > 0; o >>= 1) delta += __shfl_down_sync(FULL_MASK, delta, o);
    if (lane == 0) {
        if (!FWD && dm > 0) atomicMax(&P.ist[inst].dmax, dm);
        *(volatile int *)&TS->epoch = epoch;
        if (delta) atomicAdd(&P.ist[inst].active, delta);
        atomicAdd(&P.ist[inst].bfs_visits, 1ULL);
        if (P.trace) {
            const long long c_end = clock64();
            atomicAdd(&P.g->prof[8], (unsigned long long)(c_loaded - c_start));
            atomicAdd(&P.g->prof[9], (unsigned long long)(c_relaxed - c_loaded));
            atomicAdd(&P.g->prof[10], (unsigned long long)(c_end - c_relaxed));
            atomicAdd(&P.g->prof[11], (unsigned long long)rounds);
        }
    }
}

// --------------------------------------------------------------------------
// server mode: admission of posted instances into the running kernel
// --------------------------------------------------------------------------
__device__ __forceinline__ int flags_status(int f) {
    if (f & VF_SLOPE) return PMF_ERR_NOT_MONOTONE;
    if (f & VF_OVERFLOW) return PMF_ERR_OVERFLOW;
    if (f & VF_NEG) return PMF_ERR_INVALID_ARG;
    return PMF_OK;
}

// Set-up visit of one strip of a newly admitted instance (its capacities were
// copied in by the host, row-major with the padded pitch): padding and the
// ignored last column of w_h / last row of w_v become zero, capacities are
// checked, the lambda_0 preflow is set up (as init_kernel does for a batch)
// and the member tiles and the strip record start afresh.
template <int TH>
__device__ void setup_visit(const Params &P, int g, int inst, const DevInst &D) {
    constexpr int BR = BFS_ROWS;
    constexpr int SPAN = BR / TH;
    const TileGeo T = tile_geo(g, D, TH);
    const int lane = T.lane;
    const bool own = T.inb && !T.ghost;
    const int pitch = D.pitch;
    const size_t PS = (size_t)D.rows * pitch;
    int *base = P.planes + D.plane_off;
    int *WH = const_cast<int *>(P.img) + D.img_off, *WV = WH + PS;
    const int *L = P.lambdas + (size_t)inst * P.max_lambdas;
    const long long lam0 = __ldcg(L), lamN = __ldcg(L + D.n_lambda - 1);
    long long fsum = 0;
    int bad = 0;
#pragma unroll 1
    for (int i = 0; i < BR; ++i) {
        const int y = T.y0 + i;
        if (!own || y >= D.rows) continue;
        const size_t idx = (size_t)y * pitch + T.X;
        const bool in = y < D.H && T.X < D.W;
        const int wh = (in && T.X < D.W - 1) ? __ldcg(WH + idx) : 0;
        const int wv = (in && y < D.H - 1) ? __ldcg(WV + idx) : 0;
        const int s0 = in ? __ldcg(base + P_SRC0 * PS + idx) : 0;
        const int sl = in ? __ldcg(base + P_SLOPE * PS + idx) : 0;
        const int ct = in ? __ldcg(base + P_CT * PS + idx) : 0;
        if (wh < 0 || wv < 0 || s0 < 0 || ct < 0) bad |= VF_NEG;
        if (wh > PMF_MAX_PAIRWISE || wv > PMF_MAX_PAIRWISE || s0 > PMF_INF || ct > PMF_INF) bad |= VF_OVERFLOW;
        if (sl < 0) bad |= VF_SLOPE;
        const long long cs0 = (long long)s0 + (long long)sl * lam0, csN = (long long)s0 + (long long)sl * lamN;
        if (csN > PMF_INF) bad |= VF_OVERFLOW;
        const bool ok = s0 >= 0 && ct >= 0 && sl >= 0 && csN <= PMF_INF;
        if (!in || T.X >= D.W - 1) __stcg(WH + idx, 0);
        if (!in || y >= D.H - 1) __stcg(WV + idx, 0);
        if (!in) {
            __stcg(base + P_SRC0 * PS + idx, 0);
            __stcg(base + P_SLOPE * PS + idx, 0);
            __stcg(base + P_CT * PS + idx, 0);
        }
        int e = ok ? (int)cs0 : 0, rt = ok ? ct : 0;
        const int m = min(e, rt);
        e -= m;
        rt -= m;
        fsum += m;
        __stcg(base + P_E * PS + idx, e);
        __stcg(base + P_RT * PS + idx, rt);
        __stcg(base + P_H * PS + idx, HINF);
        __stcg(base + P_FR * PS + idx, 0);
        __stcg(base + P_FD * PS + idx, 0);
    }
    // the member tiles and the strip record start from zero counts and epochs
    int32_t *cnt = P.strip_cache + (size_t)(D.lead_base + (T.ty / SPAN) * D.tiles_x + T.tx) * STRIP_REC_WORDS +
                   RW_CNT * 32;
    if (lane < SPAN && T.ty + lane < D.tiles_y) {
        TileState *t = P.tiles + g + lane * D.tiles_x;
        *(volatile int *)&t->epoch = 0;
        *(volatile int *)&t->active = 0;
        __stcg(cnt + lane, 0);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        fsum += __shfl_down_sync(FULL_MASK, fsum, o);
        bad |= __shfl_down_sync(FULL_MASK, bad, o);
    }
    __threadfence();
    if (lane == 0) {
        if (fsum) atomicAdd(&P.ist[inst].flow, (unsigned long long)fsum);
        if (bad) {
            atomicOr(&P.ist[inst].vflags, bad);
            atomicCAS(&P.ist[inst].status, PMF_OK, flags_status(bad));
        }
    }
}

// Start a posted slot: its instance state is reset and its strips are queued
// for the set-up pass, into the same ring every running instance uses.  Run
// by the warp that took the slot from the mailbox.
template <bool SV>
__device__ void admit(const Params &P, int slot) {
    const int lane = threadIdx.x & 31;
    volatile InstState *S = P.ist + slot;
    const DevInst D = load_inst<SV>(P, slot);
    if (lane == 0) {
        S->phase = PH_SETUP;
        S->k = 0;
        S->epoch = 1;
        S->status = PMF_OK;
        S->vflags = 0;
        S->pr_budget = D.n_tiles;
        S->want_bfs = 0;
        S->lab_cap = D.hcap;
        S->pr_mark = 0;
        S->step_mark = 0;
        S->epochs = 1;
        S->lam_prev = 0;
        S->active = 0;
        S->dmax = 0;
        S->flow = 0;
        S->pr_visits = 0;
        S->bfs_visits = 0;
        S->warm_visits = 0;
        S->outstanding = 1;              // guard while the strips are queued
        __threadfence();
    }
    __syncwarp();
    enqueue_tiles(P, slot, D, false, true);
    int last = 0;
    if (lane == 0) {
        __threadfence();
        last = atomicAdd(&P.ist[slot].outstanding, -1) == 1;
    }
    if (__shfl_sync(FULL_MASK, last, 0)) transition<SV>(P, slot);
}

constexpr unsigned long long NO_TICKET = ~0ULL;
constexpr unsigned long long MB_POLL_NS = 20000;   // mailbox checks: one every 20 us at most

// server mode pop: a worker keeps its ticket across calls; while its slot is
// empty it looks at the mailbox now and then.  Returns an item, -1 to stop,
// or -2 - slot for a posted slot the warp must admit.
__device__ int ring_pop_server(const Params &P, unsigned long long &ticket) {   // one lane
    Globals *G = P.g;
    if (ticket == NO_TICKET) ticket = atomicAdd(&G->head, 1ULL);
    volatile int *slot = (volatile int *)(P.ring + (ticket & P.ring_mask));
    Mailbox *MB = P.mailbox;
    unsigned ns = 32;
    unsigned long long last_tail = ~0ULL, last_prog = ~0ULL, t_since = 0;
    int last_done = -1;
    for (unsigned polls = 1;; ++polls) {
        const int v = *slot;
        if (v != -1) {
            *slot = -1;
            __threadfence();
            ticket = NO_TICKET;
            return v;
        }
        if ((polls & 3) == 0) {
            if (ldv(&G->err)) return -1;
            const unsigned long long now = gtime_ns();
            if (now - ldv64(&G->t_start) > (unsigned long long)P.max_ns) {
                atomicOr(&G->err, GE_TIMEOUT);
                return -1;
            }
            // one warp at a time looks at the mailbox (a load over PCIe): many
            // outstanding loads of host memory hold up the SMs' memory queues
            // for the warps that are working
            const unsigned long long due = ldv64(&G->mb_next_ns);
            if (now >= due && atomicCAS(&G->mb_next_ns, due, now + MB_POLL_NS) == due) {
                int tail;
                asm volatile("ld.acquire.sys.global.b32 %0, [%1];" : "=r"(tail) : "l"(&MB->tail) : "memory");
                const int h = ldv(&G->cmd_head);
                if (h < tail && atomicCAS(&G->cmd_head, h, h + 1) == h) {
                    atomicAdd(&G->admitted, 1);
                    return -2 - *(volatile int *)&MB->ring[h % MB_CAP];
                }
                if (*(volatile int *)&MB->stop && h >= tail && ldv(&G->inst_done) >= ldv(&G->admitted))
                    return -1;
            }
            // the stall watchdog counts only while admitted work is unfinished
            const int ndone = ldv(&G->inst_done);
            const unsigned long long tl = ldv64(&G->tail), pg = ldv64(&G->progress);
            if (ndone >= ldv(&G->admitted) || tl != last_tail || ndone != last_done || pg != last_prog) {
                last_tail = tl;
                last_done = ndone;
                last_prog = pg;
                t_since = now;
            } else if (now - t_since > (unsigned long long)P.stall_ns) {
                atomicOr(&G->err, GE_STALL);
                return -1;
            }
        }
        __nanosleep(ns);
        if (ns < (unsigned)P.poll_ns) ns <<= 1;
    }
}

// --------------------------------------------------------------------------
// persistent worker
// --------------------------------------------------------------------------
constexpr int WORKER_WARPS = 4;

// MINB resident blocks per SM the register allocation must allow: 4 at tile
// height 4 (128 registers) and 2 at height 8 by default (with fewer,
// throughput-bound batches lose more than the spills cost); a second build at
// tile height 4 for 3 blocks (up to 168 registers, no spills) serves grids of
// 1 to 3 blocks per SM, where chains of dependent visits bound the launch.
// SINK: the batch holds instances whose sink capacities fall with lambda
// (their own kernels, so that the others' register allocation is untouched).
// SV: the server kernel (instances admitted from the mailbox while it runs)
template <int TH, int PO, bool SINK, bool SV, int MINB = (TH == 4 ? 4 : 2)>
__global__ void __launch_bounds__(WORKER_WARPS * 32, MINB) worker_kernel(const __grid_constant__ Params P) {
    __shared__ WarpSmem<TH> smem[WORKER_WARPS];
    // In the 4-block builds (128 registers) the rarely run warm-start pass and
    // phase change are called out of line, which keeps the hot loop's code
    // compact (instruction fetch was the top stall of the uneven batch): the
    // uneven batch runs 2 % faster although more registers spill.  The wider
    // builds keep them inline (out of line cost them 5-6 %).
    constexpr bool OOL = MINB == 4 && !SV;
    // staged strip loads: the block's buffer (dynamic shared memory, present
    // only when P.strip_stage is set) and its barrier
    extern __shared__ __align__(128) int32_t stage_buf[];
    __shared__ __align__(8) unsigned long long stage_bar;
    __shared__ int stage_lock, stage_uses;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WarpSmem<TH> &S = smem[w];
    const StripStage SS{stage_buf, &stage_bar, &stage_lock, &stage_uses};
    if (!SV && P.strip_stage) {
        if (threadIdx.x == 0) stage_init(SS);
        __syncthreads();
    }
    const int round_mode = ldv(&P.g->round_mode);
    const bool prof = P.trace != nullptr;
    unsigned long long tw = 0, tpr = 0, tbfs = 0, tfin = 0, t0 = prof ? gtime_ns() : 0;
    int next = -1;           // an item kept by the last finish, run without queueing
    unsigned chain = 0;
    unsigned long long ticket = NO_TICKET;   // server mode: a ticket kept across admissions
    for (;;) {
        int g = 0;
        if (next >= 0) {
            g = next;
            next = -1;
            // a long chain of kept items still notices a launch-wide stop,
            // and shows the stall watchdog that work is being done
            if ((++chain & 15) == 0) {
                int stop = 0;
                if (lane == 0) {
                    atomicAdd(&P.g->progress, 1ULL);
                    stop = ldv(&P.g->err);
                }
                if (__shfl_sync(FULL_MASK, stop, 0)) break;
            }
        } else {
            chain = 0;
            if constexpr (SV) {
                if (lane == 0) g = ring_pop_server(P, ticket);
            } else {
                if (lane == 0) g = round_mode ? ring_pop_round(P) : ring_pop_ticket(P);
            }
            g = __shfl_sync(FULL_MASK, g, 0);
            if (SV && g <= -2) {
                admit<SV>(P, -2 - g);
                continue;
            }
        }
        if (prof) { const unsigned long long t1 = gtime_ns(); tw += t1 - t0; t0 = t1; }
        if (g < 0) break;
        const int inst = __ldg(P.tile_inst + g);
        if (lane == 0) {
            atomicExch(&P.tiles[g].state, T_RUNNING);
            __threadfence();
        }
        __syncwarp();
        const DevInst D = load_inst<SV>(P, inst);
        // phase, k, epoch, status in one 16-byte load
        int phase, k, epoch, status;
        asm volatile("ld.volatile.global.v4.s32 {%0, %1, %2, %3}, [%4];"
                     : "=r"(phase), "=r"(k), "=r"(epoch), "=r"(status)
                     : "l"(P.ist + inst));
        bool requeue = false;
        unsigned nb = 0;
        // a relabel item must be a strip's leader tile: anything else means a
        // push/relabel item outlived its phase, which the phase changes rule out
        const bool strip = phase == PH_BFS || phase == PH_FWD || phase == PH_WARM || phase == PH_COPY ||
                           phase == PH_SETUP;
        const bool stray = strip && ((g - D.tile_base) / D.tiles_x) % (BFS_ROWS / TH) != 0;
        if (stray && lane == 0) atomicOr(&P.g->err, GE_PHASE);
        if (status == PMF_OK && phase == PH_PR) pr_visit<TH, PO, SV>(P, S, g, inst, D, k, requeue, nb);
        else if (status == PMF_OK && phase == PH_BFS && !stray)
            bfs_visit<TH, false, SV>(P, S, SS, g, inst, D, epoch, k, requeue, nb);
        else if (status == PMF_OK && phase == PH_FWD && !stray)
            bfs_visit<TH, true, SV>(P, S, SS, g, inst, D, epoch, k, requeue, nb);
        else if (status == PMF_OK && phase == PH_WARM && !stray) {
            if constexpr (OOL) warm_visit_ool<TH, SINK, SV>(P, g, inst, D, k);
            else warm_visit<TH, SINK, SV>(P, g, inst, D, k);
        }
        else if (status == PMF_OK && phase == PH_COPY && !stray) copy_visit<TH, SV>(P, g, inst, D);
        else if (SV && phase == PH_SETUP && !stray) setup_visit<TH>(P, g, inst, D);
        __threadfence();
        __syncwarp();
        if (prof) {
            const unsigned long long t1 = gtime_ns();
            if (phase == PH_PR) tpr += t1 - t0; else tbfs += t1 - t0;
            t0 = t1;
        }
        // in host-polled rounds every new item waits for the next round
        next = finish<SV, OOL>(P, g, inst, phase, requeue, nb, D, round_mode == 0);
        if (prof) { const unsigned long long t1 = gtime_ns(); tfin += t1 - t0; t0 = t1; }
    }
    if (prof && lane == 0) {
        atomicAdd(&P.g->prof[0], tw);
        atomicAdd(&P.g->prof[1], tpr);
        atomicAdd(&P.g->prof[2], tbfs);
        atomicAdd(&P.g->prof[3], tfin);
    }
}

// --------------------------------------------------------------------------
// set-up kernels
// --------------------------------------------------------------------------
__global__ void pad_image_kernel(int32_t *wh_out, int32_t *wv_out, const int32_t *w_h,
                                 const int32_t *w_v, int H, int W, int rows, int pitch,
                                 int32_t *flags) {
    const size_t n = (size_t)rows * pitch;
    int bad = 0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int y = (int)(i / pitch), x = (int)(i % pitch);
        int a = 0, b = 0;
        if (y < H && x < W - 1) a = w_h[(size_t)y * W + x];
        if (y < H - 1 && x < W) b = w_v[(size_t)y * W + x];
        if (a < 0 || b < 0) bad |= VF_NEG;
        if (a > PMF_MAX_PAIRWISE || b > PMF_MAX_PAIRWISE) bad |= VF_OVERFLOW;
        wh_out[i] = a;
        wv_out[i] = b;
    }
    if (bad) atomicOr(flags, bad);
}

__global__ void pad_terminals_kernel(int32_t *src0_out, int32_t *slope_out, int32_t *ct_out,
                                     const int32_t *src0, const int32_t *slope, const int32_t *sink,
                                     int H, int W, int rows, int pitch, int32_t *flags) {
    const size_t n = (size_t)rows * pitch;
    int bad = 0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int y = (int)(i / pitch), x = (int)(i % pitch);
        int a = 0, b = 0, c = 0;
        if (y < H && x < W) {
            const size_t j = (size_t)y * W + x;
            a = src0[j];
            b = slope[j];
            c = sink[j];
        }
        if (a < 0 || c < 0) bad |= VF_NEG;
        if (b < 0) bad |= VF_SLOPE;
        if (a > PMF_INF || c > PMF_INF) bad |= VF_OVERFLOW;
        src0_out[i] = a;
        slope_out[i] = b;
        ct_out[i] = c;
    }
    if (bad) atomicOr(flags, bad);
}

__device__ __forceinline__ int flags_to_status(int f) {
    if (f & VF_SLOPE) return PMF_ERR_NOT_MONOTONE;
    if (f & VF_OVERFLOW) return PMF_ERR_OVERFLOW;
    if (f & VF_NEG) return PMF_ERR_INVALID_ARG;
    return PMF_OK;
}

// per-solve reset: every tile queued for the first global relabel
__global__ void reset_kernel(const __grid_constant__ Params P) {
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    const size_t t0 = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    const size_t cap = (size_t)P.ring_mask + 1;
    for (size_t i = t0; i < cap; i += stride)
        if (i >= (size_t)P.n_leads_queued) P.ring[i] = -1;

    const int span = BFS_ROWS / P.tile_h;
    // one thread per tile: its instance is the last one whose first tile is
    // at or before it (instances own consecutive, non-empty tile ranges)
    for (size_t g = t0; g < (size_t)P.n_tiles_total; g += stride) {
        int lo = 0, hi = P.n_inst - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if ((size_t)__ldg(&P.inst[mid].tile_base) <= g) lo = mid;
            else hi = mid - 1;
        }
        const int tiles_x = __ldg(&P.inst[lo].tiles_x);
        const int j = (int)(g - (size_t)__ldg(&P.inst[lo].tile_base));
        const int ty = j / tiles_x, tx = j - ty * tiles_x;
        const bool lead = (ty % span) == 0;
        // a forked instance's strips are queued by its parent's copy pass
        const bool waits = __ldg(&P.inst[lo].fork_parent) >= 0;
        ((int32_t *)P.tile_inst)[g] = lo;
        TileState t;
        t.state = (lead && !waits) ? T_QUEUED : T_IDLE;
        t.epoch = 0;
        t.pad_ = 0;
        t.active = 0;
        P.tiles[g] = t;
        // every relabel strip of every instance is queued for the first
        // relabel, except those of forked instances (numbered last)
        if (lead) {
            const size_t strip = (size_t)__ldg(&P.inst[lo].lead_base) + (size_t)(ty / span) * tiles_x + tx;
            if (!waits) P.ring[strip] = (int)g;
            // the strip record's copy of its tiles' active counts starts with them, at 0
            int32_t *cnt = P.strip_cache + strip * STRIP_REC_WORDS + RW_CNT * 32;
            for (int j = 0; j < span; ++j) cnt[j] = 0;
        }
    }
    for (size_t i = t0; i < (size_t)P.n_inst; i += stride) {
        const DevInst D = P.inst[i];
        const bool waits = D.fork_parent >= 0;
        InstState s;
        s.phase = waits ? PH_WAIT : PH_BFS;
        s.k = 0;
        s.epoch = 1;
        s.vflags = P.inst_flags[i] | P.img_flags[D.image];
        s.status = flags_to_status(s.vflags);
        s.pad3_ = 0;
        s.lam_prev = 0;
        s.pad_c_ = 0;
        s.pr_mark = 0;
        s.pr_budget = D.n_tiles;
        s.dmax = 0;
        s.lab_cap = D.hcap;
        s.step_mark = 0;
        s.epochs = 1;
        s.outstanding = waits ? 0 : D.n_leads;
        s.active = 0;
        s.want_bfs = 0;
        s.flow = 0;
        s.pr_visits = 0;
        s.bfs_visits = 0;
        s.warm_visits = 0;
        P.ist[i] = s;
    }
    if (t0 == 0) {
        Globals *G = P.g;
        G->head = 0;
        G->tail = (unsigned long long)P.n_leads_queued;
        G->inst_done = 0;
        G->err = 0;
        G->round_mode = 0;
        G->round_end = G->tail;
        G->t_start = gtime_ns();
        G->progress = 0;
        G->trace_n = 0;
        for (int j = 0; j < PMF_PROFILE_COUNTERS; ++j) G->prof[j] = 0;
    }
}

// lambda_0 preflow: saturate every source arc, send what the sink arc can take
// straight to t, zero pairwise flow, labels unknown until the first BFS
__global__ void init_kernel(const __grid_constant__ Params P) {
  for (int inst = blockIdx.y; inst < P.n_inst; inst += gridDim.y) {
    const DevInst D = P.inst[inst];
    const size_t PS = (size_t)D.rows * D.pitch;
    int32_t *base = P.planes + D.plane_off;
    // a forked instance takes its state and terminals from its parent's copy
    // pass; here only its own schedule is checked against those terminals
    const bool forked = D.fork_parent >= 0;
    const int32_t *tb = forked ? P.planes + P.inst[D.fork_parent].plane_off : base;
    const int32_t *L = P.lambdas + (size_t)inst * P.max_lambdas;
    const long long lam0 = L[0], lamN = L[D.n_lambda - 1];
    long long fsum = 0;
    int bad = 0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < PS; i += (size_t)gridDim.x * blockDim.x) {
        const int s0 = tb[P_SRC0 * PS + i], sl = tb[P_SLOPE * PS + i], ct = tb[P_CT * PS + i];
        // the source capacities rise with lambda, or the sink capacities fall
        // (Section 2.1's monotone case either way): both stay within
        // [0, PMF_INF] over the whole schedule
        const long long up0 = D.slope_side ? 0 : (long long)sl * lam0, upN = D.slope_side ? 0 : (long long)sl * lamN;
        const long long dn0 = D.slope_side ? (long long)sl * lam0 : 0, dnN = D.slope_side ? (long long)sl * lamN : 0;
        const long long cs0 = (long long)s0 + up0, csN = (long long)s0 + upN;
        const long long ct0 = (long long)ct - dn0, ctN = (long long)ct - dnN;
        if (cs0 < 0 || ctN < 0) bad |= VF_NEG;
        if (csN > PMF_INF) bad |= VF_OVERFLOW;
        const bool ok = cs0 >= 0 && ctN >= 0 && csN <= PMF_INF;
        if (forked) continue;
        int e = ok ? (int)cs0 : 0;
        int rt = ok ? (int)ct0 : 0;
        const int m = min(e, rt);
        e -= m;
        rt -= m;
        fsum += m;
        base[P_E * PS + i] = e;
        base[P_RT * PS + i] = rt;
        base[P_H * PS + i] = HINF;
        base[P_FR * PS + i] = 0;
        base[P_FD * PS + i] = 0;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        fsum += __shfl_down_sync(FULL_MASK, fsum, o);
        bad |= __shfl_down_sync(FULL_MASK, bad, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (fsum) atomicAdd(&P.ist[inst].flow, (unsigned long long)fsum);
        if (bad) {
            atomicOr(&P.ist[inst].vflags, bad);
            atomicCAS(&P.ist[inst].status, PMF_OK, flags_to_status(bad));
        }
    }
  }
}

__global__ void begin_round_kernel(Globals *G) {
    G->t_start = gtime_ns();
    G->round_end = G->tail;
    G->round_mode = 1;
}

// --------------------------------------------------------------------------
// launch wrappers
// --------------------------------------------------------------------------
cudaError_t launch_pad_image(const Params &P, int image, const DevInst &d, const int32_t *w_h,
                             const int32_t *w_v, int32_t *flags, cudaStream_t s) {
    (void)P;
    (void)image;
    int32_t *wh = const_cast<int32_t *>(P.img) + d.img_off;
    const size_t n = (size_t)d.rows * d.pitch;
    const int blocks = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
    (void)cudaGetLastError();
    pad_image_kernel<<<blocks, 256, 0, s>>>(wh, wh + n, w_h, w_v, d.H, d.W, d.rows, d.pitch, flags);
    return cudaGetLastError();
}

cudaError_t launch_pad_terminals(const Params &P, int inst, const DevInst &d, const int32_t *src0,
                                 const int32_t *slope, const int32_t *sink, cudaStream_t s) {
    int32_t *base = P.planes + d.plane_off;
    const size_t n = (size_t)d.rows * d.pitch;
    const int blocks = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
    (void)cudaGetLastError();
    pad_terminals_kernel<<<blocks, 256, 0, s>>>(base + P_SRC0 * n, base + P_SLOPE * n, base + P_CT * n,
                                                src0, slope, sink, d.H, d.W, d.rows, d.pitch,
                                                P.inst_flags + inst);
    return cudaGetLastError();
}

cudaError_t launch_reset(const Params &P, cudaStream_t s) {
    const size_t n = (size_t)P.ring_mask + 1;
    const int blocks = (int)((n + 255) / 256 < 2048 ? (n + 255) / 256 : 2048);
    (void)cudaGetLastError();
    reset_kernel<<<blocks, 256, 0, s>>>(P);
    return cudaGetLastError();
}

cudaError_t launch_init(const Params &P, int max_pixels, cudaStream_t s) {
    int bx = (max_pixels + 255) / 256;
    if (bx > 64) bx = 64;
    if (bx < 1) bx = 1;
    dim3 grid(bx, P.n_inst < 65535 ? P.n_inst : 65535);
    (void)cudaGetLastError();
    init_kernel<<<grid, 256, 0, s>>>(P);
    return cudaGetLastError();
}

// --------------------------------------------------------------------------
// per-arc flow of a solved instance (phase 2 of push-relabel): the solve
// leaves a maximum preflow whose excess sits on pixels that cannot reach t;
// returning that excess to s turns it into a feasible maximum flow of the
// same value (Section 2's flow, arc by arc)
// --------------------------------------------------------------------------
constexpr int RETURN_THREADS = 512;

// One cooperative grid over the whole GPU.  Start: the preflow with every
// source arc carrying cs(p) and every sink arc ct(p) - rt(p); a pixel's excess
// is its inflow minus its outflow.  Sweep: a pixel with excess first sends it
// back along its own source arc, then back along the pair arcs that carry flow
// into it (each push lowers a positive flow towards zero).  Only a pair's
// receiving end ever changes its flow, and no flow changes sign, so the two
// ends never act on one pair at once; excess moves by atomic adds.  Every
// push lowers the sum of |flows| by its amount, so the sweeps end; the grid
// stops after a sweep in which no pixel held excess.  The sink arcs never
// change: the value stays the flow into t.  Whether a sweep saw excess goes
// to one of three flags (sweep s uses flag s % 3 and clears flag (s + 1) % 3,
// whose last readers finished two grid barriers earlier).
__global__ void __launch_bounds__(RETURN_THREADS) return_excess_kernel(
    const int32_t *E, const int32_t *RT, const int32_t *FR, const int32_t *FD, const int32_t *SRC0,
    const int32_t *SLOPE, const int32_t *CT, int lambda, int slope_side, int H, int W, int pitch, int max_sweeps,
    int32_t *f_h, int32_t *f_v, int32_t *f_s, int32_t *f_t, int32_t *status, int32_t *flags) {
    cg::grid_group grid = cg::this_grid();
    const int n = H * W;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
    for (int p = tid; p < n; p += nth) {
        const int y = p / W, x = p - y * W;
        const size_t i = (size_t)y * pitch + x;
        f_h[p] = x < W - 1 ? FR[i] : 0;
        f_v[p] = y < H - 1 ? FD[i] : 0;
        f_s[p] = slope_side ? SRC0[i] : SRC0[i] + SLOPE[i] * lambda;
        f_t[p] = E[i];                      // the excess, until the last step
    }
    if (tid == 0) flags[0] = flags[1] = flags[2] = 0;
    grid.sync();
    volatile int32_t *vh = f_h, *vv = f_v, *vs = f_s, *ve = f_t;
    int sweeps = 0;
    bool more = true;
    while (more && sweeps < max_sweeps) {
        if (tid == 0) flags[(sweeps + 1) % 3] = 0;
        bool any = false;
        for (int p = tid; p < n; p += nth) {
            const int ex = ve[p];
            if (ex <= 0) continue;
            any = true;
            const int y = p / W, x = p - y * W;
            int rem = ex;
            const int r0 = min(rem, (int)vs[p]);        // back to s
            vs[p] = vs[p] - r0;
            rem -= r0;
            if (rem > 0 && x > 0) {                     // flow arriving from the left
                const int f = vh[p - 1];
                const int d = f > 0 ? min(rem, f) : 0;
                if (d) { vh[p - 1] = f - d; atomicAdd(&f_t[p - 1], d); rem -= d; }
            }
            if (rem > 0 && x < W - 1) {                 // from the right
                const int f = -vh[p];
                const int d = f > 0 ? min(rem, f) : 0;
                if (d) { vh[p] = -(f - d); atomicAdd(&f_t[p + 1], d); rem -= d; }
            }
            if (rem > 0 && y > 0) {                     // from above
                const int f = vv[p - W];
                const int d = f > 0 ? min(rem, f) : 0;
                if (d) { vv[p - W] = f - d; atomicAdd(&f_t[p - W], d); rem -= d; }
            }
            if (rem > 0 && y < H - 1) {                 // from below
                const int f = -vv[p];
                const int d = f > 0 ? min(rem, f) : 0;
                if (d) { vv[p] = -(f - d); atomicAdd(&f_t[p + W], d); rem -= d; }
            }
            if (ex - rem) atomicSub(&f_t[p], ex - rem);
        }
        if (__syncthreads_or(any) && threadIdx.x == 0) atomicOr(&flags[sweeps % 3], 1);
        __threadfence();
        grid.sync();
        more = *(volatile int32_t *)&flags[sweeps % 3] != 0;
        ++sweeps;
    }
    grid.sync();
    for (int p = tid; p < n; p += nth) {
        const int y = p / W, x = p - y * W;
        const size_t i = (size_t)y * pitch + x;
        f_t[p] = (slope_side ? CT[i] - SLOPE[i] * lambda : CT[i]) - RT[i];
    }
    if (tid == 0) *status = more ? 1 : 0;
}

cudaError_t launch_return_excess(const Params &P, const DevInst &d, int lambda, int max_sweeps,
                                 int32_t *f_h, int32_t *f_v, int32_t *f_s, int32_t *f_t, int32_t *status,
                                 int32_t *flags, cudaStream_t s) {
    const size_t PS = (size_t)d.rows * d.pitch;
    const int32_t *base = P.planes + d.plane_off;
    int dev = 0, n_sm = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, return_excess_kernel, RETURN_THREADS, 0);
    if (e != cudaSuccess) return e;
    // every block resident at once (a cooperative launch), no more than the pixels need
    const long long need = ((long long)d.H * d.W + RETURN_THREADS - 1) / RETURN_THREADS;
    int grid = per_sm * n_sm;
    if (need < grid) grid = (int)(need < 1 ? 1 : need);
    const int32_t *E = base + P_E * PS, *RT = base + P_RT * PS, *FR = base + P_FR * PS, *FD = base + P_FD * PS;
    const int32_t *S0 = base + P_SRC0 * PS, *SL = base + P_SLOPE * PS, *CT = base + P_CT * PS;
    int lam = lambda, side = d.slope_side, H = d.H, W = d.W, pitch = d.pitch, ms = max_sweeps;
    void *args[] = {(void *)&E,  (void *)&RT,  (void *)&FR,   (void *)&FD,    (void *)&S0,  (void *)&SL,
                    (void *)&CT, (void *)&lam, (void *)&side, (void *)&H,     (void *)&W,   (void *)&pitch,
                    (void *)&ms, (void *)&f_h, (void *)&f_v,  (void *)&f_s,   (void *)&f_t, (void *)&status,
                    (void *)&flags};
    (void)cudaGetLastError();
    return cudaLaunchCooperativeKernel((const void *)return_excess_kernel, dim3(grid), dim3(RETURN_THREADS), args, 0,
                                       s);
}

// the batch kernels, by (any sink side, wide registers, tile height, push order)
static const void *batch_worker(const Params &P) {
    if (P.any_sink_side) {
        if (P.tile_h == 4) return P.chain_push ? (const void *)worker_kernel<4, 1, true, false>
                                               : (const void *)worker_kernel<4, 0, true, false>;
        return P.chain_push ? (const void *)worker_kernel<8, 1, true, false>
                            : (const void *)worker_kernel<8, 0, true, false>;
    }
    if (P.tile_h == 4 && P.wide_regs)
        return P.chain_push ? (const void *)worker_kernel<4, 1, false, false, 3>
                            : (const void *)worker_kernel<4, 0, false, false, 3>;
    if (P.tile_h == 4)
        return P.chain_push ? (const void *)worker_kernel<4, 1, false, false>
                            : (const void *)worker_kernel<4, 0, false, false>;
    return P.chain_push ? (const void *)worker_kernel<8, 1, false, false>
                        : (const void *)worker_kernel<8, 0, false, false>;
}

cudaError_t prepare_stage_kernels() {
    // static plus staging shared memory exceeds the 48 KB a kernel gets without
    // asking; set once per process, outside any stream capture
    static cudaError_t done = [] {
        const void *ks[] = {(const void *)worker_kernel<4, 1, true, false>,
                            (const void *)worker_kernel<4, 0, true, false>,
                            (const void *)worker_kernel<8, 1, true, false>,
                            (const void *)worker_kernel<8, 0, true, false>,
                            (const void *)worker_kernel<4, 1, false, false, 3>,
                            (const void *)worker_kernel<4, 0, false, false, 3>,
                            (const void *)worker_kernel<4, 1, false, false>,
                            (const void *)worker_kernel<4, 0, false, false>,
                            (const void *)worker_kernel<8, 1, false, false>,
                            (const void *)worker_kernel<8, 0, false, false>};
        for (const void *k : ks) {
            const cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, STAGE_BYTES);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }();
    return done;
}

cudaError_t launch_worker(const Params &P, int grid, cudaStream_t s) {
    (void)cudaGetLastError();
    // one kernel per tile height and push order: each holds only the sweep it runs
    const void *k = batch_worker(P);
    void *args[] = {(void *)&P};
    return cudaLaunchKernel(k, dim3(grid), dim3(WORKER_WARPS * 32), args, P.strip_stage ? STAGE_BYTES : 0, s);
}

// server mode: tile height 4, pushes along columns and rows
cudaError_t launch_server_worker(const Params &P, int grid, cudaStream_t s) {
    (void)cudaGetLastError();
    worker_kernel<4, 1, false, true><<<grid, WORKER_WARPS * 32, 0, s>>>(P);
    return cudaGetLastError();
}

cudaError_t server_occupancy(int *blocks_per_sm) {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, worker_kernel<4, 1, false, true>,
                                                         WORKER_WARPS * 32, 0);
}

// every tile idle and owned by its slot, the ring empty, every slot finished
__global__ void server_reset_kernel(const __grid_constant__ Params P, int max_tiles) {
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    const size_t t0 = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    for (size_t i = t0; i <= (size_t)P.ring_mask; i += stride) P.ring[i] = -1;
    for (size_t g = t0; g < (size_t)P.n_tiles_total; g += stride) {
        ((int32_t *)P.tile_inst)[g] = (int32_t)(g / (size_t)max_tiles);
        TileState t;
        t.state = T_IDLE;
        t.epoch = 0;
        t.pad_ = 0;
        t.active = 0;
        P.tiles[g] = t;
    }
    for (size_t i = t0; i < (size_t)P.n_inst; i += stride) {
        InstState s;
        memset(&s, 0, sizeof(s));
        s.phase = PH_DONE;
        s.status = PMF_OK;
        P.ist[i] = s;
    }
    if (t0 == 0) {
        Globals *G = P.g;
        G->head = 0;
        G->tail = 0;
        G->inst_done = 0;
        G->err = 0;
        G->round_mode = 0;
        G->round_end = 0;
        G->t_start = gtime_ns();
        G->progress = 0;
        G->trace_n = 0;
        G->cmd_head = 0;
        G->admitted = 0;
        G->mb_next_ns = 0;
        for (int j = 0; j < PMF_PROFILE_COUNTERS; ++j) G->prof[j] = 0;
    }
}

cudaError_t launch_server_reset(const Params &P, int max_tiles, cudaStream_t s) {
    (void)cudaGetLastError();
    server_reset_kernel<<<1024, 256, 0, s>>>(P, max_tiles);
    return cudaGetLastError();
}

cudaError_t launch_begin_round(const Params &P, cudaStream_t s) {
    (void)cudaGetLastError();
    begin_round_kernel<<<1, 1, 0, s>>>(P.g);
    return cudaGetLastError();
}

int worker_warps_per_block() { return WORKER_WARPS; }

cudaError_t worker_occupancy(int tile_h, int *blocks_per_sm, bool staged) {
    const size_t dyn = staged ? STAGE_BYTES : 0;
    if (tile_h == 4)
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, worker_kernel<4, 0, false, false>,
                                                             WORKER_WARPS * 32, dyn);
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, worker_kernel<8, 0, false, false>,
                                                         WORKER_WARPS * 32, dyn);
}

// Tensor maps for staged strip loads, one per instance (its planes as a 3-D
// array: pitch x rows x N_INST_PLANES, box STAGE_BOX_W x BFS_ROWS x
// STAGE_INST_PLANES) and one per image (pitch x rows x N_IMG_PLANES, box
// STAGE_BOX_W x BFS_ROWS x N_IMG_PLANES).  Reads outside a plane fill zeros.
// The row pitch is a multiple of 32 elements, so every stride is a multiple of
// 16 bytes, as the copies require.
bool encode_plane_maps(unsigned char *host_out, const int32_t *inst_base, const int32_t *img_base, int n_inst,
                       const int64_t *plane_off, const int *inst_image, int n_images, const int64_t *img_off,
                       const int *rows, const int *pitch) {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
        (void)cudaGetLastError();
    });
    if (!encode) return false;
    auto one = [&](unsigned char *dst, const int32_t *base, int r, int p, int planes, int box_planes) {
        if (p % TILE_W != 0 || (reinterpret_cast<uintptr_t>(base) & 15) != 0) return false;
        CUtensorMap m;
        const cuuint64_t dims[3] = {(cuuint64_t)p, (cuuint64_t)r, (cuuint64_t)planes};
        const cuuint64_t strides[2] = {(cuuint64_t)p * 4, (cuuint64_t)p * r * 4};
        const cuuint32_t box[3] = {(cuuint32_t)STAGE_BOX_W, (cuuint32_t)BFS_ROWS, (cuuint32_t)box_planes};
        const cuuint32_t estr[3] = {1, 1, 1};
        const CUresult rc = encode(&m, CU_TENSOR_MAP_DATA_TYPE_INT32, 3, const_cast<int32_t *>(base), dims, strides,
                                   box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                   CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (rc != CUDA_SUCCESS) return false;
        static_assert(sizeof(CUtensorMap) == TMAP_BYTES, "one tensor map per TMAP_BYTES");
        std::memcpy(dst, &m, sizeof(m));
        return true;
    };
    for (int i = 0; i < n_inst; ++i) {
        const int im = inst_image[i];
        if (!one(host_out + (size_t)i * TMAP_BYTES, inst_base + plane_off[i], rows[im], pitch[im], N_INST_PLANES,
                 STAGE_INST_PLANES))
            return false;
    }
    for (int im = 0; im < n_images; ++im)
        if (!one(host_out + (size_t)(n_inst + im) * TMAP_BYTES, img_base + img_off[im], rows[im], pitch[im],
                 N_IMG_PLANES, N_IMG_PLANES))
            return false;
    return true;
}

}  // namespace pmf
