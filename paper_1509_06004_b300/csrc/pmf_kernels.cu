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

#include "pmf.h"
#include "pmf_internal.h"

namespace pmf {

#define FULL_MASK 0xffffffffu

__device__ __forceinline__ unsigned long long gtime_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ int ldv(const int *p) { return *(const volatile int *)p; }
__device__ __forceinline__ unsigned long long ldv64(const unsigned long long *p) {
    return *(const volatile unsigned long long *)p;
}
__device__ __forceinline__ long long ldv64s(const long long *p) { return *(const volatile long long *)p; }

template <int TH>
struct WarpSmem {
    int lh[TH];    // left halo column: label
    int lw[TH];    //   w_h of the edge (x0-1) - x0
    int lf[TH];    //   flow on that edge (local copy, changed by lane 0's pushes)
    int lf0[TH];   //   its value at load
    int lout[TH];  //   excess pushed into the left halo pixel
    int rh[TH];    // right halo column: label
    int rout[TH];  //   excess pushed into the right halo pixel
    int rf0[TH];   //   lane 31's own fR at load (the right border edge)
};

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

__device__ int ring_pop(const Params &P) {   // one lane; -1 = stop
    Globals *G = P.g;
    unsigned long long last_c = ~0ULL, t_since = 0;
    unsigned ns = 64;
    for (;;) {
        if (ldv(&G->err)) return -1;
        if (gtime_ns() - ldv64(&G->t_start) > (unsigned long long)P.max_ns) {
            atomicOr(&G->err, GE_TIMEOUT);
            return -1;
        }
        unsigned long long h = ldv64(&G->head);
        unsigned long long t = ldv64(&G->tail);
        unsigned long long lim = t;
        if (G->round_mode) {
            unsigned long long re = ldv64(&G->round_end);
            if (h >= re) return -1;
            if (re < lim) lim = re;
        }
        if (h < lim) {
            if (atomicCAS(&G->head, h, h + 1) == h) {
                volatile int *slot = (volatile int *)(P.ring + (h & P.ring_mask));
                int v;
                if (!slot_wait(P, slot, false, &v)) return -1;
                *slot = -1;
                __threadfence();
                return v;
            }
            continue;
        }
        if (ldv64s(&G->pending) <= 0) return -1;
        unsigned long long c = ldv64(&G->completed);
        unsigned long long now = gtime_ns();
        if (c != last_c) { last_c = c; t_since = now; }
        else if (now - t_since > (unsigned long long)P.stall_ns) {
            atomicOr(&G->err, GE_STALL);
            return -1;
        }
        __nanosleep(ns);
        if (ns < 8192) ns <<= 1;
    }
}

// ask for tile t (same instance) to be visited; one lane
__device__ void request(const Params &P, int t, int inst) {
    int *st = &P.tiles[t].state;
    for (int it = 0; it < 1024; ++it) {
        int old = atomicCAS(st, T_IDLE, T_QUEUED);
        if (old == T_IDLE) {
            atomicAdd(&P.ist[inst].outstanding, 1);
            atomicAdd((unsigned long long *)&P.g->pending, 1ULL);
            __threadfence();
            push1(P, t);
            return;
        }
        if (old == T_QUEUED || old == T_DIRTY) return;
        // RUNNING: mark dirty so that its visitor runs it again
        int o2 = atomicCAS(st, T_RUNNING, T_DIRTY);
        if (o2 == T_RUNNING || o2 == T_DIRTY || o2 == T_QUEUED) return;
        // it went IDLE in between: retry
    }
    atomicOr(&P.g->err, GE_RING);
}

// --------------------------------------------------------------------------
// instance phase changes, run by the warp that finished the instance's last
// outstanding item (so nothing of this instance is queued or running)
// --------------------------------------------------------------------------
__device__ void enqueue_tiles(const Params &P, int inst, const DevInst &D, bool only_active) {
    const int lane = threadIdx.x & 31;
    for (int c0 = 0; c0 < D.n_tiles; c0 += 32) {
        const int t = D.tile_base + c0 + lane;
        bool sel = (c0 + lane) < D.n_tiles;
        if (sel && only_active) sel = ldv(&P.tiles[t].active) > 0;
        const unsigned m = __ballot_sync(FULL_MASK, sel);
        const int cnt = __popc(m);
        if (cnt == 0) continue;
        if (sel) P.tiles[t].state = T_QUEUED;
        unsigned long long base = 0;
        if (lane == 0) {
            atomicAdd(&P.ist[inst].outstanding, cnt);
            atomicAdd((unsigned long long *)&P.g->pending, (unsigned long long)cnt);
            __threadfence();
            base = atomicAdd(&P.g->tail, (unsigned long long)cnt);
        }
        base = __shfl_sync(FULL_MASK, base, 0);
        __threadfence();
        if (sel) {
            const unsigned long long tk = base + __popc(m & ((1u << lane) - 1u));
            volatile int *slot = (volatile int *)(P.ring + (tk & P.ring_mask));
            int dummy;
            if (slot_wait(P, slot, true, &dummy)) *slot = t;
        }
    }
}

__device__ void transition(const Params &P, int inst) {
    const int lane = threadIdx.x & 31;
    volatile InstState *S = P.ist + inst;
    const DevInst D = P.inst[inst];
    __threadfence();
    int mode = 0;   // 0 nothing, 1 all tiles, 2 tiles with active pixels
    if (lane == 0) {
        const int phase = S->phase;
        if (S->status != PMF_OK) {
            S->phase = PH_DONE;
        } else if (phase == PH_PR) {           // start a global relabel
            S->epoch = S->epoch + 1;
            S->epochs = S->epochs + 1;
            S->phase = PH_BFS;
            S->want_bfs = 0;
            S->pr_since = 0;
            mode = 1;
        } else if (phase == PH_BFS) {
            if (S->active == 0) {              // lambda step certified: record, advance
                const int k = S->k;
                P.flows[(size_t)inst * P.max_lambdas + k] = (long long)S->flow;
                S->k = k + 1;
                S->visits_step = 0;
                if (k + 1 >= D.n_lambda) {
                    S->phase = PH_DONE;
                } else {
                    S->phase = PH_PR;
                    S->pr_since = 0;
                    S->want_bfs = 0;
                    mode = 1;
                }
            } else if ((long long)S->visits_step > P.max_visits_per_tile * (long long)D.n_tiles) {
                S->status = PMF_ERR_NOT_CONVERGED;
                S->phase = PH_DONE;
            } else {
                S->phase = PH_PR;
                S->pr_since = 0;
                S->want_bfs = 0;
                mode = 2;
            }
        }
        __threadfence();
    }
    mode = __shfl_sync(FULL_MASK, mode, 0);
    if (mode) enqueue_tiles(P, inst, D, mode == 2);
}

// finish an item: wake neighbours, requeue or retire the tile, maybe change
// the instance's phase
__device__ void finish(const Params &P, int g, int inst, int phase, bool requeue, unsigned nb,
                       const DevInst &D) {
    const int lane = threadIdx.x & 31;
    int trans = 0, again = 0;
    if (lane == 0) {
        volatile InstState *IS = P.ist + inst;
        bool allow = false;
        if (IS->status == PMF_OK) {
            if (phase == PH_BFS) allow = true;
            else if (phase == PH_PR) allow = (IS->want_bfs == 0);
        }
        if (allow && nb) {
            const int lt = g - D.tile_base;
            const int ty = lt / D.tiles_x, tx = lt - ty * D.tiles_x;
            if ((nb & 1) && ty > 0) request(P, g - D.tiles_x, inst);
            if ((nb & 2) && ty < D.tiles_y - 1) request(P, g + D.tiles_x, inst);
            if ((nb & 4) && tx > 0) request(P, g - 1, inst);
            if ((nb & 8) && tx < D.tiles_x - 1) request(P, g + 1, inst);
        }
        int *st = &P.tiles[g].state;
        if (requeue && allow) {
            atomicExch(st, T_QUEUED);
            again = 1;
        } else {
            const int old = atomicCAS(st, T_RUNNING, T_IDLE);
            if (old == T_DIRTY) {
                if (allow) { atomicExch(st, T_QUEUED); again = 1; }
                else atomicExch(st, T_IDLE);
            }
        }
        if (again) {
            __threadfence();
            push1(P, g);
        } else {
            const int o = atomicSub(&P.ist[inst].outstanding, 1);
            trans = (o == 1);
        }
        atomicAdd(&P.g->completed, 1ULL);
    }
    trans = __shfl_sync(FULL_MASK, trans, 0);
    again = __shfl_sync(FULL_MASK, again, 0);
    if (trans) transition(P, inst);
    if (lane == 0 && !again) atomicAdd((unsigned long long *)&P.g->pending, ~0ULL);   // -1
}

// --------------------------------------------------------------------------
// push/relabel visit of one tile (Goldberg-Tarjan push and relabel operations,
// the solver the paper runs through NPPI, Section 3)
// --------------------------------------------------------------------------
template <int TH>
__device__ void pr_visit(const Params &P, WarpSmem<TH> &S, int g, int inst, const DevInst &D,
                         int kcur, bool &self_active, unsigned &nbmask) {
    const int lane = threadIdx.x & 31;
    const int lt = g - D.tile_base;
    const int ty = lt / D.tiles_x, tx = lt - ty * D.tiles_x;
    const int x0 = tx * TILE_W, y0 = ty * TH, x = x0 + lane;
    const int pitch = D.pitch;
    const size_t PS = (size_t)D.rows * pitch;
    int *base = P.planes + D.plane_off;
    int *E = base + P_E * PS, *Hh = base + P_H * PS, *RT = base + P_RT * PS;
    int *FR = base + P_FR * PS, *FD = base + P_FD * PS;
    const int *SLOPE = base + P_SLOPE * PS;
    const int *WH = P.img + D.img_off;
    const int *WV = WH + PS;

    int e[TH], h[TH], rt[TH], fr[TH], fd[TH], wh[TH], wv[TH], e0[TH];
    long long srt0 = 0;
#pragma unroll
    for (int i = 0; i < TH; ++i) {
        const size_t idx = (size_t)(y0 + i) * pitch + x;
        e[i] = __ldcg(E + idx);
        h[i] = __ldcg(Hh + idx);
        rt[i] = __ldcg(RT + idx);
        fr[i] = __ldcg(FR + idx);
        fd[i] = __ldcg(FD + idx);
        wh[i] = __ldg(WH + idx);
        wv[i] = __ldg(WV + idx);
        e0[i] = e[i];
        srt0 += rt[i];
    }
    const int fd0b = fd[TH - 1];

    // GGT warm start: raise the source capacities to lambda_k (Section 2.1's
    // monotone case keeps the old flow valid); the newly available source
    // capacity becomes excess, and the part the sink arc can take is sent there
    TileState *TS = P.tiles + g;
    const int tl = ldv(&TS->lam);
    if (tl < kcur) {
        const int *L = P.lambdas + (size_t)inst * P.max_lambdas;
        const int dl = L[kcur] - L[tl];
#pragma unroll
        for (int i = 0; i < TH; ++i) {
            const int sl = __ldg(SLOPE + (size_t)(y0 + i) * pitch + x);
            e[i] += sl * dl;
            const int m = min(e[i], rt[i]);
            e[i] -= m;
            rt[i] -= m;
        }
        if (lane == 0) TS->lam = kcur;
    }

    // halo
    int hT = HINF, wvT = 0, fdT = 0, hB = HINF;
    if (y0 > 0) {
        const size_t j = (size_t)(y0 - 1) * pitch + x;
        hT = __ldcg(Hh + j);
        wvT = __ldg(WV + j);
        fdT = __ldcg(FD + j);
    }
    const int fdT0 = fdT;
    if (y0 + TH < D.rows) hB = __ldcg(Hh + (size_t)(y0 + TH) * pitch + x);
    if (lane < TH) {
        const size_t j = (size_t)(y0 + lane) * pitch;
        if (x0 > 0) {
            S.lh[lane] = __ldcg(Hh + j + x0 - 1);
            S.lw[lane] = __ldg(WH + j + x0 - 1);
            S.lf[lane] = __ldcg(FR + j + x0 - 1);
        } else {
            S.lh[lane] = HINF;
            S.lw[lane] = 0;
            S.lf[lane] = 0;
        }
        S.lf0[lane] = S.lf[lane];
        S.lout[lane] = 0;
        S.rh[lane] = (x0 + TILE_W < pitch) ? __ldcg(Hh + j + x0 + TILE_W) : HINF;
        S.rout[lane] = 0;
    }
    if (lane == 31) {
#pragma unroll
        for (int i = 0; i < TH; ++i) S.rf0[i] = fr[i];
    }
    __syncwarp();

    int outU = 0, outD = 0;
    const int hcap = D.hcap;
    for (int sw = 0; sw < P.sweeps; ++sw) {
        // push phase: every active pixel sends excess to t first, then to
        // lower neighbours along residual arcs; heights are not changed here,
        // so the two ends of an edge never push against each other
#pragma unroll
        for (int i = 0; i < TH; ++i) {
            const int hp = h[i];
            int hL = __shfl_up_sync(FULL_MASK, hp, 1);
            int hR = __shfl_down_sync(FULL_MASK, hp, 1);
            int rL = __shfl_up_sync(FULL_MASK, wh[i] + fr[i], 1);
            if (lane == 0) { hL = S.lh[i]; rL = S.lw[i] + S.lf[i]; }
            if (lane == 31) hR = S.rh[i];
            const int hU = (i > 0) ? h[i - 1] : hT;
            const int hD = (i < TH - 1) ? h[i + 1] : hB;
            const int rR = wh[i] - fr[i];
            const int rD = wv[i] - fd[i];
            const int rU = (i > 0) ? (wv[i - 1] + fd[i - 1]) : (wvT + fdT);
            int ex = e[i];
            int dT = 0, dD = 0, dR = 0, dU = 0, dL = 0;
            if (ex > 0 && hp < HINF) {
                dT = min(ex, rt[i]);
                ex -= dT;
                if (ex > 0 && rD > 0 && hD < hp) { dD = min(ex, rD); ex -= dD; }
                if (ex > 0 && rR > 0 && hR < hp) { dR = min(ex, rR); ex -= dR; }
                if (ex > 0 && rU > 0 && hU < hp) { dU = min(ex, rU); ex -= dU; }
                if (ex > 0 && rL > 0 && hL < hp) { dL = min(ex, rL); ex -= dL; }
            }
            e[i] = ex;
            rt[i] -= dT;
            fr[i] += dR;
            fd[i] += dD;
            if (i < TH - 1) e[i + 1] += dD; else outD += dD;
            if (i > 0) { e[i - 1] += dU; fd[i - 1] -= dU; } else { outU += dU; fdT -= dU; }
            const int inR = __shfl_up_sync(FULL_MASK, dR, 1);
            const int inL = __shfl_down_sync(FULL_MASK, dL, 1);
            if (lane > 0) e[i] += inR;
            if (lane < 31) { e[i] += inL; fr[i] -= inL; }
            if (lane == 31) S.rout[i] += dR;
            if (lane == 0) { S.lf[i] -= dL; S.lout[i] += dL; }
        }
        // relabel phase: an active pixel without an admissible arc moves to
        // one above its lowest residual neighbour (t has label 0)
        bool act = false;
#pragma unroll
        for (int i = 0; i < TH; ++i) {
            const int hp = h[i];
            int hL = __shfl_up_sync(FULL_MASK, hp, 1);
            int hR = __shfl_down_sync(FULL_MASK, hp, 1);
            int rL = __shfl_up_sync(FULL_MASK, wh[i] + fr[i], 1);
            if (lane == 0) { hL = S.lh[i]; rL = S.lw[i] + S.lf[i]; }
            if (lane == 31) hR = S.rh[i];
            if (e[i] > 0 && hp < HINF) {
                const int hU = (i > 0) ? h[i - 1] : hT;
                const int hD = (i < TH - 1) ? h[i + 1] : hB;
                const int rU = (i > 0) ? (wv[i - 1] + fd[i - 1]) : (wvT + fdT);
                int hmin = HINF;
                if (rt[i] > 0) hmin = 0;
                if (wv[i] - fd[i] > 0) hmin = min(hmin, hD);
                if (wh[i] - fr[i] > 0) hmin = min(hmin, hR);
                if (rU > 0) hmin = min(hmin, hU);
                if (rL > 0) hmin = min(hmin, hL);
                if (hmin >= hp) h[i] = (hmin >= HINF - 1 || hmin + 1 >= hcap) ? HINF : hmin + 1;
                act |= (h[i] < HINF);
            }
        }
        if (!__any_sync(FULL_MASK, act)) break;
    }

    // write back; pixels and edges on the tile border as atomic deltas
    long long srt1 = 0;
    bool act = false;
#pragma unroll
    for (int i = 0; i < TH; ++i) {
        const size_t idx = (size_t)(y0 + i) * pitch + x;
        srt1 += rt[i];
        act |= (e[i] > 0 && h[i] < HINF);
        const bool perim = (i == 0) || (i == TH - 1) || lane == 0 || lane == 31;
        if (perim) {
            const int d = e[i] - e0[i];
            if (d) atomicAdd(E + idx, d);
        } else {
            __stcg(E + idx, e[i]);
        }
        __stcg(Hh + idx, h[i]);
        __stcg(RT + idx, rt[i]);
        if (lane == 31) {
            const int d = fr[i] - S.rf0[i];
            if (d) atomicAdd(FR + idx, d);
        } else {
            __stcg(FR + idx, fr[i]);
        }
        if (i == TH - 1) {
            const int d = fd[i] - fd0b;
            if (d) atomicAdd(FD + idx, d);
        } else {
            __stcg(FD + idx, fd[i]);
        }
    }
    if (y0 > 0) {
        const size_t j = (size_t)(y0 - 1) * pitch + x;
        if (outU) atomicAdd(E + j, outU);
        if (fdT != fdT0) atomicAdd(FD + j, fdT - fdT0);
    }
    if (outD && y0 + TH < D.rows) atomicAdd(E + (size_t)(y0 + TH) * pitch + x, outD);
    __syncwarp();
    bool lo = false, ro = false;
    if (lane < TH) {
        const size_t j = (size_t)(y0 + lane) * pitch;
        if (x0 > 0) {
            if (S.lout[lane]) { atomicAdd(E + j + x0 - 1, S.lout[lane]); lo = true; }
            if (S.lf[lane] != S.lf0[lane]) atomicAdd(FR + j + x0 - 1, S.lf[lane] - S.lf0[lane]);
        }
        if (S.rout[lane] && x0 + TILE_W < pitch) { atomicAdd(E + j + x0 + TILE_W, S.rout[lane]); ro = true; }
    }
    unsigned nb = 0;
    if (__any_sync(FULL_MASK, outU > 0)) nb |= 1;
    if (__any_sync(FULL_MASK, outD > 0)) nb |= 2;
    if (__any_sync(FULL_MASK, lo)) nb |= 4;
    if (__any_sync(FULL_MASK, ro)) nb |= 8;
    nbmask = nb;
    self_active = __any_sync(FULL_MASK, act);

    long long df = srt0 - srt1;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) df += __shfl_down_sync(FULL_MASK, df, o);
    if (lane == 0) {
        if (df) atomicAdd(&P.ist[inst].flow, (unsigned long long)df);
        atomicAdd(&P.ist[inst].pr_visits, 1ULL);
        atomicAdd(&P.ist[inst].visits_step, 1ULL);
        const int since = atomicAdd(&P.ist[inst].pr_since, 1) + 1;
        if ((long long)since * 100 >= (long long)P.relabel_pct * D.n_tiles)
            P.ist[inst].want_bfs = 1;
    }
}

// --------------------------------------------------------------------------
// global-relabel visit: one tile's share of the BFS from t over reverse
// residual arcs (exact distances by label-correcting relaxation to a fixpoint;
// unreachable pixels keep HINF).  It also writes the cut mask of the current
// lambda (1 = cannot reach t = source side) and the tile's active count.
// --------------------------------------------------------------------------
template <int TH>
__device__ void bfs_visit(const Params &P, WarpSmem<TH> &S, int g, int inst, const DevInst &D,
                          int epoch, int kcur, bool &self_again, unsigned &nbmask) {
    const int lane = threadIdx.x & 31;
    const int lt = g - D.tile_base;
    const int ty = lt / D.tiles_x, tx = lt - ty * D.tiles_x;
    const int x0 = tx * TILE_W, y0 = ty * TH, x = x0 + lane;
    const int pitch = D.pitch;
    const size_t PS = (size_t)D.rows * pitch;
    int *base = P.planes + D.plane_off;
    const int *E = base + P_E * PS, *RT = base + P_RT * PS;
    const int *FR = base + P_FR * PS, *FD = base + P_FD * PS;
    int *Hh = base + P_H * PS;
    const int *WH = P.img + D.img_off;
    const int *WV = WH + PS;
    TileState *TS = P.tiles + g;

    const bool own_valid = ldv(&TS->epoch) == epoch;
    const bool vT = ty > 0 && ldv(&P.tiles[g - D.tiles_x].epoch) == epoch;
    const bool vB = ty < D.tiles_y - 1 && ldv(&P.tiles[g + D.tiles_x].epoch) == epoch;
    const bool vL = tx > 0 && ldv(&P.tiles[g - 1].epoch) == epoch;
    const bool vR = tx < D.tiles_x - 1 && ldv(&P.tiles[g + 1].epoch) == epoch;
    __threadfence();

    int fr[TH], fd[TH], wh[TH], wv[TH], d[TH], dold[TH];
    unsigned epos = 0, rtpos = 0;
#pragma unroll
    for (int i = 0; i < TH; ++i) {
        const size_t idx = (size_t)(y0 + i) * pitch + x;
        if (__ldcg(E + idx) > 0) epos |= 1u << i;
        if (__ldcg(RT + idx) > 0) rtpos |= 1u << i;
        fr[i] = __ldcg(FR + idx);
        fd[i] = __ldcg(FD + idx);
        wh[i] = __ldg(WH + idx);
        wv[i] = __ldg(WV + idx);
        d[i] = own_valid ? __ldcg(Hh + idx) : HINF;
        dold[i] = d[i];
        if (((rtpos >> i) & 1u) && d[i] > 1) d[i] = 1;
    }
    int hT = HINF, wvT = 0, fdT = 0, hB = HINF;
    if (y0 > 0) {
        const size_t j = (size_t)(y0 - 1) * pitch + x;
        wvT = __ldg(WV + j);
        fdT = __ldcg(FD + j);
        if (vT) hT = __ldcg(Hh + j);
    }
    if (vB) hB = __ldcg(Hh + (size_t)(y0 + TH) * pitch + x);
    if (lane < TH) {
        const size_t j = (size_t)(y0 + lane) * pitch;
        if (x0 > 0) {
            S.lh[lane] = vL ? __ldcg(Hh + j + x0 - 1) : HINF;
            S.lw[lane] = __ldg(WH + j + x0 - 1);
            S.lf[lane] = __ldcg(FR + j + x0 - 1);
        } else {
            S.lh[lane] = HINF;
            S.lw[lane] = 0;
            S.lf[lane] = 0;
        }
        S.rh[lane] = vR ? __ldcg(Hh + j + x0 + TILE_W) : HINF;
    }
    __syncwarp();

    // d(p) <= d(q) + 1 for every residual arc p -> q, relaxed to the fixpoint
    bool capped = true;
    for (int it = 0; it < 64 * TH; ++it) {
        bool ch = false;
#pragma unroll
        for (int i = 0; i < TH; ++i) {          // from the row above (arc p -> up)
            const int up = (i > 0) ? d[i - 1] : hT;
            const int rU = (i > 0) ? (wv[i - 1] + fd[i - 1]) : (wvT + fdT);
            if (rU > 0 && up + 1 < d[i]) { d[i] = up + 1; ch = true; }
        }
#pragma unroll
        for (int i = TH - 1; i >= 0; --i) {     // from the row below (arc p -> down)
            const int dn = (i < TH - 1) ? d[i + 1] : hB;
            if (wv[i] - fd[i] > 0 && dn + 1 < d[i]) { d[i] = dn + 1; ch = true; }
        }
#pragma unroll
        for (int i = 0; i < TH; ++i) {
            // from the right along runs of residual arcs p -> p+1: segmented
            // min-plus scan over the warp
            int v = d[i];
            int c = (wh[i] - fr[i]) > 0;
            if (lane == 31 && c && S.rh[i] + 1 < v) v = S.rh[i] + 1;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int v2 = __shfl_down_sync(FULL_MASK, v, o);
                const int c2 = __shfl_down_sync(FULL_MASK, c, o);
                if (lane + o < 32) {
                    if (c && v2 + o < v) v = v2 + o;
                    c = c & c2;
                } else {
                    c = 0;
                }
            }
            // from the left along runs of residual arcs p -> p-1
            int rl = __shfl_up_sync(FULL_MASK, wh[i] + fr[i], 1);
            if (lane == 0) rl = S.lw[i] + S.lf[i];
            int c3 = rl > 0;
            if (lane == 0 && c3 && S.lh[i] + 1 < v) v = S.lh[i] + 1;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int v2 = __shfl_up_sync(FULL_MASK, v, o);
                const int c2 = __shfl_up_sync(FULL_MASK, c3, o);
                if (lane >= o) {
                    if (c3 && v2 + o < v) v = v2 + o;
                    c3 = c3 & c2;
                } else {
                    c3 = 0;
                }
            }
            if (v < d[i]) { d[i] = v; ch = true; }
        }
        if (!__any_sync(FULL_MASK, ch)) { capped = false; break; }
    }
    self_again = capped;

    // which neighbours can now improve: a border pixel p got a smaller label
    // than the neighbour q could have read, q -> p is residual and q's label
    // is above d(p) + 1
    bool wT = false, wB = false, wL = false, wR = false;
    if (y0 > 0) wT = d[0] < dold[0] && (wvT - fdT) > 0 && d[0] + 1 < hT;
    if (ty < D.tiles_y - 1) wB = d[TH - 1] < dold[TH - 1] && (wv[TH - 1] + fd[TH - 1]) > 0 && d[TH - 1] + 1 < hB;
    if (lane == 0 && tx > 0) {
#pragma unroll
        for (int i = 0; i < TH; ++i)
            wL |= d[i] < dold[i] && (S.lw[i] - S.lf[i]) > 0 && d[i] + 1 < S.lh[i];
    }
    if (lane == 31 && tx < D.tiles_x - 1) {
#pragma unroll
        for (int i = 0; i < TH; ++i)
            wR |= d[i] < dold[i] && (wh[i] + fr[i]) > 0 && d[i] + 1 < S.rh[i];
    }
    unsigned nb = 0;
    if (__any_sync(FULL_MASK, wT)) nb |= 1;
    if (__any_sync(FULL_MASK, wB)) nb |= 2;
    if (__any_sync(FULL_MASK, wL)) nb |= 4;
    if (__any_sync(FULL_MASK, wR)) nb |= 8;
    nbmask = nb;

    // labels, mask of lambda_k, active count
    uint8_t *M = P.masks + D.mask_off + (size_t)kcur * PS;
    int cnt = 0;
#pragma unroll
    for (int i = 0; i < TH; ++i) {
        const size_t idx = (size_t)(y0 + i) * pitch + x;
        __stcg(Hh + idx, d[i]);
        M[idx] = d[i] >= HINF ? 1 : 0;
        cnt += __popc(__ballot_sync(FULL_MASK, ((epos >> i) & 1u) && d[i] < HINF));
    }
    __threadfence();
    __syncwarp();
    if (lane == 0) {
        *(volatile int *)&TS->epoch = epoch;
        const int old = TS->active;
        TS->active = cnt;
        if (cnt != old) atomicAdd(&P.ist[inst].active, cnt - old);
        atomicAdd(&P.ist[inst].bfs_visits, 1ULL);
        atomicAdd(&P.ist[inst].visits_step, 1ULL);
    }
}

// --------------------------------------------------------------------------
// persistent worker
// --------------------------------------------------------------------------
constexpr int WORKER_WARPS = 4;

template <int TH>
__global__ void __launch_bounds__(WORKER_WARPS * 32) worker_kernel(const __grid_constant__ Params P) {
    __shared__ WarpSmem<TH> smem[WORKER_WARPS];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WarpSmem<TH> &S = smem[w];
    for (;;) {
        int g = 0;
        if (lane == 0) g = ring_pop(P);
        g = __shfl_sync(FULL_MASK, g, 0);
        if (g < 0) break;
        const int inst = P.tile_inst[g];
        const DevInst D = P.inst[inst];
        volatile InstState *IS = P.ist + inst;
        int phase = 0, status = 0, epoch = 0, k = 0;
        if (lane == 0) {
            atomicExch(&P.tiles[g].state, T_RUNNING);
            __threadfence();
            phase = IS->phase;
            status = IS->status;
            epoch = IS->epoch;
            k = IS->k;
        }
        phase = __shfl_sync(FULL_MASK, phase, 0);
        status = __shfl_sync(FULL_MASK, status, 0);
        epoch = __shfl_sync(FULL_MASK, epoch, 0);
        k = __shfl_sync(FULL_MASK, k, 0);
        __syncwarp();
        bool requeue = false;
        unsigned nb = 0;
        if (status == PMF_OK && phase == PH_PR) pr_visit<TH>(P, S, g, inst, D, k, requeue, nb);
        else if (status == PMF_OK && phase == PH_BFS) bfs_visit<TH>(P, S, g, inst, D, epoch, k, requeue, nb);
        __threadfence();
        __syncwarp();
        finish(P, g, inst, phase, requeue, nb, D);
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
    for (size_t i = t0; i < cap; i += stride) P.ring[i] = (i < (size_t)P.n_tiles_total) ? (int)i : -1;
    for (size_t i = t0; i < (size_t)P.n_tiles_total; i += stride) {
        TileState t;
        t.state = T_QUEUED;
        t.epoch = 0;
        t.lam = 0;
        t.active = 0;
        P.tiles[i] = t;
    }
    for (size_t i = t0; i < (size_t)P.n_inst; i += stride) {
        const DevInst D = P.inst[i];
        for (int j = 0; j < D.n_tiles; ++j) ((int32_t *)P.tile_inst)[D.tile_base + j] = (int)i;
        InstState s;
        s.phase = PH_BFS;
        s.k = 0;
        s.epoch = 1;
        s.outstanding = D.n_tiles;
        s.active = 0;
        s.want_bfs = 0;
        s.vflags = P.inst_flags[i] | P.img_flags[D.image];
        s.status = flags_to_status(s.vflags);
        s.flow = 0;
        s.pr_since = 0;
        s.pad_ = 0;
        s.pr_visits = 0;
        s.bfs_visits = 0;
        s.epochs = 1;
        s.visits_step = 0;
        P.ist[i] = s;
    }
    if (t0 == 0) {
        Globals G;
        G.head = 0;
        G.tail = (unsigned long long)P.n_tiles_total;
        G.round_end = G.tail;
        G.pending = P.n_tiles_total;
        G.completed = 0;
        G.err = 0;
        G.round_mode = 0;
        G.items = 0;
        G.t_start = gtime_ns();
        *P.g = G;
    }
}

// lambda_0 preflow: saturate every source arc, send what the sink arc can take
// straight to t, zero pairwise flow, labels unknown until the first BFS
__global__ void init_kernel(const __grid_constant__ Params P) {
  for (int inst = blockIdx.y; inst < P.n_inst; inst += gridDim.y) {
    const DevInst D = P.inst[inst];
    const size_t PS = (size_t)D.rows * D.pitch;
    int32_t *base = P.planes + D.plane_off;
    const int32_t *L = P.lambdas + (size_t)inst * P.max_lambdas;
    const long long lam0 = L[0], lamN = L[D.n_lambda - 1];
    long long fsum = 0;
    int bad = 0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < PS; i += (size_t)gridDim.x * blockDim.x) {
        const int s0 = base[P_SRC0 * PS + i], sl = base[P_SLOPE * PS + i], ct = base[P_CT * PS + i];
        const long long cs0 = (long long)s0 + (long long)sl * lam0;
        const long long csN = (long long)s0 + (long long)sl * lamN;
        if (cs0 < 0) bad |= VF_NEG;
        if (csN > PMF_INF) bad |= VF_OVERFLOW;
        int e = (cs0 < 0 || csN > PMF_INF) ? 0 : (int)cs0;
        int rt = ct;
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
    pad_image_kernel<<<blocks, 256, 0, s>>>(wh, wh + n, w_h, w_v, d.H, d.W, d.rows, d.pitch, flags);
    return cudaGetLastError();
}

cudaError_t launch_pad_terminals(const Params &P, int inst, const DevInst &d, const int32_t *src0,
                                 const int32_t *slope, const int32_t *sink, cudaStream_t s) {
    int32_t *base = P.planes + d.plane_off;
    const size_t n = (size_t)d.rows * d.pitch;
    const int blocks = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
    pad_terminals_kernel<<<blocks, 256, 0, s>>>(base + P_SRC0 * n, base + P_SLOPE * n, base + P_CT * n,
                                                src0, slope, sink, d.H, d.W, d.rows, d.pitch,
                                                P.inst_flags + inst);
    return cudaGetLastError();
}

cudaError_t launch_reset(const Params &P, cudaStream_t s) {
    const size_t n = (size_t)P.ring_mask + 1;
    const int blocks = (int)((n + 255) / 256 < 2048 ? (n + 255) / 256 : 2048);
    reset_kernel<<<blocks, 256, 0, s>>>(P);
    return cudaGetLastError();
}

cudaError_t launch_init(const Params &P, int max_pixels, cudaStream_t s) {
    int bx = (max_pixels + 255) / 256;
    if (bx > 64) bx = 64;
    if (bx < 1) bx = 1;
    dim3 grid(bx, P.n_inst < 65535 ? P.n_inst : 65535);
    init_kernel<<<grid, 256, 0, s>>>(P);
    return cudaGetLastError();
}

cudaError_t launch_worker(const Params &P, int grid, cudaStream_t s) {
    if (P.tile_h == 4) worker_kernel<4><<<grid, WORKER_WARPS * 32, 0, s>>>(P);
    else worker_kernel<8><<<grid, WORKER_WARPS * 32, 0, s>>>(P);
    return cudaGetLastError();
}

cudaError_t launch_begin_round(const Params &P, cudaStream_t s) {
    begin_round_kernel<<<1, 1, 0, s>>>(P.g);
    return cudaGetLastError();
}

int worker_warps_per_block() { return WORKER_WARPS; }

cudaError_t worker_occupancy(int tile_h, int *blocks_per_sm) {
    if (tile_h == 4)
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, worker_kernel<4>, WORKER_WARPS * 32, 0);
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, worker_kernel<8>, WORKER_WARPS * 32, 0);
}

}  // namespace pmf
