/*
 * pmf.h - batched parametric maximum flow / minimum cut on 4-connected image
 * grids, CUDA (sm_103a).
 *
 * The problem (Section 2 of "A Parallel Framework for Parametric Maximum Flow
 * Problems in Image Segmentation", Olaru, Florea, Sminchisescu): every pixel p
 * of an H x W image is a node joined to the source s by an arc of capacity
 * cs(p), to the sink t by an arc of capacity ct(p), and to each of its up /
 * down / left / right neighbours q by arcs p->q and q->p of capacity w(p,q).
 * A minimum s-t cut splits the pixels into a foreground (s) side and a
 * background (t) side at least cost; its cost equals the maximum flow value.
 *
 * Parametric form (Section 2.1): cs(p, lambda) = src0(p) + slope(p) * lambda
 * with slope >= 0, solved for a nondecreasing lambda schedule.  The minimum
 * cuts are then nested and the flow of lambda_k is a valid start for
 * lambda_{k+1} (Gallo-Grigoriadis-Tarjan, cited in Sections 2.1 and 3).
 *
 * Batching (Section 3.1, "supergraphs"): the paper knits many (seed, lambda)
 * problems into one graph so that one solver call fills the GPU; the minimum
 * cut of the union decomposes into the minimum cuts of the parts.  Here a
 * batch holds many independent instances (one instance = one image with one
 * set of terminal capacities and its own lambda schedule) that are solved in
 * one persistent launch without any knitting vertices.
 *
 * Outputs per solve (instance, lambda_k): the maximum flow value (int64) and a
 * uint8 mask of the MAXIMAL source set: mask[p] = 1 iff pixel p cannot reach t
 * in the residual graph of a maximum flow; this set is the union of the s
 * sides of all minimum cuts.  Both outputs are unique, so the results do not
 * depend on how the GPU schedules its work.
 *
 * Conventions
 *   - Every call returns a pmf_status and never aborts or traps.
 *   - Images are row-major int32 arrays of H*W elements, pixel (y, x) at
 *     index y*W + x.
 *   - Input pointers are borrowed: the library reads them inside the call or
 *     in stream order on the batch's stream; host buffers must stay valid
 *     until pmf_sync returns.
 *   - The caller owns the device workspace (e.g. a torch tensor) and every
 *     output buffer.  The library owns the opaque pmf_batch and a few small
 *     pinned host buffers it allocates in pmf_create_batch.
 *   - Capacities are integers: 0 <= w <= PMF_MAX_PAIRWISE, 0 <= ct <= PMF_INF,
 *     0 <= src0 + slope*lambda <= PMF_INF for every lambda of the schedule.
 *     All arithmetic is exact (int32 state, int64 flow values).
 */
#ifndef PMF_H
#define PMF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define PMF_API __attribute__((visibility("default")))
#else
#define PMF_API
#endif

#define PMF_INF (1 << 30)                 /* largest terminal capacity ("infinite") */
#define PMF_MAX_PAIRWISE ((1 << 28) - 1)  /* largest pairwise capacity */

typedef enum {
    PMF_OK = 0,
    PMF_ERR_INVALID_ARG = 1,    /* bad pointer, index, size or negative capacity */
    PMF_ERR_OUT_OF_MEMORY = 2,  /* workspace smaller than pmf_workspace_size() */
    PMF_ERR_NOT_MONOTONE = 3,   /* decreasing lambda schedule or negative slope */
    PMF_ERR_OVERFLOW = 4,       /* a capacity above PMF_INF / PMF_MAX_PAIRWISE */
    PMF_ERR_CUDA = 5,           /* a CUDA runtime call failed */
    PMF_ERR_NOT_CONVERGED = 6,  /* the device watchdog stopped this instance; or a
                                   scheduler self-check failed, and then every
                                   instance of the launch reports it */
    PMF_ERR_NOT_READY = 7       /* results requested before a finished solve */
} pmf_status;

typedef struct pmf_batch pmf_batch;     /* opaque, owned by the library */

/* Batch shape.  All arrays are host arrays, read during the call. */
typedef struct {
    int32_t n_images;
    const int32_t *img_h;       /* [n_images] rows H >= 1 */
    const int32_t *img_w;       /* [n_images] cols W >= 1 */
    int32_t n_inst;
    const int32_t *inst_image;  /* [n_inst] image index of each instance */
    int32_t max_lambdas;        /* largest schedule length solved by this batch */
    int32_t device;             /* CUDA device ordinal */
} pmf_batch_desc;

/* Solver knobs (pmf_set_tuning).  Zero fields keep the default. */
typedef struct {
    int32_t tile_h;          /* rows per tile, 4 or 8 (tiles are 32 px wide); default 8 */
    int32_t sweeps;          /* push/relabel sweeps per tile visit; default 8 */
    int32_t relabel_every;   /* a push/relabel phase may spend relabel_every% of the
                                tiles it starts with in tile visits before the next
                                global relabel; default 800 (8 visits per tile) */
    int32_t max_visits_per_tile; /* watchdog: an instance stops with
                                PMF_ERR_NOT_CONVERGED after this many visits per
                                tile per lambda step on average; default 2000 */
    int32_t mode;            /* 0 = one persistent launch fed by the device queue
                                (default); 1 = host-polled rounds, one launch per
                                round (the per-solve-launch baseline) */
    int32_t blocks_per_sm;   /* persistent grid = blocks_per_sm * SMs; default: occupancy
                                (4 at tile height 4).  At tile height 4, 1-3 run a build
                                compiled for 3 resident blocks, with more registers per
                                thread and no spills (faster chains, fewer warps) */
    int32_t use_graph;       /* 1 = replay the solve as a captured CUDA graph (default 1;
                                ignored in mode 1) */
    int32_t trace;           /* 1 = record instance phase changes (pmf_get_trace) */
    int32_t poll_ns;         /* longest sleep of an idle worker warp between polls of
                                its queue slot, ns; default 256 */
    int32_t label_slack;     /* labels more than this above the largest finite distance
                                of the last global relabel are parked until the next
                                relabel; default 16 (0 = default, -1 = off) */
    int32_t grid_blocks;     /* persistent grid size in blocks (overrides blocks_per_sm;
                                0 = auto); lets several batches share the GPU */
    int32_t push_order;      /* order of the pushes inside a sweep: 0 = every row
                                and pixel from the sweep's starting state (default);
                                1 = along columns and rows, so excess that arrives
                                can move on in the same sweep */
    int32_t relabel_extra;   /* tile visits every push/relabel phase may spend on top
                                of relabel_every% of its tiles (default 0): more room
                                for phases that start with few active tiles */
    int32_t relabel_reach;   /* a push/relabel phase may spend at least relabel_reach% of
                                the largest finite distance of the last global relabel
                                in tile visits (default 0 = no such floor): phases that
                                start with few active tiles get room to carry their
                                excess that far before the next global relabel */
    int32_t strip_stage;     /* 1 = a relabel strip's first visit of a global relabel
                                loads its 32 rows of state and capacities with two
                                tensor copies into shared memory (one buffer per
                                block) instead of per-lane loads; -1 or 0 = per-lane
                                loads (default) */
} pmf_tuning;

/* One instance phase change recorded on the device (tuning.trace = 1). */
typedef struct {
    uint64_t t_ns;           /* device %globaltimer, ns */
    int32_t inst;
    int32_t event;           /* 0 global relabel started, 1 lambda step certified,
                                2 push/relabel restarted after a relabel,
                                3 instance finished, 4 watchdog stopped it */
    int32_t k;               /* schedule index after the change */
    int32_t epoch;           /* global relabel count */
    int64_t pr_visits;       /* cumulative push/relabel tile visits */
    int64_t bfs_visits;      /* cumulative relabel tile visits */
    int64_t flow;            /* flow into t so far */
    int32_t active;          /* pixels with excess that can reach t, as of the last relabel */
    int32_t reserved;
} pmf_trace_event;

/* Per-instance counters of the last solve (pmf_get_stats). */
typedef struct {
    int64_t pr_visits;       /* push/relabel tile visits */
    int64_t bfs_visits;      /* global-relabel (BFS) strip visits */
    int64_t global_relabels; /* BFS epochs */
    int32_t lambdas_done;    /* schedule entries solved */
    int32_t status;          /* pmf_status of the instance */
    int64_t warm_visits;     /* strip visits raising the source capacities at a lambda step */
} pmf_stats;

/* Bytes of device workspace a batch of this shape needs (host-only call). */
PMF_API pmf_status pmf_workspace_size(const pmf_batch_desc *desc, size_t *bytes);

/* Create a batch over a caller-owned device workspace of at least
 * pmf_workspace_size() bytes (256-byte aligned).  cuda_stream (a cudaStream_t,
 * may be NULL for the legacy default stream) orders the set-up copies.
 * PMF_ERR_OUT_OF_MEMORY if the workspace is too small. */
PMF_API pmf_status pmf_create_batch(const pmf_batch_desc *desc, void *dev_workspace, size_t bytes,
                            void *cuda_stream, pmf_batch **out);

/* Solver knobs; takes effect at the next pmf_solve_schedule. */
PMF_API pmf_status pmf_set_tuning(pmf_batch *b, const pmf_tuning *t);
PMF_API pmf_status pmf_get_tuning(const pmf_batch *b, pmf_tuning *t);

/* Pairwise capacities of one image (Section 2: the smoothness edges).
 * w_h[y*W + x] joins (y,x)-(y,x+1), w_v[y*W + x] joins (y,x)-(y+1,x); the last
 * column of w_h and the last row of w_v are ignored.  on_device = 1: device
 * pointers (checked on the device, errors reported by pmf_sync; the arrays are
 * read by work queued on the batch's stream); 0: host pointers, copied and
 * checked on the device before the call returns (PMF_ERR_INVALID_ARG for a
 * negative capacity, PMF_ERR_OVERFLOW above the maximum); the host arrays may
 * be reused as soon as it returns.  After an error the image (or instance) is
 * marked invalid until a later call succeeds: a solve in between reports the
 * error for the instances concerned. */
PMF_API pmf_status pmf_set_capacities(pmf_batch *b, int32_t image, const int32_t *w_h,
                              const int32_t *w_v, int on_device);

/* Terminal capacities of one instance (Section 2: the unary edges; Section
 * 2.1: the lambda-dependent source side).  cs(p, lambda) = src0[p] +
 * slope[p]*lambda, ct(p) = sink[p].  slope < 0 gives PMF_ERR_NOT_MONOTONE
 * (reported first), a capacity above PMF_INF PMF_ERR_OVERFLOW, a negative one
 * PMF_ERR_INVALID_ARG.  on_device as for pmf_set_capacities. */
PMF_API pmf_status pmf_set_terminals(pmf_batch *b, int32_t inst, const int32_t *src0,
                             const int32_t *slope, const int32_t *sink, int on_device);

/* Instance dst takes the terminal capacities last set for instance src (both
 * instances of the same image), with src's validation result: one
 * device-to-device copy queued on the batch's stream, no host transfer.  For
 * one problem split into several instances, e.g. a seed's schedule cut into
 * pieces that run side by side (Section 3.1's supergraph of (seed, lambda)
 * problems).  Only the capacity planes are copied: dst keeps its own cut rule
 * and slope side (pmf_set_cut_rule, pmf_set_slope_side).  PMF_ERR_INVALID_ARG
 * for an index out of range or instances of different images; dst == src does
 * nothing. */
PMF_API pmf_status pmf_copy_terminals(pmf_batch *b, int32_t dst, int32_t src);

/* Section 3.2's s-t swap: the caller may solve an instance with s and t
 * exchanged, passing its sink capacities as src0 (slope 0) and its source
 * capacities at one lambda as sink through pmf_set_terminals (pairwise
 * capacities are symmetric, so the exchanged problem is the same grid).
 * rule = 1 tells the solver so: the flow value is unchanged, and the mask
 * pmf_get_cut(s) returns is the ORIGINAL problem's maximal source set, i.e.
 * the complement of the exchanged problem's minimal source set.  The GPU finds
 * that set after each certified step as the pixels reachable in the residual
 * graph from pixels holding excess (every minimum cut's source side contains
 * them, and they form one).  rule = 0 (default): the maximal source set of the
 * problem as given.  Takes effect at the next pmf_solve_schedule.  A
 * warm-started exchanged schedule also needs the exchanged sink capacities to
 * follow lambda: see pmf_set_slope_side.  PMF_ERR_INVALID_ARG for a bad
 * instance or rule. */
PMF_API pmf_status pmf_set_cut_rule(pmf_batch *b, int32_t inst, int32_t rule);

/* Which terminal arcs follow lambda (Section 2.1's monotone case: the factors
 * of lambda are all of one sign).  side = 0 (default): the source capacities
 * rise, cs(p, lambda) = src0 + slope * lambda, and ct(p) = sink.  side = 1:
 * the sink capacities fall, cs(p) = src0 and ct(p, lambda) = sink - slope *
 * lambda; a solve then reports PMF_ERR_INVALID_ARG for the instance if some
 * ct(p, lambda) of its schedule is negative.  Either way the maximal source
 * sets grow with lambda, so the GGT warm start carries each step's flow and
 * labels to the next: with side 1 a sink arc that carries more than its new
 * capacity gives the surplus back to its pixel as excess.  Side 1 with
 * pmf_set_cut_rule(1) solves an exchanged problem over a whole schedule: with
 * s and t exchanged, the original source capacities src0 + slope * lambda
 * become sink capacities, and they fall as lambda falls, so the exchanged
 * problem runs the original schedule backwards, with parameter
 * mu = lambda_last - lambda and sink = src0 + slope * lambda_last.  The
 * pair capacities and the planes are unchanged; only the instance's arithmetic
 * differs.  Takes effect at the next pmf_solve_schedule.  PMF_ERR_INVALID_ARG
 * for a bad instance or side. */
PMF_API pmf_status pmf_set_slope_side(pmf_batch *b, int32_t inst, int32_t side);

/* lambda-state copies (Section 3.1's supergraphs mix problems of one seed at
 * several lambdas; GGT's warm start lets each start from an earlier one's
 * flow): instance child starts from instance parent's state as it is once the
 * parent has certified step parent_step of its schedule, instead of from the
 * zero flow.  At that point, between the parent's steps, the parent's strips
 * copy its flow, labels, excess and terminal capacities into the child (the
 * child's own terminals are not used), the parent goes on with its next
 * lambda and the child with the warm start from the parent's lambda to its
 * own first lambda, so the two run side by side.  Both must be instances of
 * the same image, with the same slope side and cut rule; a parent has at most
 * one child (which may itself be a parent).  The solve checks that the
 * parent's schedule has step parent_step, that the child's first lambda is
 * not below the parent's lambda there (else PMF_ERR_NOT_MONOTONE) and that no
 * chain of forks closes on itself.  A child whose parent fails before forking
 * it finishes with the parent's status.  parent = -1 removes child's fork.
 * Takes effect at the next solve.  PMF_ERR_INVALID_ARG for bad indices, a
 * parent of another image, or a parent that already has another child. */
PMF_API pmf_status pmf_set_fork(pmf_batch *b, int32_t child, int32_t parent, int32_t parent_step);

/* Solve every instance at every lambda of its schedule.  lambdas is a host
 * array [n_inst][n_lambda] (n_lambda <= max_lambdas), nondecreasing along each
 * row (else PMF_ERR_NOT_MONOTONE, nothing launched).  Asynchronous on
 * cuda_stream; call pmf_sync before reading results.  lambda_0 starts from the
 * zero flow; each later lambda keeps the previous flow and labels (GGT warm
 * start). */
PMF_API pmf_status pmf_solve_schedule(pmf_batch *b, const int32_t *lambdas, int32_t n_lambda,
                              void *cuda_stream);

/* As pmf_solve_schedule, with a schedule length per instance (one launch for
 * instances whose lambda counts differ, Section 3.1's supergraph of uneven
 * parametric problems).  lambdas is a host array [n_inst][stride]; instance i
 * solves its first lengths[i] values, which must be nondecreasing
 * (1 <= lengths[i] <= stride <= max_lambdas; entries past lengths[i] are
 * ignored).  lengths is a host array of n_inst values.  Results of instance i
 * are indexed k < lengths[i] (pmf_get_cut / pmf_get_flow), and
 * pmf_get_cuts / pmf_get_flows return lengths[i] entries.  Errors as
 * pmf_solve_schedule; NULL lengths is PMF_ERR_INVALID_ARG. */
PMF_API pmf_status pmf_solve_schedules(pmf_batch *b, const int32_t *lambdas, const int32_t *lengths,
                                       int32_t stride, void *cuda_stream);

/* Wait for the last solve.  per_instance (host, may be NULL) receives each
 * instance's pmf_status.  Returns PMF_OK iff every instance converged. */
PMF_API pmf_status pmf_sync(pmf_batch *b, pmf_status *per_instance);

/* Which instances have finished, without waiting: while a solve runs, the
 * kernel flags each instance in mapped host memory as it finishes, so
 * done[i] = 1 (host array of n_inst bytes, may be NULL) for a finished one and
 * *n_done (may be NULL) counts them; after pmf_sync every instance of the
 * solve is reported.  A finished instance that converged can be read at once
 * (pmf_get_cut(s), pmf_get_flow(s)) while the others still run: its results are
 * final.  Its status, and any failure, come with pmf_sync. */
PMF_API pmf_status pmf_poll(pmf_batch *b, uint8_t *done, int32_t *n_done);

/* Mask of solve (inst, k): H*W bytes, 1 = source (foreground) side.
 * on_device = 1: mask is a device pointer (copied in stream order, then the
 * stream is synchronised), 0: host pointer.  PMF_ERR_NOT_READY until the
 * instance has finished and converged (pmf_poll) or after a failed one. */
PMF_API pmf_status pmf_get_cut(pmf_batch *b, int32_t inst, int32_t k, uint8_t *mask, int on_device);

/* Maximum flow value of solve (inst, k) (Section 2: equal to the minimum cut
 * cost), once the instance has finished (pmf_poll, pmf_sync). */
PMF_API pmf_status pmf_get_flow(pmf_batch *b, int32_t inst, int32_t k, int64_t *flow);

/* Every mask of instance inst: n_lambda * H * W bytes, [k][y][x], as one copy
 * and a single synchronisation (on_device as for pmf_get_cut); n_lambda is the
 * instance's schedule length in the last solve. */
PMF_API pmf_status pmf_get_cuts(pmf_batch *b, int32_t inst, uint8_t *masks, int on_device);

/* Every flow value of instance inst: its schedule length's worth of int64
 * (host pointer). */
PMF_API pmf_status pmf_get_flows(pmf_batch *b, int32_t inst, int64_t *flows);

/* Device time of the last solve, from CUDA events the library records on the
 * launching stream (pmf_sync first): solve_ms from the start of the reset
 * kernel to the end of the result copies, worker_ms the persistent worker
 * kernel alone (summed over rounds in mode 1). */
PMF_API pmf_status pmf_get_timing(pmf_batch *b, float *solve_ms, float *worker_ms);

/* Phase-change trace of the last solve (tuning.trace = 1), after pmf_sync:
 * copies up to cap records to out (host) and sets *n to the number recorded
 * (at most 65536; later events are dropped). */
PMF_API pmf_status pmf_get_trace(pmf_batch *b, pmf_trace_event *out, int32_t cap, int32_t *n);

#define PMF_PROFILE_COUNTERS 12

/* Warp-time breakdown of the last solve (tuning.trace = 1), after pmf_sync,
 * into out[PMF_PROFILE_COUNTERS] (host): out[0..3] = ns summed over worker
 * warps spent waiting for work, in push/relabel visits, in global-relabel
 * visits and retiring items; out[4] = push/relabel sweeps run; out[5..7] = SM
 * cycles (summed over visits) of the push/relabel visits' load, sweep and
 * write-back stages; out[8..10] = the same for the relabel-strip visits'
 * load, relaxation and write-back stages; out[11] = relaxation rounds run by
 * the relabel-strip visits.  All zero when tracing was off. */
PMF_API pmf_status pmf_get_profile(pmf_batch *b, uint64_t *out);

/* A feasible maximum flow of instance inst, arc by arc, at the last lambda of
 * the most recent solve (Section 2's graph; the max-flow/min-cut theorem the
 * paper cites there makes its value the minimum cut cost).  The solve itself
 * ends with a maximum preflow; this call returns the excess left on pixels
 * that cannot reach t back towards s (the second phase of push-relabel), on
 * the GPU, without changing the instance's state, masks or flow values.
 * Outputs are caller-owned DEVICE arrays of H*W int32, row-major (y*W + x):
 *   f_h  net flow from (y,x) to (y,x+1), negative = leftwards; 0 in the last column
 *   f_v  net flow from (y,x) to (y+1,x), negative = upwards; 0 in the last row
 *   f_s  flow on the arc s -> (y,x), 0 <= f_s <= cs(y,x,lambda)
 *   f_t  flow on the arc (y,x) -> t, 0 <= f_t <= ct(y,x)
 * with |f_h| <= w_h, |f_v| <= w_v, flow in = flow out at every pixel and
 * sum(f_t) = pmf_get_flow of the last lambda.  Several maximum flows exist;
 * any one is returned.  Synchronous.  PMF_ERR_NOT_READY before a finished
 * solve or for a failed instance, PMF_ERR_NOT_CONVERGED if the return did not
 * finish within its sweep limit (2^17 sweeps). */
PMF_API pmf_status pmf_get_flow_arcs(pmf_batch *b, int32_t inst, int32_t *f_h, int32_t *f_v, int32_t *f_s,
                                     int32_t *f_t);

/* ------------------------------------------------------------------------ */
/* Exact parametric search (Section 2.1: finding every breakpoint of the      */
/* parametric minimum cut is the ideal the paper names; its preset lambda     */
/* schedules approximate it).  Two device helpers; the search itself          */
/* (parametric.exact_breakpoints in the Python package) solves the problems   */
/* they build with the batch entry points.                                    */
/* ------------------------------------------------------------------------ */

/* Capacity lines of cuts (Section 2's cut cost as a function of lambda): for
 * each of n_masks source sets S_k = masks[k] | base (1 = s side; base may be
 * NULL), cap_{S_k}(lambda) = a_k + b_k * lambda with
 *   a_k = sum_{p not in S_k} src0(p) + sum_{p in S_k} sink(p)
 *         + sum over 4-neighbour pairs split by S_k of their capacity,
 *   b_k = sum_{p not in S_k} slope(p).
 * All arrays are DEVICE pointers: w_h, w_v, src0, slope, sink are H*W int32
 * (row-major, as for pmf_set_capacities / pmf_set_terminals), base is H*W
 * bytes, masks n_masks*H*W bytes ([k][y][x]); lines receives 2*n_masks int64
 * (a_k, b_k); union_out (may be NULL) receives the sets S_k as n_masks*H*W
 * bytes.  Asynchronous on cuda_stream.  PMF_ERR_INVALID_ARG for a NULL
 * pointer, a bad size or n_masks outside [1, 65535]; PMF_ERR_CUDA if the
 * launch fails. */
PMF_API pmf_status pmf_cut_lines(int32_t H, int32_t W, const int32_t *w_h, const int32_t *w_v,
                                 const int32_t *src0, const int32_t *slope, const int32_t *sink,
                                 const uint8_t *base, const uint8_t *masks, int32_t n_masks,
                                 uint8_t *union_out, int64_t *lines, void *cuda_stream);

/* The problem restricted to the pixels between two nested source sets
 * s1 <= s2 (DEVICE masks of H*W bytes, 1 = s side) at lambda = p / q, scaled
 * by q so that every capacity is an integer.  Pixels of D = s2 \ s1 keep their
 * pair capacities to each other; a pixel's pairs into s1 join its source
 * capacity and its pairs into the complement of s2 its sink capacity; every
 * other pixel gets no arcs but a sink capacity of 1 (no flow passes it, and it
 * is never in the maximal source set).  Outputs (DEVICE, H*W int32 each):
 * w_h_out, w_v_out (pairs inside D, times q), src0_out = q*(src0 + pairs
 * from s1) + p*slope, sink_out = q*(sink + pairs out of s2); solve them with
 * slope 0.  sums (DEVICE, 4 int64): [0] sum of src0_out, [1] sum of
 * sink_out over D, [2] pixels whose scaled capacities exceed PMF_INF or
 * PMF_MAX_PAIRWISE (their outputs are zeroed and the problem must not be
 * used), [3] pixels in D.  Every cut between s1 and s2 costs a constant plus
 * the restricted problem's cut, so when s1 and s2 are maximal minimum cuts at
 * lambda_1 <= p/q <= lambda_2, the restricted problem's maximal source set
 * joined with s1 is the maximal minimum cut at p/q.  Asynchronous on
 * cuda_stream.  PMF_ERR_INVALID_ARG for a NULL pointer, a bad size, q < 1,
 * p < 0 or p, q above 2^31. */
PMF_API pmf_status pmf_restrict_between(int32_t H, int32_t W, const int32_t *w_h, const int32_t *w_v,
                                        const int32_t *src0, const int32_t *slope, const int32_t *sink,
                                        const uint8_t *s1, const uint8_t *s2, int64_t p, int64_t q,
                                        int32_t *w_h_out, int32_t *w_v_out, int32_t *src0_out,
                                        int32_t *sink_out, int64_t *sums, void *cuda_stream);

/* Counters of the last solve for one instance, after pmf_sync. */
PMF_API pmf_status pmf_get_stats(pmf_batch *b, int32_t inst, pmf_stats *out);

/* Device-side pointers of the results, for zero-copy consumers: masks of
 * instance inst as [max_lambdas][rows][pitch] bytes, rows/pitch returned. */
PMF_API pmf_status pmf_get_mask_layout(pmf_batch *b, int32_t inst, const uint8_t **dev_masks,
                               int32_t *rows, int32_t *pitch);

/* Release the host side of the batch (the workspace stays the caller's). */
PMF_API void pmf_destroy_batch(pmf_batch *b);

PMF_API const char *pmf_status_string(pmf_status s);

/* ------------------------------------------------------------------------ */
/* Server: continuous batching into one running kernel (Section 3.3.1's       */
/* dynamic scheduling, where each server takes the next problem as soon as it */
/* is free, and Section 3.3.2's overlap of one request's transfers with       */
/* another's computation).  A server owns n_slots instance slots, each able   */
/* to hold one instance of up to max_h x max_w pixels and max_lambdas         */
/* lambdas, and ONE persistent kernel that solves whatever is in its device   */
/* work queue.  The host loads a request's instances into free slots (copies  */
/* on a separate stream, while the kernel runs) and posts them; an idle       */
/* worker of the running kernel takes the posted slots from a mailbox in      */
/* mapped host memory, sets them up on the device and queues their work into  */
/* the same queue every running instance uses.  Finished slots are flagged in */
/* mapped host memory (pmf_server_poll) and read back while the others run.   */
/* No call allocates or synchronises the device while the kernel runs.        */
/* ------------------------------------------------------------------------ */
typedef struct pmf_server pmf_server;   /* opaque, owned by the library */

typedef struct {
    int32_t n_slots;         /* instance slots, 1 .. 4096 */
    int32_t max_h, max_w;    /* largest image a slot holds */
    int32_t max_lambdas;     /* longest schedule a slot holds */
    int32_t device;          /* CUDA device ordinal */
} pmf_server_desc;

/* Device workspace bytes of a server (host-only call). */
PMF_API pmf_status pmf_server_workspace_size(const pmf_server_desc *desc, size_t *bytes);

/* Create a server over a caller-owned device workspace of at least
 * pmf_server_workspace_size() bytes (256-byte aligned).  Allocates a few pinned
 * and mapped host buffers and two streams of its own.  PMF_ERR_OUT_OF_MEMORY
 * if the workspace is too small. */
PMF_API pmf_status pmf_server_create(const pmf_server_desc *desc, void *dev_workspace, size_t bytes,
                                     pmf_server **out);

/* Solver knobs of the server kernel (as pmf_set_tuning; the server runs tile
 * height 4 with pushes along columns and rows, so tile_h must be 0 or 4,
 * push_order is ignored and mode must be 0).  Only before pmf_server_start. */
PMF_API pmf_status pmf_server_set_tuning(pmf_server *s, const pmf_tuning *t);

/* Launch the server kernel (it runs until pmf_server_stop, or at most
 * max_seconds, after which it stops with PMF_ERR_NOT_CONVERGED for whatever
 * is unfinished).  Every slot starts free. */
PMF_API pmf_status pmf_server_start(pmf_server *s, double max_seconds);

/* Load one instance into a free slot (Section 2's grid graph and Section
 * 2.1's schedule, as for pmf_set_capacities / pmf_set_terminals /
 * pmf_solve_schedule): HOST arrays of H*W int32 (row-major) and n_lambda
 * nondecreasing lambdas (else PMF_ERR_NOT_MONOTONE).  image_slot == slot:
 * w_h, w_v are this slot's image; image_slot != slot: the instance uses the
 * image loaded into image_slot (w_h, w_v may be NULL), which must then stay
 * loaded, posted or unread until this slot has been read.  Capacities are
 * checked on the device when the instance starts; a bad one is reported by
 * pmf_server_read as by pmf_sync.  The copies run on the server's copy stream
 * while the kernel runs.  PMF_ERR_NOT_READY for a slot posted and not yet
 * read; PMF_ERR_INVALID_ARG for a bad slot, size or pointer. */
PMF_API pmf_status pmf_server_load(pmf_server *s, int32_t slot, int32_t image_slot, int32_t H, int32_t W,
                                   const int32_t *w_h, const int32_t *w_v, const int32_t *src0,
                                   const int32_t *slope, const int32_t *sink, const int32_t *lambdas,
                                   int32_t n_lambda);

/* Admit loaded slots into the running kernel: waits for their copies, then
 * posts them to the mailbox.  PMF_ERR_INVALID_ARG if the server is not running
 * or a slot is not loaded. */
PMF_API pmf_status pmf_server_post(pmf_server *s, const int32_t *slots, int32_t n);

/* Which posted slots have finished, without waiting: done[i] = 1 (host array
 * of n_slots bytes, may be NULL); *n_done (may be NULL) counts them. */
PMF_API pmf_status pmf_server_poll(pmf_server *s, uint8_t *done, int32_t *n_done);

/* Read a finished slot's results into HOST buffers: masks n_lambda*H*W bytes
 * ([k][y][x], 1 = source side: the maximal minimum cut) and flows n_lambda
 * int64, then free the slot.  Returns the instance's status (a failed one
 * leaves the buffers untouched); PMF_ERR_NOT_READY before it has finished. */
PMF_API pmf_status pmf_server_read(pmf_server *s, int32_t slot, uint8_t *masks, int64_t *flows);

/* End the server kernel once every posted slot has finished, and wait for it.
 * PMF_ERR_NOT_CONVERGED if it had stopped on a watchdog or its time limit. */
PMF_API pmf_status pmf_server_stop(pmf_server *s);

/* Stop the kernel if it runs and release the server's host side. */
PMF_API void pmf_server_destroy(pmf_server *s);

/* ------------------------------------------------------------------------ */
/* Solve without allocating (the paper has no counterpart: this entry point   */
/* exists for callers of this library, not for the method).                   */
/* ------------------------------------------------------------------------ */
#define PMF_NOALLOC_SCRATCH_MB 24      /* device memory reserved for it when the library loads */
#define PMF_NOALLOC_MAX_PIXELS 262144  /* limit on rows*pitch: rows = H rounded up to 16,
                                          pitch = W rounded up to 32 (e.g. 512 x 512) */
#define PMF_NOALLOC_MAX_LAMBDAS 32     /* limit on the schedule length */

/* One instance (one image, one set of terminal capacities, its lambda
 * schedule) solved with no memory allocation of any kind: no cudaMalloc,
 * cudaFree, pinned or pool allocation, no allocating library routine.  It is
 * meant for callers that cannot allocate device memory themselves or let a
 * library do it: code inside a host framework that owns the whole device
 * memory budget and hands out only pre-reserved buffers, and latency-critical
 * paths where cudaMalloc's implicit device-wide synchronisation is not
 * acceptable.  All scratch (state planes, masks, work queue) lives in one
 * fixed device array of PMF_NOALLOC_SCRATCH_MB MiB that every GPU using the
 * library holds until the process exits.
 *
 * Inputs: w_h, w_v, src0, slope, sink are DEVICE pointers to H*W int32 arrays
 * (same meaning as pmf_set_capacities / pmf_set_terminals); lambdas is a HOST
 * array of n_lambda nondecreasing values.  Outputs: masks is a DEVICE buffer
 * of n_lambda*H*W bytes ([k][y][x], 1 = source side), flows a HOST array of
 * n_lambda int64 values.  Runs on cuda_stream (a cudaStream_t, NULL = legacy
 * default stream) on the current device and returns when the results are in
 * place.
 *
 * Errors: sizes beyond PMF_NOALLOC_MAX_PIXELS or PMF_NOALLOC_MAX_LAMBDAS give
 * PMF_ERR_OUT_OF_MEMORY before any GPU work; a decreasing schedule gives
 * PMF_ERR_NOT_MONOTONE; invalid capacities give the statuses pmf_sync reports
 * for a batch; a failed CUDA call gives PMF_ERR_CUDA (pmf_last_error names
 * it) after the call has waited for whatever GPU work it had queued.  The
 * solver knobs are fixed: those the autotuner picks for one-instance
 * workloads (tile height 4, pushes along columns and rows, 8 sweeps per
 * visit, relabel cadence 800 %, label slack 16).
 *
 * The first call on a device looks up the array's device address for that
 * device (cudaGetSymbolAddress); make that first call before any stream
 * capture.  The array is shared by all calls and keeps the last call's
 * contents; every call re-initialises what must start from zero.  Calls whose
 * GPU work overlapped would race on the shared array, so calls from different
 * host threads are serialised by a process-wide lock held until the call's
 * GPU work has finished. */
PMF_API pmf_status pmf_solve_noalloc(int32_t H, int32_t W, const int32_t *w_h, const int32_t *w_v,
                                     const int32_t *src0, const int32_t *slope, const int32_t *sink,
                                     const int32_t *lambdas, int32_t n_lambda, uint8_t *masks,
                                     int64_t *flows, void *cuda_stream);

/* Test hook for the error paths of pmf_solve_noalloc (no counterpart in the
 * paper).  The n-th CUDA runtime call (counting from 1) of the NEXT
 * pmf_solve_noalloc call reports a failure instead of being made, so that a
 * test can check, without any GPU fault, that the call returns
 * PMF_ERR_CUDA, names the site in pmf_last_error, and has waited for the GPU
 * work it had already queued before releasing its lock (a later call then
 * gives correct results).  n <= 0 clears it; it applies to one call only. */
PMF_API void pmf_testing_fail_noalloc_call(int32_t n);

/* Text of the last CUDA failure seen by this thread ("" if none): the call
 * site and cudaGetErrorString, for diagnostics after PMF_ERR_CUDA. */
PMF_API const char *pmf_last_error(void);

/* Library version, e.g. "pmf 0.1.0 sm_103a". */
PMF_API const char *pmf_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PMF_H */
