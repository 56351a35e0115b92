/*
 * CPU oracle for s-t maximum flow / minimum cut on 4-connected image grids.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the
 * CUDA path is checked against.  It shares no code, header, table or helper
 * with the CUDA library; only tests/, __graft_entry__.smoke() and the CPU
 * baseline leg of bench.py load it.
 *
 * What it computes (Section 2 of the paper, "Graph-Cut based Image
 * Segmentation"): the graph has a node per pixel plus the source s and the
 * sink t.  Every pixel p has an arc s->p of capacity cs(p) and an arc p->t of
 * capacity ct(p) (both kept, no folding); every pair of 4-neighbours p, q has an
 * arc p->q and an arc q->p, each of capacity w(p,q).  The cost of an s-t cut is
 * the total capacity of the arcs leaving the s side; by the max-flow/min-cut
 * theorem (Ford-Fulkerson, cited in Section 2) its minimum equals the maximum
 * flow value.  For the parametric form (Section 2.1) the source capacity is
 * cs(p, lambda) = src0(p) + slope(p) * lambda with slope >= 0, and every lambda
 * of the schedule is solved from scratch here.
 *
 * Algorithms, all in int64:
 *   - Dinic: BFS level graph from s, then blocking flow by depth-first
 *     advance/retreat with current-arc pointers; repeat until t is unreachable.
 *   - Edmonds-Karp: shortest augmenting path by BFS, one path at a time (an
 *     independent second solver for cross-checks on small/medium graphs).
 *   - Cut: the maximal source set = nodes that cannot reach t in the residual
 *     graph, found by a BFS from t over arcs u->v with residual capacity > 0
 *     walked backwards.  It is the same for every maximum flow.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

/* ------------------------------------------------------------------------ */
/* residual graph: arc 2i is the i-th input arc, arc 2i+1 its reverse (cap 0) */
/* ------------------------------------------------------------------------ */
typedef struct {
    int n;            /* nodes */
    int m;            /* residual arcs (2 x input arcs) */
    int *to;          /* to[a]   head of arc a */
    int64_t *res;     /* res[a]  residual capacity of arc a */
    int *start;       /* CSR: arcs leaving u are adj[start[u] .. start[u+1]) */
    int *adj;
} rgraph;

static void rg_free(rgraph *g) {
    free(g->to); free(g->res); free(g->start); free(g->adj);
    memset(g, 0, sizeof(*g));
}

/* returns 0 on success, -1 on allocation failure or bad arc */
static int rg_build(rgraph *g, int n, int m_in, const int *tail, const int *head,
                    const int64_t *cap) {
    memset(g, 0, sizeof(*g));
    g->n = n;
    g->m = 2 * m_in;
    g->to = (int *)malloc(sizeof(int) * (size_t)(g->m > 0 ? g->m : 1));
    g->res = (int64_t *)malloc(sizeof(int64_t) * (size_t)(g->m > 0 ? g->m : 1));
    g->start = (int *)calloc((size_t)n + 1, sizeof(int));
    g->adj = (int *)malloc(sizeof(int) * (size_t)(g->m > 0 ? g->m : 1));
    if (!g->to || !g->res || !g->start || !g->adj) { rg_free(g); return -1; }
    for (int i = 0; i < m_in; i++) {
        int u = tail[i], v = head[i];
        if (u < 0 || u >= n || v < 0 || v >= n || cap[i] < 0) { rg_free(g); return -1; }
        g->to[2 * i] = v;     g->res[2 * i] = cap[i];
        g->to[2 * i + 1] = u; g->res[2 * i + 1] = 0;
        g->start[u + 1]++;
        g->start[v + 1]++;
    }
    for (int u = 0; u < n; u++) g->start[u + 1] += g->start[u];
    int *fill = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    if (!fill) { rg_free(g); return -1; }
    memcpy(fill, g->start, sizeof(int) * (size_t)n);
    for (int a = 0; a < g->m; a++) {
        int u = g->to[a ^ 1];          /* tail of arc a */
        g->adj[fill[u]++] = a;
    }
    free(fill);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Dinic                                                                     */
/* ------------------------------------------------------------------------ */
static int dinic_levels(const rgraph *g, int s, int t, int *level, int *queue) {
    for (int u = 0; u < g->n; u++) level[u] = -1;
    int qh = 0, qt = 0;
    level[s] = 0;
    queue[qt++] = s;
    while (qh < qt) {
        int u = queue[qh++];
        for (int k = g->start[u]; k < g->start[u + 1]; k++) {
            int a = g->adj[k];
            int v = g->to[a];
            if (g->res[a] > 0 && level[v] < 0) {
                level[v] = level[u] + 1;
                queue[qt++] = v;
            }
        }
    }
    return level[t] >= 0;
}

/* One blocking flow on the level graph; path search restarts from s after
 * every augmentation, current-arc pointers persist within the phase. */
static int64_t dinic_blocking(rgraph *g, int s, int t, const int *level, int *cur,
                              int *stack) {
    int64_t total = 0;
    for (;;) {
        int top = 0, u = s;
        while (u != t) {
            int found = -1;
            while (cur[u] < g->start[u + 1]) {
                int a = g->adj[cur[u]];
                if (g->res[a] > 0 && level[g->to[a]] == level[u] + 1) { found = a; break; }
                cur[u]++;
            }
            if (found >= 0) {
                stack[top++] = found;
                u = g->to[found];
            } else {                       /* dead end: retreat one arc */
                if (top == 0) return total;
                int a = stack[--top];
                u = g->to[a ^ 1];
                cur[u]++;
            }
        }
        int64_t f = INT64_MAX;
        for (int i = 0; i < top; i++) if (g->res[stack[i]] < f) f = g->res[stack[i]];
        for (int i = 0; i < top; i++) { g->res[stack[i]] -= f; g->res[stack[i] ^ 1] += f; }
        total += f;
    }
}

static int64_t dinic(rgraph *g, int s, int t, int *err) {
    int n = g->n;
    int *level = (int *)malloc(sizeof(int) * (size_t)n);
    int *queue = (int *)malloc(sizeof(int) * (size_t)n);
    int *cur = (int *)malloc(sizeof(int) * (size_t)n);
    int *stack = (int *)malloc(sizeof(int) * (size_t)n);
    int64_t flow = 0;
    *err = 0;
    if (!level || !queue || !cur || !stack) { *err = -1; goto out; }
    while (dinic_levels(g, s, t, level, queue)) {
        for (int u = 0; u < n; u++) cur[u] = g->start[u];
        flow += dinic_blocking(g, s, t, level, cur, stack);
    }
out:
    free(level); free(queue); free(cur); free(stack);
    return flow;
}

/* ------------------------------------------------------------------------ */
/* Edmonds-Karp                                                              */
/* ------------------------------------------------------------------------ */
static int64_t edmonds_karp(rgraph *g, int s, int t, int *err) {
    int n = g->n;
    int *parc = (int *)malloc(sizeof(int) * (size_t)n);   /* arc used to reach node */
    int *queue = (int *)malloc(sizeof(int) * (size_t)n);
    int64_t flow = 0;
    *err = 0;
    if (!parc || !queue) { *err = -1; goto out; }
    for (;;) {
        for (int u = 0; u < n; u++) parc[u] = -2;
        parc[s] = -1;
        int qh = 0, qt = 0;
        queue[qt++] = s;
        while (qh < qt && parc[t] == -2) {
            int u = queue[qh++];
            for (int k = g->start[u]; k < g->start[u + 1]; k++) {
                int a = g->adj[k];
                int v = g->to[a];
                if (g->res[a] > 0 && parc[v] == -2) { parc[v] = a; queue[qt++] = v; }
            }
        }
        if (parc[t] == -2) break;
        int64_t f = INT64_MAX;
        for (int v = t; v != s; v = g->to[parc[v] ^ 1]) if (g->res[parc[v]] < f) f = g->res[parc[v]];
        for (int v = t; v != s; v = g->to[parc[v] ^ 1]) { g->res[parc[v]] -= f; g->res[parc[v] ^ 1] += f; }
        flow += f;
    }
out:
    free(parc); free(queue);
    return flow;
}

/* reach[u] = 1 iff u can reach t along arcs with residual > 0 */
static int reach_sink(const rgraph *g, int t, uint8_t *reach) {
    int *queue = (int *)malloc(sizeof(int) * (size_t)g->n);
    if (!queue) return -1;
    memset(reach, 0, (size_t)g->n);
    int qh = 0, qt = 0;
    reach[t] = 1;
    queue[qt++] = t;
    while (qh < qt) {
        int v = queue[qh++];
        for (int k = g->start[v]; k < g->start[v + 1]; k++) {
            int a = g->adj[k];          /* arc v->u; its partner a^1 is u->v */
            int u = g->to[a];
            if (!reach[u] && g->res[a ^ 1] > 0) { reach[u] = 1; queue[qt++] = u; }
        }
    }
    free(queue);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* exported: generic graphs                                                   */
/* ------------------------------------------------------------------------ */
/*
 * oracle_maxflow: maximum s-t flow of the directed graph with n nodes and m
 * arcs (tail[i] -> head[i], capacity cap[i] >= 0).  algo 0 = Dinic, 1 =
 * Edmonds-Karp.  Outputs (each may be NULL): *value, arc_flow[m] (flow on each
 * input arc), sink_reach[n] (1 iff the node reaches t in the final residual
 * graph).  Returns 0, or -1 on a bad argument / allocation failure.
 */
int oracle_maxflow(int n, int m, const int *tail, const int *head, const int64_t *cap,
                   int s, int t, int algo, int64_t *value, int64_t *arc_flow,
                   uint8_t *sink_reach) {
    if (n <= 0 || m < 0 || s < 0 || s >= n || t < 0 || t >= n || s == t) return -1;
    rgraph g;
    if (rg_build(&g, n, m, tail, head, cap) != 0) return -1;
    int err = 0;
    int64_t f = (algo == 1) ? edmonds_karp(&g, s, t, &err) : dinic(&g, s, t, &err);
    if (err) { rg_free(&g); return -1; }
    if (value) *value = f;
    if (arc_flow) for (int i = 0; i < m; i++) arc_flow[i] = cap[i] - g.res[2 * i];
    if (sink_reach && reach_sink(&g, t, sink_reach) != 0) { rg_free(&g); return -1; }
    rg_free(&g);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* exported: one grid instance at one lambda                                  */
/* ------------------------------------------------------------------------ */
/*
 * Arc list of the H x W grid graph, pixel p = y*W + x, s = H*W, t = H*W + 1.
 * Arc order: for each pixel p in raster order: s->p (cs), p->t (ct), then if
 * x+1 < W: p->p+1 and p+1->p (w_h[p]); if y+1 < H: p->p+W and p+W->p (w_v[p]).
 * Returns the number of arcs written (the caller sizes the arrays 6*H*W).
 */
int oracle_grid_arcs(int H, int W, const int32_t *w_h, const int32_t *w_v,
                     const int32_t *src0, const int32_t *slope, const int32_t *sink,
                     int64_t lambda, int *tail, int *head, int64_t *cap) {
    int N = H * W, s = N, t = N + 1, m = 0;
    for (int y = 0; y < H; y++) {
        for (int x = 0; x < W; x++) {
            int p = y * W + x;
            tail[m] = s; head[m] = p; cap[m] = (int64_t)src0[p] + (int64_t)slope[p] * lambda; m++;
            tail[m] = p; head[m] = t; cap[m] = sink[p]; m++;
            if (x + 1 < W) {
                tail[m] = p; head[m] = p + 1; cap[m] = w_h[p]; m++;
                tail[m] = p + 1; head[m] = p; cap[m] = w_h[p]; m++;
            }
            if (y + 1 < H) {
                tail[m] = p; head[m] = p + W; cap[m] = w_v[p]; m++;
                tail[m] = p + W; head[m] = p; cap[m] = w_v[p]; m++;
            }
        }
    }
    return m;
}

/*
 * oracle_grid_solve: flow value and maximal-source-set mask (mask[p] = 1 iff
 * pixel p cannot reach t) of one grid instance at one lambda, solved from
 * scratch.  Returns 0 or -1.
 */
int oracle_grid_solve(int H, int W, const int32_t *w_h, const int32_t *w_v,
                      const int32_t *src0, const int32_t *slope, const int32_t *sink,
                      int64_t lambda, int algo, int64_t *flow, uint8_t *mask) {
    if (H <= 0 || W <= 0) return -1;
    int N = H * W;
    size_t mcap = (size_t)6 * (size_t)N;
    int *tail = (int *)malloc(sizeof(int) * mcap);
    int *head = (int *)malloc(sizeof(int) * mcap);
    int64_t *cap = (int64_t *)malloc(sizeof(int64_t) * mcap);
    uint8_t *reach = (uint8_t *)malloc((size_t)N + 2);
    int rc = -1;
    if (!tail || !head || !cap || !reach) goto out;
    int m = oracle_grid_arcs(H, W, w_h, w_v, src0, slope, sink, lambda, tail, head, cap);
    if (oracle_maxflow(N + 2, m, tail, head, cap, N, N + 1, algo, flow, NULL, reach) != 0) goto out;
    if (mask) for (int p = 0; p < N; p++) mask[p] = reach[p] ? 0 : 1;
    rc = 0;
out:
    free(tail); free(head); free(cap); free(reach);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* exported: many independent solves on a pool of threads                     */
/* ------------------------------------------------------------------------ */
/* The paper's multi-core baseline runs independent seed problems on separate
 * cores with dynamic pick-up (Section 2.2); this is the same arrangement for
 * the oracle: each job is one (instance, lambda), solved from scratch. */
typedef struct {
    int n_jobs;
    const int *H, *W;
    const int32_t *const *w_h, *const *w_v, *const *src0, *const *slope, *const *sink;
    const int64_t *lambda;
    int64_t *flow;
    uint8_t *const *mask;
    int next;          /* atomic job counter */
    int failed;
} job_pool;

static void *pool_worker(void *arg) {
    job_pool *jp = (job_pool *)arg;
    for (;;) {
        int j = __atomic_fetch_add(&jp->next, 1, __ATOMIC_RELAXED);
        if (j >= jp->n_jobs) break;
        if (oracle_grid_solve(jp->H[j], jp->W[j], jp->w_h[j], jp->w_v[j], jp->src0[j],
                              jp->slope[j], jp->sink[j], jp->lambda[j], 0, &jp->flow[j],
                              jp->mask[j]) != 0)
            __atomic_store_n(&jp->failed, 1, __ATOMIC_RELAXED);
    }
    return NULL;
}

int oracle_grid_solve_jobs(int n_jobs, const int *H, const int *W,
                           const int32_t *const *w_h, const int32_t *const *w_v,
                           const int32_t *const *src0, const int32_t *const *slope,
                           const int32_t *const *sink, const int64_t *lambda,
                           int64_t *flow, uint8_t *const *mask, int n_threads) {
    job_pool jp = {n_jobs, H, W, w_h, w_v, src0, slope, sink, lambda, flow, mask, 0, 0};
    if (n_threads < 1) n_threads = 1;
    if (n_threads > 256) n_threads = 256;
    pthread_t th[256];
    int started = 0;
    for (int i = 0; i < n_threads; i++) {
        if (pthread_create(&th[i], NULL, pool_worker, &jp) != 0) break;
        started++;
    }
    if (started == 0) pool_worker(&jp);
    for (int i = 0; i < started; i++) pthread_join(th[i], NULL);
    return jp.failed ? -1 : 0;
}
