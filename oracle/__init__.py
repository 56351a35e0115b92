"""CPU oracle for grid s-t max-flow / min-cut (test infrastructure only).

Only tests/, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product (the CUDA library and its
Python binding) never does.

Contents
  * ``maxflow``          generic digraph max flow in C (Dinic or Edmonds-Karp).
  * ``grid_solve``       one grid instance, every lambda of its schedule solved
                         from scratch (Section 2.1's lambda-schedule, no warm
                         start), returning int64 flow values and uint8 masks of
                         the maximal source set.
  * ``grid_solve_many``  many grid (instance, lambda) jobs on a thread pool.
  * ``brute_force_*``    enumeration of every s-t cut of a graph with at most
                         16 non-terminal nodes (numpy, exact).
  * ``grid_solve_rational``  one grid instance at a rational lambda = p/q,
                         exact (every capacity times q).
  * ``cut_line``         the cost of a given cut as a line a + b*lambda.
  * ``brute_force_breakpoints``  every breakpoint of the minimum cut value
                         F(lambda) on a range, by enumerating all cuts of a
                         grid of at most 16 pixels (exact fractions).
  * ``grid_flow_value``  checks that per-arc flows on a grid form a feasible
                         s-t flow (capacity bounds and conservation) and
                         returns its value; ``grid_arc_flows`` gives such
                         flows from the oracle's own solver.

The definitions follow Section 2 of the paper: an s-t cut splits the nodes into
an s side and a t side, its cost is the total capacity of arcs from the s side
to the t side, and a minimum cut has least cost; the max-flow value equals it.
Where several minimum cuts exist this oracle reports the maximal s side (the
union of all minimising s sides), i.e. every pixel that cannot reach t in the
residual graph of a maximum flow.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_u8p = ctypes.POINTER(ctypes.c_uint8)


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc into oracle/_build/liboracle.so."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            L.oracle_maxflow.restype = ctypes.c_int
            L.oracle_maxflow.argtypes = [ctypes.c_int, ctypes.c_int, _i32p, _i32p, _i64p,
                                         ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         _i64p, _i64p, _u8p]
            L.oracle_grid_solve.restype = ctypes.c_int
            L.oracle_grid_solve.argtypes = [ctypes.c_int, ctypes.c_int] + [_i32p] * 5 + \
                [ctypes.c_int64, ctypes.c_int, _i64p, _u8p]
            L.oracle_grid_arcs.restype = ctypes.c_int
            L.oracle_grid_arcs.argtypes = [ctypes.c_int, ctypes.c_int] + [_i32p] * 5 + \
                [ctypes.c_int64, _i32p, _i32p, _i64p]
            pp = ctypes.POINTER(ctypes.c_void_p)
            L.oracle_grid_solve_jobs.restype = ctypes.c_int
            L.oracle_grid_solve_jobs.argtypes = [ctypes.c_int, _i32p, _i32p, pp, pp, pp, pp, pp,
                                                 _i64p, _i64p, pp, ctypes.c_int]
            _lib = L
    return _lib


def _p(a, t):
    return a.ctypes.data_as(t)


def _c32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


# ----------------------------------------------------------------------------
# generic graphs
# ----------------------------------------------------------------------------

def maxflow(n: int, tail, head, cap, s: int, t: int, algo: str = "dinic"):
    """Max flow of a digraph.  Returns (value, arc_flow[m] int64, sink_reach[n] uint8)."""
    tail = _c32(tail)
    head = _c32(head)
    cap = np.ascontiguousarray(cap, dtype=np.int64)
    m = len(tail)
    val = ctypes.c_int64(0)
    fl = np.zeros(max(m, 1), dtype=np.int64)
    reach = np.zeros(n, dtype=np.uint8)
    rc = lib().oracle_maxflow(n, m, _p(tail, _i32p), _p(head, _i32p), _p(cap, _i64p), s, t,
                              1 if algo == "ek" else 0, ctypes.byref(val), _p(fl, _i64p),
                              _p(reach, _u8p))
    if rc != 0:
        raise ValueError("oracle_maxflow: bad graph")
    return int(val.value), fl[:m], reach


def grid_arcs(H, W, w_h, w_v, src0, slope, sink, lam):
    """The oracle's arc list of one grid instance at one lambda: (tail, head, cap),
    pixel p = y*W + x, s = H*W, t = H*W + 1."""
    N = H * W
    tail = np.zeros(6 * N, np.int32)
    head = np.zeros(6 * N, np.int32)
    cap = np.zeros(6 * N, np.int64)
    arrs = [_c32(a).ravel() for a in (w_h, w_v, src0, slope, sink)]
    m = lib().oracle_grid_arcs(H, W, *[_p(a, _i32p) for a in arrs], int(lam),
                               _p(tail, _i32p), _p(head, _i32p), _p(cap, _i64p))
    return tail[:m], head[:m], cap[:m]


# ----------------------------------------------------------------------------
# grid instances
# ----------------------------------------------------------------------------

def grid_solve(H, W, w_h, w_v, src0, slope, sink, lambdas, algo: str = "dinic"):
    """Solve one grid instance at every lambda, each from scratch.
    Returns (flows int64 [m], masks uint8 [m, H, W]); mask = 1 on the s side."""
    arrs = [_c32(a).ravel() for a in (w_h, w_v, src0, slope, sink)]
    lambdas = np.asarray(lambdas, dtype=np.int64).ravel()
    flows = np.zeros(len(lambdas), np.int64)
    masks = np.zeros((len(lambdas), H, W), np.uint8)
    for k, lam in enumerate(lambdas):
        f = ctypes.c_int64(0)
        mk = masks[k]
        rc = lib().oracle_grid_solve(H, W, *[_p(a, _i32p) for a in arrs], int(lam),
                                     1 if algo == "ek" else 0, ctypes.byref(f), _p(mk, _u8p))
        if rc != 0:
            raise ValueError("oracle_grid_solve failed")
        flows[k] = f.value
    return flows, masks


def grid_solve_many(jobs, n_threads: int | None = None):
    """jobs: list of (H, W, w_h, w_v, src0, slope, sink, lambda).  Solves them on
    a pool of ``n_threads`` threads (default: all cores).  Returns (flows int64
    [n], list of uint8 [H, W] masks)."""
    n = len(jobs)
    if n_threads is None:
        n_threads = os.cpu_count() or 1
    keep = []
    Hs = np.array([j[0] for j in jobs], np.int32)
    Ws = np.array([j[1] for j in jobs], np.int32)
    ptrs = [(ctypes.c_void_p * max(n, 1))() for _ in range(6)]
    masks = []
    for i, j in enumerate(jobs):
        for a_i, a in enumerate(j[2:7]):
            a = _c32(a).ravel()
            keep.append(a)
            ptrs[a_i][i] = a.ctypes.data
        mk = np.zeros((j[0], j[1]), np.uint8)
        masks.append(mk)
        ptrs[5][i] = mk.ctypes.data
    lam = np.array([j[7] for j in jobs], np.int64)
    flows = np.zeros(max(n, 1), np.int64)
    rc = lib().oracle_grid_solve_jobs(n, _p(Hs, _i32p), _p(Ws, _i32p), *ptrs[:5],
                                      _p(lam, _i64p), _p(flows, _i64p), ptrs[5], int(n_threads))
    if rc != 0:
        raise ValueError("oracle_grid_solve_jobs failed")
    return flows[:n], masks


def solve_workload(wl, n_threads: int | None = None, instances=None):
    """Every (instance, lambda) of a Workload, from scratch.  Returns a list
    (per instance) of (flows [m], masks [m, H, W])."""
    idx = list(range(len(wl.instances))) if instances is None else list(instances)
    jobs, owner = [], []
    for i in idx:
        inst = wl.instances[i]
        im = wl.images[inst.image]
        for k, lam in enumerate(inst.lambdas):
            jobs.append((im.H, im.W, im.w_h, im.w_v, inst.src0, inst.slope, inst.sink, int(lam)))
            owner.append((i, k))
    flows, masks = grid_solve_many(jobs, n_threads)
    out = {}
    for (i, k), f, m in zip(owner, flows, masks):
        out.setdefault(i, {})[k] = (int(f), m)
    res = []
    for i in idx:
        m = len(wl.instances[i].lambdas)
        res.append((np.array([out[i][k][0] for k in range(m)], np.int64),
                    np.stack([out[i][k][1] for k in range(m)])))
    return res


# ----------------------------------------------------------------------------
# brute force (at most 16 non-terminal nodes)
# ----------------------------------------------------------------------------

def brute_force_graph(n: int, tail, head, cap, s: int, t: int):
    """Enumerate every s-t cut of a digraph whose non-terminal nodes number at
    most 16.  Returns (min cost, union of all minimising s sides as a uint8
    vector over nodes, number of minimising s sides)."""
    others = [u for u in range(n) if u != s and u != t]
    k = len(others)
    assert k <= 16, "brute force is limited to 16 non-terminal nodes"
    subsets = np.arange(1 << k, dtype=np.int64)
    side = np.zeros((n, 1 << k), dtype=np.int64)      # 1 = node on the s side
    side[s, :] = 1
    for bit, u in enumerate(others):
        side[u, :] = (subsets >> bit) & 1
    tail = np.asarray(tail, np.int64)
    head = np.asarray(head, np.int64)
    cap = np.asarray(cap, np.int64)
    cost = np.zeros(1 << k, dtype=np.int64)
    for u, v, c in zip(tail, head, cap):
        if c:
            cost += c * side[u] * (1 - side[v])
    best = int(cost.min())
    arg = np.nonzero(cost == best)[0]
    union = np.zeros(n, np.uint8)
    for bit, u in enumerate(others):
        union[u] = 1 if np.any((arg >> bit) & 1) else 0
    union[s] = 1
    return best, union, len(arg)


def brute_force_min_source_set(n: int, tail, head, cap, s: int, t: int):
    """The intersection of every minimising s side (the minimal source set of
    a minimum cut) of a digraph with at most 16 non-terminal nodes, by
    enumeration: uint8 vector over nodes."""
    others = [u for u in range(n) if u != s and u != t]
    k = len(others)
    assert k <= 16, "brute force is limited to 16 non-terminal nodes"
    subsets = np.arange(1 << k, dtype=np.int64)
    side = np.zeros((n, 1 << k), dtype=np.int64)
    side[s, :] = 1
    for bit, u in enumerate(others):
        side[u, :] = (subsets >> bit) & 1
    cost = np.zeros(1 << k, dtype=np.int64)
    for u, v, c in zip(np.asarray(tail), np.asarray(head), np.asarray(cap, np.int64)):
        if c:
            cost += c * side[u] * (1 - side[v])
    arg = np.nonzero(cost == cost.min())[0]
    inter = np.zeros(n, np.uint8)
    for bit, u in enumerate(others):
        inter[u] = 1 if np.all((arg >> bit) & 1) else 0
    inter[s] = 1
    return inter


def source_reach(n: int, tail, head, cap, flow, s: int):
    """Nodes reachable from s in the residual graph of a flow (residual of an
    arc u->v: cap - flow; of its reverse v->u: flow).  For a maximum flow this
    is the minimal source set of a minimum cut (Ford-Fulkerson)."""
    adj = [[] for _ in range(n)]
    for u, v, c, f in zip(np.asarray(tail).tolist(), np.asarray(head).tolist(),
                          np.asarray(cap, np.int64).tolist(), np.asarray(flow, np.int64).tolist()):
        if c - f > 0:
            adj[u].append(v)
        if f > 0:
            adj[v].append(u)
    seen = np.zeros(n, np.uint8)
    seen[s] = 1
    stack = [s]
    while stack:
        u = stack.pop()
        for v in adj[u]:
            if not seen[v]:
                seen[v] = 1
                stack.append(v)
    return seen


def brute_force_grid(H, W, w_h, w_v, src0, slope, sink, lam):
    """Brute-force min cut of a grid instance with H*W <= 16, its cut cost
    written straight from the definition of Section 2 (pairwise edges counted
    in the direction s side -> t side, terminal edges s->p for t-side pixels
    and p->t for s-side pixels).  Returns (min cost, maximal s-side mask [H, W],
    number of minimising sets)."""
    N = H * W
    assert N <= 16
    w_h = np.asarray(w_h, np.int64).reshape(H, W)
    w_v = np.asarray(w_v, np.int64).reshape(H, W)
    cs = (np.asarray(src0, np.int64) + np.asarray(slope, np.int64) * int(lam)).reshape(H, W)
    ct = np.asarray(sink, np.int64).reshape(H, W)
    S = np.arange(1 << N, dtype=np.int64)
    on = np.stack([(S >> p) & 1 for p in range(N)]).reshape(H, W, -1)   # 1 = s side
    cost = (cs[..., None] * (1 - on)).sum(axis=(0, 1)) + (ct[..., None] * on).sum(axis=(0, 1))
    # horizontal neighbours: an edge of capacity w in each direction
    a, b = on[:, :-1], on[:, 1:]
    cost += (w_h[:, :-1, None] * (a * (1 - b) + b * (1 - a))).sum(axis=(0, 1))
    a, b = on[:-1, :], on[1:, :]
    cost += (w_v[:-1, :, None] * (a * (1 - b) + b * (1 - a))).sum(axis=(0, 1))
    best = int(cost.min())
    arg = np.nonzero(cost == best)[0]
    union = np.zeros(N, np.uint8)
    for p in range(N):
        union[p] = 1 if np.any((arg >> p) & 1) else 0
    return best, union.reshape(H, W), len(arg)


# ----------------------------------------------------------------------------
# the parametric cut at rational lambda and its breakpoints (Section 2.1)
# ----------------------------------------------------------------------------

def _arcs_line(H, W, w_h, w_v, src0, slope, sink):
    """The arc list with each capacity as a line c0 + c1*lambda."""
    tail, head, c0 = grid_arcs(H, W, w_h, w_v, src0, slope, sink, 0)
    _, _, cl = grid_arcs(H, W, w_h, w_v, src0, slope, sink, 1)
    return tail, head, c0, cl - c0


def grid_solve_rational(H, W, w_h, w_v, src0, slope, sink, p: int, q: int, algo: str = "dinic"):
    """Maximum flow and maximal source set of one grid instance at lambda =
    p / q (q >= 1), exactly: every arc capacity c0 + c1*lambda is multiplied
    by q, giving the integer q*c0 + p*c1; scaling all capacities by q scales
    every cut's cost by q, so the minimum cuts are the same and the flow value
    is q * F(p/q).  Returns (q * F(p/q), mask uint8 [H, W], 1 = source side)."""
    p, q = int(p), int(q)
    if q < 1:
        raise ValueError("q >= 1")
    tail, head, c0, c1 = _arcs_line(H, W, w_h, w_v, src0, slope, sink)
    cap = q * c0 + p * c1
    N = H * W
    val, _, reach = maxflow(N + 2, tail, head, cap, N, N + 1, algo)
    return val, (1 - reach[:N]).astype(np.uint8).reshape(H, W)


def cut_line(H, W, w_h, w_v, src0, slope, sink, mask):
    """(a, b) with a + b*lambda = the cost of the s-t cut whose s side is s
    plus the pixels with mask = 1 (Section 2: the total capacity of the arcs
    from the s side to the t side), read off the arc list."""
    tail, head, c0, c1 = _arcs_line(H, W, w_h, w_v, src0, slope, sink)
    N = H * W
    side = np.concatenate([np.asarray(mask, np.uint8).ravel() != 0, [True, False]])
    cut = side[tail] & ~side[head]
    return int(c0[cut].sum()), int(c1[cut].sum())


def brute_force_breakpoints(H, W, w_h, w_v, src0, slope, sink, lo, hi):
    """Every breakpoint of F(lambda) = min over cuts of their cost on [lo, hi]
    for a grid of at most 16 pixels, by enumeration.  Each cut's cost is a
    line a_S + b_S*lambda (Section 2's cut cost with cs = src0 + slope*lambda),
    so F is their lower envelope.  Walking up from lo, the line in force is
    the one of least slope among those of least value, and the next breakpoint
    is the nearest crossing with a line of smaller slope.  Returns
    (breakpoints [Fraction] in (lo, hi], masks uint8 [r+1, H, W], lines
    [(a, b)]): the maximal source set (union of the minimisers) on each piece,
    from the one at lo on."""
    from fractions import Fraction
    N = H * W
    assert N <= 16
    i64 = lambda a: np.asarray(a, np.int64).reshape(H, W)
    w_h, w_v, s0, sl, ct = i64(w_h), i64(w_v), i64(src0), i64(slope), i64(sink)
    S = np.arange(1 << N, dtype=np.int64)
    on = np.stack([(S >> p) & 1 for p in range(N)]).reshape(H, W, -1)    # 1 = s side
    off = 1 - on
    a = (s0[..., None] * off).sum(axis=(0, 1)) + (ct[..., None] * on).sum(axis=(0, 1))
    x1, x2 = on[:, :-1], on[:, 1:]
    a += (w_h[:, :-1, None] * (x1 * (1 - x2) + x2 * (1 - x1))).sum(axis=(0, 1))
    y1, y2 = on[:-1, :], on[1:, :]
    a += (w_v[:-1, :, None] * (y1 * (1 - y2) + y2 * (1 - y1))).sum(axis=(0, 1))
    b = (sl[..., None] * off).sum(axis=(0, 1))
    lines = sorted({(int(x), int(y)) for x, y in zip(a, b)})

    def union_of(line):
        sel = np.nonzero((a == line[0]) & (b == line[1]))[0]
        m = np.zeros(N, np.uint8)
        for p in range(N):
            m[p] = 1 if np.any((sel >> p) & 1) else 0
        return m.reshape(H, W)

    lam = Fraction(lo)
    val = min(x + y * lam for x, y in lines)
    cur = min((l for l in lines if l[0] + l[1] * lam == val), key=lambda l: l[1])
    bps, pieces = [], [cur]
    while True:
        nxt = None
        for l in lines:
            if l[1] < cur[1]:
                x = Fraction(l[0] - cur[0], cur[1] - l[1])
                if x > lam and (nxt is None or x < nxt):
                    nxt = x
        if nxt is None or nxt > hi:
            break
        lam = nxt
        val = cur[0] + cur[1] * lam
        cur = min((l for l in lines if l[0] + l[1] * lam == val), key=lambda l: l[1])
        bps.append(lam)
        pieces.append(cur)
    return bps, np.stack([union_of(l) for l in pieces]), pieces


# ----------------------------------------------------------------------------
# per-arc flows on a grid
# ----------------------------------------------------------------------------

class FlowError(AssertionError):
    """Per-arc flows that are not a feasible s-t flow."""


def grid_flow_value(H, W, w_h, w_v, src0, slope, sink, lam, f_h, f_v, f_s, f_t) -> int:
    """Value of a grid s-t flow given per arc (Section 2's graph: arcs s->p of
    capacity cs(p) = src0 + slope*lam, p->t of capacity sink, and each pair of
    4-neighbours joined both ways with capacity w).  Flows are int arrays
    [H, W]: f_s on s->p, f_t on p->t, and on each neighbour pair its net flow,
    f_h from (y, x) to (y, x+1) and f_v from (y, x) to (y+1, x) (negative =
    the other way; a net flow between -w and w is a flow on one of the two
    opposite arcs within its capacity).

    A flow is feasible when every arc carries between zero and its capacity
    and, at every pixel, the flow in equals the flow out.  Its value is the
    total flow into t.  Raises FlowError naming the first violated condition."""
    i64 = lambda a: np.asarray(a, np.int64).reshape(H, W)
    w_h, w_v, ct = i64(w_h), i64(w_v), i64(sink)
    cs = i64(src0) + i64(slope) * int(lam)
    f_h, f_v, f_s, f_t = i64(f_h), i64(f_v), i64(f_s), i64(f_t)
    if np.any(f_s < 0) or np.any(f_s > cs):
        raise FlowError("source arc flow outside [0, cs]")
    if np.any(f_t < 0) or np.any(f_t > ct):
        raise FlowError("sink arc flow outside [0, ct]")
    if np.any(np.abs(f_h[:, :-1]) > w_h[:, :-1]) or np.any(f_h[:, -1] != 0):
        raise FlowError("horizontal pair flow above its capacity (or past the last column)")
    if np.any(np.abs(f_v[:-1, :]) > w_v[:-1, :]) or np.any(f_v[-1, :] != 0):
        raise FlowError("vertical pair flow above its capacity (or past the last row)")
    inflow = f_s.copy()
    outflow = f_t.copy()
    # a positive net pair flow leaves its first pixel and enters its second
    outflow[:, :-1] += f_h[:, :-1]
    inflow[:, 1:] += f_h[:, :-1]
    outflow[:-1, :] += f_v[:-1, :]
    inflow[1:, :] += f_v[:-1, :]
    if not np.array_equal(inflow, outflow):
        y, x = np.argwhere(inflow != outflow)[0]
        raise FlowError(f"flow not conserved at pixel ({y}, {x})")
    return int(f_t.sum())


def grid_arc_flows(H, W, w_h, w_v, src0, slope, sink, lam, algo: str = "dinic"):
    """A maximum flow of one grid instance from the oracle's digraph solver,
    in the per-pair form of ``grid_flow_value``: (value, f_h, f_v, f_s, f_t)."""
    tail, head, cap = grid_arcs(H, W, w_h, w_v, src0, slope, sink, lam)
    N = H * W
    val, fl, _ = maxflow(N + 2, tail, head, cap, N, N + 1, algo)
    f_h = np.zeros(N, np.int64)
    f_v = np.zeros(N, np.int64)
    f_s = np.zeros(N, np.int64)
    f_t = np.zeros(N, np.int64)
    for u, v, f in zip(tail.tolist(), head.tolist(), fl.tolist()):
        if u == N:
            f_s[v] += f
        elif v == N + 1:
            f_t[u] += f
        elif u // W == v // W:          # same row: a horizontal pair
            if v == u + 1:
                f_h[u] += f
            else:
                f_h[v] -= f
        elif v == u + W:                # a vertical pair
            f_v[u] += f
        else:
            f_v[v] -= f
    r = lambda a: a.reshape(H, W)
    return val, r(f_h), r(f_v), r(f_s), r(f_t)
