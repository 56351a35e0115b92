"""Pins for the CPU oracle, independent of the oracle itself.

Each check ties the oracle to something the paper or the mathematics fixes:
  * brute-force enumeration of every s-t cut (Section 2's definition of cut
    cost and minimum cut) on graphs of at most 16 non-terminal nodes;
  * the max-flow = min-cut identity (Ford-Fulkerson, cited in Section 2):
    the cost of the reported cut equals the reported flow value;
  * flow feasibility and conservation of the arc flows;
  * closed forms: no pairwise edges (each pixel is its own s-t problem), a
    1 x N chain (flow = its weakest link);
  * nestedness of the cuts for a monotone lambda schedule and concavity of
    F(lambda) (Section 2.1, after Gallo-Grigoriadis-Tarjan);
  * two independent solvers (Dinic, Edmonds-Karp) agree;
  * hand-derived worked examples under tests/golden/.
A separate test plants mistakes in a copy of the oracle's C source and checks
that these pins catch every one.
"""
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
from paper_1509_06004_b300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rand_digraph(rng, n, p_arc=0.35, cmax=9):
    tail, head, cap = [], [], []
    for u in range(n):
        for v in range(n):
            if u != v and rng.random() < p_arc:
                tail.append(u)
                head.append(v)
                cap.append(int(rng.integers(0, cmax + 1)))
    return np.array(tail, np.int32), np.array(head, np.int32), np.array(cap, np.int64)


def cut_cost_grid(mask, w_h, w_v, cs, ct):
    """Cost of the cut whose s side is {s} + {p: mask[p] = 1} (Section 2)."""
    m = mask.astype(np.int64)
    c = int((cs * (1 - m)).sum() + (ct * m).sum())
    c += int((w_h[:, :-1] * (m[:, :-1] != m[:, 1:])).sum())
    c += int((w_v[:-1, :] * (m[:-1, :] != m[1:, :])).sum())
    return c


# --------------------------------------------------------------------------
# generic graphs vs brute force
# --------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(40))
def test_digraph_dinic_ek_match_brute_force(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, 17)) + 2            # <= 16 non-terminals
    tail, head, cap = rand_digraph(rng, n)
    s, t = 0, n - 1
    best, union, _ = oracle.brute_force_graph(n, tail, head, cap, s, t)
    for algo in ("dinic", "ek"):
        val, fl, reach = oracle.maxflow(n, tail, head, cap, s, t, algo)
        assert val == best
        # maximal s side: every node that cannot reach t
        assert np.array_equal((1 - reach).astype(np.uint8)[[u for u in range(n) if u != t]],
                              union[[u for u in range(n) if u != t]])
        # feasibility and conservation
        assert np.all(fl >= 0) and np.all(fl <= cap)
        net = np.zeros(n, np.int64)
        np.add.at(net, head, fl)
        np.subtract.at(net, tail, fl)
        assert all(net[u] == 0 for u in range(n) if u not in (s, t))
        assert net[t] == val


# --------------------------------------------------------------------------
# grid instances vs brute force (<= 16 pixels)
# --------------------------------------------------------------------------

SMALL_SHAPES = [(1, 1), (1, 2), (2, 1), (1, 16), (16, 1), (2, 8), (8, 2), (4, 4), (3, 5), (5, 3), (2, 2)]


@pytest.mark.parametrize("shape", SMALL_SHAPES)
@pytest.mark.parametrize("seed", range(6))
def test_grid_matches_brute_force(shape, seed):
    H, W = shape
    rng = np.random.default_rng(1000 * seed + H * 17 + W)
    wl = inputs.random_grid(H, W, rng, wmax=6, tmax=12, p_zero=0.3, n_lambda=3, lam_max=8)
    im, inst = wl.images[0], wl.instances[0]
    flows, masks = oracle.grid_solve(H, W, im.w_h, im.w_v, inst.src0, inst.slope, inst.sink,
                                     inst.lambdas)
    for k, lam in enumerate(inst.lambdas):
        best, union, _ = oracle.brute_force_grid(H, W, im.w_h, im.w_v, inst.src0, inst.slope,
                                                 inst.sink, lam)
        assert flows[k] == best
        assert np.array_equal(masks[k], union)


def test_grid_ties_union_of_minimisers():
    """A 1x2 grid where every cut costs the same: the union of minimising s
    sides is everything, so both pixels are reported on the s side."""
    w_h = np.array([[3, 0]], np.int32)
    w_v = np.zeros((1, 2), np.int32)
    src0 = np.array([[3, 3]], np.int32)
    slope = np.zeros((1, 2), np.int32)
    sink = np.array([[3, 3]], np.int32)
    best, union, count = oracle.brute_force_grid(1, 2, w_h, w_v, src0, slope, sink, 0)
    flows, masks = oracle.grid_solve(1, 2, w_h, w_v, src0, slope, sink, [0])
    assert count > 1 and best == 6 and flows[0] == 6
    assert masks[0].tolist() == [[1, 1]] and union.tolist() == [[1, 1]]


# --------------------------------------------------------------------------
# closed forms
# --------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(4))
def test_no_pairwise_edges_closed_form(seed):
    rng = np.random.default_rng(seed)
    H, W = 37, 53
    z = np.zeros((H, W), np.int32)
    src0 = rng.integers(0, 50, (H, W)).astype(np.int32)
    slope = rng.integers(0, 3, (H, W)).astype(np.int32)
    sink = rng.integers(0, 120, (H, W)).astype(np.int32)
    lams = np.array([0, 7, 19, 40], np.int32)
    flows, masks = oracle.grid_solve(H, W, z, z, src0, slope, sink, lams)
    for k, lam in enumerate(lams):
        cs = src0.astype(np.int64) + slope.astype(np.int64) * int(lam)
        assert flows[k] == np.minimum(cs, sink).sum()
        assert np.array_equal(masks[k], (cs >= sink).astype(np.uint8))


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("vertical", [False, True])
def test_chain_closed_form(seed, vertical):
    """1 x N chain, source only at the first pixel, sink only at the last:
    flow = the weakest link; the maximal s side is everything up to the last
    weakest link."""
    rng = np.random.default_rng(seed)
    N = int(rng.integers(2, 40))
    w = rng.integers(1, 9, N - 1)
    H, W = (N, 1) if vertical else (1, N)
    w_h = np.zeros((H, W), np.int32)
    w_v = np.zeros((H, W), np.int32)
    if vertical:
        w_v[:-1, 0] = w
    else:
        w_h[0, :-1] = w
    src0 = np.zeros((H, W), np.int32)
    sink = np.zeros((H, W), np.int32)
    src0.flat[0] = inputs.INF
    sink.flat[-1] = inputs.INF
    slope = np.zeros((H, W), np.int32)
    flows, masks = oracle.grid_solve(H, W, w_h, w_v, src0, slope, sink, [0])
    assert flows[0] == w.min()
    j = int(np.nonzero(w == w.min())[0].max())
    expect = np.zeros(N, np.uint8)
    expect[:j + 1] = 1
    assert np.array_equal(masks[0].ravel(), expect)


# --------------------------------------------------------------------------
# certificates and parametric invariants on the synthetic workloads
# --------------------------------------------------------------------------

def test_c1_certificates():
    wl = inputs.single_maxflow_64()
    im, inst = wl.images[0], wl.instances[0]
    lam = int(inst.lambdas[0])
    flows, masks = oracle.grid_solve(im.H, im.W, im.w_h, im.w_v, inst.src0, inst.slope,
                                     inst.sink, inst.lambdas)
    cs = inst.src0.astype(np.int64) + inst.slope.astype(np.int64) * lam
    assert cut_cost_grid(masks[0], im.w_h.astype(np.int64), im.w_v.astype(np.int64), cs,
                         inst.sink.astype(np.int64)) == flows[0]
    # arc-level feasibility and conservation on the oracle's own arc list
    tail, head, cap = oracle.grid_arcs(im.H, im.W, im.w_h, im.w_v, inst.src0, inst.slope,
                                       inst.sink, lam)
    n = im.H * im.W + 2
    val, fl, _ = oracle.maxflow(n, tail, head, cap, n - 2, n - 1)
    assert val == flows[0]
    assert np.all(fl >= 0) and np.all(fl <= cap)
    net = np.zeros(n, np.int64)
    np.add.at(net, head, fl)
    np.subtract.at(net, tail, fl)
    assert np.all(net[:-2] == 0) and net[-1] == val
    # the seed is on the s side, the border on the t side
    y0, x0 = inst.seed_origin
    assert masks[0][y0:y0 + 5, x0:x0 + 5].all()
    assert not masks[0][0, :].any() and not masks[0][:, 0].any()


def _parametric_checks(wl, flows, masks, inst):
    im = wl.images[inst.image]
    lams = [int(x) for x in inst.lambdas]
    # nested cuts (Section 2.1): s sides grow with lambda
    for k in range(len(lams) - 1):
        assert np.all(masks[k] <= masks[k + 1])
    # F nondecreasing and concave in lambda (a minimum of affine functions)
    assert np.all(np.diff(flows) >= 0)
    for k in range(1, len(lams) - 1):
        d0 = (int(flows[k]) - int(flows[k - 1])) * (lams[k + 1] - lams[k])
        d1 = (int(flows[k + 1]) - int(flows[k])) * (lams[k] - lams[k - 1])
        assert d1 <= d0
    # every emitted cut is feasible at every lambda and tight at its own
    wh = im.w_h.astype(np.int64)
    wv = im.w_v.astype(np.int64)
    ct = inst.sink.astype(np.int64)
    for k in range(len(lams)):
        for j in range(len(lams)):
            cs = inst.src0.astype(np.int64) + inst.slope.astype(np.int64) * lams[j]
            c = cut_cost_grid(masks[k], wh, wv, cs, ct)
            assert c >= flows[j]
            if j == k:
                assert c == flows[k]


def test_parametric_small_c2_shape():
    """The C2 recipe at 60x80 (runs in well under a second)."""
    rng = np.random.default_rng(5)
    img = inputs.make_image(60, 80, 3, 0.05, rng)
    w_h, w_v = inputs.pairwise_caps(img)
    y0, x0 = inputs.random_seed_origin(60, 80, rng)
    src0, slope, sink = inputs.terminals(img, inputs.seed_square(60, 80, y0, x0))
    wl = inputs.Workload("t")
    wl.images.append(inputs.Image(60, 80, w_h, w_v, img))
    wl.instances.append(inputs.Instance(0, src0, slope, sink, inputs.lambda_schedule(12, 10, 5000)))
    inst = wl.instances[0]
    flows, masks = oracle.grid_solve(60, 80, w_h, w_v, src0, slope, sink, inst.lambdas)
    _parametric_checks(wl, flows, masks, inst)
    assert masks[0].sum() < masks[-1].sum()        # the schedule spans several cuts


@pytest.mark.parametrize("seed", range(3))
def test_dinic_equals_ek_medium(seed):
    rng = np.random.default_rng(100 + seed)
    wl = inputs.random_grid(18, 23, rng, wmax=30, tmax=60, p_zero=0.15, n_lambda=2, lam_max=40)
    im, inst = wl.images[0], wl.instances[0]
    f1, m1 = oracle.grid_solve(im.H, im.W, im.w_h, im.w_v, inst.src0, inst.slope, inst.sink,
                               inst.lambdas, "dinic")
    f2, m2 = oracle.grid_solve(im.H, im.W, im.w_h, im.w_v, inst.src0, inst.slope, inst.sink,
                               inst.lambdas, "ek")
    assert np.array_equal(f1, f2) and np.array_equal(m1, m2)


def test_thread_pool_matches_serial():
    wl = inputs.uneven_batch(n_images=2, seeds_per_image=2, n_lambda=3)
    per = oracle.solve_workload(wl, n_threads=3)
    for i, inst in enumerate(wl.instances):
        im = wl.images[inst.image]
        f, m = oracle.grid_solve(im.H, im.W, im.w_h, im.w_v, inst.src0, inst.slope, inst.sink,
                                 inst.lambdas)
        assert np.array_equal(per[i][0], f) and np.array_equal(per[i][1], m)


# --------------------------------------------------------------------------
# hand-derived worked examples
# --------------------------------------------------------------------------

def _read_golden(path):
    """Format: '# comment' lines, then 'key: v v v' lines; grids row-major."""
    d = {}
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        k, v = line.split(":", 1)
        d[k.strip()] = [int(x) for x in v.split()]
    return d


@pytest.mark.parametrize("name", sorted(f for f in os.listdir(GOLDEN) if f.endswith(".txt")))
def test_golden(name):
    d = _read_golden(os.path.join(GOLDEN, name))
    H, W = d["shape"]
    a = {k: np.array(d[k], np.int32).reshape(H, W) for k in ("w_h", "w_v", "src0", "slope", "sink")}
    lams = d["lambdas"]
    flows, masks = oracle.grid_solve(H, W, a["w_h"], a["w_v"], a["src0"], a["slope"], a["sink"],
                                     lams)
    assert flows.tolist() == d["flows"]
    assert masks.reshape(len(lams), -1).tolist() == np.array(d["masks"]).reshape(len(lams), -1).tolist()


# --------------------------------------------------------------------------
# planted mistakes: each mutant of the C source must fail a pin
# --------------------------------------------------------------------------

MUTANTS = {
    "no-reverse-residual": ("g->res[stack[i]] -= f; g->res[stack[i] ^ 1] += f;",
                            "g->res[stack[i]] -= f;"),
    "reach-forward-arc": ("if (!reach[u] && g->res[a ^ 1] > 0)", "if (!reach[u] && g->res[a] > 0)"),
    "missing-backward-pairwise": ("tail[m] = p + 1; head[m] = p; cap[m] = w_h[p]; m++;", ""),
    "slope-sign": ("(int64_t)src0[p] + (int64_t)slope[p] * lambda",
                   "(int64_t)src0[p] - (int64_t)slope[p] * lambda"),
    "mask-polarity": ("mask[p] = reach[p] ? 0 : 1;", "mask[p] = reach[p] ? 1 : 0;"),
    "sink-gets-source-cap": ("tail[m] = p; head[m] = t; cap[m] = sink[p]; m++;",
                             "tail[m] = p; head[m] = t; cap[m] = src0[p]; m++;"),
    "vertical-uses-wh": ("cap[m] = w_v[p]; m++;\n                tail[m] = p + W",
                         "cap[m] = w_h[p]; m++;\n                tail[m] = p + W"),
}


def _pins_pass(L):
    """Run a compact subset of the pins against a loaded oracle library."""
    import ctypes
    saved = oracle._lib
    oracle._lib = L
    try:
        for shape in [(4, 4), (2, 8), (3, 5), (1, 16)]:
            for seed in range(4):
                H, W = shape
                rng = np.random.default_rng(77 + seed + 7 * H)
                wl = inputs.random_grid(H, W, rng, wmax=6, tmax=12, p_zero=0.3, n_lambda=2, lam_max=8)
                im, inst = wl.images[0], wl.instances[0]
                try:
                    flows, masks = oracle.grid_solve(H, W, im.w_h, im.w_v, inst.src0, inst.slope,
                                                     inst.sink, inst.lambdas)
                except ValueError:
                    return False
                for k, lam in enumerate(inst.lambdas):
                    best, union, _ = oracle.brute_force_grid(H, W, im.w_h, im.w_v, inst.src0,
                                                             inst.slope, inst.sink, lam)
                    if flows[k] != best or not np.array_equal(masks[k], union):
                        return False
        for seed in range(20):
            rng = np.random.default_rng(seed)
            n = int(rng.integers(2, 17)) + 2
            tail, head, cap = rand_digraph(rng, n)
            best, _, _ = oracle.brute_force_graph(n, tail, head, cap, 0, n - 1)
            if oracle.maxflow(n, tail, head, cap, 0, n - 1)[0] != best:
                return False
        for seed in range(3):
            rng = np.random.default_rng(100 + seed)
            wl = inputs.random_grid(18, 23, rng, wmax=30, tmax=60, p_zero=0.15, n_lambda=2, lam_max=40)
            im, inst = wl.images[0], wl.instances[0]
            args = (im.H, im.W, im.w_h, im.w_v, inst.src0, inst.slope, inst.sink, inst.lambdas)
            f1, m1 = oracle.grid_solve(*args, "dinic")
            f2, m2 = oracle.grid_solve(*args, "ek")
            if not (np.array_equal(f1, f2) and np.array_equal(m1, m2)):
                return False
        return True
    finally:
        oracle._lib = saved


@pytest.mark.parametrize("mutant", sorted(MUTANTS))
def test_planted_mistake_is_caught(mutant):
    src = open(oracle._SRC).read()
    old, new = MUTANTS[mutant]
    assert old in src, f"mutation anchor not found for {mutant}"
    d = tempfile.mkdtemp(prefix="oracle_mut_")
    try:
        c = os.path.join(d, "m.c")
        so = os.path.join(d, "m.so")
        open(c, "w").write(src.replace(old, new, 1))
        subprocess.check_call(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-pthread", "-o", so, c])
        import ctypes
        L = ctypes.CDLL(so)
        ref = oracle.lib()
        for name in ("oracle_maxflow", "oracle_grid_solve", "oracle_grid_arcs", "oracle_grid_solve_jobs"):
            getattr(L, name).restype = getattr(ref, name).restype
            getattr(L, name).argtypes = getattr(ref, name).argtypes
        assert not _pins_pass(L), f"pins did not catch mutant {mutant}"
    finally:
        shutil.rmtree(d, ignore_errors=True)


def test_unmutated_passes_compact_pins():
    assert _pins_pass(oracle.lib())


# --------------------------------------------------------------------------
# per-arc flows: the feasibility checker against flows from both solvers, and
# against planted violations
# --------------------------------------------------------------------------
@pytest.mark.parametrize("shape,seed", [((1, 9), 0), ((9, 1), 1), ((4, 4), 2), ((7, 11), 3), ((12, 10), 4)])
@pytest.mark.parametrize("algo", ["dinic", "ek"])
def test_grid_flow_value_accepts_solver_flows(shape, seed, algo):
    H, W = shape
    wl = inputs.random_grid(H, W, np.random.default_rng(seed), n_lambda=2)
    im, inst = wl.images[0], wl.instances[0]
    for lam in inst.lambdas:
        val, f_h, f_v, f_s, f_t = oracle.grid_arc_flows(H, W, im.w_h, im.w_v, inst.src0, inst.slope,
                                                        inst.sink, int(lam), algo)
        got = oracle.grid_flow_value(H, W, im.w_h, im.w_v, inst.src0, inst.slope, inst.sink, int(lam),
                                     f_h, f_v, f_s, f_t)
        flows, _ = oracle.grid_solve(H, W, im.w_h, im.w_v, inst.src0, inst.slope, inst.sink, [int(lam)])
        assert got == val == int(flows[0])


def test_grid_flow_value_rejects_violations():
    H, W = 6, 7
    wl = inputs.random_grid(H, W, np.random.default_rng(9), p_zero=0.0)
    im, inst = wl.images[0], wl.instances[0]
    lam = int(inst.lambdas[0])
    args = (H, W, im.w_h, im.w_v, inst.src0, inst.slope, inst.sink, lam)
    val, f_h, f_v, f_s, f_t = oracle.grid_arc_flows(*args)
    assert oracle.grid_flow_value(*args, f_h, f_v, f_s, f_t) == val

    def bad(fn):
        a = [x.copy() for x in (f_h, f_v, f_s, f_t)]
        fn(a)
        with pytest.raises(oracle.FlowError):
            oracle.grid_flow_value(*args, *a)

    bad(lambda a: a[0].__setitem__((2, 3), a[0][2, 3] + 1))      # unbalanced pair flow
    bad(lambda a: a[1].__setitem__((1, 1), a[1][1, 1] - 1))
    bad(lambda a: a[2].__setitem__((0, 0), -1))                  # negative source-arc flow
    bad(lambda a: a[3].__setitem__((3, 3), a[3][3, 3] + 1))      # sink flow without supply
    bad(lambda a: a[0].__setitem__((4, W - 1), 1))               # flow past the last column
    bad(lambda a: a[1].__setitem__((H - 1, 2), 1))               # flow past the last row
    # a circulation around one square keeps conservation but may break a bound
    w_h = np.asarray(im.w_h).reshape(H, W)
    a = [x.copy() for x in (f_h, f_v, f_s, f_t)]
    a[0][1, 1] = w_h[1, 1] + 1
    with pytest.raises(oracle.FlowError):
        oracle.grid_flow_value(*args, *a)
    # and an in-bounds circulation is still a flow of the same value
    a = [x.copy() for x in (f_h, f_v, f_s, f_t)]
    c = 1
    a[0][2, 2] += c; a[1][2, 3] += c; a[0][3, 2] -= c; a[1][2, 2] -= c
    ok = (np.abs(a[0][:, :-1]) <= w_h[:, :-1]).all() and \
         (np.abs(a[1][:-1]) <= np.asarray(im.w_v).reshape(H, W)[:-1]).all()
    if ok:
        assert oracle.grid_flow_value(*args, *a) == val


# --------------------------------------------------------------------------
# the s-t swap (Section 3.2): exchanging s and t (pairwise capacities are
# symmetric) keeps the flow value, and the original maximal source set is the
# complement of the swapped problem's minimal source set
# --------------------------------------------------------------------------
@pytest.mark.parametrize("seed", range(8))
def test_min_source_set_matches_brute_force(seed):
    rng = np.random.default_rng(500 + seed)
    n = 10
    m = 30
    tail = rng.integers(0, n, m)
    head = rng.integers(0, n, m)
    keep = tail != head
    tail, head = tail[keep], head[keep]
    cap = rng.integers(0, 6, len(tail))
    val, fl, _ = oracle.maxflow(n, tail, head, cap, 0, n - 1)
    reach = oracle.source_reach(n, tail, head, cap, fl, 0)
    assert np.array_equal(reach, oracle.brute_force_min_source_set(n, tail, head, cap, 0, n - 1))


@pytest.mark.parametrize("shape,seed", [((3, 4), 0), ((4, 4), 1), ((2, 7), 2), ((6, 9), 3), ((12, 15), 4)])
def test_swap_keeps_value_and_complements_the_minimal_source_set(shape, seed):
    H, W = shape
    rng = np.random.default_rng(900 + seed)
    wl = inputs.random_grid(H, W, rng, p_zero=0.3, n_lambda=3)
    im, inst = wl.images[0], wl.instances[0]
    N = H * W
    for lam in inst.lambdas:
        cs = (np.asarray(inst.src0, np.int64) + np.asarray(inst.slope, np.int64) * int(lam)).astype(np.int32)
        f, m = oracle.grid_solve(H, W, im.w_h, im.w_v, inst.src0, inst.slope, inst.sink, [int(lam)])
        # swapped: source capacities = the sink capacities, sink capacities = cs(lambda)
        zero = np.zeros_like(cs)
        tail, head, cap = oracle.grid_arcs(H, W, im.w_h, im.w_v, inst.sink, zero, cs, 0)
        val, fl, _ = oracle.maxflow(N + 2, tail, head, cap, N, N + 1)
        assert val == int(f[0])
        minsrc = oracle.source_reach(N + 2, tail, head, cap, fl, N)[:N].reshape(H, W)
        assert np.array_equal(1 - minsrc, m[0])
        if N <= 16:
            bf = oracle.brute_force_min_source_set(N + 2, tail, head, cap, N, N + 1)[:N].reshape(H, W)
            assert np.array_equal(bf, minsrc)


# --------------------------------------------------------------------------
# the other half of Section 2.1's monotone case: sink capacities that fall
# with lambda (ct = sink - slope*lambda, cs = src0).  F is then a minimum of
# affine functions with non-positive slopes: nonincreasing and concave; the
# maximal source sets still grow with lambda
# --------------------------------------------------------------------------
@pytest.mark.parametrize("shape,seed", [((1, 1), 0), ((2, 3), 1), ((3, 4), 2), ((4, 4), 3), ((6, 9), 4),
                                        ((12, 15), 5)])
def test_falling_sink_capacities_nested_and_concave(shape, seed):
    H, W = shape
    rng = np.random.default_rng(2100 + seed)
    wl = inputs.random_grid(H, W, rng, p_zero=0.3, n_lambda=min(6, H * W + 3), lam_max=20)
    im, inst = wl.images[0], wl.instances[0]
    lams = [int(x) for x in inst.lambdas]
    sink = inst.sink.astype(np.int64) + inst.slope.astype(np.int64) * lams[-1]
    zero = np.zeros_like(inst.slope)
    flows, masks = [], []
    for lam in lams:
        ct = (sink - inst.slope.astype(np.int64) * lam).astype(np.int32)
        f, m = oracle.grid_solve(H, W, im.w_h, im.w_v, inst.src0, zero, ct, [0])
        flows.append(int(f[0]))
        masks.append(m[0])
        if H * W <= 16:
            cost, bm, _ = oracle.brute_force_grid(H, W, im.w_h, im.w_v, inst.src0, zero, ct, 0)
            assert cost == int(f[0]) and np.array_equal(bm, m[0])
    for k in range(len(lams) - 1):
        assert np.all(masks[k] <= masks[k + 1])
        assert flows[k + 1] <= flows[k]
    for k in range(1, len(lams) - 1):
        d0 = (flows[k] - flows[k - 1]) * (lams[k + 1] - lams[k])
        d1 = (flows[k + 1] - flows[k]) * (lams[k] - lams[k - 1])
        assert d1 <= d0
