"""The s-t swap (Section 3.2): the rule on the CPU, and on the GPU, solves of
the exchanged problems whose flows and masks must equal the oracle's for the
original problems (the mask comes back as the original maximal source set:
the complement of the exchanged problem's minimal source set)."""
import numpy as np
import pytest

import oracle
from paper_1509_06004_b300 import inputs, swap


def test_sign_count_rule():
    src0 = np.array([0, 0, 0, 0], np.int32)
    slope = np.array([1, 1, 1, 1], np.int32)
    sink = np.array([5, 5, 5, 1], np.int32)
    assert swap.needs_swap(src0, slope, sink, 2)          # three of four below their sink capacity
    assert not swap.needs_swap(src0, slope, sink, 5)      # no negative differences at all
    assert not swap.needs_swap(src0, slope, sink, 6)
    a, b, c = swap.swapped_terminals(src0, slope, sink, 3)
    assert np.array_equal(a, sink) and not b.any() and np.array_equal(c, src0 + 3 * slope)


def test_rule_counts_strictly():
    # at lambda 5: differences (-5+5, ..) = (0, 0, 0, 4): no negatives -> no swap
    src0 = np.zeros(4, np.int32)
    slope = np.ones(4, np.int32)
    sink = np.array([5, 5, 5, 1], np.int32)
    d = src0 + slope * 5 - sink
    assert (d < 0).sum() == 0 and not swap.needs_swap(src0, slope, sink, 5)


@pytest.mark.parametrize("shape,seed", [((1, 1), 0), ((3, 4), 1), ((4, 4), 2), ((2, 7), 3), ((6, 9), 4),
                                        ((12, 15), 5)])
def test_warm_swapped_schedule_reproduces_every_lambda(shape, seed):
    """The exchanged chain at mu_j = lambda_last - lambda_{m-1-j}, with source
    capacities ct and sink capacities sink' - slope*mu_j, is the original
    problem at lambda_{m-1-j} with s and t exchanged: same flow value, and the
    complement of its minimal source set is the original maximal source set."""
    H, W = shape
    rng = np.random.default_rng(1300 + seed)
    wl = inputs.random_grid(H, W, rng, p_zero=0.3, n_lambda=min(5, H * W + 1), lam_max=25)
    im, inst = wl.images[0], wl.instances[0]
    a, b, c, mu = swap.warm_swapped_terminals(inst.src0, inst.slope, inst.sink, inst.lambdas)
    m = len(inst.lambdas)
    assert np.all(np.diff(mu) >= 0) and mu[0] == 0
    assert np.array_equal(a, inst.sink) and np.array_equal(b, inst.slope)
    f, masks = oracle.grid_solve(H, W, im.w_h, im.w_v, inst.src0, inst.slope, inst.sink, inst.lambdas)
    N = H * W
    zero = np.zeros_like(a)
    for j in range(m):
        ct_mu = (np.asarray(c, np.int64) - np.asarray(b, np.int64) * int(mu[j])).astype(np.int32)
        assert ct_mu.min() >= 0
        tail, head, cap = oracle.grid_arcs(H, W, im.w_h, im.w_v, a, zero, ct_mu, 0)
        val, fl, _ = oracle.maxflow(N + 2, tail, head, cap, N, N + 1)
        assert val == int(f[m - 1 - j])
        minsrc = oracle.source_reach(N + 2, tail, head, cap, fl, N)[:N].reshape(H, W)
        assert np.array_equal(1 - minsrc, masks[m - 1 - j])


def test_warm_swapped_terminals_checks_its_inputs():
    z = np.zeros(4, np.int32)
    with pytest.raises(ValueError):
        swap.warm_swapped_terminals(z, z, z, [3, 2])
    with pytest.raises(ValueError):
        swap.warm_swapped_terminals(z, z, z, [])
    with pytest.raises(ValueError):
        swap.warm_swapped_terminals(np.full(4, 1 << 29, np.int32), np.full(4, 1 << 20, np.int32), z, [0, 1024])


def test_chain_rule_is_a_majority_of_the_lambdas():
    src0 = np.zeros(4, np.int32)
    slope = np.ones(4, np.int32)
    sink = np.array([5, 5, 5, 1], np.int32)
    # lambda 2 and 3 vote swap, 5 and 6 do not: a tie keeps the chain as it is
    assert not swap.chain_needs_swap(src0, slope, sink, [2, 3, 5, 6])
    assert swap.chain_needs_swap(src0, slope, sink, [2, 3, 5])
    assert not swap.chain_needs_swap(src0, slope, sink, [2, 5, 6])


@pytest.fixture(scope="module")
def gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1509_06004_b300 import build
    build.build()
    return True


def _check(wl, mode, warm=False, **tuning):
    st, res, sw = swap.solve_workload(wl, swap=mode, warm=warm, **tuning)
    ref = oracle.solve_workload(wl)
    for i, ((f, m), (of, om)) in enumerate(zip(res, ref)):
        assert all(s == 0 for s in st[i]), st[i]
        assert np.array_equal(f, of), (i, f, of)
        assert np.array_equal(m, om), (i, np.argwhere(m != om)[:5])
    return sw


@pytest.mark.gpu
@pytest.mark.parametrize("shape", [(1, 1), (1, 9), (9, 1), (7, 33), (16, 31), (33, 97), (40, 70)])
@pytest.mark.parametrize("mode", ["always", "auto"])
def test_swapped_random_grids(gpu, shape, mode):
    H, W = shape
    rng = np.random.default_rng(31 * H + W)
    wl = inputs.random_grid(H, W, rng, wmax=20, tmax=40, p_zero=0.2, n_lambda=4, lam_max=30)
    sw = _check(wl, mode)
    if mode == "always":
        assert all(all(x) for x in sw)


@pytest.mark.gpu
def test_swapped_segmentation_schedule(gpu):
    """A synthetic segmentation instance over its full lambda schedule: the
    rule swaps the low lambdas (sink-dominated) and keeps the high ones."""
    wl = inputs.parametric_320x240(n_lambda=8)
    sw = _check(wl, "auto")
    assert any(sw[0]) and not all(sw[0])


@pytest.mark.gpu
def test_cut_rule_on_a_multi_lambda_constant_problem(gpu):
    """Rule 1 on a warm-started schedule of a lambda-independent problem: the
    forward pass runs after every certified step and the next step starts
    from the same labels; every step returns the same flow and cut."""
    from paper_1509_06004_b300 import pmf
    wl = inputs.random_grid(24, 40, np.random.default_rng(5), wmax=20, tmax=40, p_zero=0.2, n_lambda=1)
    inst = wl.instances[0]
    a, b, c = swap.swapped_terminals(inst.src0, inst.slope, inst.sink, int(inst.lambdas[0]))
    sw = inputs.Workload("sw", wl.images, [inputs.Instance(0, a, b, c, np.array([3, 5, 9], np.int32))])
    bt = pmf.batch_from_workload(sw)
    bt.set_cut_rule(0, 1)
    bt.solve(np.array([[3, 5, 9]], np.int32))
    assert all(s == 0 for s in bt.sync(check=False))
    f, m = oracle.grid_solve(24, 40, wl.images[0].w_h, wl.images[0].w_v, inst.src0, inst.slope, inst.sink,
                             [int(inst.lambdas[0])])
    flows, cuts = bt.flows(0), bt.cuts(0)
    bt.close()
    assert np.all(flows == f[0])
    for k in range(3):
        assert np.array_equal(cuts[k], m[0])


@pytest.mark.gpu
@pytest.mark.parametrize("shape", [(1, 1), (1, 9), (9, 1), (7, 33), (16, 31), (33, 97), (40, 70)])
@pytest.mark.parametrize("mode", ["always", "auto"])
def test_warm_swapped_chains_random_grids(gpu, shape, mode):
    """Warm-started chains, swapped as a whole: the exchanged problem runs the
    schedule backwards with falling sink capacities, and every step's flow and
    mask must equal the oracle's for the original problem at that lambda."""
    H, W = shape
    rng = np.random.default_rng(57 * H + W)
    wl = inputs.random_grid(H, W, rng, wmax=20, tmax=40, p_zero=0.2, n_lambda=min(6, 31), lam_max=30)
    sw = _check(wl, mode, warm=True)
    if mode == "always":
        assert all(all(x) for x in sw)


@pytest.mark.gpu
@pytest.mark.parametrize("push_order", [0, 1])
def test_warm_swapped_chains_segmentation(gpu, push_order):
    """Synthetic segmentation chains over 8 lambdas, every seed swapped, with
    both push orders: parity with the oracle at every lambda."""
    wl = inputs.parametric_320x240(n_lambda=8)
    _check(wl, "always", warm=True, push_order=push_order)


@pytest.mark.gpu
def test_warm_swapped_and_plain_chains_in_one_batch(gpu):
    """Seeds of the supergraph workload (5 of them, 6 lambdas), each chain
    swapped or not by the rule; swapped and plain chains share one launch."""
    wl = inputs.supergraph_480x320()
    wl.instances = [inputs.Instance(x.image, x.src0, x.slope, x.sink, x.lambdas[::4].copy())
                    for x in wl.instances[::5]]
    sw = _check(wl, "auto", warm=True)
    _check(wl, "always", warm=True)
    assert len(sw) == 5


def test_warm_chains_host_logic_with_a_fake_batch(monkeypatch):
    """swap.solve_workload(warm=True) without a GPU: swapped chains are marked
    with cut rule 1 and slope side 1, get the reversed mu schedule, and their
    results come back reversed into the original lambda order; plain chains
    pass through untouched."""
    from paper_1509_06004_b300 import pmf
    wl = inputs.random_grid(3, 5, np.random.default_rng(3), n_lambda=4, lam_max=20)
    inst = wl.instances[0]
    wl.instances.append(inputs.Instance(0, inst.src0, inst.slope, inst.sink, inst.lambdas))
    calls = {}

    class FakeBatch:
        def __init__(self, flat):
            self.flat = flat
            calls["flat"] = flat
            calls["rule"], calls["side"] = {}, {}

        def set_cut_rule(self, j, r):
            calls["rule"][j] = r

        def set_slope_side(self, j, s):
            calls["side"][j] = s

        def solve(self, lam):
            calls["lam"] = [np.asarray(x) for x in lam]

        def sync(self, check=False):
            return [pmf.PMF_OK] * len(self.flat.instances)

        def flows(self, j):      # step k's "flow" is its own schedule value, to see the order
            return np.asarray(self.flat.instances[j].lambdas, np.int64) * 10 + j

        def cuts(self, j):
            n = len(self.flat.instances[j].lambdas)
            return np.stack([np.full((3, 5), k, np.uint8) for k in range(n)])

        def close(self):
            pass

    monkeypatch.setattr(pmf, "batch_from_workload", lambda flat, device=0, **kw: FakeBatch(flat))
    answers = iter([True, False])           # the rule swaps the first chain only
    monkeypatch.setattr(swap, "chain_needs_swap", lambda *a: next(answers))
    st, res, sw = swap.solve_workload(wl, swap="auto", warm=True)
    lam = np.asarray(inst.lambdas, np.int64)
    mu = lam[-1] - lam[::-1]
    assert sw == [[True] * 4, [False] * 4]
    assert calls["rule"] == {0: 1} and calls["side"] == {0: 1}
    assert np.array_equal(calls["lam"][0], mu) and np.array_equal(calls["lam"][1], lam)
    # swapped: result k belongs to lambda_k, i.e. to mu_{m-1-k}
    assert np.array_equal(res[0][0], (mu * 10)[::-1])
    assert [int(c[0, 0]) for c in res[0][1]] == [3, 2, 1, 0]
    assert np.array_equal(res[1][0], lam * 10 + 1)
    assert [int(c[0, 0]) for c in res[1][1]] == [0, 1, 2, 3]
    assert st == [[pmf.PMF_OK] * 4, [pmf.PMF_OK] * 4]
