"""Lambda-state copies (pmf_set_fork): a piece of a seed's schedule starts from
a copy of the previous piece's state instead of cold (GGT's warm start carried
across instances; the pieces are Section 3.1's supergraph of one seed's
problems at several lambdas).  The outputs are the unique maximum flow values
and maximal source sets, so a forked batching must give exactly the results of
one warm chain, and those of the oracle.  Host logic of the plans runs on the
CPU; everything else needs the GPU."""
import numpy as np
import pytest

import oracle
from paper_1509_06004_b300 import autotune, inputs, swap


def _synthetic(seed, H, W, n_seeds, n_lambda, lo=10, hi=5000):
    rng = np.random.default_rng(seed)
    img = inputs.make_image(H, W, 4, 0.05, rng)
    w_h, w_v = inputs.pairwise_caps(img)
    wl = inputs.Workload(f"syn{seed}")
    wl.images.append(inputs.Image(H, W, w_h, w_v, img))
    lam = inputs.lambda_schedule(n_lambda, lo, hi)
    for _ in range(n_seeds):
        y0, x0 = inputs.random_seed_origin(H, W, rng)
        s0, sl, sk = inputs.terminals(img, inputs.seed_square(H, W, y0, x0))
        wl.instances.append(inputs.Instance(0, s0, sl, sk, lam, (y0, x0)))
    return wl


# ---------------------------------------------------------------------------
# host logic (CPU)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("segments,lead", [(2, 0), (2, 3), (4, 1), (4, 4), (5, 2), (20, 0)])
def test_forked_plan_structure(segments, lead):
    """Each piece after a seed's first forks from the piece before it, at the
    step lead steps before that piece's end (clamped at its first step), and
    its first lambda is not below the parent's lambda there."""
    wl = inputs.supergraph_480x320()
    w = wl.split_forked(segments, lead)
    assert len(w.instances) == segments * len(wl.instances)
    for i, inst in enumerate(w.instances):
        if i % segments == 0:
            assert inst.fork is None
            continue
        par, step = inst.fork
        assert par == i - 1
        plen = len(w.instances[par].lambdas)
        assert step == max(0, plen - 1 - lead)
        assert inst.lambdas[0] >= w.instances[par].lambdas[step]
    res = [(np.asarray(i.lambdas, np.int64), np.zeros((len(i.lambdas), 1, 1), np.uint8)) for i in w.instances]
    g = w.gather(res, len(wl.instances))
    for s, (f, _) in enumerate(g):
        assert np.array_equal(f, wl.instances[s].lambdas)
    assert autotune.plan_name({"segments": segments, "fork": lead}, 20).startswith("fork") or segments == 1


# ---------------------------------------------------------------------------
# GPU
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1509_06004_b300 import build, pmf
    build.build()
    return pmf


def _solve(P, wl, **tuning):
    st, res = P.solve_workload(wl, **tuning)
    assert all(s == P.PMF_OK for s in st), [P.status_string(s) for s in st]
    return res


def _same(a, b):
    for (fa, ma), (fb, mb) in zip(a, b):
        assert np.array_equal(fa, fb)
        assert np.array_equal(ma, mb)


@pytest.mark.gpu
@pytest.mark.parametrize("segments,lead", [(2, 0), (2, 1), (2, 3), (4, 1), (4, 3), (8, 0)])
@pytest.mark.parametrize("tile_h", [4, 8])
def test_forked_pieces_equal_the_chain_and_the_oracle(P, segments, lead, tile_h):
    wl = _synthetic(41, 58, 93, 3, 8)
    chain = _solve(P, wl, tile_h=tile_h)
    run = wl.split_forked(segments, lead)
    got = run.gather(_solve(P, run, tile_h=tile_h, push_order=1), len(wl.instances))
    _same(chain, got)
    _same(oracle.solve_workload(wl), got)


@pytest.mark.gpu
def test_forked_segmentation_schedule_against_oracle(P):
    """A 320x240 schedule of 20 lambdas in four forked pieces, each started
    right after its predecessor's first step."""
    wl = inputs.parametric_320x240()
    run = autotune.apply_plan(wl, {"segments": 4, "fork": 4})
    got = run.gather(_solve(P, run, tile_h=4, push_order=1), 1)
    _same(oracle.solve_workload(wl), got)


@pytest.mark.gpu
def test_forked_swapped_chain(P):
    """Falling sink capacities with s and t exchanged (pmf_set_slope_side(1),
    pmf_set_cut_rule(1)): a swapped chain cut into two pieces, the second
    forked from the first after its second step, equals the unsplit chain."""
    wl = _synthetic(43, 44, 71, 1, 8)
    inst, im = wl.instances[0], wl.images[0]
    a, b, c, mu = swap.warm_swapped_terminals(inst.src0, inst.slope, inst.sink, inst.lambdas)
    sw = inputs.Workload("sw", wl.images, [inputs.Instance(0, a, b, c, mu),
                                           inputs.Instance(0, a, b, c, mu[:4]),
                                           inputs.Instance(0, a, b, c, mu[4:])])
    sw.instances[2].fork = (1, 1)
    bt = P.batch_from_workload(sw)
    for i in range(3):
        bt.set_slope_side(i, 1)
        bt.set_cut_rule(i, 1)
    bt.solve([np.asarray(x.lambdas) for x in sw.instances])
    assert all(s == 0 for s in bt.sync(check=False))
    f = np.concatenate([bt.flows(1), bt.flows(2)])
    m = np.concatenate([bt.cuts(1), bt.cuts(2)])
    assert np.array_equal(f, bt.flows(0)) and np.array_equal(m, bt.cuts(0))
    # result j of the exchanged chain belongs to lambda_{m-1-j}
    of, om = oracle.grid_solve(im.H, im.W, im.w_h, im.w_v, inst.src0, inst.slope, inst.sink, inst.lambdas)
    assert np.array_equal(f[::-1], of) and np.array_equal(m[::-1], om)
    bt.close()


@pytest.mark.gpu
def test_failed_parent_stops_its_forks(P):
    """A parent whose terminals are invalid finishes with that status, and so
    do the piece forked from it and the piece forked from that one; another
    seed in the batch is solved."""
    wl = _synthetic(44, 40, 64, 2, 6)
    bad = wl.instances[0].sink.copy()
    bad[5, 5] = -3
    wl.instances[0] = inputs.Instance(0, wl.instances[0].src0, wl.instances[0].slope, bad, wl.instances[0].lambdas)
    run = wl.split_forked(3, 1)
    # device inputs: the bad capacity is found on the device and reported by the solve
    b = P.batch_from_workload(run, device_inputs=True)
    b.solve([np.asarray(i.lambdas) for i in run.instances])
    st = b.sync(check=False)
    assert st[:3] == [P.PMF_ERR_INVALID_ARG] * 3
    assert st[3:] == [P.PMF_OK] * 3
    ref = oracle.solve_workload(wl, instances=[1])
    got = (np.concatenate([b.flows(i) for i in (3, 4, 5)]), np.concatenate([b.cuts(i) for i in (3, 4, 5)]))
    _same(ref, [got])
    b.close()


@pytest.mark.gpu
def test_fork_validation(P):
    wl = _synthetic(45, 30, 40, 1, 4)
    two = inputs.Workload("two", wl.images + wl.images, [])
    for k in range(4):
        two.instances.append(inputs.Instance(k // 2, wl.instances[0].src0, wl.instances[0].slope,
                                             wl.instances[0].sink, wl.instances[0].lambdas))
    b = P.batch_from_workload(two)
    L = P.lib()
    assert L.pmf_set_fork(b._h, 2, 0, 0) == P.PMF_ERR_INVALID_ARG      # another image
    assert L.pmf_set_fork(b._h, 0, 0, 0) == P.PMF_ERR_INVALID_ARG      # itself
    assert L.pmf_set_fork(b._h, 9, 0, 0) == P.PMF_ERR_INVALID_ARG      # no such instance
    assert L.pmf_set_fork(b._h, 1, 0, 1) == P.PMF_OK
    assert L.pmf_set_fork(b._h, 3, 2, 0) == P.PMF_OK
    lam = np.array([[10, 20, 30, 40], [20, 25, 30, 40], [10, 20, 30, 40], [10, 20, 30, 40]], np.int32)
    b.solve(lam)                                                         # fine: 1 after 0's step 1
    assert all(s == 0 for s in b.sync(check=False))
    of, om = oracle.grid_solve(30, 40, wl.images[0].w_h, wl.images[0].w_v, wl.instances[0].src0,
                               wl.instances[0].slope, wl.instances[0].sink, [20, 25, 30, 40])
    assert np.array_equal(b.flows(1), of) and np.array_equal(b.cuts(1), om)
    # the child's first lambda below the parent's lambda at the fork
    low = lam.copy()
    low[1, 0] = 15
    low[1] = np.sort(low[1])
    assert L.pmf_solve_schedule(b._h, low.ctypes.data_as(__import__("ctypes").POINTER(__import__("ctypes").c_int32)),
                                4, None) == P.PMF_ERR_NOT_MONOTONE
    # the fork step beyond the parent's schedule
    assert L.pmf_set_fork(b._h, 1, 0, 4) == P.PMF_OK
    import ctypes
    lp = lam.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    assert L.pmf_solve_schedule(b._h, lp, 4, None) == P.PMF_ERR_INVALID_ARG
    # a cycle
    assert L.pmf_set_fork(b._h, 1, 0, 0) == P.PMF_OK
    assert L.pmf_set_fork(b._h, 0, 1, 0) == P.PMF_OK
    assert L.pmf_solve_schedule(b._h, lp, 4, None) == P.PMF_ERR_INVALID_ARG
    # a second child for one parent
    assert L.pmf_set_fork(b._h, 0, -1, 0) == P.PMF_OK
    assert L.pmf_set_fork(b._h, 1, 0, 0) == P.PMF_OK
    assert L.pmf_set_fork(b._h, 1, -1, 0) == P.PMF_OK
    assert L.pmf_set_fork(b._h, 1, 0, 0) == P.PMF_OK
    b2 = P.batch_from_workload(inputs.Workload("t", wl.images, [two.instances[0]] * 3))
    assert L.pmf_set_fork(b2._h, 1, 0, 0) == P.PMF_OK
    assert L.pmf_set_fork(b2._h, 2, 0, 0) == P.PMF_ERR_INVALID_ARG
    # different slope sides
    b2.set_slope_side(1, 1)
    l3 = np.array([[10, 20]] * 3, np.int32)
    assert L.pmf_solve_schedule(b2._h, l3.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), 2, None) \
        == P.PMF_ERR_INVALID_ARG
    b.close()
    b2.close()


@pytest.mark.gpu
@pytest.mark.parametrize("grid_blocks", [1, 2, 5])
def test_forks_on_small_grids_repeated(P, grid_blocks):
    """Few blocks make the parent's copy pass, the child's start and the
    parent's next step interleave in many orders; results stay exact."""
    wl = _synthetic(46, 50, 77, 2, 8)
    ref = _solve(P, wl)
    run = wl.split_forked(4, 1)
    b = P.batch_from_workload(run, grid_blocks=grid_blocks)
    for _ in range(3):
        b.solve([np.asarray(i.lambdas) for i in run.instances])
        assert all(s == 0 for s in b.sync(check=False))
        got = run.gather([(b.flows(i), b.cuts(i)) for i in range(len(run.instances))], 2)
        _same(ref, got)
    b.close()
