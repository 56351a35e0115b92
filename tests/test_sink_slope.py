"""Falling sink capacities (pmf_set_slope_side(1)): ct(p, lambda) = sink -
slope*lambda and cs(p) = src0, the other half of Section 2.1's monotone case.
The GPU warm-starts each lambda from the last (a sink arc that carries more
than its new capacity returns the surplus to its pixel); every step's flow and
maximal source set must equal the oracle's, which solves each lambda from
scratch on the capacities written out."""
import numpy as np
import pytest

import oracle
from paper_1509_06004_b300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1509_06004_b300 import build, pmf
    build.build()
    return pmf


def falling_instance(H, W, rng, n_lambda=5, lam_max=30, wmax=20):
    """A random grid whose sink capacities fall with lambda and stay >= 0."""
    wl = inputs.random_grid(H, W, rng, wmax=wmax, tmax=40, p_zero=0.2, n_lambda=n_lambda, lam_max=lam_max)
    inst = wl.instances[0]
    lam_last = int(inst.lambdas[-1])
    sink = (inst.sink.astype(np.int64) + inst.slope.astype(np.int64) * lam_last).astype(np.int32)
    sink[rng.random((H, W)) < 0.1] = 0          # some pixels without a sink arc
    slope = np.where(sink == 0, 0, inst.slope).astype(np.int32)
    wl.instances[0] = inputs.Instance(0, inst.src0, slope, sink, inst.lambdas)
    return wl


def oracle_falling(im, inst):
    """Each lambda from scratch: cs = src0, ct = sink - slope*lambda."""
    zero = np.zeros_like(inst.slope)
    flows, masks = [], []
    for lam in inst.lambdas:
        ct = (inst.sink.astype(np.int64) - inst.slope.astype(np.int64) * int(lam)).astype(np.int32)
        f, m = oracle.grid_solve(im.H, im.W, im.w_h, im.w_v, inst.src0, zero, ct, [0])
        flows.append(int(f[0]))
        masks.append(m[0])
    return np.array(flows, np.int64), np.stack(masks)


@pytest.mark.parametrize("shape", [(1, 1), (1, 9), (9, 1), (7, 33), (16, 31), (33, 97), (40, 70)])
@pytest.mark.parametrize("tile_h,push_order", [(4, 0), (4, 1), (8, 1)])
def test_falling_sink_capacities_random_grids(P, shape, tile_h, push_order):
    H, W = shape
    rng = np.random.default_rng(4000 + 31 * H + W)
    wl = falling_instance(H, W, rng)
    b = P.batch_from_workload(wl, tile_h=tile_h, push_order=push_order)
    b.set_slope_side(0, 1)
    b.solve(np.stack([x.lambdas for x in wl.instances]).astype(np.int32))
    assert all(s == P.PMF_OK for s in b.sync(check=False))
    f, m = oracle_falling(wl.images[0], wl.instances[0])
    assert np.array_equal(b.flows(0), f), (b.flows(0), f)
    assert np.array_equal(b.cuts(0), m)
    # nested, growing source sets
    c = b.cuts(0).astype(np.int16)
    assert np.all(np.diff(c, axis=0) >= 0)
    b.close()


def test_both_sides_in_one_batch(P):
    """Rising-source and falling-sink instances on one image, one launch."""
    rng = np.random.default_rng(77)
    wl = falling_instance(24, 61, rng, n_lambda=6)
    up = inputs.random_grid(24, 61, np.random.default_rng(78), n_lambda=6)
    wl.instances.append(inputs.Instance(0, up.instances[0].src0, up.instances[0].slope, up.instances[0].sink,
                                        up.instances[0].lambdas))
    wl.instances.append(wl.instances[0])
    b = P.batch_from_workload(wl)
    b.set_slope_side(0, 1)
    b.set_slope_side(2, 1)
    b.solve(np.stack([x.lambdas for x in wl.instances]).astype(np.int32))
    assert all(s == P.PMF_OK for s in b.sync(check=False))
    im = wl.images[0]
    for i in (0, 2):
        f, m = oracle_falling(im, wl.instances[i])
        assert np.array_equal(b.flows(i), f) and np.array_equal(b.cuts(i), m)
    inst = wl.instances[1]
    f, m = oracle.grid_solve(im.H, im.W, im.w_h, im.w_v, inst.src0, inst.slope, inst.sink, inst.lambdas)
    assert np.array_equal(b.flows(1), f) and np.array_equal(b.cuts(1), m)
    # back to side 0: the same terminals are then a rising-source problem
    b.set_slope_side(2, 0)
    b.solve(np.stack([x.lambdas for x in wl.instances]).astype(np.int32))
    assert all(s == P.PMF_OK for s in b.sync(check=False))
    inst = wl.instances[2]
    f, m = oracle.grid_solve(im.H, im.W, im.w_h, im.w_v, inst.src0, inst.slope, inst.sink, inst.lambdas)
    assert np.array_equal(b.flows(2), f) and np.array_equal(b.cuts(2), m)
    b.close()


def test_negative_sink_capacity_is_reported(P):
    """A schedule that would drive a sink capacity below zero: that instance
    reports PMF_ERR_INVALID_ARG, the others are solved."""
    rng = np.random.default_rng(91)
    wl = falling_instance(12, 40, rng, n_lambda=4)
    wl.instances.append(wl.instances[0])
    b = P.batch_from_workload(wl)
    b.set_slope_side(0, 1)
    b.set_slope_side(1, 1)
    lam = np.stack([x.lambdas for x in wl.instances]).astype(np.int32)
    lam[1, -1] += 1000          # past every sink capacity with a positive slope
    b.solve(lam)
    st = b.sync(check=False)
    assert st[0] == P.PMF_OK and st[1] == P.PMF_ERR_INVALID_ARG
    with pytest.raises(P.PmfError):
        b.set_slope_side(0, 2)
    with pytest.raises(P.PmfError):
        b.set_slope_side(5, 1)
    b.close()


@pytest.mark.parametrize("shape", [(9, 1), (16, 31), (40, 70)])
def test_flow_arcs_with_falling_sink_capacities(P, shape):
    """pmf_get_flow_arcs on a side-1 instance: a feasible flow for the last
    lambda's capacities whose value is the oracle's maximum."""
    H, W = shape
    rng = np.random.default_rng(60 + H)
    wl = falling_instance(H, W, rng, n_lambda=3)
    inst, im = wl.instances[0], wl.images[0]
    b = P.batch_from_workload(wl)
    b.set_slope_side(0, 1)
    b.solve(np.stack([x.lambdas for x in wl.instances]).astype(np.int32))
    assert all(s == P.PMF_OK for s in b.sync(check=False))
    lam = int(inst.lambdas[-1])
    ct = (inst.sink.astype(np.int64) - inst.slope.astype(np.int64) * lam).astype(np.int32)
    zero = np.zeros_like(ct)
    arcs = b.flow_arcs(0)
    val = oracle.grid_flow_value(H, W, im.w_h, im.w_v, inst.src0, zero, ct, 0,
                                 arcs["f_h"], arcs["f_v"], arcs["f_s"], arcs["f_t"])
    f, _ = oracle_falling(im, inst)
    assert val == int(f[-1]) == int(b.flows(0)[-1])
    b.close()


@pytest.mark.parametrize("case", range(30))
def test_fuzz_mixed_sides_and_swapped_chains(P, case):
    """Random shapes, schedules and knobs; one batch mixes rising-source
    instances, falling-sink instances and swapped warm-started chains (side 1
    with cut rule 1, schedule run backwards); solved twice."""
    from paper_1509_06004_b300 import swap
    rng = np.random.default_rng(9000 + case)
    H, W = int(rng.integers(1, 65)), int(rng.integers(1, 97))
    n_lam = int(rng.integers(1, 7))
    base = inputs.random_grid(H, W, rng, wmax=int(rng.integers(1, 40)), tmax=40, p_zero=float(rng.uniform(0, 0.5)),
                              n_lambda=n_lam, lam_max=40)
    im = base.images[0]
    insts, kinds = [], []
    for _ in range(int(rng.integers(1, 5))):
        g = inputs.random_grid(H, W, rng, tmax=int(rng.integers(1, 60)), p_zero=float(rng.uniform(0, 0.5)),
                               n_lambda=n_lam, lam_max=40).instances[0]
        kind = int(rng.integers(0, 3))          # 0 rising source, 1 falling sink, 2 swapped chain
        if kind == 1:
            g = falling_instance_from(g)
        insts.append(g)
        kinds.append(kind)
    refs = []
    for g, kind in zip(insts, kinds):
        if kind == 1:
            refs.append(oracle_falling(im, g))
        else:
            refs.append(oracle.grid_solve(H, W, im.w_h, im.w_v, g.src0, g.slope, g.sink, g.lambdas))
    flat = inputs.Workload("fuzz", base.images, [])
    for g, kind in zip(insts, kinds):
        if kind == 2:
            a, b_, c, mu = swap.warm_swapped_terminals(g.src0, g.slope, g.sink, g.lambdas)
            flat.instances.append(inputs.Instance(0, a, b_, c, mu))
        else:
            flat.instances.append(g)
    knobs = dict(tile_h=int(rng.choice([4, 8])), push_order=int(rng.integers(0, 2)),
                 sweeps=int(rng.choice([1, 2, 4, 8, 16])), relabel_every=int(rng.choice([50, 200, 800, 1600])),
                 label_slack=int(rng.choice([0, 2, 4, 16])))
    knobs["strip_stage"] = int(rng.choice([-1, 1]))
    knobs["relabel_reach"] = int(rng.choice([0, 400, 800]))
    b = P.batch_from_workload(flat, **knobs)
    for j, kind in enumerate(kinds):
        if kind:
            b.set_slope_side(j, 1)
        if kind == 2:
            b.set_cut_rule(j, 1)
    for _ in range(2):
        b.solve(np.stack([x.lambdas for x in flat.instances]).astype(np.int32))
        st = b.sync(check=False)
        for j, (kind, (rf, rm)) in enumerate(zip(kinds, refs)):
            assert st[j] == P.PMF_OK, (j, kind, st[j])
            f, m = b.flows(j), b.cuts(j)
            if kind == 2:
                f, m = f[::-1], m[::-1]
            assert np.array_equal(f, rf), (j, kind, knobs, f, rf)
            assert np.array_equal(m, rm), (j, kind, knobs)
    b.close()


def falling_instance_from(inst):
    """The same instance with sink capacities that fall to its own at the last lambda."""
    lam_last = int(inst.lambdas[-1])
    sink = (inst.sink.astype(np.int64) + inst.slope.astype(np.int64) * lam_last).astype(np.int32)
    return inputs.Instance(inst.image, inst.src0, inst.slope, sink, inst.lambdas)
