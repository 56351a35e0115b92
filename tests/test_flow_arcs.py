"""Per-arc maximum flows (pmf_get_flow_arcs): the GPU's excess return turns
the solve's maximum preflow into a feasible flow.  Per-arc flows are not
unique, so each is checked against what fixes it: the oracle's feasibility
conditions (capacities, conservation) and its value, which must equal the
oracle's maximum-flow value.  The call must leave the instance's results
unchanged."""
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


def _check_instance(P, b, wl, i):
    inst = wl.instances[i]
    im = wl.images[inst.image]
    lam = int(inst.lambdas[-1])
    before_f, before_m = b.flows(i), b.cuts(i)
    arcs = b.flow_arcs(i)
    val = oracle.grid_flow_value(im.H, im.W, im.w_h, im.w_v, inst.src0, inst.slope, inst.sink, lam,
                                 arcs["f_h"], arcs["f_v"], arcs["f_s"], arcs["f_t"])
    f, _ = oracle.grid_solve(im.H, im.W, im.w_h, im.w_v, inst.src0, inst.slope, inst.sink, [lam])
    assert val == int(f[0]) == int(before_f[-1])
    # the instance's own results are untouched, and a second call agrees on the value
    assert np.array_equal(b.flows(i), before_f) and np.array_equal(b.cuts(i), before_m)
    again = b.flow_arcs(i)
    assert int(again["f_t"].sum()) == val
    return arcs


@pytest.mark.parametrize("shape", [(1, 1), (1, 9), (9, 1), (7, 33), (16, 31), (33, 97), (40, 70)])
@pytest.mark.parametrize("tile_h", [4, 8])
def test_random_grids(P, shape, tile_h):
    H, W = shape
    rng = np.random.default_rng(7 * H + W)
    wl = inputs.random_grid(H, W, rng, wmax=20, tmax=40, p_zero=0.3, n_lambda=3, lam_max=30)
    b = P.batch_from_workload(wl, tile_h=tile_h)
    b.solve(np.stack([x.lambdas for x in wl.instances]).astype(np.int32))
    assert all(s == P.PMF_OK for s in b.sync(check=False))
    _check_instance(P, b, wl, 0)
    b.close()


def test_synthetic_images_and_cut(P):
    """Parametric instances of the synthetic segmentation workload: besides
    feasibility and value, every pair arc from the returned source set (mask
    1) to the rest must be saturated outwards and carry nothing inwards (the
    flow saturates the minimum cut, Section 2)."""
    wl = inputs.parametric_320x240(n_lambda=6)
    b = P.batch_from_workload(wl)
    b.solve(np.stack([x.lambdas for x in wl.instances]).astype(np.int32))
    assert all(s == P.PMF_OK for s in b.sync(check=False))
    arcs = _check_instance(P, b, wl, 0)
    im = wl.images[0]
    m = b.cuts(0)[-1].astype(bool)
    w_h = np.asarray(im.w_h, np.int64).reshape(im.H, im.W)
    w_v = np.asarray(im.w_v, np.int64).reshape(im.H, im.W)
    fh, fv = arcs["f_h"].astype(np.int64), arcs["f_v"].astype(np.int64)
    a, c = m[:, :-1], m[:, 1:]
    assert np.all(fh[:, :-1][a & ~c] == w_h[:, :-1][a & ~c])
    assert np.all(fh[:, :-1][~a & c] == -w_h[:, :-1][~a & c])
    a, c = m[:-1, :], m[1:, :]
    assert np.all(fv[:-1][a & ~c] == w_v[:-1][a & ~c])
    assert np.all(fv[:-1][~a & c] == -w_v[:-1][~a & c])
    # source arcs into the sink side carry their full capacity, sink arcs of the source side too
    inst = wl.instances[0]
    cs = np.asarray(inst.src0, np.int64).reshape(im.H, im.W) + np.asarray(inst.slope, np.int64).reshape(im.H, im.W) * int(inst.lambdas[-1])
    ct = np.asarray(inst.sink, np.int64).reshape(im.H, im.W)
    assert np.all(arcs["f_s"][~m] == cs[~m])
    assert np.all(arcs["f_t"][m] == ct[m])
    b.close()


def test_batch_of_supergraph_seeds(P):
    wl = inputs.supergraph_480x320(n_lambda=4)
    wl.instances = wl.instances[:3]
    b = P.batch_from_workload(wl)
    b.solve(np.stack([x.lambdas for x in wl.instances]).astype(np.int32))
    assert all(s == P.PMF_OK for s in b.sync(check=False))
    for i in range(len(wl.instances)):
        _check_instance(P, b, wl, i)
    b.close()


def test_not_ready_before_a_solve(P):
    wl = inputs.single_maxflow_64()
    b = P.batch_from_workload(wl)
    with pytest.raises(P.PmfError) as ei:
        b.flow_arcs(0)
    assert ei.value.status == P.PMF_ERR_NOT_READY
    b.close()


def test_large_grid_properties(P):
    """A 4099 x 4100 grid (16.8 M pixels; sides that are no multiple of the
    tile, strip or pitch sizes), two lambdas: the per-arc flow is feasible by
    the oracle's conditions with the value the solver reports, its cut is
    saturated, and the two cuts are nested.  (The oracle's max-flow would take
    too long here; these properties hold at any size.)"""
    H, W = 4099, 4100
    rng = np.random.default_rng(17)
    img = inputs.make_image(H, W, 5, 0.05, rng)
    w_h, w_v = inputs.pairwise_caps(img)
    y0, x0 = inputs.random_seed_origin(H, W, rng)
    src0, slope, sink = inputs.terminals(img, inputs.seed_square(H, W, y0, x0))
    wl = inputs.Workload("large", [inputs.Image(H, W, w_h, w_v, None)],
                         [inputs.Instance(0, src0, slope, sink, np.array([40, 300], np.int32))])
    b = P.batch_from_workload(wl, push_order=1)
    b.solve(np.array([[40, 300]], np.int32))
    assert all(s == P.PMF_OK for s in b.sync(check=False))
    flows, cuts = b.flows(0), b.cuts(0)
    assert np.all(cuts[0] <= cuts[1]) and flows[0] <= flows[1]
    arcs = b.flow_arcs(0)
    val = oracle.grid_flow_value(H, W, w_h, w_v, src0, slope, sink, 300,
                                 arcs["f_h"], arcs["f_v"], arcs["f_s"], arcs["f_t"])
    assert val == int(flows[1])
    # the flow saturates the reported cut: every pair arc from the source set
    # to the rest carries its capacity outwards, so the cut's capacity is the value
    m = cuts[1].astype(bool)
    fh, fv = arcs["f_h"].astype(np.int64), arcs["f_v"].astype(np.int64)
    wh, wv = np.asarray(w_h, np.int64), np.asarray(w_v, np.int64)
    a, c = m[:, :-1], m[:, 1:]
    assert np.all(fh[:, :-1][a & ~c] == wh[:, :-1][a & ~c]) and np.all(fh[:, :-1][~a & c] == -wh[:, :-1][~a & c])
    a, c = m[:-1], m[1:]
    assert np.all(fv[:-1][a & ~c] == wv[:-1][a & ~c]) and np.all(fv[:-1][~a & c] == -wv[:-1][~a & c])
    b.close()
