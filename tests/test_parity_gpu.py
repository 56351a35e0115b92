"""CUDA path vs the CPU oracle, element by element (flows int64, masks uint8),
through the C ABI.  Both outputs are unique (the maximum flow value and the
maximal source set), so the comparison is exact."""
import numpy as np
import pytest

import oracle
from paper_1509_06004_b300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pmf():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1509_06004_b300 import build, pmf as P
    build.build()
    return P


def check_workload(P, wl, oracle_res=None, **tuning):
    st, res = P.solve_workload(wl, **tuning)
    assert all(s == P.PMF_OK for s in st), st
    if oracle_res is None:
        oracle_res = oracle.solve_workload(wl)
    for i, ((gf, gm), (of, om)) in enumerate(zip(res, oracle_res)):
        assert np.array_equal(gf, of), (i, gf, of)
        assert np.array_equal(gm, om), (i, np.argwhere(gm != om)[:10])
    return res


def test_single_64x64(pmf):
    check_workload(pmf, inputs.single_maxflow_64())


SHAPES = [(1, 1), (1, 7), (7, 1), (3, 5), (8, 32), (9, 33), (16, 31), (17, 65), (40, 70), (33, 97)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("tile_h", [4, 8])
@pytest.mark.parametrize("push_order", [0, 1])
@pytest.mark.parametrize("strip_stage", [-1, 1])
def test_random_small_grids(pmf, shape, tile_h, push_order, strip_stage):
    """strip_stage 1: relabel strips' first visits load through tensor copies
    (box columns from -4 at the left border, rows past the plane zero-filled)."""
    H, W = shape
    rng = np.random.default_rng(H * 1000 + W)
    wl = inputs.random_grid(H, W, rng, wmax=20, tmax=40, p_zero=0.2, n_lambda=4, lam_max=30)
    check_workload(pmf, wl, tile_h=tile_h, push_order=push_order, strip_stage=strip_stage)


@pytest.mark.parametrize("case", ["repeated", "zero-slope", "from-zero"])
def test_warm_start_edge_schedules(pmf, case):
    """Schedules that make the warm-start pass a no-op or near one: repeated
    lambdas (no raise), instances without any lambda dependence, a schedule
    starting at lambda = 0; against the oracle."""
    rng = np.random.default_rng({"repeated": 81, "zero-slope": 82, "from-zero": 83}[case])
    wl = inputs.Workload(case)
    for j, (H, W) in enumerate([(23, 47), (40, 33)]):
        g = inputs.random_grid(H, W, rng, wmax=20, tmax=40, p_zero=0.2, n_lambda=3, lam_max=30)
        wl.images.append(g.images[0])
        inst = g.instances[0]
        slope = np.zeros_like(inst.slope) if case == "zero-slope" else inst.slope
        if case == "repeated":
            lam = np.array([5, 5, 9, 9, 9, 20], np.int32)
        elif case == "from-zero":
            lam = np.array([0, 0, 1, 2, 30], np.int32)
        else:
            lam = np.array([3, 10, 10, 30], np.int32)
        wl.instances.append(inputs.Instance(j, inst.src0, slope, inst.sink, lam))
    check_workload(pmf, wl, tile_h=4, push_order=1)
    check_workload(pmf, wl, tile_h=8, push_order=0)


@pytest.mark.parametrize("push_order", [0, 1])
def test_ragged_schedules_mixed_sizes(pmf, push_order):
    """One launch over grids of different sizes whose schedules differ in
    length (1 to 9 lambdas): every flow and mask against the oracle."""
    rng = np.random.default_rng(77)
    wl = inputs.Workload("ragged")
    for j, (H, W) in enumerate([(9, 33), (17, 65), (40, 70), (3, 5), (33, 97)]):
        g = inputs.random_grid(H, W, rng, wmax=20, tmax=40, p_zero=0.2, n_lambda=int(rng.integers(1, 10)), lam_max=30)
        wl.images.append(g.images[0])
        for _ in range(2):
            inst = g.instances[0]
            m = int(rng.integers(1, len(inst.lambdas) + 1))
            wl.instances.append(inputs.Instance(j, inst.src0, inst.slope, inst.sink, inst.lambdas[:m]))
    assert len({len(i.lambdas) for i in wl.instances}) > 1
    check_workload(pmf, wl, tile_h=4, push_order=push_order)


@pytest.mark.parametrize("mode", ["persistent", "persistent-nograph", "rounds"])
def test_modes_on_synthetic_image(pmf, mode):
    rng = np.random.default_rng(3)
    img = inputs.make_image(70, 90, 4, 0.05, rng)
    w_h, w_v = inputs.pairwise_caps(img)
    wl = inputs.Workload("t")
    wl.images.append(inputs.Image(70, 90, w_h, w_v, img))
    lam = inputs.lambda_schedule(8, 10, 5000)
    for _ in range(3):
        y0, x0 = inputs.random_seed_origin(70, 90, rng)
        src0, slope, sink = inputs.terminals(img, inputs.seed_square(70, 90, y0, x0))
        wl.instances.append(inputs.Instance(0, src0, slope, sink, lam, (y0, x0)))
    kw = {"persistent": {}, "persistent-nograph": {"use_graph": 0}, "rounds": {"mode": 1}}[mode]
    check_workload(pmf, wl, **kw)


def test_parametric_320x240(pmf):
    wl = inputs.parametric_320x240()
    res = check_workload(pmf, wl)
    flows, masks = res[0]
    for k in range(len(flows) - 1):
        assert np.all(masks[k] <= masks[k + 1])


@pytest.mark.parametrize("case", range(24))
def test_fuzz_shapes_knobs_and_schedules(pmf, case):
    """Seeded random instances: grid shape (1 to 90 a side), capacity ranges
    and share of zero capacities, schedule length, batch size (1 to 4
    instances on up to 2 images), and solver knobs (tile height, push order,
    sweeps, relabel cadence, label slack, grid size, strip loads, budget floor).  Flows and masks must
    equal the oracle's bit for bit."""
    rng = np.random.default_rng(7000 + case)
    wl = inputs.Workload(f"fuzz{case}")
    n_img = int(rng.integers(1, 3))
    for _ in range(n_img):
        H, W = int(rng.integers(1, 91)), int(rng.integers(1, 91))
        g = inputs.random_grid(H, W, rng, wmax=int(rng.choice([3, 20, 1000])), tmax=int(rng.choice([5, 40, 2000])),
                               p_zero=float(rng.uniform(0, 0.5)), n_lambda=1)
        wl.images.append(g.images[0])
    m = int(rng.integers(1, 6))
    for _ in range(int(rng.integers(1, 5))):
        i = int(rng.integers(0, n_img))
        g = inputs.random_grid(wl.images[i].H, wl.images[i].W, rng, wmax=1, tmax=int(rng.choice([5, 40, 2000])),
                               p_zero=float(rng.uniform(0, 0.5)), n_lambda=m, lam_max=int(rng.choice([5, 50, 3000])))
        inst = g.instances[0]
        wl.instances.append(inputs.Instance(i, inst.src0, inst.slope, inst.sink, inst.lambdas))
    knobs = dict(tile_h=int(rng.choice([4, 8])), push_order=int(rng.integers(0, 2)),
                 sweeps=int(rng.choice([1, 2, 4, 8, 16])), relabel_every=int(rng.choice([50, 200, 800, 3200])),
                 label_slack=int(rng.choice([-1, 1, 4, 16])), grid_blocks=int(rng.choice([0, 1, 7, 64])))
    knobs["strip_stage"] = int(rng.choice([-1, 1]))
    knobs["relabel_reach"] = int(rng.choice([0, 400, 800, 3200]))
    check_workload(pmf, wl, **knobs)
