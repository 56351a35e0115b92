"""All integer breakpoints of a parametric minimum cut (the bisection driver
over exact solves).  The reference is brute force: the oracle solved at every
integer lambda of the range, and the lambdas where its maximal source set
changes.  The driver's logic runs on the CPU with the oracle as its solver;
the GPU test runs it on the CUDA solver."""
import numpy as np
import pytest

import oracle
from paper_1509_06004_b300 import inputs, parametric


def _instance(H, W, seed):
    rng = np.random.default_rng(seed)
    img = inputs.make_image(H, W, 3, 0.05, rng)
    w_h, w_v = inputs.pairwise_caps(img)
    y0, x0 = inputs.random_seed_origin(H, W, rng)
    src0, slope, sink = inputs.terminals(img, inputs.seed_square(H, W, y0, x0))
    return w_h, w_v, src0, slope, sink


def _oracle_solver(H, W, w_h, w_v, src0, slope, sink):
    def solve(lams):
        f, m = oracle.grid_solve(H, W, w_h, w_v, src0, slope, sink, [int(x) for x in lams])
        return f, m
    return solve


def _brute(H, W, args, lo, hi):
    f, m = oracle.grid_solve(H, W, *args, list(range(lo, hi + 1)))
    keep = [0] + [k for k in range(1, len(m)) if not np.array_equal(m[k], m[k - 1])]
    return np.array([lo + k for k in keep]), f[keep], m[keep]


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_bisection_finds_every_change_point(seed):
    H, W = 12, 14
    args = _instance(H, W, seed)
    lo, hi = 1, 600
    bp = parametric.breakpoints(H, W, *args, lo, hi, solve=_oracle_solver(H, W, *args))
    lam, f, m = _brute(H, W, args, lo, hi)
    assert np.array_equal(bp.lambdas, lam)
    assert np.array_equal(bp.flows, f)
    assert np.array_equal(bp.masks, m)
    # far fewer solves than one per lambda
    assert bp.solves <= len(lam) * int(np.ceil(np.log2(hi - lo + 1))) + 2
    # nested and growing with lambda
    for a, b in zip(bp.masks, bp.masks[1:]):
        assert np.all(b >= a) and np.any(b > a)


def test_degenerate_ranges():
    H, W = 8, 9
    args = _instance(H, W, 4)
    s = _oracle_solver(H, W, *args)
    one = parametric.breakpoints(H, W, *args, 7, 7, solve=s)
    assert list(one.lambdas) == [7] and one.solves == 1
    with pytest.raises(ValueError):
        parametric.breakpoints(H, W, *args, 9, 3, solve=s)
    # a range without any change: two solves, one set
    lam, _, _ = _brute(H, W, args, 1, 3000)
    if len(lam) > 1:
        a, b = int(lam[-1]), 3000
        flat = parametric.breakpoints(H, W, *args, a, b, solve=s)
        assert list(flat.lambdas) == [a] and flat.solves == 2


@pytest.mark.gpu
def test_gpu_breakpoints_match_brute_force():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1509_06004_b300 import build
    build.build()
    H, W = 40, 56
    args = _instance(H, W, 11)
    lo, hi = 1, 1500
    bp = parametric.breakpoints(H, W, *args, lo, hi, max_batch=64)
    lam, f, m = _brute(H, W, args, lo, hi)
    assert np.array_equal(bp.lambdas, lam)
    assert np.array_equal(bp.flows, f)
    assert np.array_equal(bp.masks, m)
