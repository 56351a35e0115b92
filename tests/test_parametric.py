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


# ---------------------------------------------------------------------------
# exact breakpoints (rational lambda*)
# ---------------------------------------------------------------------------

class OracleExact:
    """exact_breakpoints backend on the CPU oracle: the full problem solved
    exactly at each rational lambda (capacities times q, int64), cut lines
    read off the oracle's arc list."""

    def __init__(self, H, W, *args):
        self.H, self.W, self.args = H, W, args

    def _line(self, m):
        return oracle.cut_line(self.H, self.W, *self.args, m)

    def ends(self, lo, hi):
        f, m = oracle.grid_solve(self.H, self.W, *self.args, [lo, hi])
        return [m[0], m[1]], [self._line(m[0]), self._line(m[1])], [int(f[0]), int(f[1])]

    def between(self, items):
        out = []
        for s1, s2, (a1, b1), p, q in items:
            qf, m = oracle.grid_solve_rational(self.H, self.W, *self.args, p, q)
            gap = q * a1 + p * b1 - qf
            out.append(parametric.BetweenResult(False, 0) if gap == 0 else
                       parametric.BetweenResult(False, gap, m, self._line(m)))
        return out

    def host_mask(self, m):
        return np.asarray(m, np.uint8).reshape(self.H, self.W)


def _tiny(seed, H, W):
    rng = np.random.default_rng(seed)
    g = inputs.random_grid(H, W, rng, wmax=9, tmax=30, p_zero=0.2)
    im, inst = g.images[0], g.instances[0]
    return im.w_h, im.w_v, inst.src0, inst.slope, inst.sink


def test_rational_solve_and_cut_line_pinned_by_enumeration():
    """q*F(p/q) from the oracle's scaled solve equals the brute-force lower
    envelope of all cut lines at rational points; the oracle's cut lines of
    the maximal cuts equal the envelope's lines; q = 1 is the integer solve."""
    from fractions import Fraction
    for seed, (H, W) in enumerate([(3, 4), (4, 4), (2, 7), (1, 9)]):
        args = _tiny(100 + seed, H, W)
        bps, masks, lines = oracle.brute_force_breakpoints(H, W, *args, 0, 60)
        for m, l in zip(masks, lines):
            assert oracle.cut_line(H, W, *args, m) == l
        pts = sorted(set([Fraction(0), Fraction(60)] + bps + [Fraction(2 * k + 1, 6) for k in range(180)]))
        for lam in pts:
            i = sum(1 for x in bps if x <= lam)
            a, b = lines[i]
            qf, m = oracle.grid_solve_rational(H, W, *args, lam.numerator, lam.denominator)
            assert qf == a * lam.denominator + b * lam.numerator
            assert np.array_equal(m, masks[i])
        f, m = oracle.grid_solve(H, W, *args, [7])
        qf, mr = oracle.grid_solve_rational(H, W, *args, 7, 1)
        assert qf == f[0] and np.array_equal(mr, m[0])


def test_brute_force_envelope_hand_cases():
    """One pixel with cs = lambda, ct = 7: F = min(lambda, 7), one breakpoint
    at 7, the pixel joins the source side there (a tie goes to the source
    side).  Two pixels joined by w = 4, cs = lambda each, ct = 3 and 9: the
    four cuts cost 2 lambda (none on the s side), lambda + 7 ({p0}), lambda +
    13 ({p1}) and 12 (both), so F = 2 lambda up to 6 and 12 after it."""
    from fractions import Fraction
    z = np.zeros((1, 1), np.int32)
    bps, masks, lines = oracle.brute_force_breakpoints(1, 1, z, z, z, np.ones((1, 1), np.int32),
                                                       np.full((1, 1), 7, np.int32), 0, 20)
    assert bps == [Fraction(7)] and masks[:, 0, 0].tolist() == [0, 1] and lines == [(0, 1), (7, 0)]
    # 1x2: cuts {} -> 2L, {p0} -> L + 3 + 4, {p1} -> L + 9 + 4, {p0, p1} -> 12
    w_h = np.array([[4, 0]], np.int32)
    args = (w_h, np.zeros((1, 2), np.int32), np.zeros((1, 2), np.int32), np.ones((1, 2), np.int32),
            np.array([[3, 9]], np.int32))
    bps, masks, lines = oracle.brute_force_breakpoints(1, 2, *args, 0, 100)
    # 2L meets L + 7 at 7; L + 7 meets 12 at 5 < 7, so 2L meets 12 first, at 6
    assert bps == [Fraction(6)] and lines == [(0, 2), (12, 0)]
    assert masks.tolist() == [[[0, 0]], [[1, 1]]]


@pytest.mark.parametrize("seed", range(6))
def test_exact_search_matches_brute_force_envelope(seed):
    """The search (oracle backend) returns the envelope's breakpoints, pieces'
    maximal cuts and lines exactly, all verified."""
    H, W = [(3, 4), (4, 4), (2, 8), (4, 3), (1, 12), (2, 6)][seed]
    args = _tiny(200 + seed, H, W)
    lo, hi = 0, 80
    res = parametric.exact_breakpoints(H, W, *args, lo, hi, backend=OracleExact(H, W, *args))
    bps, masks, lines = oracle.brute_force_breakpoints(H, W, *args, lo, hi)
    assert res.breakpoints == bps
    assert all(res.verified)
    assert np.array_equal(res.masks, masks)
    assert [tuple(l) for l in res.lines.tolist()] == lines
    assert res.solves <= 2 * len(bps) + 2


@pytest.mark.parametrize("seed", [0, 1])
def test_exact_search_agrees_with_integer_solves(seed):
    """On a 12 x 14 grid: at every integer lambda of the range the piece's cut
    is the oracle's maximal cut and its line value the oracle's flow; at each
    breakpoint both neighbouring lines meet F (exact rational solve)."""
    H, W = 12, 14
    args = _instance(H, W, seed)
    lo, hi = 1, 600
    res = parametric.exact_breakpoints(H, W, *args, lo, hi, backend=OracleExact(H, W, *args))
    f, m = oracle.grid_solve(H, W, *args, list(range(lo, hi + 1)))
    for j, lam in enumerate(range(lo, hi + 1)):
        i = sum(1 for x in res.breakpoints if x <= lam)
        assert np.array_equal(res.masks[i], m[j])
        assert res.value(lam) == f[j]
    for i, x in enumerate(res.breakpoints):
        qf, _ = oracle.grid_solve_rational(H, W, *args, x.numerator, x.denominator)
        for a, b in (res.lines[i], res.lines[i + 1]):
            assert qf == int(a) * x.denominator + int(b) * x.numerator
    # the integer change points are the ceilings of the breakpoints
    bp = parametric.breakpoints(H, W, *args, lo, hi, solve=_oracle_solver(H, W, *args))
    import math
    assert sorted({math.ceil(x) for x in res.breakpoints}) == [int(v) for v in bp.lambdas[1:]]


@pytest.mark.gpu
@pytest.mark.parametrize("case", ["tiny", "40x56"])
def test_gpu_exact_breakpoints(case):
    """GPU search (restricted scaled problems, cut lines in the library's
    kernels) against the brute-force envelope (tiny grids) and against the
    oracle-backed search (a 40 x 56 segmentation instance)."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1509_06004_b300 import build
    build.build()
    if case == "tiny":
        for seed, (H, W) in enumerate([(3, 4), (4, 4), (2, 8), (1, 12)]):
            args = _tiny(300 + seed, H, W)
            res = parametric.exact_breakpoints(H, W, *args, 0, 80)
            bps, masks, lines = oracle.brute_force_breakpoints(H, W, *args, 0, 80)
            assert res.breakpoints == bps and all(res.verified)
            assert np.array_equal(res.masks, masks)
            assert [tuple(l) for l in res.lines.tolist()] == lines
        return
    H, W = 40, 56
    args = _instance(H, W, 11)
    res = parametric.exact_breakpoints(H, W, *args, 1, 1500)
    ref = parametric.exact_breakpoints(H, W, *args, 1, 1500, backend=OracleExact(H, W, *args))
    assert res.breakpoints == ref.breakpoints and all(res.verified)
    assert np.array_equal(res.masks, ref.masks) and np.array_equal(res.lines, ref.lines)
    assert (res.flow_lo, res.flow_hi) == (ref.flow_lo, ref.flow_hi)


def _restricted(w_h, w_v, src0, slope, sink, s1, s2, p, q):
    """The problem between two nested cuts as pmf_restrict_between documents it,
    written independently here: pixels of D = s2 minus s1 keep their pairs to
    each other, a pixel's pairs into s1 join its source capacity and its pairs
    out of s2 its sink capacity, all capacities times q at lambda = p/q; every
    other pixel gets no arcs and a unit sink capacity."""
    i64 = lambda a: np.asarray(a, np.int64)
    w_h, w_v, src0, slope, sink = map(i64, (w_h, w_v, src0, slope, sink))
    H, W = w_h.shape
    S1, S2 = np.asarray(s1) != 0, np.asarray(s2) != 0
    D = S2 & ~S1
    cs = np.zeros((H, W), np.int64)
    ct = np.ones((H, W), np.int64)
    wr = np.zeros((H, W), np.int64)
    wd = np.zeros((H, W), np.int64)
    for y in range(H):
        for x in range(W):
            if not D[y, x]:
                continue
            pin, pout = 0, 0
            for (yy, xx, w) in ((y, x + 1, w_h[y, x] if x + 1 < W else 0), (y, x - 1, w_h[y, x - 1] if x > 0 else 0),
                                (y + 1, x, w_v[y, x] if y + 1 < H else 0), (y - 1, x, w_v[y - 1, x] if y > 0 else 0)):
                if not (0 <= yy < H and 0 <= xx < W):
                    continue
                if S1[yy, xx]:
                    pin += w
                elif not S2[yy, xx]:
                    pout += w
            cs[y, x] = q * (src0[y, x] + pin) + p * slope[y, x]
            ct[y, x] = q * (sink[y, x] + pout)
            if x + 1 < W and D[y, x + 1]:
                wr[y, x] = q * w_h[y, x]
            if y + 1 < H and D[y + 1, x]:
                wd[y, x] = q * w_v[y, x]
    return wr, wd, cs, ct


@pytest.mark.parametrize("seed", range(4))
def test_restricted_problem_decomposition(seed):
    """Between the maximal cuts S1 at lambda_1 and S2 at lambda_2, the problem
    restricted to S2 minus S1 and scaled at any rational lambda* in between
    has the full problem's maximal cut at lambda* (joined with S1), and the
    gap between the sum of its source capacities and its flow is q times the
    gap between S1's line and F(lambda*) (Section 2's cut cost; the oracle
    solves both problems)."""
    from fractions import Fraction
    H, W = 10, 12
    args = _instance(H, W, 40 + seed)
    f, m = oracle.grid_solve(H, W, *args, [30, 900])
    s1, s2 = m[0], m[1]
    a1, b1 = oracle.cut_line(H, W, *args, s1)
    for lam in (Fraction(61, 2), Fraction(400, 3), Fraction(899, 1), Fraction(2137, 7)):
        p, q = lam.numerator, lam.denominator
        wr, wd, cs, ct = _restricted(*args, s1, s2, p, q)
        sub_f, sub_m = oracle.grid_solve(H, W, wr, wd, cs, np.zeros_like(cs), ct, [0])
        qf, full_m = oracle.grid_solve_rational(H, W, *args, p, q)
        assert np.array_equal((sub_m[0] != 0) | (s1 != 0), full_m != 0)
        assert int(cs.sum()) - int(sub_f[0]) == q * a1 + p * b1 - qf
