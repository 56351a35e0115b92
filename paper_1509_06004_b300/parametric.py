"""Every breakpoint of a parametric minimum cut over an integer lambda range.

In the monotone case the paper's segmentation uses (Section 2.1: source
capacities cs(p, lambda) = src0(p) + slope(p) * lambda with slope >= 0, sink
capacities fixed), the maximal minimum-cut source sets S(lambda) are nested and
grow with lambda, as Gallo, Grigoriadis and Tarjan showed; the paper names
finding all of them, instead of solving a preset schedule, as the ideal.  With
nestedness, S(a) == S(b) implies S(lambda) == S(a) for every lambda in [a, b].
So a bisection over the integers finds every integer lambda at which S
changes: an interval whose end cuts differ is split at its midpoint until it
is one apart, and one whose end cuts agree is done.  All midpoints of a round
are solved together, as independent one-lambda instances of one batch on the
GPU (the paper's lambda-supergraph, Section 3.1); the host only compares the
returned masks and picks the next midpoints.

breakpoints() returns the distinct source sets, each with the smallest integer
lambda of the range at which it is the maximal minimum cut and the flow value
there.  Solves needed: about (number of breakpoints) * log2(range) + 2.

exact_breakpoints() (below) finds the exact rational breakpoints of the
minimum cut value instead, with about two solves per breakpoint.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class Breakpoints:
    lambdas: np.ndarray       # int64 [n]: lo, then every lambda in (lo, hi] where the cut changes
    flows: np.ndarray         # int64 [n]: maximum-flow value at each of those lambdas
    masks: np.ndarray         # uint8 [n, H, W]: maximal source set from that lambda on
    solves: int               # max-flow solves run
    rounds: int               # batched rounds (including the first, at lo and hi)


class GpuBisect:
    """A solve(lambdas) -> (flows [k], masks [k] (device), lines [k, 2])
    callable for the bisection: each lambda is its own one-lambda instance of
    ONE batch that is created once (max_batch instances of the image, its
    terminals uploaded once and copied on the device) and re-run every round
    with new lambdas; unused instances repeat a lambda.  Masks stay in device
    memory; the cut lines (pmf_cut_lines) tell cuts apart, since two maximal
    cuts at different lambdas are equal exactly when their lines are."""

    def __init__(self, H, W, w_h, w_v, src0, slope, sink, device: int = 0, max_batch: int = 256, **tuning):
        import torch
        from . import pmf
        self.pmf, self.torch = pmf, torch
        self.H, self.W, self.device, self.max_batch = int(H), int(W), int(device), int(max_batch)
        self.dev = torch.device("cuda", self.device)
        d = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.int32)).to(self.dev)
        self.cap = [d(a) for a in (w_h, w_v, src0, slope, sink)]
        self.tuning = tuning
        self.b = None
        self.solves = 0

    def _ensure(self):
        if self.b is None:
            pmf = self.pmf
            b = pmf.Batch([(self.H, self.W)], [0] * self.max_batch, 1, device=self.device)
            if self.tuning:
                b.set_tuning(**self.tuning)
            b.set_capacities(0, self.cap[0], self.cap[1])
            b.set_terminals(0, self.cap[2], self.cap[3], self.cap[4])
            for i in range(1, self.max_batch):
                b.copy_terminals(i, 0)
            self.b = b
        return self.b

    def __call__(self, lams):
        import ctypes
        torch, pmf = self.torch, self.pmf
        b = self._ensure()
        flows, masks, lines = [], [], []
        for c0 in range(0, len(lams), self.max_batch):
            chunk = [int(x) for x in lams[c0:c0 + self.max_batch]]
            sched = np.array(chunk + [chunk[-1]] * (self.max_batch - len(chunk)), np.int32).reshape(-1, 1)
            b.solve(sched)
            st = b.sync(check=False)
            if any(s != pmf.PMF_OK for s in st):
                raise RuntimeError(f"breakpoint solve failed: {[pmf.status_string(s) for s in st if s]}")
            m = torch.empty((len(chunk), self.H, self.W), dtype=torch.uint8, device=self.dev)
            for i in range(len(chunk)):
                b.get_cut(i, 0, m[i])
                flows.append(b.get_flow(i, 0))
            ln = torch.empty((len(chunk), 2), dtype=torch.int64, device=self.dev)
            ptr = lambda t: ctypes.c_void_p(t.data_ptr())
            st = pmf.lib().pmf_cut_lines(self.H, self.W, *[ptr(c) for c in self.cap], ctypes.c_void_p(0), ptr(m),
                                         len(chunk), ctypes.c_void_p(0), ptr(ln),
                                         ctypes.c_void_p(torch.cuda.current_stream(self.dev).cuda_stream))
            pmf._check(st, "pmf_cut_lines")
            masks += list(m)
            lines.append(ln.cpu().numpy())
            self.solves += len(chunk)
        return np.array(flows, np.int64), masks, np.concatenate(lines)

    def close(self):
        if self.b is not None:
            self.b.close()
            self.b = None


def gpu_solver(H, W, w_h, w_v, src0, slope, sink, device: int = 0, max_batch: int = 256, **tuning):
    """The bisection's GPU solver (GpuBisect)."""
    return GpuBisect(H, W, w_h, w_v, src0, slope, sink, device=device, max_batch=max_batch, **tuning)


def breakpoints(H, W, w_h, w_v, src0, slope, sink, lo: int, hi: int, solve=None, **kw) -> Breakpoints:
    """All integer breakpoints of the instance's maximal minimum cut on [lo, hi].
    ``solve`` (lambdas -> flows, masks) defaults to the GPU solver; its results
    must be exact maximal source sets (the bisection relies on equality)."""
    lo, hi = int(lo), int(hi)
    if lo > hi:
        raise ValueError("empty lambda range")
    if np.any(np.asarray(slope) < 0):
        raise ValueError("the bisection needs nondecreasing source capacities (slope >= 0)")
    solve = solve or gpu_solver(H, W, w_h, w_v, src0, slope, sink, **kw)
    known: dict[int, tuple] = {}

    def run(lams):
        out = solve(lams)
        f, m = out[0], out[1]
        # cuts are told apart by their lines when the solver gives them, else by
        # their masks (host arrays)
        keys = out[2] if len(out) > 2 else [None] * len(lams)
        for lam, fv, mv, kv in zip(lams, f, m, keys):
            key = tuple(int(x) for x in kv) if kv is not None else np.asarray(mv, np.uint8).reshape(H, W).tobytes()
            known[int(lam)] = (int(fv), mv, key)

    run(sorted({lo, hi}))
    rounds, solves = 1, len(known)
    pending = [(lo, hi)] if hi > lo else []
    while pending:
        mids, nxt = [], []
        for a, b in pending:
            if b - a <= 1 or known[a][2] == known[b][2]:
                continue
            c = (a + b) // 2
            mids.append(c)
            nxt += [(a, c), (c, b)]
        if not mids:
            break
        run(mids)
        rounds += 1
        solves += len(mids)
        pending = nxt
    pts = sorted(known)
    keep = [pts[0]] + [b for a, b in zip(pts, pts[1:]) if known[a][2] != known[b][2]]
    host = lambda m: (m.cpu().numpy() if hasattr(m, "cpu") else np.asarray(m, np.uint8)).reshape(H, W)
    return Breakpoints(np.array(keep, np.int64), np.array([known[x][0] for x in keep], np.int64),
                       np.stack([host(known[x][1]) for x in keep]), solves, rounds)


# ----------------------------------------------------------------------------
# exact breakpoints
# ----------------------------------------------------------------------------
# The integer bisection above finds where the maximal cut changes between
# integers.  The minimum cut value F(lambda) is the lower envelope of the cut
# lines cap_S(lambda) = a_S + b_S*lambda, so its breakpoints are exact
# rationals: where the lines of consecutive maximal cuts cross.  The search
# below (the Eisner-Severance scheme for parametric minimum cuts) finds every
# one of them on [lo, hi]:
#   * solve at lo and hi: maximal cuts S_lo, S_hi and their lines;
#   * for an interval whose end cuts S1 (optimal at lambda_1) and S2 (optimal
#     at lambda_2) differ, their lines cross at lambda* = (a2 - a1)/(b1 - b2),
#     lambda_1 < lambda* <= lambda_2; solve exactly at lambda*;
#   * if F(lambda*) equals the lines' common value, no other cut is optimal
#     between them: F follows line 1 up to lambda* and line 2 after it, and
#     lambda* is a breakpoint; otherwise the maximal cut S* at lambda* lies
#     strictly between S1 and S2 and both halves are searched.
# Each solve either certifies a breakpoint or finds a new cut, so the search
# takes about twice as many solves as there are breakpoints.  The exact solve
# at a rational lambda* = p/q runs on the problem restricted to the pixels
# between S1 and S2 (every cut in between costs a constant plus its cut), with
# all capacities times q: no infinite capacities remain, so the integers fit
# the GPU's int32 state unless q is very large; such a breakpoint is reported
# as not verified (the crossing of its two cuts, with no search between them).
# All intervals of a round are solved together in one launch.

@dataclass
class ExactBreakpoints:
    breakpoints: list         # Fraction [r]: lo < lambda*_1 < ... < lambda*_r <= hi
    verified: list            # bool [r]: F(lambda*_i) checked by an exact solve
    masks: np.ndarray         # uint8 [r+1, H, W]: maximal cut on [lambda*_i, lambda*_{i+1}) (i = 0: from lo)
    lines: np.ndarray         # int64 [r+1, 2]: (a_i, b_i), cut cost a_i + b_i*lambda
    flow_lo: int              # F(lo)
    flow_hi: int              # F(hi)
    solves: int               # max-flow solves run (the two ends count as one warm-started pair)
    rounds: int               # batched rounds

    def value(self, lam):
        """F(lambda) on [lo, hi] from the lines (exact for Fraction arguments)."""
        from fractions import Fraction
        lam = Fraction(lam)
        i = sum(1 for x in self.breakpoints if x <= lam)
        a, b = (int(v) for v in self.lines[i])
        return a + b * lam


@dataclass
class BetweenResult:
    overflow: bool            # the scaled restricted problem did not fit the solver's capacity limits
    gap: int                  # q * (line value at lambda* - F(lambda*)); 0 = lambda* is a breakpoint
    mask: object = None       # the maximal cut at lambda* (backend's handle) when gap > 0
    line: tuple = None        # its (a, b)


def exact_breakpoints(H, W, w_h, w_v, src0, slope, sink, lo: int, hi: int, backend=None,
                      **kw) -> ExactBreakpoints:
    """Every breakpoint of the instance's parametric minimum cut value on
    [lo, hi], exactly, with the maximal cut and its line on each piece.
    ``backend`` (default: the GPU, ``GpuExact``) provides
      ends(lo, hi) -> ([mask_lo, mask_hi], [(a, b)] * 2, [F(lo), F(hi)]),
      between([(mask1, mask2, (a1, b1), p, q)]) -> [BetweenResult],
      host_mask(mask) -> uint8 [H, W]."""
    from fractions import Fraction
    lo, hi = int(lo), int(hi)
    if lo > hi:
        raise ValueError("empty lambda range")
    if np.any(np.asarray(slope) < 0):
        raise ValueError("the search needs nondecreasing source capacities (slope >= 0)")
    be = backend or GpuExact(H, W, w_h, w_v, src0, slope, sink, **kw)
    masks, lines, flows = be.ends(lo, hi)
    cuts = [(Fraction(lo), masks[0], tuple(int(x) for x in lines[0])),
            (Fraction(hi), masks[1], tuple(int(x) for x in lines[1]))]
    found = {}            # (i1, i2) -> (lambda*, verified) for intervals that end as a breakpoint
    pending = [(0, 1)]
    rounds, solves = 1, 1
    while pending:
        items = []
        for i1, i2 in pending:
            (a1, b1), (a2, b2) = cuts[i1][2], cuts[i2][2]
            if (a1, b1) == (a2, b2):
                continue            # the same maximal cut at both ends: none in between
            if b1 <= b2:
                raise RuntimeError("cut lines not ordered: the solver's cuts are not maximal or not nested")
            items.append((i1, i2, Fraction(a2 - a1, b1 - b2)))
        if not items:
            break
        res = be.between([(cuts[i1][1], cuts[i2][1], cuts[i1][2], lam.numerator, lam.denominator)
                          for i1, i2, lam in items])
        rounds += 1
        solves += len(items)
        pending = []
        for (i1, i2, lam), r in zip(items, res):
            if r.overflow:
                found[(i1, i2)] = (lam, False)
            elif r.gap == 0:
                found[(i1, i2)] = (lam, True)
            elif r.gap < 0:
                raise RuntimeError("a cut cheaper than the minimum: the solver's flow is not maximal")
            else:
                cuts.append((lam, r.mask, tuple(int(x) for x in r.line)))
                k = len(cuts) - 1
                pending += [(i1, k), (k, i2)]
    # the chain of distinct cuts in lambda order; a single cut if both ends agree
    order = sorted(range(len(cuts)), key=lambda i: cuts[i][0])
    if cuts[0][2] == cuts[1][2]:
        order = [0]
    bps, ver = [], []
    for i1, i2 in zip(order, order[1:]):
        lam, ok = found[(i1, i2)]
        bps.append(lam)
        ver.append(ok)
    return ExactBreakpoints(bps, ver, np.stack([be.host_mask(cuts[i][1]) for i in order]),
                            np.array([cuts[i][2] for i in order], np.int64), int(flows[0]), int(flows[-1]),
                            solves, rounds)


class GpuExact:
    """GPU backend of exact_breakpoints: the solves run through the batch
    entry points, the cut lines (pmf_cut_lines) and the restricted, scaled
    problems (pmf_restrict_between) in the library's kernels; masks stay in
    device memory until the end.  One batch of each size is created once and
    reused by every round (its workspace and inputs are rewritten on the
    device)."""

    def __init__(self, H, W, w_h, w_v, src0, slope, sink, device: int = 0, max_batch: int = 64, **tuning):
        import torch
        from . import pmf
        self.pmf, self.torch = pmf, torch
        self.H, self.W, self.device = int(H), int(W), int(device)
        self.dev = torch.device("cuda", self.device)
        d = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.int32)).to(self.dev)
        self.cap = [d(a) for a in (w_h, w_v, src0, slope, sink)]
        self.zero = torch.zeros((self.H, self.W), dtype=torch.int32, device=self.dev)
        self.max_batch = int(max_batch)
        self.tuning = tuning
        self._pool = {}

    def _ptr(self, t):
        import ctypes
        return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)

    def _stream(self):
        import ctypes
        return ctypes.c_void_p(self.torch.cuda.current_stream(self.dev).cuda_stream)

    def _lines(self, masks, base=None):
        """(the sets masks[k] | base on the device, their lines as int64 [k, 2])."""
        torch = self.torch
        k = masks.shape[0]
        uni = torch.empty_like(masks)
        lines = torch.empty((k, 2), dtype=torch.int64, device=self.dev)
        st = self.pmf.lib().pmf_cut_lines(self.H, self.W, *[self._ptr(c) for c in self.cap], self._ptr(base),
                                          self._ptr(masks), k, self._ptr(uni), self._ptr(lines), self._stream())
        self.pmf._check(st, "pmf_cut_lines")
        return uni, lines.cpu().numpy()

    def host_mask(self, m):
        return m.cpu().numpy().reshape(self.H, self.W)

    def ends(self, lo, hi):
        torch, pmf = self.torch, self.pmf
        lam = [lo] if lo == hi else [lo, hi]
        b = pmf.Batch([(self.H, self.W)], [0], len(lam), device=self.device)
        try:
            if self.tuning:
                b.set_tuning(**self.tuning)
            b.set_capacities(0, self.cap[0], self.cap[1])
            b.set_terminals(0, self.cap[2], self.cap[3], self.cap[4])
            b.solve(np.array([lam], np.int32))      # warm-started from lo to hi
            b.sync()
            m = torch.empty((len(lam), self.H, self.W), dtype=torch.uint8, device=self.dev)
            b.cuts(0, m)
            f = b.flows(0)
        finally:
            b.close()
        uni, lines = self._lines(m)
        if len(lam) == 1:
            return [uni[0], uni[0]], [lines[0], lines[0]], [f[0], f[0]]
        return [uni[0], uni[1]], [lines[0], lines[1]], [f[0], f[1]]

    def _batch(self, n):
        """A batch of n one-image instances (reused), with device buffers for
        the restricted problems' inputs."""
        torch, pmf = self.torch, self.pmf
        if n not in self._pool:
            b = pmf.Batch([(self.H, self.W)] * n, list(range(n)), 1, device=self.device)
            if self.tuning:
                b.set_tuning(**self.tuning)
            bufs = torch.zeros((n, 4, self.H, self.W), dtype=torch.int32, device=self.dev)
            sums = torch.zeros((n, 4), dtype=torch.int64, device=self.dev)
            self._pool[n] = (b, bufs, sums)
        return self._pool[n]

    def between(self, items):
        out = []
        for c0 in range(0, len(items), self.max_batch):
            out += self._between(items[c0:c0 + self.max_batch])
        return out

    def _between(self, items):
        torch, pmf = self.torch, self.pmf
        n = 1
        while n < len(items):
            n *= 2
        b, bufs, sums = self._batch(n)
        L = pmf.lib()
        for k in range(n):
            if k < len(items):
                s1, s2, _, p, q = items[k]
                st = L.pmf_restrict_between(self.H, self.W, *[self._ptr(c) for c in self.cap], self._ptr(s1),
                                            self._ptr(s2), int(p), int(q), *[self._ptr(bufs[k, j]) for j in range(4)],
                                            self._ptr(sums[k]), self._stream())
                pmf._check(st, "pmf_restrict_between")
            else:
                bufs[k].zero_()             # an unused slot solves an empty problem
            b.set_capacities(k, bufs[k, 0], bufs[k, 1])
            b.set_terminals(k, bufs[k, 2], self.zero, bufs[k, 3])
        b.solve(np.zeros((n, 1), np.int32))
        st = b.sync(check=False)
        hs = sums.cpu().numpy()
        res = []
        for k, (s1, s2, _, p, q) in enumerate(items):
            if hs[k, 2] > 0:
                res.append(BetweenResult(True, 0))
                continue
            if st[k] != pmf.PMF_OK:
                raise pmf.PmfError(st[k], "exact breakpoint solve")
            gap = int(hs[k, 0]) - b.get_flow(k, 0)
            if gap == 0:
                res.append(BetweenResult(False, 0))
                continue
            sub = torch.empty((1, self.H, self.W), dtype=torch.uint8, device=self.dev)
            b.get_cut(k, 0, sub[0])
            uni, lines = self._lines(sub, base=s1)
            res.append(BetweenResult(False, gap, uni[0], (int(lines[0, 0]), int(lines[0, 1]))))
        return res

    def close(self):
        for b, _, _ in self._pool.values():
            b.close()
        self._pool.clear()
