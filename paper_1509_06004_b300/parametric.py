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


def gpu_solver(H, W, w_h, w_v, src0, slope, sink, device: int = 0, max_batch: int = 256, **tuning):
    """A solve(lambdas) -> (flows [k], masks [k, H, W]) callable that runs each
    lambda as its own instance, max_batch instances per batch."""
    from . import inputs, pmf

    def solve(lams):
        flows, masks = [], []
        for c0 in range(0, len(lams), max_batch):
            chunk = [int(x) for x in lams[c0:c0 + max_batch]]
            wl = inputs.Workload("breakpoints", [inputs.Image(H, W, w_h, w_v, None)], [])
            for lam in chunk:
                wl.instances.append(inputs.Instance(0, src0, slope, sink, np.array([lam], np.int32)))
            st, res = pmf.solve_workload(wl, device=device, check=False, **tuning)
            if any(s != pmf.PMF_OK for s in st):
                raise RuntimeError(f"breakpoint solve failed: {[pmf.status_string(s) for s in st if s]}")
            for f, m in res:
                flows.append(int(f[0]))
                masks.append(m[0])
        return np.array(flows, np.int64), np.stack(masks) if masks else np.zeros((0, H, W), np.uint8)
    return solve


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
    known: dict[int, tuple[int, np.ndarray]] = {}

    def run(lams):
        f, m = solve(lams)
        for lam, fv, mv in zip(lams, f, m):
            known[int(lam)] = (int(fv), np.asarray(mv, np.uint8).reshape(H, W))

    run(sorted({lo, hi}))
    rounds, solves = 1, len(known)
    pending = [(lo, hi)] if hi > lo else []
    while pending:
        mids, nxt = [], []
        for a, b in pending:
            if b - a <= 1 or np.array_equal(known[a][1], known[b][1]):
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
    keep = [pts[0]] + [b for a, b in zip(pts, pts[1:]) if not np.array_equal(known[a][1], known[b][1])]
    return Breakpoints(np.array(keep, np.int64), np.array([known[x][0] for x in keep], np.int64),
                       np.stack([known[x][1] for x in keep]), solves, rounds)
