"""The s-t swap of Section 3.2 for lambda-concurrent solves.

Exchanging s and t leaves the maximum flow and the minimum cuts unchanged
(the pairwise capacities here are symmetric, so the exchanged problem is the
same grid with source capacities ct and sink capacities cs(lambda)).  The
paper applies it per graph with a sign-count rule: over the pixels, compare
the number of negative and positive differences cs - ct, and swap when the
negative ones are more.  Its purpose there is the work per iteration of a
push-relabel that processes pixels with source residual.

Here every (instance, lambda) of a workload becomes its own one-lambda
instance of one batch (the paper's lambda-supergraph), each swapped or not by
that rule.  A swapped instance is marked with pmf_set_cut_rule(1): the solver
then returns the original problem's maximal source set, as the complement of
the exchanged problem's minimal source set, which the GPU finds as the pixels
reachable from excess after the solve.
"""
from __future__ import annotations

import numpy as np


def needs_swap(src0, slope, sink, lam: int) -> bool:
    """Section 3.2's rule: more pixels with cs - ct < 0 than with cs - ct > 0."""
    d = np.asarray(src0, np.int64) + np.asarray(slope, np.int64) * int(lam) - np.asarray(sink, np.int64)
    return int((d < 0).sum()) > int((d > 0).sum())


def swapped_terminals(src0, slope, sink, lam: int):
    """Terminals of the exchanged problem at one lambda: (src0', slope', sink')
    = (ct, 0, cs(lambda))."""
    cs = np.asarray(src0, np.int64) + np.asarray(slope, np.int64) * int(lam)
    return (np.ascontiguousarray(sink, np.int32), np.zeros_like(np.asarray(sink, np.int32)),
            cs.astype(np.int32))


def solve_workload(wl, swap: str = "auto", device: int = 0, **tuning):
    """Solve every (instance, lambda) of an inputs.Workload as its own instance,
    s-t swapped by Section 3.2's rule (swap="auto"), always or never.
    Returns (statuses [n_inst][m], results [(flows [m], masks [m, H, W])],
    swapped bool [n_inst][m]) in the workload's own layout."""
    from . import inputs, pmf
    if swap not in ("auto", "always", "never"):
        raise ValueError("swap is auto, always or never")
    flat = inputs.Workload(wl.name + "/swap", wl.images, [])
    where, swapped = [], []
    for i, inst in enumerate(wl.instances):
        for k, lam in enumerate(inst.lambdas):
            sw = swap == "always" or (swap == "auto" and needs_swap(inst.src0, inst.slope, inst.sink, lam))
            if sw:
                a, b, c = swapped_terminals(inst.src0, inst.slope, inst.sink, lam)
                flat.instances.append(inputs.Instance(inst.image, a, b, c, np.array([lam], np.int32)))
            else:
                flat.instances.append(inputs.Instance(inst.image, inst.src0, inst.slope, inst.sink,
                                                      np.array([lam], np.int32)))
            where.append((i, k))
            swapped.append(sw)
    b = pmf.batch_from_workload(flat, device=device, **tuning)
    for j, sw in enumerate(swapped):
        if sw:
            b.set_cut_rule(j, 1)
    b.solve(np.stack([x.lambdas for x in flat.instances]).astype(np.int32))
    st = b.sync(check=False)
    out_st = [[None] * len(x.lambdas) for x in wl.instances]
    out_sw = [[False] * len(x.lambdas) for x in wl.instances]
    res = [(np.zeros(len(x.lambdas), np.int64),
            np.zeros((len(x.lambdas), wl.images[x.image].H, wl.images[x.image].W), np.uint8))
           for x in wl.instances]
    for j, (i, k) in enumerate(where):
        out_st[i][k] = st[j]
        out_sw[i][k] = swapped[j]
        if st[j] == pmf.PMF_OK:
            res[i][0][k] = b.flows(j)[0]
            res[i][1][k] = b.cuts(j)[0]
    b.close()
    return out_st, res, out_sw
