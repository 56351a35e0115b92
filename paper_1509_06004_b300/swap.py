"""The s-t swap of Section 3.2 for lambda-concurrent solves.

Exchanging s and t leaves the maximum flow and the minimum cuts unchanged
(the pairwise capacities here are symmetric, so the exchanged problem is the
same grid with source capacities ct and sink capacities cs(lambda)).  The
paper applies it per graph with a sign-count rule: over the pixels, compare
the number of negative and positive differences cs - ct, and swap when the
negative ones are more.  Its purpose there is the work per iteration of a
push-relabel that processes pixels with source residual.

Two batchings are built.  In the lambda-concurrent one, every (instance,
lambda) of a workload becomes its own one-lambda instance of one batch (the
paper's lambda-supergraph), each swapped or not by that rule.  In the
warm-started one, each instance keeps its whole schedule as one GGT chain, and
a swapped chain runs the exchanged problem backwards: its sink capacities
src0 + slope*lambda fall as lambda falls, which is Section 2.1's monotone case
in the parameter mu = lambda_last - lambda (pmf_set_slope_side(1)).  A
swapped instance is marked with pmf_set_cut_rule(1): the solver then returns
the original problem's maximal source set, as the complement of the exchanged
problem's minimal source set, which the GPU finds as the pixels reachable
from excess after the solve.
"""
from __future__ import annotations

import numpy as np


def needs_swap(src0, slope, sink, lam: int) -> bool:
    """Section 3.2's rule: more pixels with cs - ct < 0 than with cs - ct > 0."""
    d = np.asarray(src0, np.int64) + np.asarray(slope, np.int64) * int(lam) - np.asarray(sink, np.int64)
    return int((d < 0).sum()) > int((d > 0).sum())


def swapped_terminals(src0, slope, sink, lam: int):
    """Terminals of the exchanged problem at one lambda: (src0', slope', sink')
    = (ct, 0, cs(lambda)).  cs(lambda) must lie in [0, 2^30] (the sink
    capacities of the exchanged problem), else ValueError."""
    cs = np.asarray(src0, np.int64) + np.asarray(slope, np.int64) * int(lam)
    if cs.size and (cs.max() > (1 << 30) or cs.min() < 0):
        raise ValueError("source capacities at lambda must lie in [0, 2^30]")
    return (np.ascontiguousarray(sink, np.int32), np.zeros_like(np.asarray(sink, np.int32)),
            cs.astype(np.int32))


def warm_swapped_terminals(src0, slope, sink, lambdas):
    """The exchanged problem of a whole schedule, for a warm-started chain
    with pmf_set_slope_side(1): terminals (src0', slope', sink') = (ct, slope,
    cs(lambda_last)) and the increasing schedule mu_j = lambda_last -
    lambda_{m-1-j}.  At mu_j its source capacities are ct and its sink
    capacities sink' - slope*mu_j = cs(lambda_{m-1-j}): the original problem at
    lambda_{m-1-j} with s and t exchanged, so result j belongs to
    lambda_{m-1-j}."""
    lam = np.asarray(lambdas, np.int64)
    if lam.ndim != 1 or lam.size == 0 or np.any(np.diff(lam) < 0):
        raise ValueError("lambdas must be a nonempty nondecreasing schedule")
    top = np.asarray(src0, np.int64) + np.asarray(slope, np.int64) * int(lam[-1])
    if top.size and (top.max() > (1 << 30) or top.min() < 0):
        raise ValueError("source capacities at the last lambda must lie in [0, 2^30]")
    mu = (lam[-1] - lam[::-1]).astype(np.int32)
    return (np.ascontiguousarray(sink, np.int32), np.ascontiguousarray(slope, np.int32),
            top.astype(np.int32), mu)


def chain_needs_swap(src0, slope, sink, lambdas) -> bool:
    """Section 3.2's rule for a warm-started chain: swap when the rule says so
    for more than half of its lambdas."""
    votes = sum(needs_swap(src0, slope, sink, int(l)) for l in lambdas)
    return 2 * votes > len(lambdas)


def solve_workload(wl, swap: str = "auto", device: int = 0, warm: bool = False, **tuning):
    """Solve an inputs.Workload s-t swapped by Section 3.2's rule
    (swap="auto"), always or never.  warm=False: every (instance, lambda) is
    its own instance, swapped or not on its own.  warm=True: every instance is
    one warm-started chain over its schedule, swapped or not as a whole (see
    chain_needs_swap).  Returns (statuses [n_inst][m], results [(flows [m],
    masks [m, H, W])], swapped bool [n_inst][m]) in the workload's own layout."""
    from . import inputs, pmf
    if swap not in ("auto", "always", "never"):
        raise ValueError("swap is auto, always or never")
    if warm:
        return _solve_chains(wl, swap, device, tuning)
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


def _solve_chains(wl, swap, device, tuning):
    """solve_workload(warm=True): one warm-started instance per chain."""
    from . import inputs, pmf
    flat = inputs.Workload(wl.name + "/swap-chains", wl.images, [])
    swapped = []
    for inst in wl.instances:
        sw = swap == "always" or (swap == "auto" and chain_needs_swap(inst.src0, inst.slope, inst.sink,
                                                                      inst.lambdas))
        if sw:
            a, b, c, mu = warm_swapped_terminals(inst.src0, inst.slope, inst.sink, inst.lambdas)
            flat.instances.append(inputs.Instance(inst.image, a, b, c, mu))
        else:
            flat.instances.append(inst)
        swapped.append(sw)
    b = pmf.batch_from_workload(flat, device=device, **tuning)
    for j, sw in enumerate(swapped):
        if sw:
            b.set_cut_rule(j, 1)
            b.set_slope_side(j, 1)
    b.solve([np.asarray(x.lambdas, np.int32) for x in flat.instances])
    st = b.sync(check=False)
    out_st, res, out_sw = [], [], []
    for j, (inst, sw) in enumerate(zip(wl.instances, swapped)):
        m = len(inst.lambdas)
        img = wl.images[inst.image]
        out_st.append([st[j]] * m)
        out_sw.append([sw] * m)
        if st[j] == pmf.PMF_OK:
            f, c = b.flows(j), b.cuts(j)
            if sw:
                f, c = f[::-1], c[::-1]
            res.append((np.ascontiguousarray(f), np.ascontiguousarray(c)))
        else:
            res.append((np.zeros(m, np.int64), np.zeros((m, img.H, img.W), np.uint8)))
    b.close()
    return out_st, res, out_sw
