"""Autotuner: batching mode and solver knobs for a class of workloads.

The solve's speed depends on how a seed's lambda schedule is spread over
instances and on the kernel knobs, and the best choice shifts with image size,
instance count and schedule length:

* ``segments`` — each seed's schedule is cut into this many consecutive
  pieces, each its own warm-started instance (1 = one lambda-sequential chain
  per seed; schedule length = every (seed, lambda) cold, the paper's
  lambda-supergraph); more pieces give the GPU more independent work, fewer
  keep more warm-start reuse;
* ``interleave`` — each seed's schedule is dealt round-robin into this many
  pieces (piece j: lambda_j, lambda_{j+P}, ...): every piece starts cold at one
  of the smallest lambdas and neighbouring lambdas of a seed run side by side;
* ``fork`` — with ``segments`` > 1: each piece after a seed's first starts
  from a copy of the previous piece's state (pmf_set_fork) taken ``fork``
  steps before that piece's end, instead of cold (-1 = cold pieces);
* ``tile_h`` (rows per tile), ``push_order`` (pushes from the sweep's starting
  state, or along columns and rows), ``sweeps`` (push/relabel sweeps per tile visit),
  ``relabel_every`` (visit budget of a push/relabel phase, percent of its
  tiles), ``relabel_extra`` (visits added to every phase's budget),
  ``relabel_reach`` (a phase's budget floor, percent of the last relabel's
  largest distance),
  ``label_slack`` (parking threshold above the last exact distance),
  ``poll_ns`` (longest sleep of an idle warp between polls of its queue slot) and
  ``blocks_per_sm`` (4 resident blocks, or 3 with more registers each).

``tune`` times candidates on the GPU by coordinate descent inside a time
budget; choices are cached in a JSON file keyed by (GPU name, workload class).
Results never depend on the choice (outputs are unique), only speed does.
"""
from __future__ import annotations

import json
import math
import os
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
CACHE_PATH = os.path.join(HERE, "tuned.json")

DEFAULTS = {"tile_h": 4, "sweeps": 8, "relabel_every": 800, "label_slack": 16, "push_order": 0, "relabel_extra": 0,
            "poll_ns": 256, "blocks_per_sm": 0, "relabel_reach": 0, "strip_stage": -1}
SPACE = {
    "tile_h": [4, 8],
    "push_order": [0, 1],
    "sweeps": [2, 4, 8, 16],
    "relabel_every": [200, 400, 800, 1600, 3200, 6400],
    "label_slack": [2, 4, 8, 16, 32],
    "relabel_extra": [0, 64, 256, 1024],
    "relabel_reach": [0, 400, 800],
    "poll_ns": [256, 1024, 4096],
    # 0: the occupancy (4 blocks per SM at tile height 4); 3: the build with
    # the fourth block's registers (no spills)
    "blocks_per_sm": [0, 3],
}


def apply_plan(wl, plan: dict):
    """The workload as a plan batches it: each seed's schedule dealt into
    ``plan["interleave"]`` round-robin pieces, then each piece cut into
    ``plan["segments"]`` consecutive ones (both default to 1).  Every piece
    records which lambdas of which seed it holds (``Workload.gather``)."""
    w = wl
    il = int(plan.get("interleave", 1) or 1)
    if il > 1:
        w = w.split_interleaved(il)
    seg = int(plan.get("segments", 1) or 1)
    fork = int(plan.get("fork", -1))
    if seg > 1 and fork >= 0:
        w = w.split_forked(seg, fork)
    elif seg > 1:
        w = w.split_segments(seg)
    return w


def schedules(wl) -> list:
    """Per-instance lambda schedules of a workload (they may differ in length)."""
    return [np.asarray(i.lambdas, np.int32) for i in wl.instances]


def plan_name(plan: dict, m: int) -> str:
    """Short name of a batching plan for a schedule of m lambdas: m2 (one
    warm chain per seed), m1 (every (seed, lambda) cold), segN, ilvN."""
    seg, il = int(plan.get("segments", 1) or 1), int(plan.get("interleave", 1) or 1)
    fork = int(plan.get("fork", -1))
    if il > 1:
        return f"ilv{il}" + (f"-seg{seg}" if seg > 1 else "")
    if seg > 1 and fork >= 0:
        return f"fork{seg}x{fork}"
    return "m2" if seg == 1 else ("m1" if seg == m else f"seg{seg}")


def bench_plan(wl, device: int = 0) -> dict:
    """The plan and knobs the benchmark runs a workload with: the autotuner's
    cached choice for this GPU and workload class, else the defaults with one
    warm chain per seed."""
    c = cached(wl, device)
    out = {"segments": 1, "interleave": 1, "fork": -1, **DEFAULTS}
    if c is not None:
        for k in out:
            if k in c:
                out[k] = c[k]
    return out


def knobs_of(plan: dict) -> dict:
    """The solver knobs of a plan (pmf_set_tuning fields)."""
    return {k: plan[k] for k in DEFAULTS if k in plan}


def divisors(m: int) -> list[int]:
    return [d for d in range(1, m + 1) if m % d == 0]


def _bucket(v: float) -> int:
    """Power-of-two bucket (as an exponent) of a positive size."""
    return int(round(math.log2(max(1.0, float(v)))))


def workload_class(wl) -> str:
    """Key of the workload's class: mean image size, instance count and
    schedule length, each bucketed to a power of two (the lambda count exactly)."""
    px = np.mean([wl.images[i.image].H * wl.images[i.image].W for i in wl.instances])
    lens = sorted({len(i.lambdas) for i in wl.instances})
    return f"px2^{_bucket(px)}-inst2^{_bucket(len(wl.instances))}-lam{'/'.join(map(str, lens))}"


def gpu_name(device: int = 0) -> str:
    import torch
    return torch.cuda.get_device_name(device)


def load_cache(path: str = CACHE_PATH) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save_cache(cache: dict, path: str = CACHE_PATH) -> None:
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def cached(wl, device: int = 0, path: str = CACHE_PATH) -> dict | None:
    return load_cache(path).get(f"{gpu_name(device)}|{workload_class(wl)}")


def gpu_measure(wl, segments, knobs: dict, reps: int = 3, device: int = 0) -> float:
    """Median device time (ms) of ``reps`` solves (after one warm-up) of the
    workload cut into ``segments`` pieces per seed (an int), or batched by a
    plan ({"segments", "interleave"})."""
    import torch
    from . import pmf
    plan = segments if isinstance(segments, dict) else {"segments": segments}
    w = apply_plan(wl, plan)
    stream = torch.cuda.Stream(device=device)
    b = pmf.batch_from_workload(w, device=device, stream=stream, **knobs)
    lam = schedules(w)
    ts = []
    try:
        for r in range(reps + 1):
            b.solve(lam, stream=stream)
            st = b.sync(check=False)
            if any(s != pmf.PMF_OK for s in st):
                return float("inf")
            if r:
                ts.append(b.timing()[0])
    finally:
        b.close()
    return float(np.median(ts))


INTERLEAVE = [2, 3, 4, 5, 6, 8, 10]


def plans_for(m: int) -> list[dict]:
    """Batching plans tried for a schedule of m lambdas: consecutive pieces
    (every divisor of m) and round-robin pieces (a few strides)."""
    out = [{"segments": d, "interleave": 1, "fork": -1} for d in divisors(m)]
    out += [{"segments": 1, "interleave": p, "fork": -1} for p in INTERLEAVE if p < m]
    # forked pieces: each piece after the first starts from its predecessor's
    # state, taken right after the predecessor's first step or halfway
    for d in divisors(m):
        if 1 < d < m:
            L = m // d
            for lead in sorted({L - 1, L // 2}):
                if lead >= 1:
                    out.append({"segments": d, "interleave": 1, "fork": lead})
    return out


def tune(wl, measure=None, budget_s: float = 90.0, reps: int = 3, log=None) -> dict:
    """Coordinate descent over the batching plan (``segments`` /
    ``interleave``) then each knob of SPACE, starting from one warm chain per
    seed and DEFAULTS; stops when a full pass brings no gain or the time
    budget is spent.  ``measure(wl, plan, knobs) -> ms`` defaults to
    gpu_measure.  Returns {"segments", "interleave", knobs..., "ms"}."""
    measure = measure or (lambda w, p, k: gpu_measure(w, p, k, reps=reps))
    m = min(len(i.lambdas) for i in wl.instances)
    plans = plans_for(m)
    t_end = time.monotonic() + budget_s
    seen: dict = {}

    def cost(p, k):
        key = (tuple(sorted(p.items())), tuple(sorted(k.items())))
        if key not in seen:
            seen[key] = measure(wl, dict(p), dict(k))
            if log:
                log(f"plan={plan_name(p, m)} {k} -> {seen[key]:.2f} ms")
        return seen[key]

    best_p, best_k = plans[0], dict(DEFAULTS)
    best = cost(best_p, best_k)
    improved = True
    while improved and time.monotonic() < t_end:
        improved = False
        for p in plans:
            if time.monotonic() >= t_end:
                break
            c = cost(p, best_k)
            if c < best:
                best, best_p, improved = c, p, True
        for name, vals in SPACE.items():
            for v in vals:
                if time.monotonic() >= t_end:
                    break
                k = dict(best_k)
                k[name] = v
                c = cost(best_p, k)
                if c < best:
                    best, best_k, improved = c, k, True
    out = {**best_p, **best_k, "ms": best}
    return out


def tune_and_cache(wl, device: int = 0, budget_s: float = 90.0, path: str = CACHE_PATH, log=None) -> dict:
    res = tune(wl, measure=lambda w, p, k: gpu_measure(w, p, k, reps=3, device=device), budget_s=budget_s, log=log)
    cache = load_cache(path)
    res["class"] = workload_class(wl)
    cache[f"{gpu_name(device)}|{workload_class(wl)}"] = res
    save_cache(cache, path)
    return res


if __name__ == "__main__":
    import argparse
    import sys
    sys.path.insert(0, os.path.dirname(HERE))
    from paper_1509_06004_b300 import inputs
    ap = argparse.ArgumentParser(description="tune and cache the solver settings for a workload")
    ap.add_argument("--workload", default="supergraph-480x320",
                    choices=["supergraph-480x320", "parametric-320x240", "uneven-64", "single-64x64"])
    ap.add_argument("--budget", type=float, default=90.0)
    a = ap.parse_args()
    wl = {"supergraph-480x320": inputs.supergraph_480x320, "parametric-320x240": inputs.parametric_320x240,
          "uneven-64": inputs.uneven_batch, "single-64x64": inputs.single_maxflow_64}[a.workload]()
    print(json.dumps(tune_and_cache(wl, budget_s=a.budget, log=lambda s: print(s, flush=True))))
