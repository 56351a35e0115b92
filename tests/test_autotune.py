"""Autotuner logic on the CPU with a synthetic cost model (no GPU)."""
import os

import numpy as np

from paper_1509_06004_b300 import autotune, inputs


def test_divisors_and_class():
    assert autotune.divisors(20) == [1, 2, 4, 5, 10, 20]
    wl = inputs.supergraph_480x320(n_lambda=20)
    k = autotune.workload_class(wl)
    assert k == "px2^17-inst2^5-lam20"
    assert autotune.workload_class(wl.split_lambdas()) == "px2^17-inst2^9-lam1"


def test_coordinate_descent_finds_separable_minimum():
    wl = inputs.single_maxflow_64()
    wl.instances[0].lambdas = np.arange(1, 13, dtype=np.int32)   # 12 lambdas: segments 1..12
    target = {"segments": 4, "tile_h": 8, "push_order": 1, "sweeps": 16, "relabel_every": 400, "label_slack": 32,
              "relabel_extra": 256, "relabel_reach": 800, "poll_ns": 1024, "blocks_per_sm": 3}

    def cost(w, p, k):
        assert p["interleave"] == 1 or p["segments"] == 1
        c = abs(np.log2(p["segments"]) - np.log2(target["segments"])) + (p["interleave"] - 1)
        for name in autotune.SPACE:
            c += abs(autotune.SPACE[name].index(k[name]) - autotune.SPACE[name].index(target[name]))
        return 10.0 + c

    res = autotune.tune(wl, measure=cost, budget_s=30)
    assert {k: res[k] for k in target} == target
    assert res["interleave"] == 1
    assert res["ms"] == 10.0


def test_descent_picks_round_robin_pieces():
    """A cost that favours dealing each schedule into three round-robin pieces
    is found, and the plan batches the workload that way."""
    wl = inputs.single_maxflow_64()
    wl.instances[0].lambdas = np.arange(1, 13, dtype=np.int32)

    def cost(w, p, k):
        return 5.0 + abs(p["interleave"] - 3) + 0.5 * (p["segments"] - 1)

    res = autotune.tune(wl, measure=cost, budget_s=30)
    assert res["interleave"] == 3 and res["segments"] == 1
    w = autotune.apply_plan(wl, res)
    assert [list(i.lambdas) for i in w.instances] == [[1, 4, 7, 10], [2, 5, 8, 11], [3, 6, 9, 12]]
    assert autotune.plan_name(res, 12) == "ilv3"


def test_gather_restores_every_plan():
    """Pieces of every plan put back per seed give the original schedules."""
    wl = inputs.supergraph_480x320()
    m = len(wl.instances[0].lambdas)
    for p in autotune.plans_for(m):
        w = autotune.apply_plan(wl, p)
        fake = [(np.asarray(i.lambdas, np.int64) * 3 + i.origin[0] if i.origin else np.asarray(i.lambdas, np.int64) * 3,
                 np.asarray(i.lambdas, np.uint8).reshape(-1, 1, 1)) for i in w.instances]
        g = w.gather(fake, len(wl.instances))
        for s, (f, mk) in enumerate(g):
            assert np.array_equal(f, wl.instances[s].lambdas.astype(np.int64) * 3 + (s if (p["segments"] > 1 or p["interleave"] > 1) else 0))
            assert np.array_equal(mk.ravel(), wl.instances[s].lambdas.astype(np.uint8))


def test_cache_round_trip(tmp_path):
    p = os.path.join(tmp_path, "t.json")
    c = autotune.load_cache(p)
    assert c == {}
    c["gpu|cls"] = {"segments": 5, **autotune.DEFAULTS, "ms": 1.0}
    autotune.save_cache(c, p)
    assert autotune.load_cache(p)["gpu|cls"]["segments"] == 5
