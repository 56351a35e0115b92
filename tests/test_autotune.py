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
              "relabel_extra": 256, "poll_ns": 1024}

    def cost(w, s, k):
        c = abs(np.log2(s) - np.log2(target["segments"]))
        for name in autotune.SPACE:
            c += abs(autotune.SPACE[name].index(k[name]) - autotune.SPACE[name].index(target[name]))
        return 10.0 + c

    res = autotune.tune(wl, measure=cost, budget_s=30)
    assert {k: res[k] for k in target} == target
    assert res["ms"] == 10.0


def test_cache_round_trip(tmp_path):
    p = os.path.join(tmp_path, "t.json")
    c = autotune.load_cache(p)
    assert c == {}
    c["gpu|cls"] = {"segments": 5, **autotune.DEFAULTS, "ms": 1.0}
    autotune.save_cache(c, p)
    assert autotune.load_cache(p)["gpu|cls"]["segments"] == 5
