"""The C-ABI library loads and exports every entry point its header declares;
host-only calls behave (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1509_06004_b300 import build as pbuild
from paper_1509_06004_b300 import pmf

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    pbuild.build()


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "pmf.h")).read()
    return sorted(set(re.findall(r"PMF_API[^;]*?\b(pmf_[a-z_]+)\s*\(", txt, re.S)))


def test_header_declares_what_binding_lists():
    assert declared_symbols() == sorted(pmf.EXPORTS)


def test_library_exports_every_declared_symbol():
    L = ctypes.CDLL(pmf.LIB_PATH)
    for name in declared_symbols():
        assert hasattr(L, name), name


def test_no_internal_symbols_exported():
    out = os.popen(f"nm -D --defined-only {pmf.LIB_PATH}").read()
    names = {l.split()[-1] for l in out.splitlines() if " T " in l}
    assert names == set(declared_symbols())


def test_version_and_status_strings():
    assert b"sm_103a" in pmf.lib().pmf_version()
    for s in range(8):
        assert pmf.status_string(s) not in ("", "unknown status")


def test_workspace_size_host_only():
    n1 = pmf.workspace_size([(64, 64)], [0], 1)
    n2 = pmf.workspace_size([(64, 64)], [0, 0], 1)
    n3 = pmf.workspace_size([(64, 64)], [0], 20)
    # 8 int32 planes of 64x64 per instance, masks per lambda
    assert n2 - n1 >= 8 * 64 * 64 * 4
    assert n3 - n1 >= 19 * 64 * 64
    big = pmf.workspace_size([(320, 480)], [0] * 500, 1)
    assert big >= 500 * 320 * 480 * (8 * 4 + 1)


@pytest.mark.parametrize("bad", ["no-images", "bad-image-index", "zero-lambdas", "neg-shape"])
def test_workspace_size_rejects_bad_desc(bad):
    shapes, ii, ml = [(10, 10)], [0], 2
    if bad == "no-images":
        shapes = []
    elif bad == "bad-image-index":
        ii = [1]
    elif bad == "zero-lambdas":
        ml = 0
    elif bad == "neg-shape":
        shapes = [(0, 5)]
    with pytest.raises(pmf.PmfError) as ei:
        pmf.workspace_size(shapes, ii, ml)
    assert ei.value.status == pmf.PMF_ERR_INVALID_ARG


def test_null_arguments_are_rejected_without_gpu():
    L = pmf.lib()
    assert L.pmf_workspace_size(None, None) == pmf.PMF_ERR_INVALID_ARG
    assert L.pmf_sync(None, None) == pmf.PMF_ERR_INVALID_ARG
    assert L.pmf_get_flow(None, 0, 0, None) == pmf.PMF_ERR_INVALID_ARG
    assert L.pmf_get_flow_arcs(None, 0, None, None, None, None) == pmf.PMF_ERR_INVALID_ARG
    assert L.pmf_copy_terminals(None, 0, 0) == pmf.PMF_ERR_INVALID_ARG
    assert L.pmf_set_cut_rule(None, 0, 1) == pmf.PMF_ERR_INVALID_ARG
    assert L.pmf_set_slope_side(None, 0, 1) == pmf.PMF_ERR_INVALID_ARG
    assert L.pmf_solve_schedules(None, None, None, 1, None) == pmf.PMF_ERR_INVALID_ARG
    L.pmf_destroy_batch(None)
