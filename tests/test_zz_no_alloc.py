"""pmf_solve_noalloc: the single-instance solve for callers that cannot
allocate device memory (it keeps its scratch in a fixed device array reserved
when the library loads).  Its results must equal those of the batch entry
points (pmf_create_batch + pmf_solve_schedule) exactly, call after call, since
the shared array keeps the previous call's contents.

This file is named to be collected last, so that a run stopping at the first
failure has already run every other test."""
import ctypes

import numpy as np
import pytest

from paper_1509_06004_b300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pmf():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1509_06004_b300 import build, pmf as P
    build.build()
    return P


def _small_parametric(seed, H, W, n_lambda):
    rng = np.random.default_rng(seed)
    img = inputs.make_image(H, W, 4, 0.05, rng)
    w_h, w_v = inputs.pairwise_caps(img)
    y0, x0 = inputs.random_seed_origin(H, W, rng)
    src0, slope, sink = inputs.terminals(img, inputs.seed_square(H, W, y0, x0))
    wl = inputs.Workload(f"noalloc-{seed}")
    wl.images.append(inputs.Image(H, W, w_h, w_v, img))
    wl.instances.append(inputs.Instance(0, src0, slope, sink, inputs.lambda_schedule(n_lambda, 10, 5000)))
    return wl


def _noalloc(P, wl):
    import torch
    im, inst = wl.images[0], wl.instances[0]
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.int32)).cuda()
    args = [dev(a) for a in (im.w_h, im.w_v, inst.src0, inst.slope, inst.sink)]
    lam = np.ascontiguousarray(inst.lambdas, np.int32)
    n = len(lam)
    masks = torch.zeros((n, im.H, im.W), dtype=torch.uint8, device="cuda")
    flows = np.zeros(n, np.int64)
    stream = torch.cuda.current_stream().cuda_stream
    st = P.lib().pmf_solve_noalloc(im.H, im.W, *[ctypes.c_void_p(a.data_ptr()) for a in args],
                                   lam.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), n,
                                   ctypes.c_void_p(masks.data_ptr()),
                                   flows.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                   ctypes.c_void_p(stream))
    return st, flows, masks.cpu().numpy()


def test_noalloc_equals_batch_entry_points_two_calls(pmf):
    # two different instances in a row: the second call must not see the first's state
    for seed, H, W, n in ((11, 120, 160, 12), (12, 97, 133, 20)):
        wl = _small_parametric(seed, H, W, n)
        st, flows, masks = _noalloc(pmf, wl)
        assert st == pmf.PMF_OK, pmf.status_string(st)
        ref_st, ref = pmf.solve_workload(wl)
        assert ref_st == [pmf.PMF_OK]
        assert np.array_equal(flows, ref[0][0])
        assert np.array_equal(masks, ref[0][1])


def test_noalloc_rejects_sizes_beyond_its_limit(pmf):
    z = ctypes.c_void_p(8)          # never dereferenced: the size check comes first
    lam = np.array([10], np.int32)
    flows = np.zeros(1, np.int64)
    st = pmf.lib().pmf_solve_noalloc(1024, 1024, z, z, z, z, z,
                                     lam.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), 1, z,
                                     flows.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), None)
    assert st == pmf.PMF_ERR_OUT_OF_MEMORY
    lam40 = np.arange(40, dtype=np.int32)
    flows40 = np.zeros(40, np.int64)
    st = pmf.lib().pmf_solve_noalloc(16, 16, z, z, z, z, z,
                                     lam40.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), 40, z,
                                     flows40.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), None)
    assert st == pmf.PMF_ERR_OUT_OF_MEMORY
