"""pmf_solve_noalloc: the single-instance solve for callers that cannot
allocate device memory (it keeps its scratch in a fixed device array reserved
when the library loads).  Its results must equal the CPU oracle's and those of
the batch entry points (pmf_create_batch + pmf_solve_schedule) exactly, call
after call, since the shared array keeps the previous call's contents.

This file is named to be collected last, so that a run stopping at the first
failure has already run every other test."""
import ctypes

import numpy as np
import pytest

import oracle
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


def _noalloc(P, wl, w_h=None):
    import torch
    im, inst = wl.images[0], wl.instances[0]
    if w_h is not None:
        im = inputs.Image(im.H, im.W, w_h, im.w_v)
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


def test_noalloc_equals_oracle_and_batch_entry_points_two_calls(pmf):
    # two different instances in a row: the second call must not see the first's state
    for seed, H, W, n in ((11, 120, 160, 12), (12, 97, 133, 20)):
        wl = _small_parametric(seed, H, W, n)
        st, flows, masks = _noalloc(pmf, wl)
        assert st == pmf.PMF_OK, pmf.status_string(st)
        (of, om), = oracle.solve_workload(wl)
        assert np.array_equal(flows, of)
        assert np.array_equal(masks, om)
        ref_st, ref = pmf.solve_workload(wl)
        assert ref_st == [pmf.PMF_OK]
        assert np.array_equal(flows, ref[0][0])
        assert np.array_equal(masks, ref[0][1])


def test_noalloc_allocates_nothing(pmf):
    """After a first call (which looks up the array's address), further calls
    leave the device's free memory unchanged."""
    import torch
    wl = _small_parametric(13, 64, 96, 6)
    assert _noalloc(pmf, wl)[0] == pmf.PMF_OK
    # the test's own tensors are allocated before the measured call
    im, inst = wl.images[0], wl.instances[0]
    dev = [torch.from_numpy(np.ascontiguousarray(a, np.int32)).cuda()
           for a in (im.w_h, im.w_v, inst.src0, inst.slope, inst.sink)]
    masks = torch.zeros((6, im.H, im.W), dtype=torch.uint8, device="cuda")
    flows = np.zeros(6, np.int64)
    lam = np.ascontiguousarray(inst.lambdas, np.int32)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    st = pmf.lib().pmf_solve_noalloc(im.H, im.W, *[ctypes.c_void_p(a.data_ptr()) for a in dev],
                                     lam.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), 6,
                                     ctypes.c_void_p(masks.data_ptr()),
                                     flows.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), None)
    torch.cuda.synchronize()
    assert st == pmf.PMF_OK
    assert torch.cuda.mem_get_info()[0] == free0


def test_noalloc_reports_invalid_capacities(pmf):
    """A negative pairwise capacity gives PMF_ERR_INVALID_ARG (found on the
    device by the padding kernel); the next call is correct again."""
    wl = _small_parametric(14, 50, 70, 4)
    bad = wl.images[0].w_h.copy()
    bad[10, 10] = -5
    st, _, _ = _noalloc(pmf, wl, w_h=bad)
    assert st == pmf.PMF_ERR_INVALID_ARG
    st, flows, masks = _noalloc(pmf, wl)
    assert st == pmf.PMF_OK
    (of, om), = oracle.solve_workload(wl)
    assert np.array_equal(flows, of) and np.array_equal(masks, om)


@pytest.mark.parametrize("fail_at", [1, 3, 6, 10, 11, 14, 16, 18])
def test_noalloc_cuda_failure_is_reported_and_recovered(pmf, fail_at):
    """A CUDA call made to fail on the host (the test hook skips it and
    reports an error; nothing faults on the GPU) returns PMF_ERR_CUDA with the
    site in pmf_last_error, after the call has waited for the work it had
    queued; the next call on the same stream then gives the oracle's results."""
    wl = _small_parametric(15, 60, 90, 5)
    pmf.lib().pmf_testing_fail_noalloc_call(fail_at)
    st, _, _ = _noalloc(pmf, wl)
    assert st == pmf.PMF_ERR_CUDA
    assert b"injected failure" in pmf.lib().pmf_last_error()
    st, flows, masks = _noalloc(pmf, wl)
    assert st == pmf.PMF_OK
    (of, om), = oracle.solve_workload(wl)
    assert np.array_equal(flows, of) and np.array_equal(masks, om)


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
