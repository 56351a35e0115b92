"""GPU tests beyond plain parity: batch invariance (Section 3.1's decomposition
argument: each instance's minimum cut is the same alone or inside a larger
batch), independence from the launch configuration, the batching modes, the
input paths, sampled parity on large images, edge cases and every error status of the C ABI."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1509_06004_b300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1509_06004_b300 import build, pmf
    build.build()
    return pmf


def _solve(P, wl, **tuning):
    st, res = P.solve_workload(wl, **tuning)
    assert all(s == P.PMF_OK for s in st), [P.status_string(s) for s in st]
    return res


def _same(a, b):
    for (fa, ma), (fb, mb) in zip(a, b):
        assert np.array_equal(fa, fb)
        assert np.array_equal(ma, mb)


def _synthetic(seed, H, W, n_seeds, n_lambda, lo=10, hi=5000):
    rng = np.random.default_rng(seed)
    img = inputs.make_image(H, W, 4, 0.05, rng)
    w_h, w_v = inputs.pairwise_caps(img)
    wl = inputs.Workload(f"syn{seed}")
    wl.images.append(inputs.Image(H, W, w_h, w_v, img))
    lam = inputs.lambda_schedule(n_lambda, lo, hi)
    for _ in range(n_seeds):
        y0, x0 = inputs.random_seed_origin(H, W, rng)
        s0, sl, sk = inputs.terminals(img, inputs.seed_square(H, W, y0, x0))
        wl.instances.append(inputs.Instance(0, s0, sl, sk, lam, (y0, x0)))
    return wl


# ---------------------------------------------------------------------------
# invariance
# ---------------------------------------------------------------------------

def test_alone_equals_in_mixed_batch(P):
    a = _synthetic(1, 61, 83, 2, 6)
    b = _synthetic(2, 40, 150, 3, 6)
    mixed = inputs.Workload("mixed", a.images + b.images, [])
    for inst in a.instances:
        mixed.instances.append(inst)
    for inst in b.instances:
        mixed.instances.append(inputs.Instance(1, inst.src0, inst.slope, inst.sink, inst.lambdas))
    # reverse order too
    rev = inputs.Workload("rev", mixed.images, mixed.instances[::-1])
    ra, rb, rm, rr = _solve(P, a), _solve(P, b), _solve(P, mixed), _solve(P, rev)
    _same(ra + rb, rm)
    _same(rm, rr[::-1])


@pytest.mark.parametrize("knobs", [dict(tile_h=4), dict(sweeps=1), dict(sweeps=32), dict(relabel_every=50),
                                   dict(relabel_every=5000), dict(label_slack=-1), dict(label_slack=1),
                                   dict(blocks_per_sm=1), dict(poll_ns=8192), dict(grid_blocks=1),
                                   dict(grid_blocks=3), dict(grid_blocks=37), dict(grid_blocks=197, tile_h=4),
                                   dict(push_order=1), dict(push_order=1, tile_h=4, sweeps=2)])
def test_launch_configuration_does_not_change_results(P, knobs):
    wl = _synthetic(3, 70, 96, 3, 8)
    _same(_solve(P, wl), _solve(P, wl, **knobs))


def test_batching_modes_agree(P):
    wl = _synthetic(4, 64, 90, 2, 8)
    base = _solve(P, wl)
    for segs in (2, 4, 8):
        split = _solve(P, wl.split_segments(segs))
        # reassemble: instance i of the split workload holds piece i % segs of seed i // segs
        for s in range(len(wl.instances)):
            f = np.concatenate([split[s * segs + j][0] for j in range(segs)])
            m = np.concatenate([split[s * segs + j][1] for j in range(segs)])
            assert np.array_equal(f, base[s][0]) and np.array_equal(m, base[s][1])


@pytest.mark.parametrize("stride", [2, 3, 5, 8])
def test_round_robin_pieces_agree(P, stride):
    """Schedules dealt round-robin into pieces (piece j: lambda_j,
    lambda_{j+stride}, ...; pieces of unequal length in one launch) give the
    unsplit results once put back in schedule order."""
    wl = _synthetic(24, 66, 101, 3, 8)
    base = _solve(P, wl)
    run = wl.split_interleaved(stride)
    got = run.gather(_solve(P, run), len(wl.instances))
    _same(base, got)


@pytest.mark.parametrize("pieces", [[1, 7], [3, 5], [2, 1, 5], [5, 2, 1], [1, 1, 1, 1, 4]])
def test_uneven_pieces_agree(P, pieces):
    """Schedules cut into pieces of different lengths (one launch with
    per-instance schedule lengths) give the unsplit results."""
    wl = _synthetic(14, 58, 95, 2, 8)
    base = _solve(P, wl)
    split = _solve(P, wl.split_pieces(pieces))
    n = len(pieces)
    for s in range(len(wl.instances)):
        assert [len(split[s * n + j][0]) for j in range(n)] == pieces
        f = np.concatenate([split[s * n + j][0] for j in range(n)])
        m = np.concatenate([split[s * n + j][1] for j in range(n)])
        assert np.array_equal(f, base[s][0]) and np.array_equal(m, base[s][1])


def test_copied_terminals_equal_uploaded_ones(P):
    """Pieces of one seed share its terminal arrays, so the binding uploads
    them once and copies them on the device (pmf_copy_terminals); the results
    equal those of separate uploads."""
    wl = _synthetic(16, 44, 70, 2, 6).split_segments(3)
    shared = _solve(P, wl)
    sep = inputs.Workload("sep", wl.images, [inputs.Instance(i.image, i.src0.copy(), i.slope.copy(), i.sink.copy(),
                                                             i.lambdas) for i in wl.instances])
    _same(shared, _solve(P, sep))
    b = P.batch_from_workload(_synthetic(17, 20, 30, 2, 2))
    L = P.lib()
    assert L.pmf_copy_terminals(b._h, 0, 2) == P.PMF_ERR_INVALID_ARG
    assert L.pmf_copy_terminals(b._h, -1, 0) == P.PMF_ERR_INVALID_ARG
    assert L.pmf_copy_terminals(b._h, 1, 1) == P.PMF_OK
    b.close()
    two = inputs.Workload("two", _synthetic(18, 20, 30, 1, 2).images + _synthetic(19, 24, 30, 1, 2).images, [])
    two.instances = [inputs.Instance(0, *([np.zeros((20, 30), np.int32)] * 3), np.array([1, 2], np.int32)),
                     inputs.Instance(1, *([np.zeros((24, 30), np.int32)] * 3), np.array([1, 2], np.int32))]
    b = P.batch_from_workload(two)
    assert L.pmf_copy_terminals(b._h, 1, 0) == P.PMF_ERR_INVALID_ARG   # different images
    b.close()


def test_poll_reads_finished_instances_during_the_solve(P):
    """Instances read as soon as pmf_poll reports them finished (while larger
    ones still run) equal the results after pmf_sync and the oracle's."""
    import torch
    small = _synthetic(20, 24, 40, 3, 4)
    big = _synthetic(21, 200, 300, 2, 12)
    wl = inputs.Workload("mix", small.images + big.images, list(small.instances))
    for inst in big.instances:
        wl.instances.append(inputs.Instance(1, inst.src0, inst.slope, inst.sink, inst.lambdas))
    b = P.batch_from_workload(wl)
    early = {}
    b.solve([i.lambdas for i in wl.instances])
    ev = torch.cuda.Event()
    ev.record(torch.cuda.current_stream())
    while len(early) < len(wl.instances):
        fresh = [i for i in np.nonzero(b.poll())[0] if i not in early]
        for i in fresh:
            early[i] = (b.flows(i), b.cuts(i))
        if not fresh and ev.query():
            break
    assert b.sync() == [P.PMF_OK] * len(wl.instances)
    assert b.poll().all()
    ref = oracle.solve_workload(wl, instances=list(early))
    for (i, (f, m)), (of, om) in zip(early.items(), ref):
        assert np.array_equal(f, b.flows(i)) and np.array_equal(m, b.cuts(i))
        assert np.array_equal(f, of) and np.array_equal(m, om)
    b.close()


def test_ragged_schedules_status_codes_and_reuse(P):
    """pmf_solve_schedules: argument checks, entries past an instance's length
    ignored, and a batch alternating between ragged and uniform schedules."""
    wl = _synthetic(15, 36, 50, 3, 6)
    b = P.batch_from_workload(wl)
    lam = np.stack([i.lambdas for i in wl.instances]).astype(np.int32)
    lengths = np.array([6, 2, 4], np.int32)
    i32p = ctypes.POINTER(ctypes.c_int32)
    L = P.lib()
    padded = lam.copy()
    padded[1, 2:] = 1                     # past instance 1's length: ignored even though decreasing
    assert L.pmf_solve_schedules(b._h, padded.ctypes.data_as(i32p), lengths.ctypes.data_as(i32p), 6, None) == 0
    b.lengths = [int(x) for x in lengths]
    assert b.sync(check=False) == [P.PMF_OK] * 3
    for i in range(3):
        of, om = oracle.grid_solve(36, 50, wl.images[0].w_h, wl.images[0].w_v, wl.instances[i].src0,
                                   wl.instances[i].slope, wl.instances[i].sink, lam[i, :lengths[i]])
        assert np.array_equal(b.flows(i), of) and np.array_equal(b.cuts(i), om)
    with pytest.raises(P.PmfError) as e:  # beyond the instance's own schedule
        b.get_flow(1, 2)
    assert e.value.status == P.PMF_ERR_INVALID_ARG
    bad = lengths.copy()
    bad[0] = 7                            # longer than the stride
    assert L.pmf_solve_schedules(b._h, lam.ctypes.data_as(i32p), bad.ctypes.data_as(i32p), 6, None) \
        == P.PMF_ERR_INVALID_ARG
    bad[0] = 0
    assert L.pmf_solve_schedules(b._h, lam.ctypes.data_as(i32p), bad.ctypes.data_as(i32p), 6, None) \
        == P.PMF_ERR_INVALID_ARG
    assert L.pmf_solve_schedules(b._h, lam.ctypes.data_as(i32p), None, 6, None) == P.PMF_ERR_INVALID_ARG
    dec = lam.copy()
    dec[2, 1], dec[2, 2] = dec[2, 2], dec[2, 1]
    assert L.pmf_solve_schedules(b._h, dec.ctypes.data_as(i32p), lengths.ctypes.data_as(i32p), 6, None) \
        == P.PMF_ERR_NOT_MONOTONE
    # back to one length for all, then ragged again through the binding
    b.solve(lam)
    b.sync()
    assert all(len(b.flows(i)) == 6 for i in range(3))
    b.solve([lam[0, :1], lam[1], lam[2, :3]])
    b.sync()
    assert [len(b.flows(i)) for i in range(3)] == [1, 6, 3]
    assert b.cuts(2).shape == (3, 36, 50)
    b.close()


def test_repeated_solves_and_device_inputs(P):
    wl = _synthetic(5, 50, 77, 2, 5)
    b = P.batch_from_workload(wl)
    lam = np.stack([i.lambdas for i in wl.instances])
    outs = []
    for _ in range(3):
        b.solve(lam)
        b.sync()
        outs.append([(b.flows(i), b.cuts(i)) for i in range(len(wl.instances))])
    b.close()
    _same(outs[0], outs[1])
    _same(outs[0], outs[2])
    bd = P.batch_from_workload(wl, device_inputs=True)
    bd.solve(lam)
    bd.sync()
    _same(outs[0], [(bd.flows(i), bd.cuts(i)) for i in range(len(wl.instances))])
    # masks read into device memory
    import torch
    H, W = wl.images[0].H, wl.images[0].W
    dm = torch.empty((len(lam[0]), H, W), dtype=torch.uint8, device="cuda")
    bd.cuts(0, dm)
    assert np.array_equal(dm.cpu().numpy(), outs[0][0][1])
    bd.close()


# ---------------------------------------------------------------------------
# large images (sampled; the benchmarked workloads are compared in full in
# test_parity_bench_configs.py)
# ---------------------------------------------------------------------------

def test_large_image_sampled(P):
    """A 770 x 1010 image (no side a multiple of the tile or strip sizes):
    sampled flows and masks equal the oracle's; cuts nested, flows
    nondecreasing along each schedule."""
    wl = _synthetic(77, 770, 1010, 2, 3, lo=20, hi=400)
    res = _solve(P, wl, push_order=1)
    rng = np.random.default_rng(2)
    for i, k in ((0, int(rng.integers(0, 3))), (1, int(rng.integers(0, 3)))):
        inst = wl.instances[i]
        im = wl.images[inst.image]
        of, om = oracle.grid_solve(im.H, im.W, im.w_h, im.w_v, inst.src0, inst.slope, inst.sink,
                                   [inst.lambdas[k]])
        assert res[i][0][k] == of[0]
        assert np.array_equal(res[i][1][k], om[0])
    for f, m in res:
        assert np.all(np.diff(f) >= 0)
        assert np.all(m[:-1] <= m[1:])


def test_uneven_batch_sampled(P):
    wl = inputs.uneven_batch(n_images=6, seeds_per_image=2, n_lambda=6)
    res = _solve(P, wl)
    rng = np.random.default_rng(1)
    for i in rng.choice(len(wl.instances), size=4, replace=False):
        inst = wl.instances[i]
        im = wl.images[inst.image]
        k = int(rng.integers(0, len(inst.lambdas)))
        of, om = oracle.grid_solve(im.H, im.W, im.w_h, im.w_v, inst.src0, inst.slope, inst.sink,
                                   [inst.lambdas[k]])
        assert res[i][0][k] == of[0]
        assert np.array_equal(res[i][1][k], om[0])


# ---------------------------------------------------------------------------
# edge cases
# ---------------------------------------------------------------------------

def _single(H, W, w_h, w_v, src0, slope, sink, lams):
    wl = inputs.Workload("edge")
    wl.images.append(inputs.Image(H, W, np.asarray(w_h, np.int32).reshape(H, W),
                                  np.asarray(w_v, np.int32).reshape(H, W)))
    wl.instances.append(inputs.Instance(0, np.asarray(src0, np.int32).reshape(H, W),
                                        np.asarray(slope, np.int32).reshape(H, W),
                                        np.asarray(sink, np.int32).reshape(H, W),
                                        np.asarray(lams, np.int32)))
    return wl


@pytest.mark.parametrize("case", ["zeros", "all-source", "all-sink", "equal-lambdas", "max-caps",
                                  "one-pixel", "one-row", "one-column", "checker-ties"])
def test_edge_cases(P, case):
    rng = np.random.default_rng(7)
    H, W = 23, 41
    z = np.zeros((H, W), np.int32)
    w = rng.integers(0, 50, (H, W)).astype(np.int32)
    lams = [0, 3, 9]
    if case == "zeros":
        wl = _single(H, W, z, z, z, z, z, lams)
    elif case == "all-source":
        wl = _single(H, W, w, w, np.full((H, W), 100, np.int32), z + 1, z, lams)
    elif case == "all-sink":
        wl = _single(H, W, w, w, z, z, np.full((H, W), 100, np.int32), lams)
    elif case == "equal-lambdas":
        wl = _single(H, W, w, w, rng.integers(0, 30, (H, W)), z + 2, rng.integers(0, 60, (H, W)), [5, 5, 5, 7, 7])
    elif case == "max-caps":
        big = np.full((H, W), inputs.INF, np.int32)
        wl = _single(H, W, np.full((H, W), (1 << 28) - 1, np.int32), w, big - 10, z + 1, big, [0, 5, 10])
    elif case == "one-pixel":
        wl = _single(1, 1, [0], [0], [7], [1], [9], [0, 1, 2, 3])
    elif case == "one-row":
        wl = _single(1, 97, rng.integers(0, 9, 97), np.zeros(97), rng.integers(0, 9, 97), np.ones(97),
                     rng.integers(0, 20, 97), lams)
    elif case == "one-column":
        wl = _single(97, 1, np.zeros(97), rng.integers(0, 9, 97), rng.integers(0, 9, 97), np.ones(97),
                     rng.integers(0, 20, 97), lams)
    else:  # ties everywhere
        cs = np.full((H, W), 5, np.int32)
        wl = _single(H, W, z + 3, z + 3, cs, z, cs, [0])
    res = _solve(P, wl)
    inst, im = wl.instances[0], wl.images[0]
    of, om = oracle.grid_solve(im.H, im.W, im.w_h, im.w_v, inst.src0, inst.slope, inst.sink, inst.lambdas)
    assert np.array_equal(res[0][0], of)
    assert np.array_equal(res[0][1], om)


# ---------------------------------------------------------------------------
# error statuses (host-made failures only; nothing faults or hangs the GPU)
# ---------------------------------------------------------------------------

def test_status_codes(P):
    import torch
    wl = _synthetic(9, 32, 40, 2, 3)
    b = P.batch_from_workload(wl)
    lam = np.stack([i.lambdas for i in wl.instances])
    with pytest.raises(P.PmfError) as e:          # results before any solve
        b.get_flow(0, 0)
    assert e.value.status == P.PMF_ERR_NOT_READY
    with pytest.raises(P.PmfError) as e:          # decreasing schedule
        b.solve(lam[:, ::-1].copy())
    assert e.value.status == P.PMF_ERR_NOT_MONOTONE
    with pytest.raises(P.PmfError) as e:          # more lambdas than the batch holds
        b.solve(np.concatenate([lam, lam], axis=1))
    assert e.value.status == P.PMF_ERR_INVALID_ARG
    im, inst = wl.images[0], wl.instances[0]
    bad = inst.slope.copy()
    bad[3, 3] = -1
    with pytest.raises(P.PmfError) as e:          # negative slope, host path
        b.set_terminals(0, inst.src0, bad, inst.sink)
    assert e.value.status == P.PMF_ERR_NOT_MONOTONE
    big = im.w_h.copy()
    big[1, 1] = (1 << 28)
    with pytest.raises(P.PmfError) as e:          # pairwise capacity above the maximum
        b.set_capacities(0, big, im.w_v)
    assert e.value.status == P.PMF_ERR_OVERFLOW
    # device path: detected on the GPU, reported per instance by pmf_sync
    b.set_terminals(0, torch.from_numpy(inst.src0).cuda(), torch.from_numpy(bad).cuda(),
                    torch.from_numpy(inst.sink).cuda())
    src_over = wl.instances[1].src0.copy()
    yy, xx = np.argwhere(wl.instances[1].slope == 1)[0]
    src_over[yy, xx] = inputs.INF - 1             # + slope * lambda_max > INF
    b.set_terminals(1, torch.from_numpy(src_over).cuda(), torch.from_numpy(wl.instances[1].slope).cuda(),
                    torch.from_numpy(wl.instances[1].sink).cuda())
    b.solve(lam)
    st = b.sync(check=False)
    assert st == [P.PMF_ERR_NOT_MONOTONE, P.PMF_ERR_OVERFLOW]
    assert b.poll().all()                         # failed instances are finished too
    with pytest.raises(P.PmfError) as e:          # ... but have nothing to read
        b.get_flow(1, 0)
    assert e.value.status == P.PMF_ERR_NOT_READY
    b.copy_terminals(1, 0)                        # a copy carries the validation result
    b.solve(lam)
    assert b.sync(check=False) == [P.PMF_ERR_NOT_MONOTONE, P.PMF_ERR_NOT_MONOTONE]
    b.close()
    # workspace too small
    d, keep = P._desc([(32, 40)], [0], 3, 0)
    need = P.workspace_size([(32, 40)], [0], 3)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    h = ctypes.c_void_p(0)
    st = P.lib().pmf_create_batch(ctypes.byref(d), ctypes.c_void_p(ws.data_ptr()), need - 256, None, ctypes.byref(h))
    assert st == P.PMF_ERR_OUT_OF_MEMORY


def test_watchdog_stops_an_instance_without_a_gpu_fault(P):
    # a tiny visit budget: the device watchdog must end the solve with
    # NOT_CONVERGED for the hard instance while the trivial one still finishes
    hard = _synthetic(10, 96, 128, 1, 4, lo=20, hi=80)
    z = np.zeros((96, 128), np.int32)
    wl = inputs.Workload("wd", hard.images, [hard.instances[0],
                                             inputs.Instance(0, z + 3, z, z + 5, hard.instances[0].lambdas)])
    b = P.batch_from_workload(wl, max_visits_per_tile=1, relabel_every=50)
    b.solve(np.stack([i.lambdas for i in wl.instances]))
    st = b.sync(check=False)
    b.close()
    assert st[0] == P.PMF_ERR_NOT_CONVERGED
    assert st[1] in (P.PMF_OK, P.PMF_ERR_NOT_CONVERGED)


def test_trace_and_profile(P):
    wl = _synthetic(11, 48, 64, 2, 4)
    b = P.batch_from_workload(wl, trace=1)
    b.solve(np.stack([i.lambdas for i in wl.instances]))
    b.sync()
    ev = b.trace()
    done = [e for e in ev if e["event"] == 3]
    assert sorted(e["inst"] for e in done) == [0, 1]
    steps = [e for e in ev if e["event"] == 1]
    assert len(steps) == 2 * 4
    prof = b.profile()
    assert prof["pr_ns"] > 0 and prof["bfs_ns"] > 0
    sm, wm = b.timing()
    assert sm >= wm > 0
    b.close()


def test_concurrent_batches_on_separate_streams(P):
    """Several batches solving at once on their own streams (as the serving
    loop runs them) give each batch's results unchanged."""
    import torch
    wls = [_synthetic(20 + j, 90 + 7 * j, 120 - 5 * j, 3, 6) for j in range(4)]
    ref = [_solve(P, w) for w in wls]
    for grid in (148, 37):
        streams = [torch.cuda.Stream() for _ in wls]
        bs = []
        for w, s in zip(wls, streams):
            with torch.cuda.stream(s):
                b = P.batch_from_workload(w, stream=s, grid_blocks=grid, tile_h=4)
            bs.append(b)
        for w, s, b in zip(wls, streams, bs):
            b.solve(np.stack([i.lambdas for i in w.instances]), stream=s)
        for w, b, r in zip(wls, bs, ref):
            assert all(x == P.PMF_OK for x in b.sync(check=False))
            _same(r, [(b.flows(i), b.cuts(i)) for i in range(len(w.instances))])
            b.close()


def test_race_repeated_small_grids(P):
    """Many repetitions under few workers (the interleavings change from run
    to run): flows must equal the oracle's every time.  This caught a tile
    being queued twice while a phase change was still releasing tiles."""
    wl = _synthetic(3, 70, 96, 3, 8)
    ref = oracle.solve_workload(wl)
    for rep in range(12):
        for grid in (1, 2, 5):
            res = _solve(P, wl, grid_blocks=grid, tile_h=4 if rep % 2 else 8)
            for (f, m), (of, om) in zip(res, ref):
                assert np.array_equal(f, of), (rep, grid)
                assert np.array_equal(m, om), (rep, grid)
