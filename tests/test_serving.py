"""Serving: admission logic on the CPU (fake backend, virtual clock) and, on
the GPU, continuous batching whose per-request results equal the results of
solving each request alone."""
import numpy as np
import pytest

from paper_1509_06004_b300 import inputs, serving


class FakeBackend:
    """Requests take a fixed virtual duration; memory is a byte counter."""

    def __init__(self, clock, budget, dur=0.1):
        self.clock, self.budget, self.dur = clock, budget, dur
        self.used = 0

    def bytes(self, req):
        return req.nbytes

    def reserve(self, req):
        if self.used + req.nbytes > self.budget:
            return None
        self.used += req.nbytes
        return req.nbytes

    def release(self, tok):
        self.used -= tok

    def in_use(self):
        return self.used

    def start(self, req, slot, tok):
        return self.clock.t + self.dur

    def done(self, h):
        return self.clock.t >= h

    def finish(self, h, collect):
        return None, None


class Clock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += max(dt, 1e-4)


class Req:
    def __init__(self, t, nbytes, px=100):
        self.arrival_s, self.nbytes = t, nbytes
        self.workload = type("W", (), {"pixel_solves": px})()


def test_scheduler_slots_budget_and_fifo():
    clk = Clock()
    be = FakeBackend(clk, budget=100)
    reqs = [Req(0.00, 40), Req(0.01, 40), Req(0.02, 40), Req(0.03, 10), Req(0.5, 90)]
    st = serving.Scheduler(be, slots=3, budget_bytes=100).run(reqs, clock=clk, sleep=clk.sleep)
    c = {x.index: x for x in st.completed}
    assert len(c) == 5
    assert st.peak_bytes <= 100 and st.max_concurrent <= 3
    # the third 40-byte request waits for memory; request 3 (10 bytes) waits behind it (FCFS)
    assert c[2].admit_s >= c[0].done_s - 1e-9
    assert c[3].admit_s >= c[2].admit_s
    # a request arriving while others run is admitted as soon as they free memory
    assert c[4].admit_s >= 0.5
    assert all(x.latency_s >= 0.1 - 1e-9 for x in st.completed)


def test_summary_skips_warmup_requests():
    """Latency figures cover only the requests after the warm-up ones; the
    throughput covers the whole run."""
    clk = Clock()
    be = FakeBackend(clk, budget=100, dur=0.1)
    reqs = [Req(0.0, 10) for _ in range(4)] + [Req(1.0, 10) for _ in range(4)]
    st = serving.Scheduler(be, slots=4, budget_bytes=100).run(reqs, realtime=True, clock=clk, sleep=clk.sleep)
    full, part = st.summary(), st.summary(skip=4)
    assert full["requests"] == 8 and part["requests"] == 4
    assert part["pixel_solves_per_s"] == full["pixel_solves_per_s"]
    assert part["p50_ms"] <= full["p99_ms"]


def test_scheduler_rejects_oversized_request():
    clk = Clock()
    with pytest.raises(ValueError):
        serving.Scheduler(FakeBackend(clk, 50), 2, 50).run([Req(0.0, 60)], clock=clk, sleep=clk.sleep)


def test_device_arena_first_fit_and_merge():
    a = serving.DeviceArena(4096)
    x = a.alloc(1000)
    y = a.alloc(1000)
    z = a.alloc(1000)
    assert x[0] == 0 and y[0] == 1024 and z[0] == 2048
    assert a.alloc(2000) is None
    a.release(y)
    a.release(x)
    assert a.free[0] == (0, 2048)
    a.release(z)
    assert a.free == [(0, 4096)] and a.in_use == 0


@pytest.mark.gpu
@pytest.mark.parametrize("live", [True, False])
def test_continuous_batching_equals_alone(live):
    """Requests served while others run (live: admitted into one running
    server kernel; else: one launch per request on its own stream) give
    exactly the results of solving each request alone."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1509_06004_b300 import build, pmf
    build.build()
    reqs = inputs.serving_stream(rate_per_s=1000.0, n_requests=8, seed=3, max_side=256)
    for r in reqs:       # keep the test short: 4 seeds, 6 lambdas
        r.workload.instances = r.workload.instances[:4]
        for inst in r.workload.instances:
            inst.lambdas = inst.lambdas[:6]
    st = serving.serve(reqs, slots=3, budget_bytes=1 << 30, realtime=True, collect=True, segments=2, live=live)
    assert st.max_concurrent >= 2
    for c, r in zip(st.completed, reqs):
        status, alone = pmf.solve_workload(r.workload)
        assert all(s == pmf.PMF_OK for s in status)
        for (fa, ma), f, m in zip(alone, c.flows, c.masks):
            assert np.array_equal(fa, f) and np.array_equal(ma, m)


@pytest.mark.gpu
def test_serving_large_mix_repeated():
    """Four concurrent large requests at a time (images up to 800 px wide),
    served three times over: every request must finish with the same flows
    and masks each time, equal to solving it alone, and a sample equal to the
    oracle.  Large, sparse phases are where a phase change queues its tiles
    for longest, so this is the mix most likely to expose a scheduling race."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle
    from paper_1509_06004_b300 import build, pmf
    build.build()
    reqs = inputs.serving_stream(rate_per_s=1000.0, n_requests=10, seed=5, max_side=800)
    for r in reqs:       # bounded test time: at most 8 seeds, 10 lambdas per request
        r.workload.instances = r.workload.instances[:8]
        for inst in r.workload.instances:
            inst.lambdas = inst.lambdas[:10]
    runs = [serving.serve(reqs, slots=4, budget_bytes=8 << 30, realtime=False, collect=True, segments=5, live=live)
            for live in (True, True, False)]
    assert runs[0].max_concurrent >= 2
    for i, r in enumerate(reqs):
        status, alone = pmf.solve_workload(r.workload)
        assert all(s == pmf.PMF_OK for s in status)
        for run in runs:
            c = run.completed[i]
            for (fa, ma), f, m in zip(alone, c.flows, c.masks):
                assert np.array_equal(fa, f) and np.array_equal(ma, m)
    rng = np.random.default_rng(0)
    for _ in range(2):
        i = int(rng.integers(len(reqs)))
        wl = reqs[i].workload
        j = int(rng.integers(len(wl.instances)))
        inst = wl.instances[j]
        im = wl.images[inst.image]
        k = int(rng.integers(len(inst.lambdas)))
        f, m = oracle.grid_solve(im.H, im.W, im.w_h, im.w_v, inst.src0, inst.slope, inst.sink,
                                 [int(inst.lambdas[k])])
        c = runs[-1].completed[i]
        assert int(c.flows[j][k]) == int(f[0])
        assert np.array_equal(c.masks[j][k].reshape(-1), np.asarray(m[0]).reshape(-1))


@pytest.mark.gpu
def test_server_slots_bad_inputs_and_reuse():
    """The server kernel keeps running across requests: a slot loaded with a
    negative capacity reports PMF_ERR_INVALID_ARG while its neighbours are
    solved; the freed slots then take new instances (one sharing another
    slot's image), whose results equal the oracle's; a slot can be read only
    once it has finished; the server stops cleanly."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle
    from paper_1509_06004_b300 import build, pmf
    build.build()
    reqs = inputs.serving_stream(rate_per_s=1000.0, n_requests=3, seed=8, max_side=240)
    srv = pmf.Server(6, 180, 240, 12)
    srv.start(120.0)
    try:
        wl = reqs[0].workload
        im = wl.images[0]
        bad = wl.instances[1].sink.copy()
        bad[3, 3] = -1
        srv.load(0, 0, im.w_h, im.w_v, wl.instances[0].src0, wl.instances[0].slope, wl.instances[0].sink,
                 wl.instances[0].lambdas[:5])
        srv.load(1, 0, None, None, wl.instances[1].src0, wl.instances[1].slope, bad, wl.instances[1].lambdas[:5])
        assert srv.read(0, check=False)[0] == pmf.PMF_ERR_NOT_READY     # loaded, not posted
        srv.post([0, 1])
        import time
        t0 = time.time()
        while not (srv.poll()[0] and srv.poll()[1]) and time.time() - t0 < 60:
            time.sleep(0.001)
        st0, f0, m0 = srv.read(0)
        assert st0 == pmf.PMF_OK
        assert srv.read(1, check=False)[0] == pmf.PMF_ERR_INVALID_ARG
        inst = wl.instances[0]
        of, om = oracle.grid_solve(im.H, im.W, im.w_h, im.w_v, inst.src0, inst.slope, inst.sink, inst.lambdas[:5])
        assert np.array_equal(f0, of) and np.array_equal(m0, om)
        # reuse: another request's image in slot 1, shared by slot 0
        wl2 = reqs[1].workload
        im2 = wl2.images[0]
        for s, j in ((1, 0), (0, 1)):
            i2 = wl2.instances[j]
            srv.load(s, 1, im2.w_h if s == 1 else None, im2.w_v if s == 1 else None, i2.src0, i2.slope, i2.sink,
                     i2.lambdas[:7])
        srv.post([1, 0])
        t0 = time.time()
        while not (srv.poll()[0] and srv.poll()[1]) and time.time() - t0 < 60:
            time.sleep(0.001)
        for s, j in ((1, 0), (0, 1)):
            st, f, m = srv.read(s)
            i2 = wl2.instances[j]
            of, om = oracle.grid_solve(im2.H, im2.W, im2.w_h, im2.w_v, i2.src0, i2.slope, i2.sink, i2.lambdas[:7])
            assert np.array_equal(f, of) and np.array_equal(m, om)
    finally:
        assert srv.stop() == pmf.PMF_OK
        srv.close()


@pytest.mark.gpu
def test_lone_request_gets_the_whole_gpu():
    """A lone request on the live server takes about as long as solving it
    alone end to end in one batch launch that has the whole GPU (host inputs
    uploaded, solve, every mask and flow read back), within a margin for the
    admission path: no static share of the SMs holds it back."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import time
    from paper_1509_06004_b300 import build, pmf
    build.build()
    req = inputs.serving_stream(rate_per_s=10.0, n_requests=1, seed=11, max_side=640)[0]
    req.arrival_s = 0.0
    wl = req.workload
    im = wl.images[0]
    b = pmf.batch_from_workload(wl, tile_h=4, push_order=1, label_slack=8)
    lam = np.stack([i.lambdas for i in wl.instances])
    ts = []
    for _ in range(4):
        t0 = time.perf_counter()
        b.set_capacities(0, im.w_h, im.w_v)
        for i, inst in enumerate(wl.instances):
            b.set_terminals(i, inst.src0, inst.slope, inst.sink)
        b.solve(lam)
        b.sync()
        for i in range(len(wl.instances)):
            b.flows(i)
            b.cuts(i)
        ts.append(time.perf_counter() - t0)
    b.close()
    alone = float(np.median(ts[1:]))
    st = [serving.serve([req], slots=1, budget_bytes=4 << 30, realtime=False) for _ in range(3)]
    live = float(np.median([s.completed[0].latency_s for s in st]))
    assert live < 1.5 * alone + 0.02, (live, alone)


@pytest.mark.gpu
def test_c5_stream_on_the_live_server_against_oracle():
    """The serving workload's own stream (Poisson arrivals at 50 requests/s,
    images up to 800x600, 4-32 seeds, 10-30 lambdas; its first 12 requests,
    which arrive within 0.3 s and so run mixed on the live server): every seed
    of every request equals solving that request alone in one batch launch,
    and the first seed of every request equals the oracle at every lambda
    (Section 2's exact cut: flows and maximal source sets)."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle
    from paper_1509_06004_b300 import build, pmf
    build.build()
    reqs = inputs.serving_stream(50.0, 12, seed=0, max_side=800)
    st = serving.serve(reqs, slots=16, budget_bytes=16 << 30, realtime=True, collect=True)
    assert st.max_concurrent >= 4
    for c, r in zip(st.completed, reqs):
        wl = r.workload
        status, alone = pmf.solve_workload(wl, tile_h=4, push_order=1, label_slack=8)
        assert all(s == pmf.PMF_OK for s in status)
        for (fa, ma), f, m in zip(alone, c.flows, c.masks):
            assert np.array_equal(fa, f) and np.array_equal(ma, m)
        (of, om), = oracle.solve_workload(wl, instances=[0])
        assert np.array_equal(c.flows[0], of)
        assert np.array_equal(c.masks[0], om)


class FakeServer:
    """Stands in for pmf.Server: slots finish when the test says so."""

    def __init__(self, n):
        self.n, self.loaded, self.posted, self.finished, self.images = n, set(), set(), set(), {}

    def load(self, slot, image_slot, w_h, w_v, src0, slope, sink, lambdas):
        assert slot not in self.posted
        assert (w_h is not None) == (slot == image_slot)
        self.loaded.add(slot)
        self.images[slot] = image_slot

    def post(self, slots):
        assert all(s in self.loaded for s in slots)
        self.posted.update(slots)

    def poll(self):
        return np.array([s in self.finished for s in range(self.n)])

    def read(self, slot, check=True):
        assert slot in self.finished
        self.finished.discard(slot)
        self.posted.discard(slot)
        self.loaded.discard(slot)
        return 0, np.zeros(1, np.int64), np.zeros((1, 1, 1), np.uint8)


def test_live_backend_slot_bookkeeping():
    """Each seed of a request takes a free slot, the first one holding the
    image and the others using it; a request waits for enough free slots;
    it is done when all its slots are; reading frees them."""
    be = serving.LiveBackend.__new__(serving.LiveBackend)
    from paper_1509_06004_b300 import pmf
    be.pmf, be.server, be.n_slots, be.slot_bytes = pmf, FakeServer(5), 5, 100
    be.free = list(range(5))[::-1]
    reqs = inputs.serving_stream(rate_per_s=100.0, n_requests=3, seed=4, max_side=200)
    for r, k in zip(reqs, (3, 2, 4)):
        r.workload.instances = r.workload.instances[:k]
    t0 = be.reserve(reqs[0])
    t1 = be.reserve(reqs[1])
    assert sorted(t0 + t1) == [0, 1, 2, 3, 4] and be.in_use() == 500
    assert be.reserve(reqs[2]) is None                   # 4 seeds, no slot free
    h0 = be.start(reqs[0], 0, t0)
    assert all(be.server.images[s] == t0[0] for s in t0)
    assert not be.done(h0)
    be.server.finished.update(t0[:2])
    assert not be.done(h0)
    be.server.finished.update(t0)
    assert be.done(h0)
    be.finish(h0, collect=True)
    be.release(t0)
    assert be.bytes(reqs[2]) == 400 and be.reserve(reqs[2]) is None   # 3 free, 4 needed
    be.release(t1)
    t2 = be.reserve(reqs[2])
    assert len(t2) == 4 and len(set(t2)) == 4
