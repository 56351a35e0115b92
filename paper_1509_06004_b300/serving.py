"""Serving loop: continuous batching of parametric segmentation requests.

Each request is one image with its seeds and its lambda schedule (the paper's
per-image figure-ground stage, Section 4).  Requests arrive over time; the
server keeps up to ``slots`` of them on the GPU at once, and their work
overlaps on the device.  A request is admitted (first come, first served) as
soon as a slot is free AND its device memory fits in what is left of the
budget; its residual state stays resident on the device across its whole
lambda schedule; when it finishes its masks and flows are read back, its slot
and memory are released and the next waiting request is admitted at once.  This is the GPU analogue of
the paper's dynamic scheduler, which hands the next supergraph to whichever
server frees up first (Section 3.3.1), and of its overlap of one call's
transfer with another's computation (Section 3.3.2).

The scheduler is plain host logic over a backend; tests use a fake backend on
the CPU.  Two GPU backends:

* ``LiveBackend`` (the default): ONE server kernel (pmf_server_*) keeps running;
  a request's seeds are loaded into free instance slots while it runs and
  posted to it, an idle worker of the kernel admits them into the device work
  queue that every running instance shares, and finished slots are read back
  while the others run.  A lone request gets the whole GPU; several mix in
  one queue, with no static share of the SMs.
* ``GpuBackend``: each request as its own batch and persistent launch on a
  stream of its own, with a fixed share of the SMs per slot.

Latency of a request = completion (results on the host) - arrival.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Completed:
    index: int
    arrival_s: float
    admit_s: float
    done_s: float
    pixel_solves: int
    flows: list | None = None
    masks: list | None = None

    @property
    def latency_s(self) -> float:
        return self.done_s - self.arrival_s


@dataclass
class ServeStats:
    completed: list = field(default_factory=list)
    makespan_s: float = 0.0
    peak_bytes: int = 0
    max_concurrent: int = 0

    def summary(self, skip: int = 0) -> dict:
        """Latency percentiles over the requests with index >= skip (the
        first ones warm the stream up); throughput over the whole run."""
        meas = [c for c in self.completed if c.index >= skip]
        lat = np.array([c.latency_s for c in meas]) * 1e3
        pix = sum(c.pixel_solves for c in self.completed)
        return {"requests": len(meas),
                "p50_ms": float(np.percentile(lat, 50)) if len(lat) else None,
                "p99_ms": float(np.percentile(lat, 99)) if len(lat) else None,
                "mean_ms": float(lat.mean()) if len(lat) else None,
                "pixel_solves_per_s": pix / self.makespan_s if self.makespan_s > 0 else None,
                "makespan_s": self.makespan_s, "peak_bytes": self.peak_bytes,
                "max_concurrent": self.max_concurrent}


class DeviceArena:
    """First-fit byte ranges of one pre-reserved buffer: request workspaces
    come from here, so admitting a request never allocates (allocation would
    synchronise the device and stall the requests already running)."""

    ALIGN = 256

    def __init__(self, size: int):
        self.size = int(size)
        self.free = [(0, self.size)]          # sorted (offset, length)

    def alloc(self, n: int):
        n = (int(n) + self.ALIGN - 1) // self.ALIGN * self.ALIGN
        for k, (off, ln) in enumerate(self.free):
            if ln >= n:
                if ln == n:
                    self.free.pop(k)
                else:
                    self.free[k] = (off + n, ln - n)
                return off, n
        return None

    def release(self, tok) -> None:
        off, n = tok
        k = 0
        while k < len(self.free) and self.free[k][0] < off:
            k += 1
        self.free.insert(k, (off, n))
        if k + 1 < len(self.free) and off + n == self.free[k + 1][0]:
            self.free[k] = (off, n + self.free[k + 1][1])
            self.free.pop(k + 1)
        if k > 0 and self.free[k - 1][0] + self.free[k - 1][1] == self.free[k][0]:
            self.free[k - 1] = (self.free[k - 1][0], self.free[k - 1][1] + self.free[k][1])
            self.free.pop(k)

    @property
    def in_use(self) -> int:
        return self.size - sum(ln for _, ln in self.free)


class Scheduler:
    """Admission and completion bookkeeping, independent of the GPU."""

    def __init__(self, backend, slots: int, budget_bytes: int):
        assert slots >= 1
        self.backend = backend
        self.slots = slots
        self.budget = int(budget_bytes)

    def run(self, requests, realtime: bool = True, collect: bool = False,
            clock=time.perf_counter, sleep=time.sleep) -> ServeStats:
        """requests: list of objects with .arrival_s and .workload.
        realtime=False releases every request at t = 0."""
        pending = collections.deque(sorted(enumerate(requests), key=lambda r: r[1].arrival_s))
        waiting = collections.deque()
        active = {}                      # slot -> (index, request, handle, admit time, reservation)
        free_slots = list(range(self.slots))
        st = ServeStats()
        t0 = clock()
        while pending or waiting or active:
            now = clock() - t0
            while pending and (not realtime or pending[0][1].arrival_s <= now):
                waiting.append(pending.popleft())
            progressed = False
            for slot in list(active):
                i, req, h, t_admit, tok = active[slot]
                if self.backend.done(h):
                    res = self.backend.finish(h, collect)
                    t_done = clock() - t0
                    st.completed.append(Completed(i, req.arrival_s if realtime else 0.0, t_admit, t_done,
                                                  req.workload.pixel_solves,
                                                  *(res if collect else (None, None))))
                    del active[slot]
                    free_slots.append(slot)
                    self.backend.release(tok)
                    progressed = True
            while waiting and free_slots:
                i, req = waiting[0]
                if self.backend.bytes(req) > self.budget:
                    raise ValueError(f"request {i} needs more than the whole memory budget")
                tok = self.backend.reserve(req)
                if tok is None:
                    break                # first come, first served: wait for memory
                waiting.popleft()
                slot = free_slots.pop()
                h = self.backend.start(req, slot, tok)
                active[slot] = (i, req, h, clock() - t0, tok)
                st.peak_bytes = max(st.peak_bytes, self.backend.in_use())
                st.max_concurrent = max(st.max_concurrent, len(active))
                progressed = True
            if not progressed:
                nxt = pending[0][1].arrival_s - (clock() - t0) if (pending and realtime and not waiting) else 0.0
                sleep(min(nxt, 0.002) if nxt > 0 else 0.0002)
        st.makespan_s = clock() - t0
        st.completed.sort(key=lambda c: c.index)
        return st


class GpuBackend:
    """Runs each request as one batch of the CUDA solver on a slot's stream,
    its workspace taken from a device arena of the budget's size."""

    def __init__(self, slots: int, budget_bytes: int, device: int = 0, segments: int | None = None,
                 tuning: dict | None = None):
        import torch
        from . import pmf
        self.torch, self.pmf = torch, pmf
        self.device = device
        self.streams = [torch.cuda.Stream(device=device) for _ in range(slots)]
        self.segments = segments
        self.tuning = dict(tuning or {})
        # knobs measured best for this request mix on a B300 (60 requests up to
        # 800x600, 4 slots): chain-ordered pushes, label slack 8, and each seed's
        # schedule as one warm-started chain (segments=None)
        self.tuning.setdefault("tile_h", 4)          # 4 resident blocks per SM at this tile height
        self.tuning.setdefault("push_order", 1)
        self.tuning.setdefault("label_slack", 8)
        if "grid_blocks" not in self.tuning:
            n_sm = torch.cuda.get_device_properties(device).multi_processor_count
            # the slots share the SMs: every slot's persistent grid fits at once
            self.tuning["grid_blocks"] = max(1, (4 * n_sm) // slots)
        self.arena = DeviceArena(budget_bytes)
        self.buf = torch.empty(self.arena.size, dtype=torch.uint8, device=f"cuda:{device}")

    def _plan(self, wl):
        """Cut each seed's schedule into the largest number of equal pieces
        that divides it and does not exceed ``segments``."""
        m = min(len(i.lambdas) for i in wl.instances)
        s = max(d for d in range(1, (self.segments or 1) + 1) if m % d == 0)
        return (wl.split_segments(s) if s > 1 else wl), s

    def bytes(self, req) -> int:
        w, _ = self._plan(req.workload)
        return self.pmf.workspace_size([(im.H, im.W) for im in w.images], [i.image for i in w.instances],
                                       max(len(i.lambdas) for i in w.instances), self.device)

    def reserve(self, req):
        return self.arena.alloc(self.bytes(req))

    def release(self, tok) -> None:
        self.arena.release(tok)

    def in_use(self) -> int:
        return self.arena.in_use

    def start(self, req, slot, tok):
        w, s = self._plan(req.workload)
        stream = self.streams[slot]
        off, n = tok
        with self.torch.cuda.stream(stream):
            b = self.pmf.batch_from_workload(w, device=self.device, stream=stream,
                                             workspace=self.buf[off:off + n], **self.tuning)
            lam = np.stack([i.lambdas for i in w.instances]).astype(np.int32)
            b.solve(lam, stream=stream)
            ev = self.torch.cuda.Event()
            ev.record(stream)
        return (b, ev, w, s, req)

    def done(self, h) -> bool:
        return h[1].query()

    def finish(self, h, collect: bool):
        b, ev, w, s, req = h
        st = b.sync(check=False)
        if any(x != self.pmf.PMF_OK for x in st):
            b.close()
            raise RuntimeError(f"request failed: {[self.pmf.status_string(x) for x in st]}")
        flows, masks = [], []
        for i in range(len(req.workload.instances)):     # reassemble the pieces of each seed
            flows.append(np.concatenate([b.flows(i * s + j) for j in range(s)]))
            masks.append(np.concatenate([b.cuts(i * s + j) for j in range(s)]))
        b.close()
        return (flows, masks) if collect else (None, None)


class LiveBackend:
    """Requests as instances of one running server kernel: each seed of a
    request takes an instance slot (the first one holds the request's image,
    the others use it), the slots are loaded while the kernel runs and posted
    to it together; the request is done when all its slots are, and its slots
    are freed when it has been read.  Admission is by free slots: the server
    has as many as the memory budget holds (at most ``max_slots``)."""

    def __init__(self, budget_bytes: int, device: int = 0, max_h: int = 600, max_w: int = 800,
                 max_lambdas: int = 30, max_slots: int = 512, tuning: dict | None = None,
                 max_seconds: float = 900.0):
        from . import pmf
        self.pmf = pmf
        per = pmf.server_workspace_size(2, max_h, max_w, max_lambdas, device) - \
            pmf.server_workspace_size(1, max_h, max_w, max_lambdas, device)
        self.slot_bytes = per
        n = int(max(1, min(max_slots, budget_bytes // max(per, 1))))
        tuning = dict(tuning or {})
        tuning.setdefault("label_slack", 8)
        self.server = pmf.Server(n, max_h, max_w, max_lambdas, device, **tuning)
        self.server.start(max_seconds)
        self.free = list(range(n))[::-1]
        self.n_slots = n
        self._done = None

    def bytes(self, req) -> int:
        return len(req.workload.instances) * self.slot_bytes

    def reserve(self, req):
        k = len(req.workload.instances)
        if k > self.n_slots:
            raise ValueError("a request with more seeds than the server has slots")
        if len(self.free) < k:
            return None
        return [self.free.pop() for _ in range(k)]

    def release(self, tok) -> None:
        self.free.extend(tok)

    def in_use(self) -> int:
        return (self.n_slots - len(self.free)) * self.slot_bytes

    def start(self, req, slot, tok):
        wl = req.workload
        im = wl.images[0]
        for j, inst in enumerate(wl.instances):
            first = j == 0
            self.server.load(tok[j], tok[0], im.w_h if first else None, im.w_v if first else None,
                             inst.src0, inst.slope, inst.sink, inst.lambdas)
        self.server.post(tok)
        return (tok, req)

    def done(self, h) -> bool:
        d = self.server.poll()
        return bool(all(d[s] for s in h[0]))

    def finish(self, h, collect: bool):
        tok, req = h
        flows, masks, bad = [], [], []
        for s in tok:
            st, f, m = self.server.read(s, check=False)
            bad.append(st)
            flows.append(f)
            masks.append(m)
        if any(x != self.pmf.PMF_OK for x in bad):
            raise RuntimeError(f"request failed: {[self.pmf.status_string(x) for x in bad]}")
        return (flows, masks) if collect else (None, None)

    def close(self) -> int:
        st = self.server.stop()
        self.server.close()
        return st


def serve(requests, slots: int = 16, budget_bytes: int = 64 << 30, device: int = 0, realtime: bool = True,
          collect: bool = False, segments: int | None = None, tuning: dict | None = None,
          live: bool = True, max_slots: int = 512) -> ServeStats:
    """Serve a request stream with continuous batching; returns ServeStats.
    live=True: one running server kernel, at most ``slots`` requests admitted
    at once (and as many seeds as the budget's instance slots hold);
    live=False: one batch and launch per request, ``slots`` of them at once."""
    if live:
        max_h = max(r.workload.images[0].H for r in requests)
        max_w = max(r.workload.images[0].W for r in requests)
        max_l = max(len(i.lambdas) for r in requests for i in r.workload.instances)
        backend = LiveBackend(budget_bytes, device, max_h, max_w, max_l, max_slots, tuning)
        try:
            return Scheduler(backend, slots, budget_bytes).run(requests, realtime=realtime, collect=collect)
        finally:
            if backend.close() != 0:
                raise RuntimeError("the server kernel stopped on a watchdog")
    backend = GpuBackend(slots, budget_bytes, device, segments, tuning)
    return Scheduler(backend, slots, budget_bytes).run(requests, realtime=realtime, collect=collect)
