"""ctypes binding of libpmf.so (the C ABI declared in include/pmf.h).

Argument marshalling only: every step of the solve runs in the library's CUDA
kernels.  PyTorch provides the device workspace and the stream.  There is no
CPU fallback: if the library is missing or no GPU is present the calls raise.

    b = Batch([(H, W)], inst_image=[0, 0], max_lambdas=20)
    b.set_capacities(0, w_h, w_v)               # numpy (host) or torch.cuda tensors
    b.set_terminals(0, src0, slope, sink)
    b.solve(lambdas)                            # [n_inst][n_lambda], nondecreasing rows
    b.sync()
    flow = b.get_flow(inst, k); mask = b.get_cut(inst, k)
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpmf.so")

PMF_OK = 0
PMF_ERR_INVALID_ARG = 1
PMF_ERR_OUT_OF_MEMORY = 2
PMF_ERR_NOT_MONOTONE = 3
PMF_ERR_OVERFLOW = 4
PMF_ERR_CUDA = 5
PMF_ERR_NOT_CONVERGED = 6
PMF_ERR_NOT_READY = 7
PMF_INF = 1 << 30
PMF_MAX_PAIRWISE = (1 << 28) - 1

# every entry point declared in include/pmf.h
EXPORTS = ["pmf_workspace_size", "pmf_create_batch", "pmf_set_tuning", "pmf_get_tuning",
           "pmf_set_capacities", "pmf_set_terminals", "pmf_copy_terminals", "pmf_solve_schedule", "pmf_solve_schedules", "pmf_sync", "pmf_poll",
           "pmf_get_cut", "pmf_get_flow", "pmf_get_cuts", "pmf_get_flows", "pmf_get_timing",
           "pmf_get_stats", "pmf_get_trace", "pmf_get_profile", "pmf_get_mask_layout",
           "pmf_destroy_batch", "pmf_status_string", "pmf_version", "pmf_last_error",
           "pmf_solve_noalloc", "pmf_get_flow_arcs", "pmf_set_cut_rule",
           "pmf_set_slope_side", "pmf_testing_fail_noalloc_call", "pmf_cut_lines",
           "pmf_restrict_between", "pmf_set_fork", "pmf_server_workspace_size", "pmf_server_create",
           "pmf_server_set_tuning", "pmf_server_start", "pmf_server_load", "pmf_server_post", "pmf_server_poll",
           "pmf_server_read", "pmf_server_stop", "pmf_server_destroy"]


class PmfError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = f"{where}: {status_string(status)} (status {status})"
        if status == PMF_ERR_CUDA:
            try:
                msg += f" [{lib().pmf_last_error().decode()}]"
            except Exception:
                pass
        super().__init__(msg)


class BatchDesc(ctypes.Structure):
    _fields_ = [("n_images", ctypes.c_int32), ("img_h", ctypes.POINTER(ctypes.c_int32)),
                ("img_w", ctypes.POINTER(ctypes.c_int32)), ("n_inst", ctypes.c_int32),
                ("inst_image", ctypes.POINTER(ctypes.c_int32)), ("max_lambdas", ctypes.c_int32),
                ("device", ctypes.c_int32)]


class Tuning(ctypes.Structure):
    _fields_ = [("tile_h", ctypes.c_int32), ("sweeps", ctypes.c_int32),
                ("relabel_every", ctypes.c_int32), ("max_visits_per_tile", ctypes.c_int32),
                ("mode", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32),
                ("use_graph", ctypes.c_int32), ("trace", ctypes.c_int32),
                ("poll_ns", ctypes.c_int32), ("label_slack", ctypes.c_int32),
                ("grid_blocks", ctypes.c_int32), ("push_order", ctypes.c_int32),
                ("relabel_extra", ctypes.c_int32), ("relabel_reach", ctypes.c_int32),
                ("strip_stage", ctypes.c_int32)]


class ServerDesc(ctypes.Structure):
    _fields_ = [("n_slots", ctypes.c_int32), ("max_h", ctypes.c_int32), ("max_w", ctypes.c_int32),
                ("max_lambdas", ctypes.c_int32), ("device", ctypes.c_int32)]


class TraceEvent(ctypes.Structure):
    _fields_ = [("t_ns", ctypes.c_uint64), ("inst", ctypes.c_int32), ("event", ctypes.c_int32),
                ("k", ctypes.c_int32), ("epoch", ctypes.c_int32), ("pr_visits", ctypes.c_int64),
                ("bfs_visits", ctypes.c_int64), ("flow", ctypes.c_int64), ("active", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


TRACE_EVENTS = {0: "relabel", 1: "step-done", 2: "push-relabel", 3: "done", 4: "not-converged"}


class Stats(ctypes.Structure):
    _fields_ = [("pr_visits", ctypes.c_int64), ("bfs_visits", ctypes.c_int64),
                ("global_relabels", ctypes.c_int64), ("lambdas_done", ctypes.c_int32),
                ("status", ctypes.c_int32), ("warm_visits", ctypes.c_int64)]


_lib = None
_lock = threading.Lock()


def lib(path: str | None = None):
    """Load libpmf.so (built by ``python -m paper_1509_06004_b300.build``)."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                raise RuntimeError(f"libpmf.so not found at {p}; build it with "
                                   "`python -m paper_1509_06004_b300.build` (no CPU fallback exists)")
            L = ctypes.CDLL(p)
            vp = ctypes.c_void_p
            i32 = ctypes.c_int32
            i32p = ctypes.POINTER(ctypes.c_int32)
            L.pmf_workspace_size.argtypes = [ctypes.POINTER(BatchDesc), ctypes.POINTER(ctypes.c_size_t)]
            L.pmf_create_batch.argtypes = [ctypes.POINTER(BatchDesc), vp, ctypes.c_size_t, vp,
                                           ctypes.POINTER(vp)]
            L.pmf_set_tuning.argtypes = [vp, ctypes.POINTER(Tuning)]
            L.pmf_get_tuning.argtypes = [vp, ctypes.POINTER(Tuning)]
            L.pmf_set_capacities.argtypes = [vp, i32, vp, vp, ctypes.c_int]
            L.pmf_set_terminals.argtypes = [vp, i32, vp, vp, vp, ctypes.c_int]
            L.pmf_copy_terminals.argtypes = [vp, i32, i32]
            L.pmf_solve_schedule.argtypes = [vp, i32p, i32, vp]
            L.pmf_solve_schedules.argtypes = [vp, i32p, i32p, i32, vp]
            L.pmf_sync.argtypes = [vp, ctypes.POINTER(ctypes.c_int)]
            L.pmf_poll.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_int32)]
            L.pmf_get_cut.argtypes = [vp, i32, i32, vp, ctypes.c_int]
            L.pmf_get_flow.argtypes = [vp, i32, i32, ctypes.POINTER(ctypes.c_int64)]
            L.pmf_get_stats.argtypes = [vp, i32, ctypes.POINTER(Stats)]
            L.pmf_get_cuts.argtypes = [vp, i32, vp, ctypes.c_int]
            L.pmf_get_flows.argtypes = [vp, i32, ctypes.POINTER(ctypes.c_int64)]
            L.pmf_get_flow_arcs.argtypes = [vp, i32, vp, vp, vp, vp]
            L.pmf_set_cut_rule.argtypes = [vp, i32, i32]
            L.pmf_set_slope_side.argtypes = [vp, i32, i32]
            L.pmf_set_fork.argtypes = [vp, i32, i32, i32]
            L.pmf_get_timing.argtypes = [vp, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float)]
            L.pmf_get_profile.argtypes = [vp, ctypes.POINTER(ctypes.c_uint64)]
            L.pmf_get_trace.argtypes = [vp, ctypes.POINTER(TraceEvent), i32, i32p]
            L.pmf_get_mask_layout.argtypes = [vp, i32, ctypes.POINTER(vp), i32p, i32p]
            L.pmf_destroy_batch.argtypes = [vp]
            L.pmf_destroy_batch.restype = None
            L.pmf_status_string.argtypes = [ctypes.c_int]
            L.pmf_status_string.restype = ctypes.c_char_p
            L.pmf_version.argtypes = []
            L.pmf_version.restype = ctypes.c_char_p
            L.pmf_solve_noalloc.argtypes = [i32, i32, vp, vp, vp, vp, vp, i32p, i32, vp,
                                            ctypes.POINTER(ctypes.c_int64), vp]
            L.pmf_cut_lines.argtypes = [i32, i32, vp, vp, vp, vp, vp, vp, vp, i32, vp, vp, vp]
            L.pmf_restrict_between.argtypes = [i32, i32, vp, vp, vp, vp, vp, vp, vp, ctypes.c_int64,
                                               ctypes.c_int64, vp, vp, vp, vp, vp, vp]
            sdp = ctypes.POINTER(ServerDesc)
            L.pmf_server_workspace_size.argtypes = [sdp, ctypes.POINTER(ctypes.c_size_t)]
            L.pmf_server_create.argtypes = [sdp, vp, ctypes.c_size_t, ctypes.POINTER(vp)]
            L.pmf_server_set_tuning.argtypes = [vp, ctypes.POINTER(Tuning)]
            L.pmf_server_start.argtypes = [vp, ctypes.c_double]
            L.pmf_server_load.argtypes = [vp, i32, i32, i32, i32, vp, vp, vp, vp, vp, vp, i32]
            L.pmf_server_post.argtypes = [vp, vp, i32]
            L.pmf_server_poll.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_int32)]
            L.pmf_server_read.argtypes = [vp, i32, vp, vp]
            L.pmf_server_stop.argtypes = [vp]
            L.pmf_server_destroy.argtypes = [vp]
            L.pmf_server_destroy.restype = None
            L.pmf_testing_fail_noalloc_call.argtypes = [i32]
            L.pmf_testing_fail_noalloc_call.restype = None
            L.pmf_last_error.argtypes = []
            L.pmf_last_error.restype = ctypes.c_char_p
            for name in EXPORTS:
                if name not in ("pmf_destroy_batch", "pmf_status_string", "pmf_version", "pmf_last_error",
                                "pmf_testing_fail_noalloc_call", "pmf_server_destroy"):
                    getattr(L, name).restype = ctypes.c_int
            _lib = L
    return _lib


def status_string(s: int) -> str:
    try:
        return lib().pmf_status_string(int(s)).decode()
    except RuntimeError:
        return "unknown"


def _check(st: int, where: str):
    if st != PMF_OK:
        raise PmfError(st, where)


def _desc(shapes, inst_image, max_lambdas, device):
    Hs = np.ascontiguousarray([s[0] for s in shapes], np.int32)
    Ws = np.ascontiguousarray([s[1] for s in shapes], np.int32)
    ii = np.ascontiguousarray(inst_image, np.int32)
    d = BatchDesc(len(shapes), Hs.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                  Ws.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), len(ii),
                  ii.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), int(max_lambdas), int(device))
    return d, (Hs, Ws, ii)


def workspace_size(shapes, inst_image, max_lambdas: int, device: int = 0) -> int:
    """Device bytes a batch of this shape needs (no GPU needed)."""
    d, keep = _desc(shapes, inst_image, max_lambdas, device)
    n = ctypes.c_size_t(0)
    _check(lib().pmf_workspace_size(ctypes.byref(d), ctypes.byref(n)), "pmf_workspace_size")
    return int(n.value)


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(int(stream.cuda_stream))


class Batch:
    """One batch of grid instances sharing a device workspace."""

    def __init__(self, shapes, inst_image, max_lambdas: int, device: int = 0, stream=None,
                 workspace=None):
        import torch
        self.shapes = [(int(h), int(w)) for h, w in shapes]
        self.inst_image = [int(i) for i in inst_image]
        self.max_lambdas = int(max_lambdas)
        self.device = int(device)
        d, self._keep = _desc(self.shapes, self.inst_image, self.max_lambdas, self.device)
        n = ctypes.c_size_t(0)
        _check(lib().pmf_workspace_size(ctypes.byref(d), ctypes.byref(n)), "pmf_workspace_size")
        self.workspace_bytes = int(n.value)
        if workspace is None:
            workspace = torch.empty(self.workspace_bytes, dtype=torch.uint8, device=f"cuda:{self.device}")
        self.workspace = workspace
        self.stream = stream
        h = ctypes.c_void_p(0)
        _check(lib().pmf_create_batch(ctypes.byref(d), ctypes.c_void_p(workspace.data_ptr()),
                                      self.workspace_bytes, _stream_ptr(stream), ctypes.byref(h)),
               "pmf_create_batch")
        self._h = h
        self.n_lambda = 0
        self.lengths = [0] * len(self.inst_image)

    # -- set-up ------------------------------------------------------------------
    @staticmethod
    def _arg(a):
        """(pointer, on_device, keep-alive) for a numpy array or a torch tensor."""
        try:
            import torch
            if isinstance(a, torch.Tensor):
                if a.dtype != torch.int32:
                    a = a.to(torch.int32)
                a = a.contiguous()
                if a.is_cuda:
                    return ctypes.c_void_p(a.data_ptr()), 1, a
                a = a.numpy()
        except ImportError:
            pass
        a = np.ascontiguousarray(a, np.int32)
        return ctypes.c_void_p(a.ctypes.data), 0, a

    def set_capacities(self, image: int, w_h, w_v):
        (p1, d1, k1), (p2, d2, k2) = self._arg(w_h), self._arg(w_v)
        if d1 != d2:
            raise ValueError("w_h and w_v must both be host or both be device arrays")
        st = lib().pmf_set_capacities(self._h, int(image), p1, p2, d1)
        self._pin = (k1, k2)
        _check(st, "pmf_set_capacities")

    def set_terminals(self, inst: int, src0, slope, sink):
        args = [self._arg(a) for a in (src0, slope, sink)]
        if len({a[1] for a in args}) != 1:
            raise ValueError("src0, slope and sink must all be host or all be device arrays")
        st = lib().pmf_set_terminals(self._h, int(inst), args[0][0], args[1][0], args[2][0], args[0][1])
        self._pin2 = [a[2] for a in args]
        _check(st, "pmf_set_terminals")

    def copy_terminals(self, dst: int, src: int):
        """Instance dst takes instance src's terminal capacities (same image),
        copied on the device (pmf_copy_terminals)."""
        _check(lib().pmf_copy_terminals(self._h, int(dst), int(src)), "pmf_copy_terminals")

    def set_tuning(self, **kw):
        t = Tuning()
        _check(lib().pmf_get_tuning(self._h, ctypes.byref(t)), "pmf_get_tuning")
        for k, v in kw.items():
            if not hasattr(t, k):
                raise KeyError(k)
            setattr(t, k, int(v))
        _check(lib().pmf_set_tuning(self._h, ctypes.byref(t)), "pmf_set_tuning")

    def tuning(self) -> dict:
        t = Tuning()
        _check(lib().pmf_get_tuning(self._h, ctypes.byref(t)), "pmf_get_tuning")
        return {f: getattr(t, f) for f, _ in Tuning._fields_}

    # -- solve -------------------------------------------------------------------
    def solve(self, lambdas, stream=None):
        """lambdas: one schedule for every instance (1-D), a [n_inst][m] array,
        or a list of per-instance 1-D schedules of different lengths
        (pmf_solve_schedules)."""
        strm = _stream_ptr(stream if stream is not None else self.stream)
        if isinstance(lambdas, (list, tuple)) and len({len(np.ravel(x)) for x in lambdas}) > 1:
            rows = [np.ascontiguousarray(np.ravel(x), np.int32) for x in lambdas]
            if len(rows) != len(self.inst_image):
                raise ValueError("one schedule per instance")
            stride = max(len(r) for r in rows)
            lam = np.zeros((len(rows), stride), np.int32)
            for i, r in enumerate(rows):
                lam[i, :len(r)] = r
            lengths = np.array([len(r) for r in rows], np.int32)
            self.n_lambda = stride
            self.lengths = [int(x) for x in lengths]
            self._lam = (lam, lengths)
            st = lib().pmf_solve_schedules(self._h, lam.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                           lengths.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), stride, strm)
            _check(st, "pmf_solve_schedules")
            return
        lam = np.ascontiguousarray(lambdas, np.int32)
        if lam.ndim == 1:
            lam = np.broadcast_to(lam, (len(self.inst_image), lam.shape[0])).copy()
        self.n_lambda = int(lam.shape[1])
        self.lengths = [self.n_lambda] * len(self.inst_image)
        self._lam = lam
        st = lib().pmf_solve_schedule(self._h, lam.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                      self.n_lambda, strm)
        _check(st, "pmf_solve_schedule")

    def poll(self) -> np.ndarray:
        """Finished instances of the running (or last) solve, without waiting:
        a bool array; finished ones that converged can be read already."""
        done = np.zeros(len(self.inst_image), np.uint8)
        n = ctypes.c_int32(0)
        _check(lib().pmf_poll(self._h, ctypes.c_void_p(done.ctypes.data), ctypes.byref(n)), "pmf_poll")
        return done.astype(bool)

    def sync(self, check: bool = True):
        per = (ctypes.c_int * len(self.inst_image))()
        st = lib().pmf_sync(self._h, per)
        if check:
            _check(st, "pmf_sync")
        return [int(x) for x in per]

    # -- results -----------------------------------------------------------------
    def get_flow(self, inst: int, k: int) -> int:
        f = ctypes.c_int64(0)
        _check(lib().pmf_get_flow(self._h, int(inst), int(k), ctypes.byref(f)), "pmf_get_flow")
        return int(f.value)

    def get_cut(self, inst: int, k: int, out=None):
        H, W = self.shapes[self.inst_image[inst]]
        if out is None:
            out = np.empty((H, W), np.uint8)
        try:
            import torch
            if isinstance(out, torch.Tensor):
                assert out.is_cuda and out.dtype == torch.uint8 and out.is_contiguous() and out.numel() == H * W
                _check(lib().pmf_get_cut(self._h, int(inst), int(k), ctypes.c_void_p(out.data_ptr()), 1),
                       "pmf_get_cut")
                return out
        except ImportError:
            pass
        assert out.dtype == np.uint8 and out.flags.c_contiguous and out.size == H * W
        _check(lib().pmf_get_cut(self._h, int(inst), int(k), ctypes.c_void_p(out.ctypes.data), 0),
               "pmf_get_cut")
        return out

    def flows(self, inst: int) -> np.ndarray:
        out = np.empty(self.lengths[inst], np.int64)
        _check(lib().pmf_get_flows(self._h, int(inst), out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))),
               "pmf_get_flows")
        return out

    def set_cut_rule(self, inst: int, rule: int) -> None:
        """rule 1: the instance's terminals were passed with s and t swapped
        (see pmf_set_cut_rule); cuts then come back for the original problem."""
        _check(lib().pmf_set_cut_rule(self._h, int(inst), int(rule)), "pmf_set_cut_rule")

    def set_fork(self, child: int, parent: int, parent_step: int) -> None:
        """child starts from parent's state once parent has certified its
        step parent_step (see pmf_set_fork); parent = -1 removes the fork."""
        _check(lib().pmf_set_fork(self._h, int(child), int(parent), int(parent_step)), "pmf_set_fork")

    def set_slope_side(self, inst: int, side: int) -> None:
        """0: source capacities src0 + slope*lambda rise with lambda (default);
        1: sink capacities sink - slope*lambda fall (see pmf_set_slope_side)."""
        _check(lib().pmf_set_slope_side(self._h, int(inst), int(side)), "pmf_set_slope_side")

    def flow_arcs(self, inst: int) -> dict:
        """A feasible maximum flow of the instance at its last lambda, per arc:
        {"f_h", "f_v", "f_s", "f_t"} as int32 host arrays [H, W] (see
        pmf_get_flow_arcs).  The arrays are computed in device memory."""
        import torch
        H, W = self.shapes[self.inst_image[inst]]
        bufs = torch.empty((4, H, W), dtype=torch.int32, device=f"cuda:{self.device}")
        ptr = [ctypes.c_void_p(bufs[j].data_ptr()) for j in range(4)]
        _check(lib().pmf_get_flow_arcs(self._h, int(inst), *ptr), "pmf_get_flow_arcs")
        a = bufs.cpu().numpy()
        return {"f_h": a[0], "f_v": a[1], "f_s": a[2], "f_t": a[3]}

    def cuts(self, inst: int, out=None) -> np.ndarray:
        """All masks of an instance, [its schedule length, H, W] (numpy host
        array, or a contiguous uint8 CUDA tensor for a device copy)."""
        H, W = self.shapes[self.inst_image[inst]]
        m = self.lengths[inst]
        if out is None:
            out = np.empty((m, H, W), np.uint8)
        try:
            import torch
            if isinstance(out, torch.Tensor):
                assert out.is_cuda and out.dtype == torch.uint8 and out.is_contiguous()
                assert out.numel() == m * H * W
                _check(lib().pmf_get_cuts(self._h, int(inst), ctypes.c_void_p(out.data_ptr()), 1), "pmf_get_cuts")
                return out
        except ImportError:
            pass
        assert out.dtype == np.uint8 and out.flags.c_contiguous and out.size == m * H * W
        _check(lib().pmf_get_cuts(self._h, int(inst), ctypes.c_void_p(out.ctypes.data), 0), "pmf_get_cuts")
        return out

    def timing(self) -> tuple[float, float]:
        """(solve_ms, worker_ms) of the last solve, from library-recorded CUDA events."""
        a, w = ctypes.c_float(0), ctypes.c_float(0)
        _check(lib().pmf_get_timing(self._h, ctypes.byref(a), ctypes.byref(w)), "pmf_get_timing")
        return float(a.value), float(w.value)

    def trace(self) -> list[dict]:
        """Phase-change events of the last solve (needs set_tuning(trace=1))."""
        n = ctypes.c_int32(0)
        _check(lib().pmf_get_trace(self._h, None, 0, ctypes.byref(n)), "pmf_get_trace")
        buf = (TraceEvent * max(1, n.value))()
        _check(lib().pmf_get_trace(self._h, buf, n.value, ctypes.byref(n)), "pmf_get_trace")
        return [{f: getattr(buf[i], f) for f, _ in TraceEvent._fields_} for i in range(n.value)]

    def profile(self) -> dict:
        """Warp-time breakdown of the last solve (needs set_tuning(trace=1))."""
        keys = ["wait_ns", "pr_ns", "bfs_ns", "retire_ns", "sweeps", "pr_load_cyc", "pr_sweep_cyc",
                "pr_store_cyc", "bfs_load_cyc", "bfs_relax_cyc", "bfs_store_cyc", "bfs_rounds"]
        a = (ctypes.c_uint64 * len(keys))()
        _check(lib().pmf_get_profile(self._h, a), "pmf_get_profile")
        return {k: int(a[i]) for i, k in enumerate(keys)}

    def stats(self, inst: int) -> dict:
        s = Stats()
        _check(lib().pmf_get_stats(self._h, int(inst), ctypes.byref(s)), "pmf_get_stats")
        return {f: getattr(s, f) for f, _ in Stats._fields_}

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().pmf_destroy_batch(self._h)
            self._h = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def server_workspace_size(n_slots: int, max_h: int, max_w: int, max_lambdas: int, device: int = 0) -> int:
    """Device bytes of a server (no GPU needed)."""
    d = ServerDesc(n_slots, max_h, max_w, max_lambdas, device)
    n = ctypes.c_size_t(0)
    _check(lib().pmf_server_workspace_size(ctypes.byref(d), ctypes.byref(n)), "pmf_server_workspace_size")
    return int(n.value)


class Server:
    """A running server kernel with instance slots (pmf_server_*): load
    instances into free slots and post them while it runs; poll and read
    finished ones."""

    def __init__(self, n_slots: int, max_h: int, max_w: int, max_lambdas: int, device: int = 0,
                 workspace=None, **tuning):
        import torch
        self.n_slots, self.max_h, self.max_w, self.max_lambdas = int(n_slots), int(max_h), int(max_w), int(max_lambdas)
        self.device = int(device)
        d = ServerDesc(self.n_slots, self.max_h, self.max_w, self.max_lambdas, self.device)
        self.workspace_bytes = server_workspace_size(n_slots, max_h, max_w, max_lambdas, device)
        if workspace is None:
            workspace = torch.empty(self.workspace_bytes, dtype=torch.uint8, device=f"cuda:{self.device}")
        self.workspace = workspace
        h = ctypes.c_void_p(0)
        _check(lib().pmf_server_create(ctypes.byref(d), ctypes.c_void_p(workspace.data_ptr()), self.workspace_bytes,
                                       ctypes.byref(h)), "pmf_server_create")
        self._h = h
        self.shape = {}
        self._keep = {}
        if tuning:
            t = Tuning()
            for k, v in tuning.items():
                setattr(t, k, int(v))
            _check(lib().pmf_server_set_tuning(self._h, ctypes.byref(t)), "pmf_server_set_tuning")

    def start(self, max_seconds: float = 600.0):
        _check(lib().pmf_server_start(self._h, float(max_seconds)), "pmf_server_start")

    def load(self, slot: int, image_slot: int, w_h, w_v, src0, slope, sink, lambdas):
        c = lambda a: np.ascontiguousarray(a, np.int32) if a is not None else None
        src0, slope, sink = c(src0), c(slope), c(sink)
        H, W = src0.shape
        w_h, w_v = c(w_h), c(w_v)
        lam = np.ascontiguousarray(lambdas, np.int32)
        p = lambda a: ctypes.c_void_p(a.ctypes.data) if a is not None else ctypes.c_void_p(0)
        st = lib().pmf_server_load(self._h, int(slot), int(image_slot), H, W, p(w_h), p(w_v), p(src0), p(slope),
                                   p(sink), lam.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), len(lam))
        _check(st, "pmf_server_load")
        self.shape[int(slot)] = (H, W, len(lam))

    def post(self, slots):
        a = np.ascontiguousarray(slots, np.int32)
        _check(lib().pmf_server_post(self._h, ctypes.c_void_p(a.ctypes.data), len(a)), "pmf_server_post")

    def poll(self) -> np.ndarray:
        done = np.zeros(self.n_slots, np.uint8)
        _check(lib().pmf_server_poll(self._h, ctypes.c_void_p(done.ctypes.data), None), "pmf_server_poll")
        return done.astype(bool)

    def read(self, slot: int, check: bool = True):
        """(status, flows [m], masks [m, H, W]) of a finished slot; frees it."""
        H, W, m = self.shape[int(slot)]
        masks = np.empty((m, H, W), np.uint8)
        flows = np.empty(m, np.int64)
        st = lib().pmf_server_read(self._h, int(slot), ctypes.c_void_p(masks.ctypes.data),
                                   ctypes.c_void_p(flows.ctypes.data))
        if check:
            _check(st, "pmf_server_read")
        return st, flows, masks

    def stop(self) -> int:
        return lib().pmf_server_stop(self._h)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().pmf_server_destroy(self._h)
            self._h = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def batch_from_workload(wl, device: int = 0, stream=None, device_inputs: bool = False,
                        workspace=None, **tuning) -> Batch:
    """A Batch holding every image and instance of an inputs.Workload, with all
    capacities uploaded (host path, or device path if device_inputs); the
    workspace is allocated unless a uint8 CUDA tensor of enough bytes is given."""
    import torch
    max_l = max(len(i.lambdas) for i in wl.instances)
    b = Batch([(im.H, im.W) for im in wl.images], [i.image for i in wl.instances], max_l,
              device=device, stream=stream, workspace=workspace)
    if tuning:
        b.set_tuning(**tuning)
    conv = (lambda a: torch.from_numpy(np.ascontiguousarray(a, np.int32)).to(f"cuda:{device}")) \
        if device_inputs else (lambda a: a)
    for i, im in enumerate(wl.images):
        b.set_capacities(i, conv(im.w_h), conv(im.w_v))
    # pieces of one problem (the same terminal arrays) are uploaded once; a
    # forked piece takes its parent's terminals with its state
    first = {}
    for i, inst in enumerate(wl.instances):
        fork = getattr(inst, "fork", None)
        if fork is not None:
            b.set_fork(i, fork[0], fork[1])
            continue
        key = (inst.image, id(inst.src0), id(inst.slope), id(inst.sink))
        if key in first:
            b.copy_terminals(i, first[key])
        else:
            b.set_terminals(i, conv(inst.src0), conv(inst.slope), conv(inst.sink))
            first[key] = i
    return b


def solve_workload(wl, device: int = 0, check: bool = True, **tuning):
    """Solve every instance of a Workload in one batch (schedules may differ in
    length).  Returns (per-instance statuses, list of (flows [m_i], masks
    [m_i, H, W]))."""
    b = batch_from_workload(wl, device=device, **tuning)
    b.solve([np.asarray(i.lambdas) for i in wl.instances])
    st = b.sync(check=check)
    res = []
    for i in range(len(wl.instances)):
        if st[i] == PMF_OK:
            res.append((b.flows(i), b.cuts(i)))
        else:
            res.append((None, None))
    b.close()
    return st, res
