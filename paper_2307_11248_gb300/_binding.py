"""Thin ctypes binding of ``libqap.so`` (include/qap.h).

Argument marshalling only: every step of the search runs in the CUDA
library.  Function names follow the C-ABI.  There is no fallback: if the
library cannot be built or loaded, or no CUDA device is usable, the calls
raise.
"""
from __future__ import annotations

import ctypes
import threading

import numpy as np

from . import build as _build

OK, EINVAL, EOVERFLOW, ENOMEM, ECUDA, ETIMEOUT, EUNSUPPORTED = range(7)
FORCE_INT64 = 1
LAUNCH_PERSISTENT, LAUNCH_PLAIN = 0, 1
TABU_PAIR, TABU_UNIT_LOC, TABU_UNIT = 0, 1, 2
PHASE_X_AUTO, PHASE_X_DOTS = 0, 1

_lock = threading.Lock()
_lib = None


class QapError(RuntimeError):
    def __init__(self, status, where):
        msg = f"{where}: {strerror(status)}"
        if status == ECUDA:
            msg += f" ({last_error()})"
        super().__init__(msg)
        self.status = status


class Tenure(ctypes.Structure):
    _fields_ = [("tmin", ctypes.c_int32), ("tmax", ctypes.c_int32), ("period", ctypes.c_int32)]


class CtxInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("delta_bytes", ctypes.c_int32),
                ("sym_flow", ctypes.c_int32), ("sym_dist", ctypes.c_int32),
                ("bound", ctypes.c_int64), ("flow_bytes", ctypes.c_int32),
                ("dist_bytes", ctypes.c_int32)]


class SearchParams(ctypes.Structure):
    _fields_ = [("starts", ctypes.c_int32), ("walk_base", ctypes.c_uint32),
                ("descend", ctypes.c_int32), ("max_descent", ctypes.c_int32),
                ("iters", ctypes.c_int32), ("tenure", Tenure), ("aspiration", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("launch", ctypes.c_int32),
                ("threads_per_walk", ctypes.c_int32), ("tenure_per_n", ctypes.c_int32),
                ("criterion", ctypes.c_int32), ("freq_penalty", ctypes.c_int32),
                ("phase_x", ctypes.c_int32)]


class WalkOutputs(ctypes.Structure):
    _fields_ = [(name, ctypes.c_void_p) for name in
                ("best_p", "best_cost", "final_cost", "best_iter", "iters_done", "status",
                 "descent_moves", "hash", "descent_hash", "freq")]


class ServerConfig(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("mem_bytes", ctypes.c_int64)]


class RequestTimes(ctypes.Structure):
    _fields_ = [("queued_us", ctypes.c_double), ("device_us", ctypes.c_double),
                ("total_us", ctypes.c_double), ("kernel_start_us", ctypes.c_double),
                ("kernel_end_us", ctypes.c_double)]


class ServerStats(ctypes.Structure):
    _fields_ = [(name, ctypes.c_int64) for name in
                ("submitted", "completed", "pending", "in_flight", "arena_bytes", "arena_used",
                 "peak_in_flight")]


class PlanInfo(ctypes.Structure):
    _fields_ = [(name, ctypes.c_int32) for name in
                ("threads_per_walk", "pairs_per_thread", "smem_bytes", "grid", "ctas_per_sm",
                 "sms", "classes", "products", "workspace")]


class TuneResult(ctypes.Structure):
    _fields_ = [("nmin", ctypes.c_int32), ("nmax", ctypes.c_int32), ("instances", ctypes.c_int32),
                ("candidates", ctypes.c_int32), ("threads_per_walk", ctypes.c_int32),
                ("pairs_per_thread", ctypes.c_int32), ("workspace", ctypes.c_int32),
                ("products", ctypes.c_int32), ("trial_ms", ctypes.c_float),
                ("rule_ms", ctypes.c_float)]


class ClassInfo(ctypes.Structure):
    _fields_ = [(name, ctypes.c_int32) for name in
                ("nmin", "nmax", "instances", "walks", "threads_per_walk", "pairs_per_thread",
                 "products", "workspace", "grid", "ctas_per_sm", "smem_bytes", "delta_bytes",
                 "flow_bytes", "dist_bytes")] + \
               [("last_ms", ctypes.c_float)]


OUTPUT_FIELDS = {  # name -> (dtype, per-walk shape multiplier uses n)
    "best_p": (np.int32, True), "best_cost": (np.int64, False), "final_cost": (np.int64, False),
    "best_iter": (np.int32, False), "iters_done": (np.int32, False), "status": (np.int32, False),
    "descent_moves": (np.int32, False), "hash": (np.uint64, False),
    "descent_hash": (np.uint64, False),
}


def lib():
    """Build (if stale) and load the CUDA library."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            L = ctypes.CDLL(path)
            vp, i32, u32, u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint32, ctypes.c_uint64
            st = ctypes.c_int
            L.qap_create.argtypes = [vp, vp, i32, u32, ctypes.POINTER(vp)]
            L.qap_create.restype = st
            L.qap_destroy.argtypes = [vp]
            L.qap_destroy.restype = None
            L.qap_info.argtypes = [vp, ctypes.POINTER(CtxInfo)]
            L.qap_info.restype = st
            L.qap_strerror.argtypes = [st]
            L.qap_strerror.restype = ctypes.c_char_p
            L.qap_last_error.argtypes = []
            L.qap_last_error.restype = ctypes.c_char_p
            L.qap_cost.argtypes = [vp, i32, vp, vp]
            L.qap_cost.restype = st
            L.qap_search.argtypes = [vp, ctypes.POINTER(SearchParams), vp,
                                     ctypes.POINTER(WalkOutputs)]
            L.qap_search.restype = st
            L.qap_search_async.argtypes = [vp, ctypes.POINTER(SearchParams), vp,
                                           ctypes.POINTER(WalkOutputs), vp]
            L.qap_search_async.restype = st
            L.qap_plan.argtypes = [vp, ctypes.POINTER(SearchParams), ctypes.POINTER(PlanInfo)]
            L.qap_plan.restype = st
            L.qap_2opt.argtypes = [vp, i32, u64, i32, vp, vp, vp]
            L.qap_2opt.restype = st
            L.qap_tabu.argtypes = [vp, i32, i32, Tenure, i32, u64, vp, vp, vp, vp]
            L.qap_tabu.restype = st
            L.qap_batch_create.argtypes = [i32, vp, vp, vp, u32, ctypes.POINTER(vp)]
            L.qap_batch_create.restype = st
            L.qap_batch_destroy.argtypes = [vp]
            L.qap_batch_destroy.restype = None
            L.qap_batch_info.argtypes = [vp, vp, vp, vp]
            L.qap_batch_info.restype = st
            L.qap_batch_plan.argtypes = [vp, ctypes.POINTER(SearchParams),
                                         ctypes.POINTER(PlanInfo)]
            L.qap_batch_plan.restype = st
            L.qap_best_walks.argtypes = [vp, i32, i32, vp]
            L.qap_best_walks.restype = st
            L.qap_batch_autotune.argtypes = [vp, ctypes.POINTER(SearchParams), i32,
                                             ctypes.POINTER(TuneResult), i32,
                                             ctypes.POINTER(i32)]
            L.qap_batch_autotune.restype = st
            L.qap_batch_set_timing.argtypes = [vp, i32]
            L.qap_batch_set_timing.restype = st
            L.qap_batch_classes.argtypes = [vp, ctypes.POINTER(SearchParams),
                                            ctypes.POINTER(ClassInfo), i32, ctypes.POINTER(i32),
                                            vp]
            L.qap_batch_classes.restype = st
            L.qap_batch_search.argtypes = [vp, ctypes.POINTER(SearchParams),
                                           ctypes.POINTER(WalkOutputs), i32]
            L.qap_batch_search.restype = st
            L.qap_batch_search_async.argtypes = [vp, ctypes.POINTER(SearchParams),
                                                 ctypes.POINTER(WalkOutputs), i32, vp]
            L.qap_batch_search_async.restype = st
            L.qap_batch_search_noalloc.argtypes = [vp, ctypes.POINTER(SearchParams),
                                                   ctypes.POINTER(WalkOutputs), i32, vp]
            L.qap_batch_search_noalloc.restype = st
            L.qap_server_create.argtypes = [ctypes.POINTER(ServerConfig), ctypes.POINTER(vp)]
            L.qap_server_create.restype = st
            L.qap_server_submit.argtypes = [vp, vp, vp, i32, u32, ctypes.POINTER(SearchParams),
                                            ctypes.POINTER(u64)]
            L.qap_server_submit.restype = st
            L.qap_server_wait.argtypes = [vp, u64, i32, ctypes.POINTER(WalkOutputs),
                                          ctypes.POINTER(RequestTimes)]
            L.qap_server_wait.restype = st
            L.qap_server_get_stats.argtypes = [vp, ctypes.POINTER(ServerStats)]
            L.qap_server_get_stats.restype = st
            L.qap_server_destroy.argtypes = [vp]
            L.qap_server_destroy.restype = None
            _lib = L
    return _lib


def strerror(status):
    return lib().qap_strerror(status).decode()


def last_error():
    return lib().qap_last_error().decode()


def _check(status, where):
    if status != OK:
        raise QapError(status, where)


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else ctypes.c_void_p(0)


def make_params(starts, *, seed=0, iters=0, tenure=(1, 1, 0), aspiration=True, descend=False,
                max_descent=-1, walk_base=0, launch=LAUNCH_PERSISTENT, threads_per_walk=0,
                tenure_per_n=False, criterion=0, freq_penalty=0, phase_x=PHASE_X_AUTO):
    """Search parameters.  With tenure_per_n, `tenure` is given in hundredths
    of each instance's n (e.g. (90, 110, 200) is [0.9n, 1.1n] redrawn every
    2n; (10, 33, 0) is the paper's [0.1n, 0.33n] drawn per move).
    ``criterion`` is TABU_PAIR, TABU_UNIT_LOC or TABU_UNIT; ``freq_penalty``
    the frequency-based diversification weight (0 = off); ``phase_x`` is
    PHASE_X_AUTO (maintained products where they apply) or PHASE_X_DOTS."""
    return SearchParams(int(starts), int(walk_base), int(bool(descend)), int(max_descent),
                        int(iters), Tenure(*[int(t) for t in tenure]), int(bool(aspiration)),
                        int(seed) & (2**64 - 1), int(launch), int(threads_per_walk),
                        int(bool(tenure_per_n)), int(criterion), int(freq_penalty),
                        int(phase_x))


# ---------------------------------------------------------------------------
# entry points (same names as the C-ABI)
# ---------------------------------------------------------------------------

def qap_create(F, D, flags=0):
    F = np.ascontiguousarray(F, dtype=np.int64)
    D = np.ascontiguousarray(D, dtype=np.int64)
    n = F.shape[0]
    if F.shape != (n, n) or D.shape != (n, n):
        raise ValueError("F and D must be n x n")
    h = ctypes.c_void_p()
    _check(lib().qap_create(_ptr(F), _ptr(D), n, flags, ctypes.byref(h)), "qap_create")
    return h


def qap_destroy(h):
    lib().qap_destroy(h)


def qap_info(h):
    info = CtxInfo()
    _check(lib().qap_info(h, ctypes.byref(info)), "qap_info")
    return {k: getattr(info, k) for k, _ in CtxInfo._fields_}


def qap_cost(h, perms):
    P = np.ascontiguousarray(perms, dtype=np.int32)
    if P.ndim == 1:
        P = P[None, :]
    out = np.zeros(P.shape[0], dtype=np.int64)
    _check(lib().qap_cost(h, P.shape[0], _ptr(P), _ptr(out)), "qap_cost")
    return out


def qap_plan(h, params):
    info = PlanInfo()
    _check(lib().qap_plan(h, ctypes.byref(params), ctypes.byref(info)), "qap_plan")
    return {k: getattr(info, k) for k, _ in PlanInfo._fields_}


def qap_search(h, params, starts=None, n=None, freq=False):
    """Blocking search with host buffers; returns a dict of numpy arrays
    (with ``freq``, also the W x n x n frequency memory)."""
    if n is None:
        n = qap_info(h)["n"]
    W = params.starts
    st = None
    if starts is not None:
        st = np.ascontiguousarray(starts, dtype=np.int32)
        if st.shape != (W, n):
            raise ValueError("starts must be W x n")
    out = {k: np.zeros((W, n) if per_n else W, dtype=dt)
           for k, (dt, per_n) in OUTPUT_FIELDS.items()}
    ptrs = {k: out[k].ctypes.data for k in OUTPUT_FIELDS}
    if freq:
        out["freq"] = np.zeros((W, n, n), dtype=np.int32)
        ptrs["freq"] = out["freq"].ctypes.data
    o = WalkOutputs(**ptrs)
    _check(lib().qap_search(h, ctypes.byref(params), _ptr(st), ctypes.byref(o)), "qap_search")
    return out


def qap_search_async(h, params, d_starts, d_out, stream):
    """Stream-ordered search on device pointers.

    d_starts: device pointer (int) or 0; d_out: dict name -> device pointer
    (int; missing names are NULL); stream: cudaStream_t as an int."""
    o = WalkOutputs(**{k: int(d_out.get(k, 0) or 0) for k in list(OUTPUT_FIELDS) + ["freq"]})
    _check(lib().qap_search_async(h, ctypes.byref(params), ctypes.c_void_p(int(d_starts or 0)),
                                  ctypes.byref(o), ctypes.c_void_p(int(stream or 0))),
           "qap_search_async")


def qap_2opt(h, starts, seed, max_iters=-1, n=None):
    if n is None:
        n = qap_info(h)["n"]
    best_p = np.zeros((starts, n), dtype=np.int32)
    best_cost = np.zeros(starts, dtype=np.int64)
    moves = np.zeros(starts, dtype=np.int32)
    _check(lib().qap_2opt(h, starts, int(seed), max_iters, _ptr(best_p), _ptr(best_cost),
                          _ptr(moves)), "qap_2opt")
    return best_p, best_cost, moves


def qap_best_walks(best_cost, walks):
    """Index of the best walk of each group of `walks` consecutive entries
    (lowest cost, ties to the lowest walk index), through the C-ABI."""
    c = np.ascontiguousarray(best_cost, dtype=np.int64).reshape(-1)
    if walks < 1 or c.size % walks:
        raise QapError(EINVAL, "qap_best_walks")
    groups = c.size // walks
    idx = np.zeros(groups, dtype=np.int32)
    _check(lib().qap_best_walks(_ptr(c), groups, int(walks), _ptr(idx)), "qap_best_walks")
    return idx


def qap_tabu(h, starts, iters, tenure, aspiration, seed, n=None):
    if n is None:
        n = qap_info(h)["n"]
    best_p = np.zeros((starts, n), dtype=np.int32)
    best_cost = np.zeros(starts, dtype=np.int64)
    best_iter = np.zeros(starts, dtype=np.int32)
    status = np.zeros(starts, dtype=np.int32)
    _check(lib().qap_tabu(h, starts, iters, Tenure(*tenure), int(bool(aspiration)), int(seed),
                          _ptr(best_p), _ptr(best_cost), _ptr(best_iter), _ptr(status)),
           "qap_tabu")
    return best_p, best_cost, best_iter, status


# ---------------------------------------------------------------------------
# convenience: an instance handle and torch device buffers
# ---------------------------------------------------------------------------

class Instance:
    """Owns one qap_ctx; use as a context manager or call close()."""

    def __init__(self, F, D, force_int64=False):
        self.n = int(np.asarray(F).shape[0])
        self.h = qap_create(F, D, FORCE_INT64 if force_int64 else 0)
        self.info = qap_info(self.h)

    def close(self):
        if self.h is not None:
            qap_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def cost(self, perms):
        return qap_cost(self.h, perms)

    def plan(self, params):
        return qap_plan(self.h, params)

    def search(self, params, starts=None, freq=False):
        return qap_search(self.h, params, starts, n=self.n, freq=freq)

    def device_outputs(self, walks, device="cuda"):
        """torch tensors for every output of a search of `walks` walks."""
        import torch
        tdt = {np.int32: torch.int32, np.int64: torch.int64, np.uint64: torch.int64}
        return {k: torch.zeros((walks, self.n) if per_n else walks, dtype=tdt[dt], device=device)
                for k, (dt, per_n) in OUTPUT_FIELDS.items()}

    def search_async(self, params, outs, starts=None, stream=None):
        """Stream-ordered search into torch tensors from device_outputs()."""
        import torch
        if stream is None:
            stream = torch.cuda.current_stream()
        d_out = {k: v.data_ptr() for k, v in outs.items()}
        qap_search_async(self.h, params, starts.data_ptr() if starts is not None else 0, d_out,
                         stream.cuda_stream)


# ---------------------------------------------------------------------------
# batches of instances
# ---------------------------------------------------------------------------

def qap_batch_create(Fs, Ds, flags=0):
    Fs = [np.ascontiguousarray(F, dtype=np.int64) for F in Fs]
    Ds = [np.ascontiguousarray(D, dtype=np.int64) for D in Ds]
    count = len(Fs)
    ns = np.array([F.shape[0] for F in Fs], dtype=np.int32)
    fptrs = (ctypes.c_void_p * count)(*[F.ctypes.data for F in Fs])
    dptrs = (ctypes.c_void_p * count)(*[D.ctypes.data for D in Ds])
    h = ctypes.c_void_p()
    _check(lib().qap_batch_create(count, fptrs, dptrs, _ptr(ns), flags, ctypes.byref(h)),
           "qap_batch_create")
    return h


def qap_batch_destroy(h):
    lib().qap_batch_destroy(h)


def qap_batch_info(h):
    c, m, d = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(lib().qap_batch_info(h, ctypes.byref(c), ctypes.byref(m), ctypes.byref(d)),
           "qap_batch_info")
    return {"count": c.value, "nmax": m.value, "delta_bytes": d.value}


def qap_batch_plan(h, params):
    info = PlanInfo()
    _check(lib().qap_batch_plan(h, ctypes.byref(params), ctypes.byref(info)), "qap_batch_plan")
    return {k: getattr(info, k) for k, _ in PlanInfo._fields_}


def qap_batch_autotune(h, params, trial_iters=200, max_classes=64):
    """Autotune a batch's launch plans; returns one dict per size class."""
    res = (TuneResult * max_classes)()
    nres = ctypes.c_int32(0)
    _check(lib().qap_batch_autotune(h, ctypes.byref(params), int(trial_iters), res, max_classes,
                                    ctypes.byref(nres)), "qap_batch_autotune")
    return [{k: getattr(res[i], k) for k, _ in TuneResult._fields_}
            for i in range(min(nres.value, max_classes))]


def qap_batch_search(h, params, p_stride, freq=False):
    """Blocking batch search; rows i * starts + k; best_p rows of p_stride
    (with ``freq``, also W x p_stride x p_stride frequency memories)."""
    W = qap_batch_info(h)["count"] * params.starts
    out = {k: np.zeros((W, p_stride) if per_n else W, dtype=dt)
           for k, (dt, per_n) in OUTPUT_FIELDS.items()}
    ptrs = {k: out[k].ctypes.data for k in OUTPUT_FIELDS}
    if freq:
        out["freq"] = np.zeros((W, p_stride, p_stride), dtype=np.int32)
        ptrs["freq"] = out["freq"].ctypes.data
    o = WalkOutputs(**ptrs)
    _check(lib().qap_batch_search(h, ctypes.byref(params), ctypes.byref(o), p_stride),
           "qap_batch_search")
    return out


def qap_batch_search_async(h, params, d_out, p_stride, stream):
    o = WalkOutputs(**{k: int(d_out.get(k, 0) or 0) for k in list(OUTPUT_FIELDS) + ["freq"]})
    _check(lib().qap_batch_search_async(h, ctypes.byref(params), ctypes.byref(o), p_stride,
                                        ctypes.c_void_p(int(stream or 0))),
           "qap_batch_search_async")


def qap_batch_set_timing(h, on):
    _check(lib().qap_batch_set_timing(h, 1 if on else 0), "qap_batch_set_timing")


def qap_batch_classes(h, params, count):
    """The size classes of a batch search: a list of dicts (last_ms is the
    last timed launch's device time, or -1) and the class of each instance."""
    nc = ctypes.c_int32()
    _check(lib().qap_batch_classes(h, ctypes.byref(params), None, 0, ctypes.byref(nc), None),
           "qap_batch_classes")
    arr = (ClassInfo * max(1, nc.value))()
    of = np.zeros(count, dtype=np.int32)
    _check(lib().qap_batch_classes(h, ctypes.byref(params), arr, nc.value, ctypes.byref(nc),
                                   _ptr(of)), "qap_batch_classes")
    return ([{k: getattr(arr[i], k) for k, _ in ClassInfo._fields_} for i in range(nc.value)],
            of)


def qap_batch_search_noalloc(h, params, d_out, p_stride, stream):
    """qap_batch_search_async without any allocation inside the call (its
    work queue and tables live in a static device array); see qap.h."""
    o = WalkOutputs(**{k: int(d_out.get(k, 0) or 0) for k in OUTPUT_FIELDS})
    _check(lib().qap_batch_search_noalloc(h, ctypes.byref(params), ctypes.byref(o), p_stride,
                                          ctypes.c_void_p(int(stream or 0))),
           "qap_batch_search_noalloc")


class Batch:
    """Owns one qap_batch (many instances searched in one launch)."""

    def __init__(self, Fs, Ds, force_int64=False):
        self.ns = [int(np.asarray(F).shape[0]) for F in Fs]
        self.h = qap_batch_create(Fs, Ds, FORCE_INT64 if force_int64 else 0)
        self.info = qap_batch_info(self.h)
        self.p_stride = self.info["nmax"]

    def close(self):
        if self.h is not None:
            qap_batch_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def plan(self, params):
        return qap_batch_plan(self.h, params)

    def autotune(self, params, trial_iters=200):
        return qap_batch_autotune(self.h, params, trial_iters)

    def search(self, params, freq=False):
        return qap_batch_search(self.h, params, self.p_stride, freq=freq)

    def set_timing(self, on):
        qap_batch_set_timing(self.h, on)

    def classes(self, params):
        return qap_batch_classes(self.h, params, self.info["count"])

    def device_outputs(self, walks, device="cuda"):
        import torch
        W = self.info["count"] * walks
        tdt = {np.int32: torch.int32, np.int64: torch.int64, np.uint64: torch.int64}
        return {k: torch.zeros((W, self.p_stride) if per_n else W, dtype=tdt[dt], device=device)
                for k, (dt, per_n) in OUTPUT_FIELDS.items()}

    def search_async(self, params, outs, stream=None):
        import torch
        if stream is None:
            stream = torch.cuda.current_stream()
        qap_batch_search_async(self.h, params, {k: v.data_ptr() for k, v in outs.items()},
                               self.p_stride, stream.cuda_stream)


# ---------------------------------------------------------------------------
# serving loop
# ---------------------------------------------------------------------------

def qap_server_create(slots=64, mem_bytes=1 << 30):
    h = ctypes.c_void_p()
    _check(lib().qap_server_create(ctypes.byref(ServerConfig(slots, 0, mem_bytes)),
                                   ctypes.byref(h)), "qap_server_create")
    return h


def qap_server_submit(h, F, D, params, flags=0):
    F = np.ascontiguousarray(F, dtype=np.int64)
    D = np.ascontiguousarray(D, dtype=np.int64)
    t = ctypes.c_uint64()
    _check(lib().qap_server_submit(h, _ptr(F), _ptr(D), F.shape[0], flags, ctypes.byref(params),
                                   ctypes.byref(t)), "qap_server_submit")
    return t.value


def qap_server_wait(h, ticket, n, walks, timeout_ms=60000):
    """Results dict (numpy) and times dict of a finished request."""
    out = {k: np.zeros((walks, n) if per_n else walks, dtype=dt)
           for k, (dt, per_n) in OUTPUT_FIELDS.items()}
    o = WalkOutputs(**{k: out[k].ctypes.data for k in OUTPUT_FIELDS})
    tm = RequestTimes()
    _check(lib().qap_server_wait(h, ticket, int(timeout_ms), ctypes.byref(o), ctypes.byref(tm)),
           "qap_server_wait")
    return out, {k: getattr(tm, k) for k, _ in RequestTimes._fields_}


def qap_server_get_stats(h):
    st = ServerStats()
    _check(lib().qap_server_get_stats(h, ctypes.byref(st)), "qap_server_get_stats")
    return {k: getattr(st, k) for k, _ in ServerStats._fields_}


def qap_server_destroy(h):
    lib().qap_server_destroy(h)


class Server:
    """Owns one qap_server."""

    def __init__(self, slots=64, mem_bytes=1 << 30):
        self.h = qap_server_create(slots, mem_bytes)
        self._shape = {}

    def submit(self, F, D, params, force_int64=False):
        t = qap_server_submit(self.h, F, D, params, FORCE_INT64 if force_int64 else 0)
        self._shape[t] = (int(np.asarray(F).shape[0]), params.starts)
        return t

    def wait(self, ticket, timeout_ms=60000):
        n, walks = self._shape[ticket]
        res = qap_server_wait(self.h, ticket, n, walks, timeout_ms)
        del self._shape[ticket]
        return res

    def stats(self):
        return qap_server_get_stats(self.h)

    def close(self):
        if self.h is not None:
            qap_server_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
