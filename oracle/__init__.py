"""Python binding of the CPU oracle (``qap_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers.  The GPU library in
``paper_2307_11248_gb300`` never imports this package.

The oracle is plain scalar C with int64 arithmetic and overflow checks; see
``qap_oracle.c`` for which passage of the paper each function follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qap_oracle.c")
_HDR = os.path.join(_HERE, "qap_oracle.h")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")

REF, FAST, CHECK = 0, 1, 2
TABU_PAIR, TABU_UNIT_LOC, TABU_UNIT = 0, 1, 2
OK, EOVERFLOW, EINVAL, EMISMATCH = 0, 1, 2, 3
STREAM_START, STREAM_TENURE = 0, 1

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` with gcc."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= newest:
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-Wall",
           "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Tenure(ctypes.Structure):
    _fields_ = [("tmin", ctypes.c_int32), ("tmax", ctypes.c_int32),
                ("period", ctypes.c_int32)]


class _Rules(ctypes.Structure):
    _fields_ = [("criterion", ctypes.c_int32), ("penalty", ctypes.c_int32)]


class _WalkResult(ctypes.Structure):
    _fields_ = [("best_cost", ctypes.c_int64), ("final_cost", ctypes.c_int64),
                ("best_iter", ctypes.c_int32), ("iters_done", ctypes.c_int32),
                ("status", ctypes.c_int32), ("hash", ctypes.c_uint64)]


def _p(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else ctypes.c_void_p(0)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            vp, i32, u32, i64, u64 = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint32,
                                      ctypes.c_int64, ctypes.c_uint64)
            L.orc_philox4x32_10.argtypes = [vp, vp, vp]
            L.orc_draw.argtypes = [u64, u32, u32, u32]
            L.orc_draw.restype = u32
            L.orc_bounded.argtypes = [u32, u32]
            L.orc_bounded.restype = u32
            L.orc_start_perm.argtypes = [u64, u32, ctypes.c_int, vp]
            L.orc_tenure.argtypes = [ctypes.POINTER(_Tenure), u64, u32, i32]
            L.orc_tenure.restype = i32
            L.orc_hash_init.restype = u64
            L.orc_hash_move.argtypes = [u64, ctypes.c_int, ctypes.c_int]
            L.orc_hash_move.restype = u64
            L.orc_cost.argtypes = [vp, vp, ctypes.c_int, vp, vp]
            L.orc_cost.restype = i64
            L.orc_delta.argtypes = [vp, vp, ctypes.c_int, vp, ctypes.c_int, ctypes.c_int, vp]
            L.orc_delta.restype = i64
            L.orc_2opt.argtypes = [vp, vp, ctypes.c_int, vp, i32, ctypes.c_int, vp, i32,
                                   ctypes.POINTER(_WalkResult)]
            L.orc_tabu.argtypes = [vp, vp, ctypes.c_int, vp, i32, ctypes.POINTER(_Tenure),
                                   ctypes.c_int, ctypes.POINTER(_Rules), u64, u32, ctypes.c_int,
                                   vp, vp, vp, ctypes.POINTER(_WalkResult)]
            L.orc_run_walks.argtypes = [vp, vp, ctypes.c_int, i32, vp, vp, ctypes.c_int, i32,
                                        i32, ctypes.POINTER(_Tenure), ctypes.c_int,
                                        ctypes.POINTER(_Rules), u64, ctypes.c_int, ctypes.c_int,
                                        vp, vp, vp, vp, vp, vp, vp, vp, vp]
            L.orc_brute_force.argtypes = [vp, vp, ctypes.c_int, vp, vp]
            L.orc_brute_force.restype = i64
            L.orc_num_threads.restype = ctypes.c_int
            _lib = L
    return _lib


def _mat(M, n=None):
    M = np.ascontiguousarray(M, dtype=np.int64)
    assert M.ndim == 2 and M.shape[0] == M.shape[1]
    if n is not None:
        assert M.shape[0] == n
    return M


def _check(err):
    if err == EOVERFLOW:
        raise OverflowError("oracle: int64 overflow")
    if err == EINVAL:
        raise ValueError("oracle: invalid argument")
    if err == EMISMATCH:
        raise AssertionError("oracle: O(1) delta update disagrees with Eq. 2")
    if err:
        raise RuntimeError(f"oracle error {err}")


def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def draw(seed, walk, stream, idx):
    return int(lib().orc_draw(seed, walk, stream, idx))


def bounded(x, m):
    return int(lib().orc_bounded(x, m))


def start_perm(seed, walk, n):
    p = np.zeros(n, dtype=np.int32)
    lib().orc_start_perm(seed, walk, n, _p(p))
    return p


def tenure(tmin, tmax, period, seed, walk, it):
    t = _Tenure(tmin, tmax, period)
    return int(lib().orc_tenure(ctypes.byref(t), seed, walk, it))


def hash_moves(moves):
    L = lib()
    h = L.orc_hash_init()
    for r, s in moves:
        h = L.orc_hash_move(h, int(r), int(s))
    return int(h)


def cost(F, D, p):
    F = _mat(F); D = _mat(D, F.shape[0])
    p = np.ascontiguousarray(p, dtype=np.int32)
    err = ctypes.c_int(0)
    c = lib().orc_cost(_p(F), _p(D), F.shape[0], _p(p), ctypes.byref(err))
    _check(err.value)
    return int(c)


def delta(F, D, p, r, s):
    F = _mat(F); D = _mat(D, F.shape[0])
    p = np.ascontiguousarray(p, dtype=np.int32)
    err = ctypes.c_int(0)
    d = lib().orc_delta(_p(F), _p(D), F.shape[0], _p(p), r, s, ctypes.byref(err))
    _check(err.value)
    return int(d)


def two_opt(F, D, p, max_iters=-1, mode=FAST, moves_cap=0):
    """Best-improvement 2opt from p; returns (p_local_min, result dict).

    With ``moves_cap > 0`` the dict also holds ``moves``, the first
    ``moves_cap`` applied moves as (r, s) rows."""
    F = _mat(F); D = _mat(D, F.shape[0])
    p = np.array(p, dtype=np.int32, copy=True)
    res = _WalkResult()
    mv = np.full((max(moves_cap, 0), 2), -1, dtype=np.int32) if moves_cap > 0 else None
    _check(lib().orc_2opt(_p(F), _p(D), F.shape[0], _p(p), max_iters, mode, _p(mv),
                          moves_cap, ctypes.byref(res)))
    d = _res_dict(res)
    if mv is not None:
        d["moves"] = mv[:min(moves_cap, d["iters_done"])]
    return p, d


def tabu(F, D, p, iters, tmin, tmax, period, aspiration, seed, walk, mode=FAST,
         want_freq=False, criterion=TABU_PAIR, penalty=0):
    """Tabu search from p; returns (final_p, best_p, result dict[, freq]).

    The dict holds ``moves``, the applied moves as (r, s) rows.  ``criterion``
    picks the tabu rule (TABU_PAIR, TABU_UNIT_LOC, TABU_UNIT) and ``penalty``
    the frequency penalty on non-improving moves."""
    F = _mat(F); D = _mat(D, F.shape[0])
    n = F.shape[0]
    p = np.array(p, dtype=np.int32, copy=True)
    best_p = np.zeros(n, dtype=np.int32)
    freq = np.zeros((n, n), dtype=np.int32) if want_freq else None
    mv = np.full((max(iters, 0), 2), -1, dtype=np.int32)
    res = _WalkResult()
    tn = _Tenure(tmin, tmax, period)
    rules = _Rules(criterion, penalty)
    _check(lib().orc_tabu(_p(F), _p(D), n, _p(p), iters, ctypes.byref(tn), int(aspiration),
                          ctypes.byref(rules), seed, walk, mode, _p(best_p), _p(freq), _p(mv),
                          ctypes.byref(res)))
    d = _res_dict(res)
    d["moves"] = mv[:d["iters_done"]]
    out = (p, best_p, d)
    return out + (freq,) if want_freq else out


def _res_dict(res):
    return dict(best_cost=res.best_cost, final_cost=res.final_cost, best_iter=res.best_iter,
                iters_done=res.iters_done, status=res.status, hash=res.hash)


def run_walks(F, D, walks, *, seed, iters=0, tenure=(1, 1, 0), aspiration=True,
              descend=False, max_descent=-1, walk_ids=None, starts=None, mode=FAST,
              threads=0, criterion=TABU_PAIR, penalty=0):
    """Run `walks` independent searches of one instance (OpenMP over walks).

    Walk w draws its start permutation and tenures with walk id
    ``walk_ids[w]`` (default w).  ``descend`` runs 2opt to a local minimum
    first; ``iters`` is the tabu iteration budget (0 with ``descend`` gives
    plain 2opt).  Returns a dict of numpy arrays.
    """
    F = _mat(F); D = _mat(D, F.shape[0])
    n = F.shape[0]
    ids = None
    if walk_ids is not None:
        ids = np.ascontiguousarray(walk_ids, dtype=np.uint32)
        assert ids.shape == (walks,)
    st = None
    if starts is not None:
        st = np.ascontiguousarray(starts, dtype=np.int32)
        assert st.shape == (walks, n)
    out = dict(
        best_p=np.zeros((walks, n), dtype=np.int32),
        best_cost=np.zeros(walks, dtype=np.int64),
        final_cost=np.zeros(walks, dtype=np.int64),
        best_iter=np.zeros(walks, dtype=np.int32),
        iters_done=np.zeros(walks, dtype=np.int32),
        status=np.zeros(walks, dtype=np.int32),
        hash=np.zeros(walks, dtype=np.uint64),
        descent_hash=np.zeros(walks, dtype=np.uint64),
        descent_moves=np.zeros(walks, dtype=np.int32),
    )
    tn = _Tenure(*tenure)
    rules = _Rules(criterion, penalty)
    err = lib().orc_run_walks(
        _p(F), _p(D), n, walks, _p(ids), _p(st), int(descend), max_descent, iters,
        ctypes.byref(tn), int(aspiration), ctypes.byref(rules), seed, mode, threads,
        _p(out["best_p"]), _p(out["best_cost"]), _p(out["final_cost"]), _p(out["best_iter"]),
        _p(out["iters_done"]), _p(out["status"]), _p(out["hash"]), _p(out["descent_hash"]),
        _p(out["descent_moves"]))
    _check(err)
    return out


def brute_force(F, D):
    """Exact optimum by enumerating all n! permutations (n <= 10)."""
    F = _mat(F); D = _mat(D, F.shape[0])
    n = F.shape[0]
    p = np.zeros(n, dtype=np.int32)
    err = ctypes.c_int(0)
    c = lib().orc_brute_force(_p(F), _p(D), n, _p(p), ctypes.byref(err))
    _check(err.value)
    return int(c), p


def num_threads():
    return int(lib().orc_num_threads())
