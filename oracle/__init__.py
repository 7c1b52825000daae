"""CPU oracle for StaticGreedy / StaticGreedyDU (Cheng et al., CIKM'13).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and
the benchmark's CPU-baseline leg may import this package.  It shares no
code with the GPU library (``paper_1212_4779_gb300``) and imports nothing
from it; the only module both sides use is the seeded graph generator
``paper_1212_4779_gb300.inputs``, which holds none of the method's
arithmetic.

The arithmetic lives in ``sg_oracle.c`` (plain C, OpenMP over sources),
built on demand into ``oracle/_build/`` with gcc; ``brute.py`` is an
independent pure-Python brute force for tiny graphs.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sg_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libsg_oracle.so")
_lock = threading.Lock()
_lib = None

UIC, WIC = 0, 1
LITERAL, COVER, DU, CELF = 0, 1, 2, 3
OR_OK, OR_EINVAL, OR_ENOMEM, OR_EINVARIANT = 0, -1, -2, -3


def build(force: bool = False) -> str:
    """Compile ``sg_oracle.c`` into ``oracle/_build/libsg_oracle.so``."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.run(["gcc", "-O2", "-std=c11", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"],
                       check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(os.environ.get("SG_ORACLE_LIB") or build())
        P = ctypes.c_void_p
        i64, i32, u64, dbl, cint = ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64, ctypes.c_double, ctypes.c_int
        lib.or_splitmix64.restype = u64
        lib.or_splitmix64.argtypes = [u64]
        lib.or_live.restype = cint
        lib.or_live.argtypes = [u64, ctypes.c_uint32, u64, u64]
        lib.or_canon_coo.restype = cint
        lib.or_canon_coo.argtypes = [i64, i64, P, P, P, P, P]
        lib.or_thresholds.restype = cint
        lib.or_thresholds.argtypes = [cint, dbl, i64, P, P, P]
        lib.or_select.restype = cint
        lib.or_select.argtypes = [cint, i64, P, P, P, i32, i32, u64, cint, P, P, P, P, P, P, P]
        lib.or_init_gains.restype = cint
        lib.or_init_gains.argtypes = [i64, P, P, P, i32, i32, u64, cint, P, P, P, P]
        lib.or_spread.restype = i64
        lib.or_spread.argtypes = [i64, P, P, P, i32, u64, i32, P, cint, P, P, P]
        lib.or_reach_sums.restype = cint
        lib.or_reach_sums.argtypes = [i64, P, P, P, i32, u64, i32, P, cint, P, P, P, P]
        lib.or_live_masks.restype = cint
        lib.or_live_masks.argtypes = [i64, P, i32, u64, P, P, P]
        lib.or_live_range.restype = cint
        lib.or_live_range.argtypes = [u64, ctypes.c_uint32, u64, u64, u64]
        lib.or_lt_intervals.restype = cint
        lib.or_lt_intervals.argtypes = [i64, P, P, P, P, P]
        lib.or_coupled_ids.restype = cint
        lib.or_coupled_ids.argtypes = [i64, P, P, P]
        _lib = lib
        return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _threads(nthreads):
    return int(nthreads) if nthreads else (os.cpu_count() or 1)


class OracleError(RuntimeError):
    pass


def _check(rc, what):
    if rc != OR_OK:
        raise OracleError(f"{what}: oracle status {rc}")


def splitmix64(x: int) -> int:
    return int(_load().or_splitmix64(ctypes.c_uint64(x & 0xFFFFFFFFFFFFFFFF)))


def live(seed: int, r: int, e: int, thr: int) -> bool:
    return bool(_load().or_live(seed, r, e, thr))


def live_range(seed: int, r: int, key: int, lo: int, hi: int) -> bool:
    return bool(_load().or_live_range(seed, r, key, lo, hi))


class Graph:
    """Canonical graph (CSR) with per-arc thresholds for one cascade model."""

    def __init__(self, n, src, dst, model="uic", p=0.0):
        """model: "uic", "wic", "uic_undirected" (uniform cascade on a
        symmetric graph with one coin per undirected edge: both arcs hash the
        lower of their two canonical arc ids), or "lt" (the linear threshold
        model's live-edge form with weights 1/d_v: each node keeps at most one
        in-arc, chosen by one draw per node and snapshot)."""
        lib = _load()
        src = np.ascontiguousarray(src, dtype=np.int32)
        dst = np.ascontiguousarray(dst, dtype=np.int32)
        self.n = int(n)
        rp = np.zeros(self.n + 1, dtype=np.int64)
        col = np.zeros(max(1, src.size), dtype=np.int32)
        m = ctypes.c_int64(0)
        _check(lib.or_canon_coo(self.n, src.size, _ptr(src), _ptr(dst), _ptr(rp), _ptr(col),
                                ctypes.byref(m)), "canonicalise")
        self.m = int(m.value)
        self.rp = rp
        self.col = np.ascontiguousarray(col[: self.m])
        if self.col.size == 0:
            self.col = np.zeros(1, dtype=np.int32)
        self.model = model
        self.p = float(p)
        self.thr = np.zeros(max(1, self.m), dtype=np.uint64)
        _check(lib.or_thresholds(WIC if model == "wic" else UIC, self.p, self.n, _ptr(self.rp),
                                 _ptr(self.col), _ptr(self.thr)), "thresholds")
        self.cid = None
        self.lo = None
        if model == "lt":
            self.cid = np.zeros(max(1, self.m), dtype=np.int64)
            self.lo = np.zeros(max(1, self.m), dtype=np.uint64)
            _check(lib.or_lt_intervals(self.n, _ptr(self.rp), _ptr(self.col), _ptr(self.cid), _ptr(self.lo),
                                       _ptr(self.thr)), "lt_intervals")
        if model == "uic_undirected":
            self.cid = np.zeros(max(1, self.m), dtype=np.int64)
            if lib.or_coupled_ids(self.n, _ptr(self.rp), _ptr(self.col), _ptr(self.cid)) != 0:
                raise OracleError("uic_undirected needs a symmetric graph (every arc's reverse present)")

    def _cid(self):
        return _ptr(self.cid) if self.cid is not None else None

    def _lo(self):
        return _ptr(self.lo) if self.lo is not None else None

    def select(self, R, k, seed, mode=DU, nthreads=None, want_init=False, want_hist=False):
        """Greedy seeds by Algorithm 1 (LITERAL/COVER) or Algorithm 2 (DU).
        Returns dict(seeds, gains, counters[, s_init][, s_hist])."""
        lib = _load()
        seeds = np.zeros(k, dtype=np.int32)
        gains = np.zeros(k, dtype=np.int64)
        cnt = np.zeros(4, dtype=np.uint64)
        s_init = np.zeros(self.n, dtype=np.int64) if want_init else None
        s_hist = np.zeros((k, self.n), dtype=np.int64) if want_hist else None
        rc = lib.or_select(mode, self.n, _ptr(self.rp), _ptr(self.col), _ptr(self.thr), R, k,
                           ctypes.c_uint64(seed), _threads(nthreads), _ptr(seeds), _ptr(gains),
                           _ptr(s_init) if want_init else None, _ptr(s_hist) if want_hist else None,
                           _ptr(cnt), self._cid(), self._lo())
        _check(rc, "select")
        out = dict(seeds=seeds, gains=gains, counters=cnt[:3], evals=int(cnt[3]))
        if want_init:
            out["s_init"] = s_init
        if want_hist:
            out["s_hist"] = s_hist
        return out

    def init_gains(self, R, seed, r0=0, r1=None, nthreads=None):
        """(s_v over snapshots r0..r1-1, init snapshot-edge count)."""
        lib = _load()
        r1 = R if r1 is None else r1
        s = np.zeros(self.n, dtype=np.int64)
        ed = ctypes.c_uint64(0)
        _check(lib.or_init_gains(self.n, _ptr(self.rp), _ptr(self.col), _ptr(self.thr), r0, r1,
                                 ctypes.c_uint64(seed), _threads(nthreads), _ptr(s), ctypes.byref(ed), self._cid(),
                                 self._lo()),
               "init_gains")
        return s, int(ed.value)

    def spread(self, R, seed, S, nthreads=None, want_edges=False):
        """f(S) = sum_r |R(G'_r, S)| (and, with want_edges, the snapshot-edge
        count sum_r sum over R(G'_r, S) of out-degrees)."""
        S = np.ascontiguousarray(S, dtype=np.int32)
        ed = ctypes.c_uint64(0)
        v = _load().or_spread(self.n, _ptr(self.rp), _ptr(self.col), _ptr(self.thr), R,
                              ctypes.c_uint64(seed), S.size, _ptr(S), _threads(nthreads), ctypes.byref(ed),
                              self._cid(), self._lo())
        if v < 0:
            raise OracleError(f"spread: oracle status {v}")
        return (int(v), int(ed.value)) if want_edges else int(v)

    def reach_sums(self, R, seed, vs, nthreads=None):
        """(sum_r |R(G'_r, v)| for v in vs, their init snapshot-edge count)."""
        vs = np.ascontiguousarray(vs, dtype=np.int32)
        out = np.zeros(vs.size, dtype=np.int64)
        ed = ctypes.c_uint64(0)
        _check(_load().or_reach_sums(self.n, _ptr(self.rp), _ptr(self.col), _ptr(self.thr), R,
                                     ctypes.c_uint64(seed), vs.size, _ptr(vs), _threads(nthreads),
                                     _ptr(out), ctypes.byref(ed), self._cid(), self._lo()), "reach_sums")
        return out, int(ed.value)

    def live_masks(self, R, seed):
        """uint64[m, W]: bit b of word w = coin of arc e in snapshot 64w+b."""
        W = (R + 63) // 64
        masks = np.zeros((max(1, self.m), W), dtype=np.uint64)
        _check(_load().or_live_masks(self.m, _ptr(self.thr), R, ctypes.c_uint64(seed), _ptr(masks),
                                     self._cid(), self._lo()), "live_masks")
        return masks[: self.m]
