"""Python binding of the C ABI in ``include/sg.h`` (``_build/libsg.so``).

Argument marshalling only: every step of the selection path runs in the
library's CUDA kernels.  PyTorch supplies device memory (its caching
allocator is registered as the library's allocator) and streams.  The
module-level functions carry the C names; :class:`Graph` wraps a handle.

There is no CPU fallback: if the compiled library is missing or no GPU is
visible, every call raises :class:`SGError`.
"""

from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_build", "libsg.so")

SG_OK, SG_EINVAL, SG_ENOMEM, SG_ECUDA, SG_ETIMEOUT, SG_EBUSY, SG_EINTERNAL = range(7)
SG_UIC, SG_WIC, SG_UIC_UNDIRECTED, SG_LT = 0, 1, 2, 3
_STATUS = {0: "SG_OK", 1: "SG_EINVAL", 2: "SG_ENOMEM", 3: "SG_ECUDA", 4: "SG_ETIMEOUT", 5: "SG_EBUSY",
           6: "SG_EINTERNAL"}

# exported entry points, as declared in include/sg.h
EXPORTS = ("sg_workspace_create", "sg_workspace_bytes", "sg_workspace_free", "sg_select_ws", "sg_select_batch",
           "sg_batch_capture", "sg_batch_launch", "sg_batch_free", "sg_server_create", "sg_server_submit",
           "sg_server_poll", "sg_server_counts", "sg_server_destroy",
           "sg_set_allocator", "sg_set_heavy_threshold", "sg_set_engine_limits", "sg_set_landmarks",
           "sg_set_snapshot_lists", "sg_set_forward_lists", "sg_set_mask_cache", "sg_set_walk_groups", "sg_set_direction", "sg_set_scc_condensation", "sg_argmax_noalloc", "sg_load_graph", "sg_load_graph_coo", "sg_graph_info", "sg_graph_trim", "sg_select",
           "sg_select_state", "sg_init_gains", "sg_spread", "sg_select_celf", "sg_live_masks", "sg_graph_csr", "sg_free_graph", "sg_last_error", "sg_version",
           "sg_debug_inject_flags", "sg_debug_set_wait_limit", "sg_get_tuning", "sg_set_tuning", "sg_autotune")


class SGError(RuntimeError):
    def __init__(self, status, msg=""):
        self.status = status
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")


class sg_cascade(ctypes.Structure):
    _fields_ = [("model", ctypes.c_int32), ("p", ctypes.c_double)]


class sg_stats(ctypes.Structure):
    _fields_ = [("init_edges", ctypes.c_uint64), ("fwd_edges", ctypes.c_uint64), ("rev_edges", ctypes.c_uint64),
                ("init_tier2_tasks", ctypes.c_uint64), ("init_tier3_tasks", ctypes.c_uint64),
                ("rev_tier2_tasks", ctypes.c_uint64), ("rev_tier3_tasks", ctypes.c_uint64),
                ("rev_tasks", ctypes.c_uint64), ("du_entries", ctypes.c_uint64),
                ("ms_index", ctypes.c_float), ("ms_init", ctypes.c_float), ("ms_init_tier1", ctypes.c_float),
                ("ms_rounds", ctypes.c_float), ("ms_fwd", ctypes.c_float), ("ms_total", ctypes.c_float),
                ("status_flags", ctypes.c_int32), ("kernel_launches", ctypes.c_int32),
                ("heavy_index", ctypes.c_int32), ("mask_cache", ctypes.c_int32),
                ("work_keys", (ctypes.c_uint64 * 3) * 2), ("work_elems", (ctypes.c_uint64 * 3) * 2),
                ("ms_landmarks", ctypes.c_float), ("ms_init_tier2", ctypes.c_float),
                ("ms_init_tier3", ctypes.c_float), ("reserved2", ctypes.c_int32),
                ("list_elems", ctypes.c_uint64 * 3)]

    def as_dict(self):
        out = {}
        for k, _ in self._fields_:
            v = getattr(self, k)
            out[k] = [list(row) for row in v] if k.startswith("work_") else (list(v) if k == "list_elems" else v)
        return out


class sg_tuning(ctypes.Structure):
    _fields_ = [("walk_groups", ctypes.c_int32), ("direction_mode", ctypes.c_int32),
                ("direction_div", ctypes.c_int32), ("tier1_keys", ctypes.c_int32), ("tier2_keys", ctypes.c_int32),
                ("landmarks", ctypes.c_int32), ("scc", ctypes.c_int32), ("forward_lists", ctypes.c_int32),
                ("word_major", ctypes.c_int32), ("tier1_direct", ctypes.c_int32)]

    def as_dict(self):
        return {name: int(getattr(self, name)) for name, _ in self._fields_}


class sg_query(ctypes.Structure):
    _fields_ = [("graph", ctypes.c_void_p), ("ws", ctypes.c_void_p), ("R", ctypes.c_int32), ("k", ctypes.c_int32),
                ("cascade", sg_cascade), ("seed", ctypes.c_uint64), ("out_seeds", ctypes.c_void_p),
                ("out_gains", ctypes.c_void_p), ("status", ctypes.c_int),
                ("tuning", ctypes.POINTER(sg_tuning))]


class sg_server_cfg(ctypes.Structure):
    _fields_ = [("max_running", ctypes.c_int32), ("memory_budget", ctypes.c_size_t), ("k_cap", ctypes.c_int32)]


_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_RELEASE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)

_lock = threading.Lock()
_lib = None
_hooks = None


def library_path() -> str:
    return _LIB_PATH


def lib() -> ctypes.CDLL:
    """Load ``libsg.so`` (built by ``paper_1212_4779_gb300.build``)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_LIB_PATH):
            raise SGError(SG_ECUDA, f"CUDA library not built: {_LIB_PATH} is missing "
                                    "(run `python -c 'import __graft_entry__ as g; g.build()'`)")
        L = ctypes.CDLL(_LIB_PATH)
        P, i32, i64, u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
        L.sg_set_allocator.argtypes = [_ALLOC_FN, _RELEASE_FN, P]
        L.sg_set_heavy_threshold.argtypes = [i32]
        L.sg_set_engine_limits.argtypes = [i32, i32]
        L.sg_set_landmarks.argtypes = [i32]
        L.sg_set_snapshot_lists.argtypes = [i32]
        L.sg_set_mask_cache.argtypes = [i32]
        L.sg_set_forward_lists.argtypes = [i32]
        L.sg_set_walk_groups.argtypes = [i32]
        L.sg_set_direction.argtypes = [i32, i32]
        L.sg_set_scc_condensation.argtypes = [i32]
        L.sg_graph_trim.argtypes = [P]
        L.sg_debug_inject_flags.argtypes = [i32]
        L.sg_debug_set_wait_limit.argtypes = [i64]
        L.sg_get_tuning.argtypes = [ctypes.POINTER(sg_tuning)]
        L.sg_set_tuning.argtypes = [ctypes.POINTER(sg_tuning)]
        L.sg_autotune.argtypes = [P, i32, i32, sg_cascade, u64, P, ctypes.c_char_p, ctypes.POINTER(sg_tuning),
                                  ctypes.POINTER(ctypes.c_double)]
        L.sg_spread.argtypes = [P, i32, sg_cascade, u64, P, i32, P, ctypes.POINTER(i64), ctypes.POINTER(u64)]
        L.sg_select_celf.argtypes = [P, i32, i32, sg_cascade, u64, P, P, P, ctypes.POINTER(i64), P]
        L.sg_argmax_noalloc.argtypes = [P, i64, P, P, P]
        L.sg_load_graph.argtypes = [i64, i64, P, P, ctypes.c_int, P, ctypes.POINTER(P)]
        L.sg_load_graph_coo.argtypes = [i64, i64, P, P, ctypes.c_int, P, ctypes.POINTER(P)]
        L.sg_graph_info.argtypes = [P, ctypes.POINTER(i64), ctypes.POINTER(i64)]
        L.sg_select.argtypes = [P, i32, i32, sg_cascade, u64, P, P, P, ctypes.POINTER(sg_stats)]
        L.sg_select_state.argtypes = [P, i32, i32, sg_cascade, u64, P, P, P, P, P]
        L.sg_init_gains.argtypes = [P, i32, sg_cascade, u64, P, P, ctypes.POINTER(u64)]
        L.sg_live_masks.argtypes = [P, i32, sg_cascade, u64, P, P]
        L.sg_graph_csr.argtypes = [P, P, P, P]
        L.sg_free_graph.argtypes = [P]
        L.sg_free_graph.restype = None
        L.sg_workspace_create.argtypes = [P, i32, i32, P, ctypes.POINTER(P)]
        L.sg_workspace_bytes.argtypes = [P, i32, i32, ctypes.POINTER(ctypes.c_size_t)]
        L.sg_workspace_free.argtypes = [P]
        L.sg_workspace_free.restype = None
        L.sg_select_ws.argtypes = [P, P, i32, i32, sg_cascade, u64, P, P, P, ctypes.POINTER(sg_stats)]
        L.sg_select_batch.argtypes = [i32, ctypes.POINTER(sg_query), i32, P]
        L.sg_batch_capture.argtypes = [i32, ctypes.POINTER(sg_query), i32, P, ctypes.POINTER(P)]
        L.sg_batch_launch.argtypes = [P, P]
        L.sg_batch_free.argtypes = [P]
        L.sg_batch_free.restype = None
        L.sg_server_create.argtypes = [ctypes.POINTER(sg_server_cfg), ctypes.POINTER(P)]
        L.sg_server_submit.argtypes = [P, P, i32, i32, sg_cascade, u64, ctypes.POINTER(i64)]
        L.sg_server_poll.argtypes = [P, i64, ctypes.POINTER(i32), P, P, ctypes.POINTER(ctypes.c_double)]
        L.sg_server_counts.argtypes = [P, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i64)]
        L.sg_server_destroy.argtypes = [P]
        L.sg_server_destroy.restype = None
        L.sg_last_error.restype = ctypes.c_char_p
        L.sg_version.restype = ctypes.c_char_p
        for name in ("sg_workspace_create", "sg_workspace_bytes", "sg_select_ws", "sg_select_batch",
                     "sg_batch_capture", "sg_batch_launch", "sg_server_create", "sg_server_submit",
                     "sg_server_poll", "sg_server_counts", "sg_set_allocator", "sg_set_heavy_threshold", "sg_set_engine_limits", "sg_set_landmarks",
                     "sg_set_snapshot_lists", "sg_set_forward_lists", "sg_set_mask_cache", "sg_set_walk_groups", "sg_set_direction", "sg_set_scc_condensation", "sg_argmax_noalloc", "sg_load_graph", "sg_load_graph_coo", "sg_graph_info", "sg_select",
                     "sg_select_state", "sg_init_gains", "sg_spread", "sg_select_celf", "sg_live_masks", "sg_graph_csr",
                     "sg_debug_inject_flags", "sg_debug_set_wait_limit", "sg_get_tuning", "sg_set_tuning",
                     "sg_autotune"):
            getattr(L, name).restype = ctypes.c_int
        _lib = L
        return L


def _check(rc):
    if rc != SG_OK:
        raise SGError(rc, lib().sg_last_error().decode(errors="replace"))


def _require_gpu():
    import torch

    if not torch.cuda.is_available():
        raise SGError(SG_ECUDA, "no CUDA device visible; the library has no CPU path")
    return torch


def use_torch_allocator(enable: bool = True):
    """Route the library's device allocations through PyTorch's caching
    allocator (on by default once a GPU call is made)."""
    global _hooks
    L = lib()
    if not enable:
        _check(L.sg_set_allocator(_ALLOC_FN(), _RELEASE_FN(), None))
        _hooks = None
        return
    torch = _require_gpu()

    def _alloc(nbytes, stream, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))
        except Exception:  # noqa: BLE001 - reported to C as NULL (SG_ENOMEM)
            return None

    def _release(ptr, nbytes, stream, ctx):
        try:
            torch.cuda.caching_allocator_delete(int(ptr))
        except Exception:  # noqa: BLE001
            pass

    hooks = (_ALLOC_FN(_alloc), _RELEASE_FN(_release))
    _check(L.sg_set_allocator(hooks[0], hooks[1], None))
    _hooks = hooks


def _ensure_ready():
    torch = _require_gpu()
    if _hooks is None and os.environ.get("SG_TORCH_ALLOC", "1") != "0":
        use_torch_allocator(True)
    return torch


def _stream_ptr(stream):
    if stream is None:
        import torch

        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _addr(a):
    """(address, is_device) of a numpy array or torch tensor (contiguous)."""
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data, 0
    if not a.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return a.data_ptr(), int(a.is_cuda)


def _cascade(model, p):
    m = {"uic": SG_UIC, "wic": SG_WIC, "uic_undirected": SG_UIC_UNDIRECTED, "lt": SG_LT, SG_UIC: SG_UIC,
         SG_WIC: SG_WIC, SG_UIC_UNDIRECTED: SG_UIC_UNDIRECTED, SG_LT: SG_LT}[model]
    return sg_cascade(m, float(p))


# ------------------------------------------------------------- C-named calls


def sg_version() -> str:
    return lib().sg_version().decode()


def sg_last_error() -> str:
    return lib().sg_last_error().decode(errors="replace")


def sg_set_allocator(alloc=None, release=None):
    """Install Python callables ``alloc(nbytes, stream) -> int`` and
    ``release(ptr, nbytes, stream)`` as the device allocator; with no
    arguments restore the library default (cudaMallocAsync)."""
    global _hooks
    if alloc is None and release is None:
        _check(lib().sg_set_allocator(_ALLOC_FN(), _RELEASE_FN(), None))
        _hooks = None
        return
    hooks = (_ALLOC_FN(lambda nb, st, ctx: alloc(int(nb), int(st or 0))),
             _RELEASE_FN(lambda ptr, nb, st, ctx: release(int(ptr), int(nb), int(st or 0))))
    _check(lib().sg_set_allocator(hooks[0], hooks[1], None))
    _hooks = hooks


def sg_set_heavy_threshold(min_degree: int):
    """Heavy-row live-index threshold for graphs loaded afterwards (0: off)."""
    _check(lib().sg_set_heavy_threshold(int(min_degree)))


def sg_set_engine_limits(tier1_keys: int = 256, tier2_keys: int = 2048):
    """Visited-set sizes at which tasks move to the next engine tier."""
    _check(lib().sg_set_engine_limits(int(tier1_keys), int(tier2_keys)))


def sg_set_snapshot_lists(enable: int = 1):
    """Per-snapshot live in-lists of heavy rows for the reverse pass (0: off)."""
    _check(lib().sg_set_snapshot_lists(int(enable)))


def sg_set_forward_lists(enable: int = 1):
    """Forward per-snapshot live lists for sparse initial-gain expansions (0: off)."""
    _check(lib().sg_set_forward_lists(int(enable)))


def sg_set_direction(mode: int = 1, divisor: int = 4):
    """Walk levels: 0 top-down only, 1 bottom-up past n/divisor frontier nodes, 2 bottom-up after level 0."""
    _check(lib().sg_set_direction(int(mode), int(divisor)))


def sg_set_scc_condensation(enable: int = 1):
    """Initial-gain sources inside a landmark's SCC skip that snapshot's walk (0: off)."""
    _check(lib().sg_set_scc_condensation(int(enable)))


def sg_set_walk_groups(groups: int = 32):
    """Blocks per 64-snapshot word of the forward and landmark walks (8/16/32/64)."""
    _check(lib().sg_set_walk_groups(int(groups)))


def sg_set_mask_cache(enable: int = 0):
    """Live-mask cache: evaluate every arc's coins once per query (1) or hash
    in registers during the traversals (0, the default)."""
    _check(lib().sg_set_mask_cache(int(enable)))


def sg_argmax_noalloc(s, out_id, out_gain, stream=None):
    """Argmax of a device int64 gain tensor into device int32/int64 outputs
    without any allocation (for callers that cannot allocate at that
    point, e.g. while recording a CUDA graph)."""
    _check(lib().sg_argmax_noalloc(ctypes.c_void_p(_addr(s)[0]), int(s.numel()), _stream_ptr(stream),
                                   ctypes.c_void_p(_addr(out_id)[0]), ctypes.c_void_p(_addr(out_gain)[0])))


def sg_set_landmarks(count: int = 8):
    """Landmark reach sets for the initial gains (0: off, up to 8)."""
    _check(lib().sg_set_landmarks(int(count)))


def sg_load_graph(n, m, row_ptr, col, stream=None):
    """CSR load; ``row_ptr`` int64[n+1] and ``col`` int32[m] as numpy arrays
    or torch tensors (host or device).  Returns the opaque handle."""
    _ensure_ready()
    rp_a, rp_dev = _addr(row_ptr)
    col_a, col_dev = _addr(col)
    if rp_dev != col_dev:
        raise ValueError("row_ptr and col must both be host or both be device memory")
    h = ctypes.c_void_p()
    _check(lib().sg_load_graph(int(n), int(m), ctypes.c_void_p(rp_a), ctypes.c_void_p(col_a), rp_dev,
                               _stream_ptr(stream), ctypes.byref(h)))
    return h


def sg_load_graph_coo(n, m, src, dst, stream=None):
    _ensure_ready()
    s_a, s_dev = _addr(src)
    d_a, d_dev = _addr(dst)
    if s_dev != d_dev:
        raise ValueError("src and dst must both be host or both be device memory")
    h = ctypes.c_void_p()
    _check(lib().sg_load_graph_coo(int(n), int(m), ctypes.c_void_p(s_a), ctypes.c_void_p(d_a), s_dev,
                                   _stream_ptr(stream), ctypes.byref(h)))
    return h


def sg_debug_inject_flags(flags: int):
    """Testing hook: the next query plants `flags` into its device flags."""
    _check(lib().sg_debug_inject_flags(int(flags)))


def sg_get_tuning():
    t = sg_tuning()
    _check(lib().sg_get_tuning(ctypes.byref(t)))
    return t


def sg_set_tuning(t):
    _check(lib().sg_set_tuning(ctypes.byref(t)))


def sg_autotune(h, R, k, model="uic", p=0.0, seed=0, stream=None, cache_path=None):
    """Fastest knobs for one query (results unchanged); returns (sg_tuning, ms per select)."""
    t = sg_tuning()
    ms = ctypes.c_double(0.0)
    _check(lib().sg_autotune(h, int(R), int(k), _cascade(model, p), ctypes.c_uint64(seed & (2**64 - 1)),
                             _stream_ptr(stream), cache_path.encode() if cache_path else None, ctypes.byref(t),
                             ctypes.byref(ms)))
    return t, ms.value


def sg_debug_set_wait_limit(polls: int):
    """Testing hook: polls a bounded device wait makes before giving up (0: default)."""
    _check(lib().sg_debug_set_wait_limit(int(polls)))


def sg_graph_trim(h):
    """Free the graph's own workspace (the graph stays resident)."""
    _check(lib().sg_graph_trim(h))


def sg_graph_info(h):
    n, m = ctypes.c_int64(), ctypes.c_int64()
    _check(lib().sg_graph_info(h, ctypes.byref(n), ctypes.byref(m)))
    return n.value, m.value


def sg_select(h, R, k, model, p, seed, out_seeds, out_gains, stream=None, stats=False):
    """Run StaticGreedyDU; writes ``out_seeds`` (int32[k]) and ``out_gains``
    (int64[k]) (numpy or torch, host or device).  Returns stats dict or None."""
    st = sg_stats() if stats else None
    _check(lib().sg_select(h, int(R), int(k), _cascade(model, p), ctypes.c_uint64(seed & (2**64 - 1)),
                           _stream_ptr(stream), ctypes.c_void_p(_addr(out_seeds)[0]),
                           ctypes.c_void_p(_addr(out_gains)[0]), ctypes.byref(st) if stats else None))
    return st.as_dict() if stats else None


def sg_select_state(h, R, k, model, p, seed, out_seeds, out_gains, out_s, out_cov, stream=None):
    """sg_select, then Algorithm 2's state after the k rounds: ``out_s``
    (int64[n]: marginal gains of non-seeds, seeds negative) and ``out_cov``
    (uint64[ceil(R/64) * n]: coverage bits of the seeds)."""
    _check(lib().sg_select_state(h, int(R), int(k), _cascade(model, p), ctypes.c_uint64(seed & (2**64 - 1)),
                                 _stream_ptr(stream), ctypes.c_void_p(_addr(out_seeds)[0]),
                                 ctypes.c_void_p(_addr(out_gains)[0]), ctypes.c_void_p(_addr(out_s)[0]),
                                 ctypes.c_void_p(_addr(out_cov)[0])))


def sg_init_gains(h, R, model, p, seed, out_s, stream=None, want_edges=False):
    ed = ctypes.c_uint64(0)
    _check(lib().sg_init_gains(h, int(R), _cascade(model, p), ctypes.c_uint64(seed & (2**64 - 1)),
                               _stream_ptr(stream), ctypes.c_void_p(_addr(out_s)[0]),
                               ctypes.byref(ed) if want_edges else None))
    return ed.value if want_edges else None


def sg_select_celf(h, R, k, model, p, seed, out_seeds, out_gains, stream=None, stats=False):
    """StaticGreedyCELF: same outputs as sg_select; returns (evaluations,
    stats dict or None)."""
    st = sg_stats() if stats else None
    ev = ctypes.c_int64(0)
    _check(lib().sg_select_celf(h, int(R), int(k), _cascade(model, p), ctypes.c_uint64(seed & (2**64 - 1)),
                                _stream_ptr(stream), ctypes.c_void_p(_addr(out_seeds)[0]),
                                ctypes.c_void_p(_addr(out_gains)[0]), ctypes.byref(ev),
                                ctypes.byref(st) if stats else None))
    return ev.value, (st.as_dict() if stats else None)


def sg_spread(h, R, model, p, seed, S, stream=None):
    """(sum_r |R(G'_r, S)|, snapshot-edge count) over R snapshots of hash
    seed ``seed``; S is any int sequence, numpy or torch (host or device)."""
    if not hasattr(S, "data_ptr"):
        S = np.ascontiguousarray(np.asarray(S, dtype=np.int32))
    total = ctypes.c_int64(0)
    edges = ctypes.c_uint64(0)
    n_s = int(S.numel() if hasattr(S, "numel") else S.size)
    _check(lib().sg_spread(h, int(R), _cascade(model, p), ctypes.c_uint64(seed & (2**64 - 1)),
                           ctypes.c_void_p(_addr(S)[0] if n_s else 0), n_s, _stream_ptr(stream),
                           ctypes.byref(total), ctypes.byref(edges)))
    return total.value, edges.value


def sg_live_masks(h, R, model, p, seed, out_masks, stream=None):
    _check(lib().sg_live_masks(h, int(R), _cascade(model, p), ctypes.c_uint64(seed & (2**64 - 1)),
                               _stream_ptr(stream), ctypes.c_void_p(_addr(out_masks)[0])))


def sg_graph_csr(h, row_ptr, col, stream=None):
    _check(lib().sg_graph_csr(h, _stream_ptr(stream), ctypes.c_void_p(_addr(row_ptr)[0]),
                              ctypes.c_void_p(_addr(col)[0])))


def sg_free_graph(h):
    if h:
        lib().sg_free_graph(h)


def sg_workspace_create(h, R_max, k_max, stream=None):
    w = ctypes.c_void_p()
    _check(lib().sg_workspace_create(h, int(R_max), int(k_max), _stream_ptr(stream), ctypes.byref(w)))
    return w


def sg_workspace_bytes(h, R_max, k_max):
    b = ctypes.c_size_t()
    _check(lib().sg_workspace_bytes(h, int(R_max), int(k_max), ctypes.byref(b)))
    return b.value


def sg_workspace_free(w):
    if w:
        lib().sg_workspace_free(w)


def sg_select_ws(h, w, R, k, model, p, seed, out_seeds, out_gains, stream=None, stats=False):
    st = sg_stats() if stats else None
    _check(lib().sg_select_ws(h, w, int(R), int(k), _cascade(model, p), ctypes.c_uint64(seed & (2**64 - 1)),
                              _stream_ptr(stream), ctypes.c_void_p(_addr(out_seeds)[0]),
                              ctypes.c_void_p(_addr(out_gains)[0]), ctypes.byref(st) if stats else None))
    return st.as_dict() if stats else None


def _queries(items):
    """items: (graph handle, workspace or None, R, k, model, p, seed, seeds_out, gains_out[, sg_tuning])."""
    arr = (sg_query * len(items))()
    keep = []
    for i, it in enumerate(items):
        h, w, R, k, model, p, seed, so, go = it[:9]
        tun = it[9] if len(it) > 9 else None
        arr[i] = sg_query(h, w, int(R), int(k), _cascade(model, p), ctypes.c_uint64(seed & (2**64 - 1)),
                          ctypes.c_void_p(_addr(so)[0]), ctypes.c_void_p(_addr(go)[0]), 0,
                          ctypes.pointer(tun) if tun is not None else None)
        keep.append(tun)
    arr._tunings = keep  # alive as long as the array
    return arr


def sg_select_batch(items, concurrency=8, stream=None):
    """Run a batch of queries concurrently; returns the per-query statuses."""
    arr = _queries(items)
    rc = lib().sg_select_batch(len(items), arr, int(concurrency), _stream_ptr(stream))
    _check(rc)
    return [arr[i].status for i in range(len(items))]


def sg_batch_capture(items, concurrency=8, stream=None):
    arr = _queries(items)
    b = ctypes.c_void_p()
    _check(lib().sg_batch_capture(len(items), arr, int(concurrency), _stream_ptr(stream), ctypes.byref(b)))
    return b


def sg_batch_launch(b, stream=None):
    _check(lib().sg_batch_launch(b, _stream_ptr(stream)))


def sg_batch_free(b):
    if b:
        lib().sg_batch_free(b)


def sg_server_create(max_running=8, memory_budget=0, k_cap=128):
    _ensure_ready()
    cfg = sg_server_cfg(int(max_running), int(memory_budget), int(k_cap))
    sv = ctypes.c_void_p()
    _check(lib().sg_server_create(ctypes.byref(cfg), ctypes.byref(sv)))
    return sv


def sg_server_submit(sv, h, R, k, model, p, seed):
    rid = ctypes.c_int64()
    _check(lib().sg_server_submit(sv, h, int(R), int(k), _cascade(model, p), ctypes.c_uint64(seed & (2**64 - 1)),
                                  ctypes.byref(rid)))
    return rid.value


def sg_server_poll(sv, rid, k):
    """(done, seeds, gains, latency_ms); seeds/gains None while pending."""
    done = ctypes.c_int32()
    lat = ctypes.c_double()
    seeds = np.zeros(k, dtype=np.int32)
    gains = np.zeros(k, dtype=np.int64)
    _check(lib().sg_server_poll(sv, int(rid), ctypes.byref(done), ctypes.c_void_p(seeds.ctypes.data),
                                ctypes.c_void_p(gains.ctypes.data), ctypes.byref(lat)))
    if not done.value:
        return False, None, None, None
    return True, seeds, gains, lat.value


def sg_server_counts(sv):
    q, r, f = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(lib().sg_server_counts(sv, ctypes.byref(q), ctypes.byref(r), ctypes.byref(f)))
    return q.value, r.value, f.value


def sg_server_destroy(sv):
    if sv:
        lib().sg_server_destroy(sv)


# --------------------------------------------------------------- convenience


@dataclass
class Selection:
    seeds: np.ndarray
    gains: np.ndarray
    stats: dict | None


class Graph:
    """A graph resident on the GPU (wraps an ``sg_graph`` handle)."""

    def __init__(self, handle):
        self._h = handle
        self.n, self.m = sg_graph_info(handle)

    @classmethod
    def from_coo(cls, n, src, dst, stream=None):
        src = np.ascontiguousarray(src, dtype=np.int32) if isinstance(src, np.ndarray) else src
        dst = np.ascontiguousarray(dst, dtype=np.int32) if isinstance(dst, np.ndarray) else dst
        return cls(sg_load_graph_coo(n, len(src), src, dst, stream))

    @classmethod
    def from_csr(cls, n, row_ptr, col, stream=None):
        row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64) if isinstance(row_ptr, np.ndarray) else row_ptr
        col = np.ascontiguousarray(col, dtype=np.int32) if isinstance(col, np.ndarray) else col
        return cls(sg_load_graph(n, len(col), row_ptr, col, stream))

    @property
    def handle(self):
        return self._h

    def select(self, R, k, model="uic", p=0.0, seed=0, stream=None, stats=False):
        """Seeds and integer gains (numpy, host) of StaticGreedyDU."""
        seeds = np.zeros(k, dtype=np.int32)
        gains = np.zeros(k, dtype=np.int64)
        st = sg_select(self._h, R, k, model, p, seed, seeds, gains, stream, stats)
        return Selection(seeds, gains, st)

    def select_state(self, R, k, model="uic", p=0.0, seed=0, stream=None):
        """(Selection, s int64[n], cov uint64[W, n]) after the k rounds."""
        W = (R + 63) // 64
        seeds = np.zeros(k, dtype=np.int32)
        gains = np.zeros(k, dtype=np.int64)
        s = np.zeros(self.n, dtype=np.int64)
        cov = np.zeros((W, self.n), dtype=np.uint64)
        sg_select_state(self._h, R, k, model, p, seed, seeds, gains, s, cov, stream)
        return Selection(seeds, gains, None), s, cov

    def init_gains(self, R, model="uic", p=0.0, seed=0, stream=None):
        s = np.zeros(self.n, dtype=np.int64)
        edges = sg_init_gains(self._h, R, model, p, seed, s, stream, want_edges=True)
        return s, edges

    def select_celf(self, R, k, model="uic", p=0.0, seed=0, stream=None, stats=False):
        """StaticGreedyCELF; returns (Selection, evaluations)."""
        seeds = np.zeros(k, dtype=np.int32)
        gains = np.zeros(k, dtype=np.int64)
        ev, st = sg_select_celf(self._h, R, k, model, p, seed, seeds, gains, stream, stats)
        return Selection(seeds, gains, st), ev

    def trim(self):
        """Release the device memory of this graph's own workspace."""
        sg_graph_trim(self._h)

    def spread(self, R, model, p, seed, S, stream=None):
        """(sum_r |R(G'_r, S)|, snapshot-edge count) on R fresh snapshots."""
        return sg_spread(self._h, R, model, p, seed, S, stream)

    def live_masks(self, R, model="uic", p=0.0, seed=0, stream=None):
        W = (R + 63) // 64
        out = np.zeros((max(1, self.m), W), dtype=np.uint64)
        sg_live_masks(self._h, R, model, p, seed, out, stream)
        return out[: self.m]

    def csr(self):
        rp = np.zeros(self.n + 1, dtype=np.int64)
        col = np.zeros(max(1, self.m), dtype=np.int32)
        sg_graph_csr(self._h, rp, col)
        return rp, col[: self.m]

    def close(self):
        if self._h:
            sg_free_graph(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
