"""Thin Python binding of the GRNND C ABI (include/grnnd.h).

Argument marshalling only: every step of the build and the search runs in the
CUDA kernels of ``libgrnnd.so``.  PyTorch supplies device memory and the
current stream.  When the library is missing the calls raise; there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "libgrnnd.so")
HEADER = os.path.join(os.path.dirname(_PKG), "include", "grnnd.h")

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, EBUSY = 0, -1, -2, -3, -4, -5
L2SQ, IP = 0, 1
FP32, BF16, FP8 = 0, 1, 2
ORDER_RANDOM, ORDER_ASC, ORDER_DESC = 0, 1, 2
EMPTY = 0xFFFFFFFFFFFFFFFF

_lock = threading.Lock()
_lib = None


class GrnndError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"grnnd status {status}: {msg}")
        self.status = status


class Tuning(ctypes.Structure):
    """grnnd_tuning: lane-group routing by pool size and CTAs-per-SM caps of the join."""
    _fields_ = [("group_max", ctypes.c_int32 * 3), ("warp_ctas_per_sm", ctypes.c_int32),
                ("team_ctas_per_sm", ctypes.c_int32), ("row_copies", ctypes.c_int32), ("ms", ctypes.c_float)]

    def as_dict(self):
        return {"group_max": list(self.group_max), "warp_ctas_per_sm": self.warp_ctas_per_sm,
                "team_ctas_per_sm": self.team_ctas_per_sm, "row_copies": self.row_copies, "ms": self.ms}


def tuning(group_max=(8, 16, 32), warp_ctas_per_sm=0, team_ctas_per_sm=0, row_copies=0) -> Tuning:
    t = Tuning()
    for c in range(3):
        t.group_max[c] = group_max[c]
    t.warp_ctas_per_sm, t.team_ctas_per_sm, t.row_copies = warp_ctas_per_sm, team_ctas_per_sm, row_copies
    return t


class Params(ctypes.Structure):
    _fields_ = [("S", ctypes.c_int32), ("R", ctypes.c_int32), ("T1", ctypes.c_int32), ("T2", ctypes.c_int32),
                ("rho", ctypes.c_float), ("seed", ctypes.c_uint64), ("metric", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("order", ctypes.c_int32), ("final_prune", ctypes.c_int32),
                ("stream", ctypes.c_void_p), ("hbm_budget", ctypes.c_uint64), ("tuning", ctypes.POINTER(Tuning))]


class KernelTime(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int64), ("ms", ctypes.c_double)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_int32), ("hbm_budget", ctypes.c_uint64), ("max_batch_queries", ctypes.c_int64)]


class RequestInfo(ctypes.Structure):
    _fields_ = [("id", ctypes.c_int64), ("kind", ctypes.c_int32), ("state", ctypes.c_int32),
                ("status", ctypes.c_int32), ("batch", ctypes.c_int32), ("index", ctypes.c_int64),
                ("units", ctypes.c_int64), ("bytes", ctypes.c_uint64), ("t_submit", ctypes.c_double),
                ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double), ("message", ctypes.c_char * 128)]

    def as_dict(self):
        return {"id": self.id, "kind": ("build", "search")[self.kind], "state": self.state, "status": self.status,
                "batch": self.batch, "index": self.index, "units": self.units, "bytes": self.bytes,
                "t_submit": self.t_submit, "t_admit": self.t_admit, "t_done": self.t_done,
                "message": self.message.decode(errors="replace")}


_SIGS = {
    "grnnd_profile_begin": (ctypes.c_int, []),
    "grnnd_profile_begin_only": (ctypes.c_int, [ctypes.c_char_p]),
    "grnnd_profile_end": (ctypes.c_int, [ctypes.POINTER(KernelTime), ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]),
    # name: (restype, argtypes)
    "grnnd_params_default": (None, [ctypes.POINTER(Params)]),
    "grnnd_build": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                   ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64,
                                   ctypes.POINTER(ctypes.c_void_p)]),
    "grnnd_build_ex": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.POINTER(Params),
                                      ctypes.POINTER(ctypes.c_void_p)]),
    "grnnd_search": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                    ctypes.c_void_p]),
    "grnnd_graph_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32),
                                        ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]),
    "grnnd_graph_view": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p),
                                        ctypes.POINTER(ctypes.c_void_p)]),
    "grnnd_graph_copy": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "grnnd_graph_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32]),
    "grnnd_free": (None, [ctypes.c_void_p]),
    "grnnd_last_error": (ctypes.c_char_p, []),
    "grnnd_pool_init": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                       ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_void_p]),
    "grnnd_workspace_size": (ctypes.c_size_t, [ctypes.c_int64, ctypes.c_int32]),
    "grnnd_join_round": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                        ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int32,
                                        ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p]),
    "grnnd_quantized_size": (ctypes.c_size_t, [ctypes.c_int64, ctypes.c_int32, ctypes.c_int32]),
    "grnnd_quantize": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                      ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    "grnnd_join_round_q": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                          ctypes.c_int32, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int32,
                                          ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int32,
                                          ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p]),
    "grnnd_final_prune_q": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                           ctypes.c_int32, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int32,
                                           ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int32,
                                           ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_size_t, ctypes.c_void_p]),
    "grnnd_set_stream": (None, [ctypes.c_void_p]),
    "grnnd_get_stream": (ctypes.c_void_p, []),
    "grnnd_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p,
                                      ctypes.c_int32, ctypes.POINTER(Params), ctypes.POINTER(Tuning)]),
    "grnnd_autotune_pool": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int64,
                                           ctypes.POINTER(Params), ctypes.c_void_p, ctypes.c_int32, ctypes.c_float,
                                           ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                                           ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float)]),
    "grnnd_build_batch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                         ctypes.c_void_p, ctypes.c_void_p]),
    "grnnd_workspace_status": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int64, ctypes.c_int32,
                                              ctypes.c_void_p]),
    "grnnd_reverse_sample": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int32, ctypes.c_float, ctypes.c_void_p,
                                            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p]),
    "grnnd_final_prune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                         ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int32,
                                         ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                         ctypes.c_void_p]),
    "grnnd_pair_dist": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                       ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]),
    "grnnd_entry_workspace_size": (ctypes.c_size_t, [ctypes.c_int64, ctypes.c_int32]),
    "grnnd_entry_point": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                         ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    "grnnd_entry_point_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                                 ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]),
    "grnnd_search_graph": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                          ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                          ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_void_p]),
    "grnnd_brute_knn": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                       ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_void_p]),
    "grnnd_keys_to_graph": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_void_p, ctypes.c_void_p]),
    "grnnd_server_create": (ctypes.c_int, [ctypes.POINTER(ServerConfig), ctypes.POINTER(ctypes.c_void_p)]),
    "grnnd_server_submit_build": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                                 ctypes.POINTER(Params), ctypes.POINTER(ctypes.c_int64)]),
    "grnnd_server_submit_search": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64,
                                                  ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                                  ctypes.POINTER(ctypes.c_int64)]),
    "grnnd_server_wait": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_double,
                                         ctypes.POINTER(RequestInfo)]),
    "grnnd_server_index": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(ctypes.c_void_p)]),
    "grnnd_server_release": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64]),
    "grnnd_server_status": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint64),
                                           ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_int32),
                                           ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]),
    "grnnd_server_destroy": (None, [ctypes.c_void_p]),
    "grnnd_set_memory_cache": (ctypes.c_int, [ctypes.c_uint64]),
    "grnnd_selftest_bounded_wait": (ctypes.c_int, [ctypes.c_uint32, ctypes.c_void_p]),
}


def lib(path: str | None = None):
    """Loads libgrnnd.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None and path is None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"{p} is missing: build it with `python -m paper_2510_02774_gb300.build`")
        L = ctypes.CDLL(p)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        if path is None:
            _lib = L
        return L


def _check(rc: int):
    if rc != OK:
        msg = lib().grnnd_last_error()
        raise GrnndError(rc, msg.decode() if msg else "")


# ---------------------------------------------------------------------------------------
# torch helpers (device memory and streams only)
# ---------------------------------------------------------------------------------------

def profile_begin(only=None):
    """Starts per-kernel CUDA-event timing of this thread's library launches; `only` (a list
    of kernel names) limits the timing to those kernels."""
    if only:
        _check(lib().grnnd_profile_begin_only(",".join(only).encode()))
    else:
        _check(lib().grnnd_profile_begin())


def profile_end() -> dict:
    """Stops timing; returns {kernel name: (launches, total ms)}."""
    buf = (KernelTime * 64)()
    n = ctypes.c_int32()
    _check(lib().grnnd_profile_end(buf, 64, ctypes.byref(n)))
    return {buf[i].name.decode(): (int(buf[i].launches), float(buf[i].ms)) for i in range(min(n.value, 64))}


def _torch():
    import torch
    return torch


def _stream_ptr(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t) -> ctypes.c_void_p:
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def device_points(X, device="cuda"):
    """Copies points (numpy or torch, n x d float32) into a device tensor of shape
    (n, ld) with ld = d rounded up to 4 and zero padding.  Returns (tensor, d)."""
    torch = _torch()
    Xt = torch.as_tensor(np.ascontiguousarray(X, dtype=np.float32)) if isinstance(X, np.ndarray) else X
    n, d = Xt.shape
    ld = (d + 3) & ~3
    out = torch.zeros((n, ld), dtype=torch.float32, device=device)
    out[:, :d] = Xt.to(device=device, dtype=torch.float32)
    return out, d


def workspace(n: int, R: int, device="cuda"):
    torch = _torch()
    nb = int(lib().grnnd_workspace_size(n, R))
    return torch.empty(nb, dtype=torch.uint8, device=device)


# ---------------------------------------------------------------------------------------
# Whole build and search
# ---------------------------------------------------------------------------------------

@dataclass
class Graph:
    handle: ctypes.c_void_p
    n: int
    d: int
    R: int
    entry: int

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            try:
                lib().grnnd_free(h)
            except Exception:
                pass
            self.handle = ctypes.c_void_p(0)

    def to_numpy(self):
        """(ids n x R int32 -1 padded, dists n x R float32, deg n int32) on the host."""
        ids = np.empty((self.n, self.R), np.int32)
        dists = np.empty((self.n, self.R), np.float32)
        deg = np.empty(self.n, np.int32)
        _check(lib().grnnd_graph_copy(self.handle, ids.ctypes.data_as(ctypes.c_void_p),
                                      dists.ctypes.data_as(ctypes.c_void_p), deg.ctypes.data_as(ctypes.c_void_p)))
        return ids, dists, deg

    def stats(self):
        out = np.zeros(8, np.int64)
        lib().grnnd_graph_stats(self.handle, out.ctypes.data_as(ctypes.c_void_p), 8)
        keys = ["rounds", "vertices_with_new", "rows_gathered", "pair_distances", "pairs_fired", "proposals",
                "merged", "rechecks"]
        return dict(zip(keys, out.tolist()))

    def search(self, queries, k: int = 10, beam: int = 64):
        """Candidate-list search; queries numpy (host) or torch (host or device)."""
        return search(self, queries, k, beam)


def set_memory_cache(nbytes: int) -> None:
    """grnnd_set_memory_cache: keep up to nbytes of freed build memory on the current device
    for the next build (0 turns the cache off and releases it)."""
    _check(lib().grnnd_set_memory_cache(int(nbytes)))


def params(S=16, R=32, T1=4, T2=8, rho=0.6, seed=0, metric=L2SQ, precision=FP32, order=ORDER_RANDOM,
           final_prune=True, stream=None, hbm_budget=0, tuning=None) -> Params:
    p = Params()
    lib().grnnd_params_default(ctypes.byref(p))
    p.S, p.R, p.T1, p.T2, p.rho, p.seed = S, R, T1, T2, rho, seed
    p.metric, p.precision, p.order, p.final_prune = metric, precision, order, int(bool(final_prune))
    p.stream = stream
    p.hbm_budget = hbm_budget
    if tuning is not None:
        p.tuning = ctypes.pointer(tuning)
    return p


def build(points, S=16, R=32, T1=4, T2=8, rho=0.6, seed=0, metric=L2SQ, precision=FP32, order=ORDER_RANDOM,
          final_prune=True, stream=None, hbm_budget=0, tuning=None) -> Graph:
    """grnnd_build_ex on numpy (host) or torch (host or device) points of shape (n, d).
    With torch CUDA points the build runs on the current torch stream."""
    if isinstance(points, np.ndarray):
        pts = np.ascontiguousarray(points, dtype=np.float32)
        ptr = pts.ctypes.data_as(ctypes.c_void_p)
        st = None
    else:
        pts = points.contiguous()
        ptr = ctypes.c_void_p(pts.data_ptr())
        st = _stream_ptr(stream).value if pts.is_cuda else None
    n, d = pts.shape
    p = params(S, R, T1, T2, rho, seed, metric, precision, order, final_prune, st, hbm_budget, tuning)
    h = ctypes.c_void_p()
    _check(lib().grnnd_build_ex(ptr, n, d, ctypes.byref(p), ctypes.byref(h)))
    n_, d_, R_, e_ = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(lib().grnnd_graph_info(h, ctypes.byref(n_), ctypes.byref(d_), ctypes.byref(R_), ctypes.byref(e_)))
    return Graph(h, n_.value, d_.value, R_.value, e_.value)


def _graph_of(h) -> Graph:
    n_, d_, R_, e_ = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(lib().grnnd_graph_info(h, ctypes.byref(n_), ctypes.byref(d_), ctypes.byref(R_), ctypes.byref(e_)))
    return Graph(h, n_.value, d_.value, R_.value, e_.value)


def build_batch(points, offsets, S=16, R=32, T1=4, T2=8, rho=0.6, seed=0, metric=L2SQ, precision=FP32,
                order=ORDER_RANDOM, final_prune=True, stream=None, hbm_budget=0, tuning=None) -> list:
    """grnnd_build_batch: independent builds of the row ranges [offsets[b], offsets[b+1]) of
    `points` (numpy or torch, shape (n, d)) in one pass; returns one Graph per build."""
    if isinstance(points, np.ndarray):
        pts = np.ascontiguousarray(points, dtype=np.float32)
        ptr = pts.ctypes.data_as(ctypes.c_void_p)
        st = None
    else:
        pts = points.contiguous()
        ptr = ctypes.c_void_p(pts.data_ptr())
        st = _stream_ptr(stream).value if pts.is_cuda else None
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    nb = len(off) - 1
    p = params(S, R, T1, T2, rho, seed, metric, precision, order, final_prune, st, hbm_budget, tuning)
    hs = (ctypes.c_void_p * nb)()
    _check(lib().grnnd_build_batch(ptr, off.ctypes.data_as(ctypes.c_void_p), nb, pts.shape[1], ctypes.byref(p),
                                   ctypes.cast(hs, ctypes.c_void_p)))
    return [_graph_of(ctypes.c_void_p(hs[b])) for b in range(nb)]


def autotune(points, S=16, R=32, T1=4, T2=8, rho=0.6, seed=0, metric=L2SQ, precision=FP32, order=ORDER_RANDOM,
             final_prune=True, stream=None, offsets=None) -> Tuning:
    """grnnd_autotune on a sample of the workload (numpy or torch rows; with offsets, a batch
    of builds); returns the Tuning."""
    if isinstance(points, np.ndarray):
        pts = np.ascontiguousarray(points, dtype=np.float32)
        ptr = pts.ctypes.data_as(ctypes.c_void_p)
        st = None
    else:
        pts = points.contiguous()
        ptr = ctypes.c_void_p(pts.data_ptr())
        st = _stream_ptr(stream).value if pts.is_cuda else None
    p = params(S, R, T1, T2, rho, seed, metric, precision, order, final_prune, st)
    t = Tuning()
    off = None if offsets is None else np.ascontiguousarray(offsets, dtype=np.int64)
    _check(lib().grnnd_autotune(ptr, pts.shape[0], pts.shape[1],
                                None if off is None else off.ctypes.data_as(ctypes.c_void_p),
                                0 if off is None else len(off) - 1, ctypes.byref(p), ctypes.byref(t)))
    return t


def autotune_pool(points, nq: int, candidates, recall_target: float = 0.95, k: int = 10, beam: int = 64,
                  S=16, R=32, T1=4, T2=8, rho=0.6, seed=0, metric=L2SQ, precision=FP32, order=ORDER_RANDOM,
                  final_prune=True, stream=None, tuning=None):
    """grnnd_autotune_pool: the pool capacity R among `candidates` for builds like this one
    (the last nq rows of `points` are the held-out queries); returns (R, recall, build ms)."""
    if isinstance(points, np.ndarray):
        pts = np.ascontiguousarray(points, dtype=np.float32)
        ptr = pts.ctypes.data_as(ctypes.c_void_p)
        st = None
    else:
        pts = points.contiguous()
        ptr = ctypes.c_void_p(pts.data_ptr())
        st = _stream_ptr(stream).value if pts.is_cuda else None
    p = params(S, R, T1, T2, rho, seed, metric, precision, order, final_prune, st, 0, tuning)
    cand = np.ascontiguousarray(candidates, dtype=np.int32)
    r, rec, ms = ctypes.c_int32(), ctypes.c_float(), ctypes.c_float()
    _check(lib().grnnd_autotune_pool(ptr, pts.shape[0], pts.shape[1], nq, ctypes.byref(p),
                                     cand.ctypes.data_as(ctypes.c_void_p), len(cand), recall_target, k, beam,
                                     ctypes.byref(r), ctypes.byref(rec), ctypes.byref(ms)))
    return r.value, rec.value, ms.value


def search(graph: Graph, queries, k: int = 10, beam: int = 64):
    if isinstance(queries, np.ndarray):
        q = np.ascontiguousarray(queries, dtype=np.float32)
        out = np.empty((q.shape[0], k), np.int32)
        _check(lib().grnnd_search(graph.handle, q.ctypes.data_as(ctypes.c_void_p), q.shape[0], k, beam,
                                  out.ctypes.data_as(ctypes.c_void_p)))
        return out
    torch = _torch()
    q = queries.contiguous().to(torch.float32)
    out = torch.empty((q.shape[0], k), dtype=torch.int32, device=q.device)
    L = lib()
    prev = L.grnnd_get_stream()
    if q.is_cuda:  # the search runs on the current torch stream
        L.grnnd_set_stream(_stream_ptr())
    try:
        _check(L.grnnd_search(graph.handle, _ptr(q), q.shape[0], k, beam, _ptr(out)))
    finally:
        L.grnnd_set_stream(prev)
    return out


# ---------------------------------------------------------------------------------------
# Step-level calls on torch device tensors (X is (n, ld) float32 from device_points)
# ---------------------------------------------------------------------------------------

def pool_init(X, d: int, S: int, R: int, seed: int, metric: int = L2SQ, stream=None):
    torch = _torch()
    n, ld = X.shape
    keys = torch.empty((n, R), dtype=torch.int64, device=X.device)
    deg = torch.empty(n, dtype=torch.int32, device=X.device)
    _check(lib().grnnd_pool_init(_ptr(X), n, d, ld, metric, S, R, seed, _ptr(keys), _ptr(deg), _stream_ptr(stream)))
    return keys, deg


def quantize(X, d: int, precision: int, stream=None):
    """Quantized copy of device points X (n x ld) for the BF16 / FP8 step calls (a uint8 tensor)."""
    torch = _torch()
    n, ld = X.shape
    nb = lib().grnnd_quantized_size(n, d, precision)
    if nb == 0:
        raise GrnndError(EINVAL, "precision must be BF16 or FP8")
    q = torch.empty(nb + 256, dtype=torch.uint8, device=X.device)
    off = (-q.data_ptr()) % 256
    q = q[off:off + nb]
    _check(lib().grnnd_quantize(_ptr(X), n, d, ld, precision, _ptr(q), nb, _stream_ptr(stream)))
    return q


def join_round(X, d: int, keys, deg, seed: int, t1: int, t2: int, order: int = ORDER_RANDOM, metric: int = L2SQ,
               ws=None, stats=None, stream=None, inplace: bool = False, precision: int = FP32, qpoints=None):
    """One round; with inplace=True the pool tensors are updated and returned.  In the BF16 /
    FP8 forms `qpoints` is the copy from quantize(X, d, precision)."""
    torch = _torch()
    n, ld = X.shape
    R = keys.shape[1]
    ws = workspace(n, R, X.device) if ws is None else ws
    k2 = keys if inplace else torch.empty_like(keys)
    d2 = deg if inplace else torch.empty_like(deg)
    qn = 0 if qpoints is None else qpoints.numel()
    _check(lib().grnnd_join_round_q(_ptr(X), n, d, ld, metric, precision, _ptr(qpoints), qn, R, _ptr(keys), _ptr(deg),
                                    seed, t1, t2, order, _ptr(k2), _ptr(d2), _ptr(ws), ws.numel(), _ptr(stats),
                                    _stream_ptr(stream)))
    return k2, d2


def reverse_sample(keys, deg, rho: float, ws=None, stats=None, stream=None, inplace: bool = False):
    torch = _torch()
    n, R = keys.shape
    ws = workspace(n, R, keys.device) if ws is None else ws
    k2 = keys if inplace else torch.empty_like(keys)
    d2 = deg if inplace else torch.empty_like(deg)
    _check(lib().grnnd_reverse_sample(n, R, ctypes.c_float(rho), _ptr(keys), _ptr(deg), _ptr(k2), _ptr(d2), _ptr(ws),
                                      ws.numel(), _ptr(stats), _stream_ptr(stream)))
    return k2, d2


def workspace_status(ws, n: int, R: int, stream=None) -> None:
    """Raise GrnndError if a device-side wait of the last step on `ws` gave up (synchronises)."""
    _check(lib().grnnd_workspace_status(_ptr(ws), ws.numel(), n, R, _stream_ptr(stream)))


def final_prune(X, d: int, keys, deg, seed: int, t1: int, order: int = ORDER_RANDOM, metric: int = L2SQ, ws=None,
                stream=None, precision: int = FP32, qpoints=None):
    torch = _torch()
    n, ld = X.shape
    R = keys.shape[1]
    ws = workspace(n, R, X.device) if ws is None else ws
    k2 = torch.empty_like(keys)
    d2 = torch.empty_like(deg)
    qn = 0 if qpoints is None else qpoints.numel()
    _check(lib().grnnd_final_prune_q(_ptr(X), n, d, ld, metric, precision, _ptr(qpoints), qn, R, _ptr(keys),
                                     _ptr(deg), seed, t1, order, _ptr(k2), _ptr(d2), _ptr(ws), ws.numel(),
                                     _stream_ptr(stream)))
    return k2, d2


def pair_dist(X, d: int, pairs, metric: int = L2SQ, stream=None):
    torch = _torch()
    n, ld = X.shape
    pairs = pairs.to(device=X.device, dtype=torch.int32).contiguous()
    out = torch.empty(pairs.shape[0], dtype=torch.float32, device=X.device)
    _check(lib().grnnd_pair_dist(_ptr(X), n, d, ld, metric, _ptr(pairs), pairs.shape[0], _ptr(out), _stream_ptr(stream)))
    return out


def entry_point(X, d: int, metric: int = L2SQ, stream=None) -> int:
    torch = _torch()
    n, ld = X.shape
    ws = torch.empty(int(lib().grnnd_entry_workspace_size(n, d)), dtype=torch.uint8, device=X.device)
    e = torch.empty(1, dtype=torch.int32, device=X.device)
    _check(lib().grnnd_entry_point(_ptr(X), n, d, ld, metric, _ptr(e), _ptr(ws), ws.numel(), _stream_ptr(stream)))
    return int(e.item())


def entry_point_noalloc(X, d: int, metric: int = L2SQ, out=None, stream=None) -> int:
    """Search entry computed with the library's fixed device scratch (no allocation by
    the library; `out` may be a caller-provided device int32 tensor of one element)."""
    torch = _torch()
    n, ld = X.shape
    e = torch.empty(1, dtype=torch.int32, device=X.device) if out is None else out
    _check(lib().grnnd_entry_point_noalloc(_ptr(X), n, d, ld, metric, _ptr(e), _stream_ptr(stream)))
    return int(e.item())


def search_graph(X, d: int, gids, gdeg, entry: int, Q, k: int, beam: int, metric: int = L2SQ, stream=None):
    torch = _torch()
    n, ld = X.shape
    R = gids.shape[1]
    nq, ldq = Q.shape
    ids = torch.empty((nq, k), dtype=torch.int32, device=X.device)
    dd = torch.empty((nq, k), dtype=torch.float32, device=X.device)
    _check(lib().grnnd_search_graph(_ptr(X), n, d, ld, metric, _ptr(gids), _ptr(gdeg), R, entry, _ptr(Q), nq, ldq, k,
                                    beam, _ptr(ids), _ptr(dd), _stream_ptr(stream)))
    return ids, dd


def brute_knn(X, d: int, Q, k: int, metric: int = L2SQ, stream=None):
    torch = _torch()
    n, ld = X.shape
    nq, ldq = Q.shape
    ids = torch.empty((nq, k), dtype=torch.int32, device=X.device)
    dd = torch.empty((nq, k), dtype=torch.float32, device=X.device)
    _check(lib().grnnd_brute_knn(_ptr(X), n, d, ld, metric, _ptr(Q), nq, ldq, k, _ptr(ids), _ptr(dd),
                                 _stream_ptr(stream)))
    return ids, dd


def keys_to_graph(keys):
    torch = _torch()
    n, R = keys.shape
    ids = torch.empty((n, R), dtype=torch.int32, device=keys.device)
    dd = torch.empty((n, R), dtype=torch.float32, device=keys.device)
    _check(lib().grnnd_keys_to_graph(n, R, _ptr(keys), _ptr(ids), _ptr(dd), _stream_ptr()))
    return ids, dd


# ---------------------------------------------------------------------------------------
# Host-side decoding of pool keys (for comparisons in tests and reports)
# ---------------------------------------------------------------------------------------

def decode_keys(keys) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """keys (n, R) int64/uint64 -> (ids int32 -1 for empty, dist float32, old uint8)."""
    k = np.asarray(keys).view(np.uint64) if np.asarray(keys).dtype != np.uint64 else np.asarray(keys)
    empty = k == np.uint64(EMPTY)
    ob = (k >> np.uint64(32)).astype(np.uint32)
    neg = (ob & np.uint32(0x80000000)) == 0
    bits = np.where(neg, ~ob, ob & np.uint32(0x7FFFFFFF)).astype(np.uint32)
    dist = bits.view(np.float32)
    ids = ((k >> np.uint64(1)) & np.uint64(0x7FFFFFFF)).astype(np.int32)
    old = (k & np.uint64(1)).astype(np.uint8)
    ids[empty] = -1
    dist = np.where(empty, np.float32(np.inf), dist).astype(np.float32)
    old[empty] = 0
    return ids, dist, old


def encode_keys(ids, dist, old) -> np.ndarray:
    """Inverse of decode_keys: (ids, float32 dist, old) -> uint64 keys (EMPTY where id < 0)."""
    ids = np.asarray(ids, np.int64)
    d32 = np.asarray(dist, np.float32)
    bits = d32.view(np.uint32)
    ob = np.where((bits & np.uint32(0x80000000)) != 0, ~bits, bits | np.uint32(0x80000000)).astype(np.uint64)
    k = (ob << np.uint64(32)) | (ids.astype(np.uint64) << np.uint64(1)) | np.asarray(old, np.uint64)
    return np.where(ids < 0, np.uint64(EMPTY), k).astype(np.uint64)


def header_functions() -> list[str]:
    """Names of every function declared in include/grnnd.h."""
    import re
    with open(HEADER) as f:
        txt = f.read()
    return sorted(set(re.findall(r"GRNND_API\s+[\w\s\*]*?\b(grnnd_\w+)\s*\(", txt)))


# ---------------------------------------------------------------------------------------
# Serving loop
# ---------------------------------------------------------------------------------------

class Server:
    """grnnd_server_*: build and search requests served concurrently on `slots` streams under
    an HBM budget.  Buffers handed to submit_* are kept alive here until their request is
    waited for."""

    def __init__(self, slots: int = 4, hbm_budget: int = 8 << 30, max_batch_queries: int = 0):
        cfg = ServerConfig(slots, hbm_budget, max_batch_queries)
        self.handle = ctypes.c_void_p()
        _check(lib().grnnd_server_create(ctypes.byref(cfg), ctypes.byref(self.handle)))
        self._keep = {}
        self._lock = threading.Lock()

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            lib().grnnd_server_destroy(self.handle)
            self.handle = ctypes.c_void_p(0)
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _rows(x):
        if isinstance(x, np.ndarray):
            a = np.ascontiguousarray(x, dtype=np.float32)
            return a, a.ctypes.data_as(ctypes.c_void_p)
        a = x.contiguous()
        return a, ctypes.c_void_p(a.data_ptr())

    def submit_build(self, points, **kw) -> int:
        """Queues a build of points (numpy or torch, (n, d)); kw as for build().  Returns the
        request id, which is also the index id."""
        a, ptr = self._rows(points)
        p = params(**kw)
        rid = ctypes.c_int64()
        _check(lib().grnnd_server_submit_build(self.handle, ptr, a.shape[0], a.shape[1], ctypes.byref(p),
                                               ctypes.byref(rid)))
        with self._lock:
            self._keep[rid.value] = (a, p, kw.get("tuning"))
        return rid.value

    def submit_search(self, index: int, queries, k: int = 10, beam: int = 64, out=None) -> int:
        """Queues a search of `queries` on index `index`; the result lands in `out` (numpy
        int32 (nq, k) by default, or a torch tensor), returned by result()."""
        a, ptr = self._rows(queries)
        if out is None:
            out = np.empty((a.shape[0], k), np.int32)
        optr = out.ctypes.data_as(ctypes.c_void_p) if isinstance(out, np.ndarray) else ctypes.c_void_p(out.data_ptr())
        rid = ctypes.c_int64()
        _check(lib().grnnd_server_submit_search(self.handle, index, ptr, a.shape[0], k, beam, optr,
                                                ctypes.byref(rid)))
        with self._lock:
            self._keep[rid.value] = (a, out)
        return rid.value

    def wait(self, rid: int, timeout: float = -1.0) -> dict:
        """Waits for request rid; returns its info dict (with 'out' for a search).  Raises
        GrnndError if the request failed (or TimeoutError if it is not done in time)."""
        info = RequestInfo()
        rc = lib().grnnd_server_wait(self.handle, rid, timeout, ctypes.byref(info))
        d = info.as_dict()
        if rc == ETIMEOUT and d["state"] != 2:
            raise TimeoutError(f"request {rid} not done")
        with self._lock:
            keep = self._keep.pop(rid, None)
        if d["kind"] == "search" and keep is not None:
            d["out"] = keep[1]
        if rc != OK:
            raise GrnndError(rc, d["message"])
        return d

    def graph(self, index: int):
        """(ids, dists, deg) numpy copies and the entry of a resident index."""
        h = ctypes.c_void_p()
        _check(lib().grnnd_server_index(self.handle, index, ctypes.byref(h)))
        n_, d_, R_, e_ = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check(lib().grnnd_graph_info(h, ctypes.byref(n_), ctypes.byref(d_), ctypes.byref(R_), ctypes.byref(e_)))
        ids = np.empty((n_.value, R_.value), np.int32)
        dists = np.empty((n_.value, R_.value), np.float32)
        deg = np.empty(n_.value, np.int32)
        _check(lib().grnnd_graph_copy(h, ids.ctypes.data_as(ctypes.c_void_p), dists.ctypes.data_as(ctypes.c_void_p),
                                      deg.ctypes.data_as(ctypes.c_void_p)))
        return ids, dists, deg, e_.value

    def release(self, index: int):
        _check(lib().grnnd_server_release(self.handle, index))

    def status(self) -> dict:
        u, pk = ctypes.c_uint64(), ctypes.c_uint64()
        q, r, i = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check(lib().grnnd_server_status(self.handle, ctypes.byref(u), ctypes.byref(pk), ctypes.byref(q),
                                         ctypes.byref(r), ctypes.byref(i)))
        return {"bytes_in_use": u.value, "peak_bytes": pk.value, "queued": q.value, "running": r.value,
                "indices": i.value}

