"""ctypes front end of the FP64 GRNND oracle (``grnnd_oracle.c``).

TEST INFRASTRUCTURE ONLY.  The test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The CUDA library never
imports this module and shares no code with it.

The pool representation used here is three (n, R) arrays plus a degree vector:
``ids`` (int32, -1 for an empty slot), ``dist`` (float64, +inf for empty),
``old`` (uint8) and ``deg`` (int32).  Row v holds its first ``deg[v]`` entries
sorted by (dist, id), as Alg 4 / Sec 3.5 of the paper keep them.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "grnnd_oracle.c")
_SRC_MT = os.path.join(_HERE, "grnnd_oracle_mt.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libgrnnd_oracle.so")
_LIB_MT_PATH = os.path.join(_OUT_DIR, "libgrnnd_oracle_mt.so")
_lock = threading.Lock()
_lib = None
_lib_mt = None

# -ffp-contract=off: no fused multiply-add, so x86 and Arm hosts agree bit for bit.
_CFLAGS = ["-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math"]


def _stale(lib, srcs):
    return not os.path.exists(lib) or any(os.path.getmtime(lib) < os.path.getmtime(s) for s in srcs)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into ``oracle/_build`` (idempotent), and the library of
    its multi-threaded build driver (the oracle's source plus ``grnnd_oracle_mt.c``)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or _stale(_LIB_PATH, [_SRC]):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.run(["gcc", *_CFLAGS, "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, _LIB_PATH)
    if force or _stale(_LIB_MT_PATH, [_SRC, _SRC_MT]):
        tmp = _LIB_MT_PATH + f".tmp{os.getpid()}"
        subprocess.run(["gcc", *_CFLAGS, "-pthread", "-o", tmp, _SRC, _SRC_MT, "-lm"], check=True)
        os.replace(tmp, _LIB_MT_PATH)
    return _LIB_PATH


def _p(t):
    return ctypes.POINTER(t)


def lib():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        L = ctypes.CDLL(build())
        i32, i64, u64, f32, f64, u8 = (ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64,
                                       ctypes.c_float, ctypes.c_double, ctypes.c_uint8)
        L.orc_splitmix64.argtypes = [u64]
        L.orc_splitmix64.restype = u64
        L.orc_hash.argtypes = [u64, u64, u64, u64, u64]
        L.orc_hash.restype = u64
        L.orc_dist.argtypes = [_p(f32), _p(f32), i32, i32]
        L.orc_dist.restype = f64
        L.orc_init.argtypes = [_p(f32), i64, i32, i32, i32, i32, u64, f64,
                               _p(i32), _p(f64), _p(u8), _p(i32), _p(u8)]
        L.orc_visit_order.argtypes = [u64, i32, i32, i64, i32, _p(i32), i32, _p(i32)]
        L.orc_visit_order.restype = None
        L.orc_prune.argtypes = [_p(f32), i32, i32, i32, _p(i32), _p(f64), _p(u8), _p(i32), i32,
                                f64, _p(u8), _p(i32), _p(f64), _p(i64)]
        L.orc_round.argtypes = [_p(f32), i64, i32, i32, i32, _p(i32), _p(f64), _p(u8), _p(i32),
                                u64, i32, i32, i32, i32, f64,
                                _p(i32), _p(f64), _p(u8), _p(i32), _p(u8), _p(i64)]
        L.orc_reverse.argtypes = [i64, i32, f32, _p(i32), _p(f64), _p(u8), _p(i32),
                                  _p(i32), _p(f64), _p(u8), _p(i32), _p(u8)]
        L.orc_final_prune.argtypes = [_p(f32), i64, i32, i32, i32, _p(i32), _p(f64), _p(u8), _p(i32),
                                      u64, i32, i32, i32, f64, _p(i32), _p(f64), _p(i32), _p(u8)]
        L.orc_build.argtypes = [_p(f32), i64, i32, i32, i32, i32, i32, i32, f32, u64, i32, i32, i32,
                                _p(i32), _p(f64), _p(i32), _p(i64)]
        L.orc_merge.argtypes = [i64, i32, i64, _p(i32), _p(i32), _p(f64), _p(u8),
                                _p(i32), _p(f64), _p(u8), _p(i32)]
        L.orc_brute_knn.argtypes = [_p(f32), i64, i32, i32, _p(f32), i64, i32, _p(i32), _p(f64)]
        L.orc_entry.argtypes = [_p(f32), i64, i32, i32]
        L.orc_entry.restype = i64
        L.orc_search.argtypes = [_p(i32), _p(i32), i32, _p(f32), i64, i32, i32, i64, _p(f32), i64,
                                 i32, i32, _p(i32), _p(f64), _p(i64)]
        for name in ("orc_init", "orc_prune", "orc_round", "orc_reverse", "orc_final_prune",
                     "orc_build", "orc_merge", "orc_brute_knn", "orc_search"):
            getattr(L, name).restype = ctypes.c_int
        _lib = L
        return L


def _ptr(a: np.ndarray, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _f32(X) -> np.ndarray:
    return np.ascontiguousarray(X, dtype=np.float32)


def _check(rc: int, what: str):
    if rc != 0:
        raise ValueError(f"oracle {what} failed with status {rc}")


@dataclass
class Pool:
    ids: np.ndarray   # (n, R) int32, -1 empty
    dist: np.ndarray  # (n, R) float64
    old: np.ndarray   # (n, R) uint8
    deg: np.ndarray   # (n,) int32

    @property
    def n(self):
        return self.ids.shape[0]

    @property
    def R(self):
        return self.ids.shape[1]

    def copy(self) -> "Pool":
        return Pool(self.ids.copy(), self.dist.copy(), self.old.copy(), self.deg.copy())

    @staticmethod
    def empty(n: int, R: int) -> "Pool":
        return Pool(np.full((n, R), -1, np.int32), np.full((n, R), np.inf), np.zeros((n, R), np.uint8),
                    np.zeros(n, np.int32))


def _pool_args(p: Pool):
    return (_ptr(p.ids, ctypes.c_int32), _ptr(p.dist, ctypes.c_double), _ptr(p.old, ctypes.c_uint8),
            _ptr(p.deg, ctypes.c_int32))


def splitmix64(z: int) -> int:
    return int(lib().orc_splitmix64(ctypes.c_uint64(z & (2**64 - 1))))


def counter_hash(seed: int, t1: int, t2: int, v: int, x: int) -> int:
    M = 2**64 - 1
    return int(lib().orc_hash(seed & M, t1 & M, t2 & M, v & M, x & M))


def dist(x, y, metric: int = 0) -> float:
    x, y = _f32(x), _f32(y)
    return float(lib().orc_dist(_ptr(x, ctypes.c_float), _ptr(y, ctypes.c_float), x.shape[-1], metric))


def init(X, S: int, R: int, seed: int, metric: int = 0, tol: float = 0.0):
    """Alg 3 initialisation.  Returns (pool, flags)."""
    X = _f32(X)
    n, d = X.shape
    p = Pool.empty(n, R)
    flags = np.zeros(n, np.uint8)
    _check(lib().orc_init(_ptr(X, ctypes.c_float), n, d, metric, S, R, seed, tol, *_pool_args(p),
                          _ptr(flags, ctypes.c_uint8)), "init")
    return p, flags


def visit_order(seed: int, t1: int, t2: int, v: int, ids, order: int = 0) -> np.ndarray:
    ids = np.ascontiguousarray(ids, dtype=np.int32)
    perm = np.zeros(len(ids), np.int32)
    lib().orc_visit_order(seed, t1, t2, v, len(ids), _ptr(ids, ctypes.c_int32), order,
                          _ptr(perm, ctypes.c_int32))
    return perm


def prune(X, ids, dists, perm, old=None, metric: int = 0, skip_old: bool = False, tol: float = 0.0):
    """Eq 2 prune of one pool in visit order ``perm``.

    Returns (alive[m] bool, killer[m] int (-1 for survivors), kdist[m], flagged, n_eval)."""
    X = _f32(X)
    ids = np.ascontiguousarray(ids, np.int32)
    dists = np.ascontiguousarray(dists, np.float64)
    m = len(ids)
    old = np.zeros(m, np.uint8) if old is None else np.ascontiguousarray(old, np.uint8)
    perm = np.ascontiguousarray(perm, np.int32)
    alive = np.zeros(m, np.uint8)
    killer = np.zeros(m, np.int32)
    kd = np.zeros(m, np.float64)
    ne = np.zeros(1, np.int64)
    f = lib().orc_prune(_ptr(X, ctypes.c_float), X.shape[1], metric, m, _ptr(ids, ctypes.c_int32),
                        _ptr(dists, ctypes.c_double), _ptr(old, ctypes.c_uint8), _ptr(perm, ctypes.c_int32),
                        int(skip_old), tol, _ptr(alive, ctypes.c_uint8), _ptr(killer, ctypes.c_int32),
                        _ptr(kd, ctypes.c_double), _ptr(ne, ctypes.c_int64))
    return alive.astype(bool), killer, kd, bool(f), int(ne[0])


def round_(X, pool: Pool, seed: int, t1: int, t2: int, order: int = 0, metric: int = 0,
           skip_old: bool = False, tol: float = 0.0):
    """One round of Alg 4 (pool1 -> pool2).  Returns (pool2, flags, stats[3])."""
    X = _f32(X)
    n, d = X.shape
    out = Pool.empty(n, pool.R)
    flags = np.zeros(n, np.uint8)
    stats = np.zeros(3, np.int64)
    _check(lib().orc_round(_ptr(X, ctypes.c_float), n, d, metric, pool.R, *_pool_args(pool), seed, t1, t2,
                           order, int(skip_old), tol, *_pool_args(out), _ptr(flags, ctypes.c_uint8),
                           _ptr(stats, ctypes.c_int64)), "round")
    return out, flags, stats


def reverse(pool: Pool, rho: float):
    """Sec 3.6 reverse-edge sampling + merge.  Returns (pool', flags)."""
    out = Pool.empty(pool.n, pool.R)
    flags = np.zeros(pool.n, np.uint8)
    _check(lib().orc_reverse(pool.n, pool.R, ctypes.c_float(rho), *_pool_args(pool), *_pool_args(out),
                             _ptr(flags, ctypes.c_uint8)), "reverse")
    return out, flags


def merge(n: int, R: int, target, ids, dists, old):
    """C6 merge of a proposal list into n fixed-capacity pools of R slots."""
    target = np.ascontiguousarray(target, np.int32)
    ids = np.ascontiguousarray(ids, np.int32)
    dists = np.ascontiguousarray(dists, np.float64)
    old = np.ascontiguousarray(old, np.uint8)
    out = Pool.empty(n, R)
    _check(lib().orc_merge(n, R, len(target), _ptr(target, ctypes.c_int32), _ptr(ids, ctypes.c_int32),
                           _ptr(dists, ctypes.c_double), _ptr(old, ctypes.c_uint8), *_pool_args(out)), "merge")
    return out


def final_prune(X, pool: Pool, seed: int, t1: int, order: int = 0, metric: int = 0,
                skip_old: bool = False, tol: float = 0.0):
    """C11 final prune.  Returns (gids (n,R), gdist (n,R), gdeg (n,), flags)."""
    X = _f32(X)
    n, d = X.shape
    gids = np.full((n, pool.R), -1, np.int32)
    gd = np.full((n, pool.R), np.inf)
    gdeg = np.zeros(n, np.int32)
    flags = np.zeros(n, np.uint8)
    _check(lib().orc_final_prune(_ptr(X, ctypes.c_float), n, d, metric, pool.R, *_pool_args(pool), seed, t1,
                                 order, int(skip_old), tol, _ptr(gids, ctypes.c_int32), _ptr(gd, ctypes.c_double),
                                 _ptr(gdeg, ctypes.c_int32), _ptr(flags, ctypes.c_uint8)), "final_prune")
    return gids, gd, gdeg, flags


def build_graph(X, S: int, R: int, T1: int, T2: int, rho: float = 0.6, seed: int = 0, metric: int = 0,
                order: int = 0, skip_old: bool = False, final_prune: bool = True):
    """Alg 3 end to end.  Returns (gids, gdist, gdeg, stats[3])."""
    X = _f32(X)
    n, d = X.shape
    gids = np.full((n, R), -1, np.int32)
    gd = np.full((n, R), np.inf)
    gdeg = np.zeros(n, np.int32)
    stats = np.zeros(3, np.int64)
    _check(lib().orc_build(_ptr(X, ctypes.c_float), n, d, metric, S, R, T1, T2, ctypes.c_float(rho), seed,
                           order, int(skip_old), int(final_prune), _ptr(gids, ctypes.c_int32),
                           _ptr(gd, ctypes.c_double), _ptr(gdeg, ctypes.c_int32), _ptr(stats, ctypes.c_int64)),
           "build")
    return gids, gd, gdeg, stats


def lib_mt():
    global _lib_mt
    with _lock:
        if _lib_mt is not None:
            return _lib_mt
        build()
        L = ctypes.CDLL(_LIB_MT_PATH)
        i32, i64, u64, f32 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_float
        L.orc_build_mt.argtypes = [_p(f32), i64, i32, i32, i32, i32, i32, i32, f32, u64, i32, i32, i32, i32,
                                   _p(i32), _p(ctypes.c_double), _p(i32), _p(i64)]
        L.orc_build_mt.restype = ctypes.c_int
        _lib_mt = L
        return L


def build_graph_mt(X, S: int, R: int, T1: int, T2: int, rho: float = 0.6, seed: int = 0, metric: int = 0,
                   order: int = 0, skip_old: bool = False, final_prune: bool = True, threads: int = 1):
    """build_graph with the per-vertex prunes and the per-target merges split over `threads`
    host threads (grnnd_oracle_mt.c); the same results at any thread count."""
    X = _f32(X)
    n, d = X.shape
    gids = np.full((n, R), -1, np.int32)
    gd = np.full((n, R), np.inf)
    gdeg = np.zeros(n, np.int32)
    stats = np.zeros(3, np.int64)
    _check(lib_mt().orc_build_mt(_ptr(X, ctypes.c_float), n, d, metric, S, R, T1, T2, ctypes.c_float(rho), seed,
                                 order, int(skip_old), int(final_prune), int(threads), _ptr(gids, ctypes.c_int32),
                                 _ptr(gd, ctypes.c_double), _ptr(gdeg, ctypes.c_int32), _ptr(stats, ctypes.c_int64)),
           "build_mt")
    return gids, gd, gdeg, stats


def brute_knn(X, Q, k: int, metric: int = 0):
    """Exact k-NN by (dist, id).  Returns (ids (nq,k), dist (nq,k))."""
    X, Q = _f32(X), _f32(Q)
    nq = Q.shape[0]
    ids = np.zeros((nq, k), np.int32)
    dd = np.zeros((nq, k), np.float64)
    _check(lib().orc_brute_knn(_ptr(X, ctypes.c_float), X.shape[0], X.shape[1], metric, _ptr(Q, ctypes.c_float),
                               nq, k, _ptr(ids, ctypes.c_int32), _ptr(dd, ctypes.c_double)), "brute_knn")
    return ids, dd


def entry(X, metric: int = 0) -> int:
    X = _f32(X)
    return int(lib().orc_entry(_ptr(X, ctypes.c_float), X.shape[0], X.shape[1], metric))


def search(gids, gdeg, X, Q, k: int, beam: int, entry_id: int, metric: int = 0):
    """Candidate-list search.  Returns (ids (nq,k), dist (nq,k), n_distance_evals)."""
    X, Q = _f32(X), _f32(Q)
    gids = np.ascontiguousarray(gids, np.int32)
    gdeg = np.ascontiguousarray(gdeg, np.int32)
    nq = Q.shape[0]
    ids = np.zeros((nq, k), np.int32)
    dd = np.zeros((nq, k), np.float64)
    ne = np.zeros(1, np.int64)
    _check(lib().orc_search(_ptr(gids, ctypes.c_int32), _ptr(gdeg, ctypes.c_int32), gids.shape[1],
                            _ptr(X, ctypes.c_float), X.shape[0], X.shape[1], metric, entry_id,
                            _ptr(Q, ctypes.c_float), nq, k, beam, _ptr(ids, ctypes.c_int32),
                            _ptr(dd, ctypes.c_double), _ptr(ne, ctypes.c_int64)), "search")
    return ids, dd, int(ne[0])


def recall_at_k(found_ids, true_ids) -> float:
    """Recall@k (Sec 2.1): fraction of the true k nearest ids that were returned."""
    found_ids = np.asarray(found_ids)
    true_ids = np.asarray(true_ids)
    k = true_ids.shape[1]
    hit = 0
    for f, t in zip(found_ids, true_ids):
        hit += len(set(f[f >= 0].tolist()) & set(t.tolist()))
    return hit / (k * len(true_ids))
