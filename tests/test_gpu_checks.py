"""The checked build (-DGRNND_CHECKS=1: device bounds checks on the indices the kernels read
from pools, records and redirect slots, reported through the step's status word instead of
a fault).  compute-sanitizer does not run on this pool; this build is its stand-in: whole
builds of every form and metric, batched builds, the step calls and the serving loop run
through it with no check firing and give the normal library's graphs."""
import ctypes

import numpy as np
import pytest

from paper_2510_02774_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_02774_gb300 import build as B
    B.build()
    from paper_2510_02774_gb300 import grnnd
    grnnd.lib()
    return grnnd


@pytest.fixture(scope="module")
def LC(G):
    from paper_2510_02774_gb300 import build as B
    return G.lib(B.build(checks=True))  # a second handle on the checked library


def _build_checked(G, LC, X, **kw):
    X = np.ascontiguousarray(X, np.float32)
    p = G.params(**kw)
    h = ctypes.c_void_p()
    rc = LC.grnnd_build_ex(X.ctypes.data_as(ctypes.c_void_p), X.shape[0], X.shape[1], ctypes.byref(p),
                           ctypes.byref(h))
    assert rc == 0, LC.grnnd_last_error()
    n, R = X.shape[0], kw["R"]
    ids = np.empty((n, R), np.int32)
    dist = np.empty((n, R), np.float32)
    deg = np.empty(n, np.int32)
    assert LC.grnnd_graph_copy(h, ids.ctypes.data_as(ctypes.c_void_p), dist.ctypes.data_as(ctypes.c_void_p),
                               deg.ctypes.data_as(ctypes.c_void_p)) == 0
    LC.grnnd_free(h)
    return ids, dist, deg


@pytest.mark.parametrize("precision,metric,d,S,R", [(0, 0, 24, 16, 32), (1, 0, 128, 32, 64), (2, 1, 40, 16, 48),
                                                    (0, 0, 200, 32, 64), (1, 1, 96, 24, 40)])
def test_checked_build_is_silent_and_equal(G, LC, precision, metric, d, S, R):
    X = synth.small_integers(6000, d, -8, 8, seed=d + S)
    kw = dict(S=S, R=R, T1=2, T2=5, seed=3, precision=precision, metric=metric)
    want = G.build(X, **kw).to_numpy()
    got = _build_checked(G, LC, X, **kw)
    for a, b in zip(got, want):
        assert (a == b).all()


def test_checked_continuous_and_batched(G, LC):
    X = synth.gaussian_mixture(5000, 64, seed=4)
    kw = dict(S=16, R=32, T1=3, T2=4, seed=7, precision=1)
    want = G.build(X, **kw).to_numpy()
    got = _build_checked(G, LC, X, **kw)
    for a, b in zip(got, want):
        assert (a == b).all()
    off = (ctypes.c_int64 * 4)(0, 1000, 3500, 5000)
    p = G.params(**kw)
    hs = (ctypes.c_void_p * 3)()
    Xc = np.ascontiguousarray(X, np.float32)
    assert LC.grnnd_build_batch(Xc.ctypes.data_as(ctypes.c_void_p), off, 3, 64, ctypes.byref(p),
                                ctypes.cast(hs, ctypes.c_void_p)) == 0, LC.grnnd_last_error()
    for b in range(3):
        deg = np.empty(off[b + 1] - off[b], np.int32)
        assert LC.grnnd_graph_copy(ctypes.c_void_p(hs[b]), None, None, deg.ctypes.data_as(ctypes.c_void_p)) == 0
        one = G.build(X[off[b]:off[b + 1]], **kw).to_numpy()
        assert (deg == one[2]).all()
        LC.grnnd_free(ctypes.c_void_p(hs[b]))
