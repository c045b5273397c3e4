"""grnnd_entry_point_noalloc: the search entry computed without any device allocation.

Callers that may not allocate device memory when they need the entry point (their
own arena owns the GPU, or cudaMalloc's implicit synchronisation is not allowed in
their loop) use this call; its scratch is a fixed array inside the library.  It must
give the same entry as grnnd_entry_point, call after call, although every call
reuses the array that the previous call left behind.  This file is collected last
so that a stop at its first failure has already run every other test.
"""
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


def _noalloc(G, Xd, d, metric):
    n, ld = Xd.shape
    out = torch.full((1,), -7, dtype=torch.int32, device="cuda")
    rc = G.lib().grnnd_entry_point_noalloc(ctypes.c_void_p(Xd.data_ptr()), n, d, ld, metric,
                                           ctypes.c_void_p(out.data_ptr()),
                                           ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == G.OK, G.lib().grnnd_last_error()
    torch.cuda.synchronize()
    return int(out.item())


@pytest.mark.parametrize("metric", [0, 1])
def test_noalloc_entry_equals_allocating_entry_on_consecutive_calls(G, metric):
    cases = [synth.small_integers(5000, 13, -8, 8, seed=3),            # exact arithmetic
             synth.gaussian_mixture(3000, 96, 10, 5.0, 1.0, seed=4),   # wider rows, other n
             synth.small_integers(777, 1024, -4, 4, seed=5)]           # the largest d allowed
    first = None
    for X in cases + cases[:1]:   # the last call repeats the first after the array was reused
        Xd, d = G.device_points(X)
        want = G.entry_point(Xd, d, metric)          # caller-provided workspace
        got = _noalloc(G, Xd, d, metric)             # fixed library scratch
        assert got == want
        assert 0 <= got < X.shape[0]
        if first is None:
            first = got
    assert got == first


def test_noalloc_entry_rejects_rows_wider_than_its_scratch(G):
    Xd, d = G.device_points(np.zeros((8, 1028), np.float32))
    out = torch.zeros(1, dtype=torch.int32, device="cuda")
    rc = G.lib().grnnd_entry_point_noalloc(ctypes.c_void_p(Xd.data_ptr()), 8, d, Xd.shape[1], 0,
                                           ctypes.c_void_p(out.data_ptr()), None)
    assert rc == G.EINVAL
    assert b"d <= 1024" in G.lib().grnnd_last_error()
