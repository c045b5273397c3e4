"""The C-ABI library builds, loads, exports every declared entry point, and rejects
bad arguments before touching the GPU (no compute calls: runs without a GPU)."""
import ctypes
import subprocess

import numpy as np
import pytest

from paper_2510_02774_gb300 import build as B
from paper_2510_02774_gb300 import grnnd as G


@pytest.fixture(scope="module")
def L():
    B.build()
    return G.lib()


def test_every_declared_symbol_is_exported(L):
    declared = G.header_functions()
    assert len(declared) >= 20
    out = subprocess.run(["nm", "-D", "--defined-only", G.LIB_PATH], capture_output=True, text=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if " T " in l}
    missing = [f for f in declared if f not in exported]
    assert not missing, missing
    assert set(declared) == set(G._SIGS), "binding and header disagree"
    for f in declared:
        assert hasattr(L, f)


def test_defaults(L):
    p = G.Params()
    L.grnnd_params_default(ctypes.byref(p))
    assert (p.S, p.R, p.T1, p.T2, p.final_prune, p.metric, p.precision, p.order) == (16, 32, 4, 8, 1, 0, 0, 0)
    assert abs(p.rho - 0.6) < 1e-7


@pytest.mark.parametrize("kw,frag", [
    (dict(S=8, R=4), "S"),          # S > R
    (dict(S=2, R=257), "R"),        # R above the largest pool (256)
    (dict(S=2, R=1), "R"),
    (dict(S=2, R=4, T1=0), "T1"),
    (dict(S=2, R=4, rho=1.5), "rho"),
    (dict(S=2, R=4, metric=7), "metric"),
    (dict(S=2, R=4, order=9), "order"),
    (dict(S=2, R=4, precision=3), "precision"),   # FP32, BF16 and FP8 only
])
def test_build_rejects_bad_params_before_any_launch(L, kw, frag):
    X = np.zeros((10, 3), np.float32)
    with pytest.raises(G.GrnndError) as e:
        G.build(X, **kw)
    assert e.value.status == G.EINVAL
    assert frag in str(e.value)


def test_build_rejects_too_few_points(L):
    with pytest.raises(G.GrnndError) as e:
        G.build(np.zeros((1, 4), np.float32), S=1, R=2)
    assert e.value.status == G.EINVAL
    with pytest.raises(G.GrnndError) as e:   # S > n - 1
        G.build(np.zeros((4, 4), np.float32), S=4, R=8)
    assert e.value.status == G.EINVAL


def test_step_calls_validate_layout(L):
    null = ctypes.c_void_p(0)
    bad = ctypes.c_void_p(16 * 1000 + 4)  # not 16-byte aligned
    rc = L.grnnd_pool_init(bad, 10, 3, 4, 0, 2, 4, 0, null, null, null)
    assert rc == G.EINVAL and b"aligned" in L.grnnd_last_error()
    rc = L.grnnd_pool_init(ctypes.c_void_p(1 << 20), 10, 5, 5, 0, 2, 4, 0, null, null, null)
    assert rc == G.EINVAL and b"ld" in L.grnnd_last_error()
    rc = L.grnnd_search(null, null, 1, 1, 1, null)
    assert rc == G.EINVAL
    rc = L.grnnd_workspace_status(null, 1 << 30, 10, 4, null)
    assert rc == G.EINVAL and b"workspace" in L.grnnd_last_error()
    rc = L.grnnd_workspace_status(ctypes.c_void_p(1 << 20), 16, 10, 4, null)  # far too small
    assert rc == G.EINVAL


def test_workspace_size_scales(L):
    a = L.grnnd_workspace_size(1000, 32)
    b = L.grnnd_workspace_size(2000, 32)
    assert a > 1000 * 32 * 20 and b > a


def test_key_codec_orders_like_dist_then_id():
    ids = np.array([[3, 1, 2, -1]], np.int32)
    d = np.array([[0.5, 0.5, -2.0, 0.0]], np.float32)
    k = G.encode_keys(ids, d, np.array([[1, 0, 0, 0]]))
    i2, d2, o2 = G.decode_keys(k)
    assert (i2 == ids).all() and (o2 == [[1, 0, 0, 0]]).all()
    assert d2[0, :3].tolist() == [0.5, 0.5, -2.0]
    order = np.argsort(k[0, :3])
    assert order.tolist() == [2, 1, 0]  # (-2, 2) < (0.5, 1) < (0.5, 3)


def test_build_batch_validates_before_any_launch(L):
    import ctypes
    p = G.params(S=4, R=8)
    null = ctypes.c_void_p(0)
    hs = (ctypes.c_void_p * 3)()
    pts = ctypes.c_void_p(1 << 20)
    ok = (ctypes.c_int64 * 4)(0, 10, 20, 30)
    assert L.grnnd_build_batch(pts, ok, 3, 4, ctypes.byref(p), null) == G.EINVAL
    assert L.grnnd_build_batch(pts, ok, 0, 4, ctypes.byref(p), hs) == G.EINVAL
    bad0 = (ctypes.c_int64 * 4)(1, 10, 20, 30)
    assert L.grnnd_build_batch(pts, bad0, 3, 4, ctypes.byref(p), hs) == G.EINVAL
    assert b"offsets[0]" in L.grnnd_last_error()
    tiny = (ctypes.c_int64 * 4)(0, 10, 11, 30)  # a build of one point
    assert L.grnnd_build_batch(pts, tiny, 3, 4, ctypes.byref(p), hs) == G.EINVAL
    small = (ctypes.c_int64 * 4)(0, 10, 14, 30)  # S = 4 needs 5 points
    assert L.grnnd_build_batch(pts, small, 3, 4, ctypes.byref(p), hs) == G.EINVAL
    assert all(h is None for h in hs)


def test_autotune_pool_is_validated(L):
    import ctypes
    pts = ctypes.c_void_p(1 << 20)
    p = G.params(S=8, R=16)
    out = (ctypes.c_int32(), ctypes.c_float(), ctypes.c_float())
    for cands, nq, tgt, k, beam in [((), 10, 0.9, 10, 64), ((1,), 10, 0.9, 10, 64), ((16, 257), 10, 0.9, 10, 64),
                                    ((16,), 0, 0.9, 10, 64), ((16,), 98, 0.9, 10, 64), ((16,), 10, 0.0, 10, 64),
                                    ((16,), 10, 1.5, 10, 64), ((16,), 10, 0.9, 0, 64), ((16,), 10, 0.9, 33, 64),
                                    ((16,), 10, 0.9, 10, 8), ((16,), 10, 0.9, 10, 257)]:
        c = (ctypes.c_int32 * max(1, len(cands)))(*cands)
        rc = L.grnnd_autotune_pool(pts, 100, 4, nq, ctypes.byref(p), c, len(cands), tgt, k, beam,
                                   *(ctypes.byref(x) for x in out))
        assert rc == G.EINVAL, (cands, nq, tgt, k, beam)


def test_tuning_is_validated(L):
    import ctypes
    pts = ctypes.c_void_p(1 << 20)
    h = ctypes.c_void_p()
    for gm, w in [((9, 16, 32), 0), ((8, 17, 32), 0), ((8, 16, 33), 0), ((-1, 16, 32), 0), ((8, 16, 32), -1)]:
        t = G.tuning(gm, w, 0)
        p = G.params(S=4, R=8, tuning=t)
        assert L.grnnd_build_ex(pts, 100, 4, ctypes.byref(p), ctypes.byref(h)) == G.EINVAL
        assert b"tuning" in L.grnnd_last_error()
    for rc in (-1, 3):
        p = G.params(S=4, R=8, tuning=G.tuning(row_copies=rc))
        assert L.grnnd_build_ex(pts, 100, 4, ctypes.byref(p), ctypes.byref(h)) == G.EINVAL
        assert b"row_copies" in L.grnnd_last_error()


def test_server_validates_before_any_cuda_call(L):
    import ctypes
    h = ctypes.c_void_p()
    for cfg in [G.ServerConfig(0, 1 << 30, 0), G.ServerConfig(65, 1 << 30, 0), G.ServerConfig(2, 0, 0),
                G.ServerConfig(2, 1 << 30, -1)]:
        assert L.grnnd_server_create(ctypes.byref(cfg), ctypes.byref(h)) == G.EINVAL
        assert h.value is None
    rid = ctypes.c_int64()
    p = G.params(S=4, R=8)
    assert L.grnnd_server_submit_build(None, ctypes.c_void_p(1 << 20), 100, 4, ctypes.byref(p),
                                       ctypes.byref(rid)) == G.EINVAL
    assert L.grnnd_server_submit_search(None, 1, ctypes.c_void_p(1 << 20), 1, 1, 1, ctypes.c_void_p(1 << 20),
                                        ctypes.byref(rid)) == G.EINVAL
    assert L.grnnd_server_wait(None, 1, 0.0, None) == G.EINVAL
    assert L.grnnd_server_release(None, 1) == G.EINVAL


def test_current_stream_is_per_thread(L):
    import threading
    assert L.grnnd_get_stream() is None
    L.grnnd_set_stream(ctypes.c_void_p(0x1234))
    seen = []
    t = threading.Thread(target=lambda: seen.append(L.grnnd_get_stream()))
    t.start()
    t.join()
    try:
        assert seen == [None]                 # another thread keeps its own (NULL) stream
        assert L.grnnd_get_stream() == 0x1234
    finally:
        L.grnnd_set_stream(None)
    assert L.grnnd_get_stream() is None


def test_quantized_step_calls_validate(L):
    assert L.grnnd_quantized_size(100, 33, G.BF16) >= 100 * 48 * 2 + 100 * 8  # rows of 48 BF16, row terms
    assert L.grnnd_quantized_size(100, 33, G.FP8) >= 100 * 64 + 100 * 8       # rows of 64 e4m3 bytes
    assert L.grnnd_quantized_size(100, 33, G.FP32) == 0
    buf = ctypes.create_string_buffer(1 << 16)
    rc = L.grnnd_quantize(ctypes.c_void_p(256), 100, 33, 36, G.FP32, buf, len(buf), None)
    assert rc == G.EINVAL and b"precision" in L.grnnd_last_error()
    # a precision form without its quantized rows is rejected before any launch
    rc = L.grnnd_join_round_q(ctypes.c_void_p(256), 100, 33, 36, 0, G.BF16, None, 0, 16, ctypes.c_void_p(256),
                              ctypes.c_void_p(256), 1, 1, 1, 0, ctypes.c_void_p(256), ctypes.c_void_p(256),
                              ctypes.c_void_p(256), 1 << 30, None, None)
    assert rc == G.EINVAL and b"quantized" in L.grnnd_last_error()


def test_profile_filter_is_host_state(L):
    """grnnd_profile_begin_only parses its name list on the host; with no launch in between,
    grnnd_profile_end reports no kernel, and neither call touches the GPU."""
    G.profile_begin(only=["rnd_join_warp", "rnd_join_team"])
    assert G.profile_end() == {}
    G.profile_begin()
    assert G.profile_end() == {}
    for names in (None, b"", b",,select,"):
        assert L.grnnd_profile_begin_only(names) == 0
        assert G.profile_end() == {}
