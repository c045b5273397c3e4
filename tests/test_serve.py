"""Serving loop (grnnd_server_*): continuous batching of build and search requests on
concurrent streams under an HBM budget.  Every result must be the same as the same
request run alone (bit for bit: builds and searches are deterministic), whatever else is
in flight."""
import time

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


def _alone(G, X, kw, queries):
    g = G.build(X, **kw)
    return g.to_numpy(), g.entry, [g.search(Q, k, beam) for Q, k, beam in queries]


def _mix(seed):
    """Builds of different sizes, dimensions, forms and metrics, each with searches."""
    g = np.random.default_rng(seed)
    cases = []
    for i, (n, d, prec, metric) in enumerate([(3000, 24, 0, 0), (1200, 40, 1, 0), (5000, 16, 1, 1), (800, 96, 2, 0),
                                              (2500, 33, 0, 1)]):
        X = synth.small_integers(n, d, -8, 8, seed=seed * 10 + i)
        kw = dict(S=8 + 4 * (i % 3), R=16 + 8 * (i % 3), T1=2, T2=3, seed=i, precision=prec, metric=metric)
        queries = []
        for j in range(3):
            nq = int(g.integers(1, 200))
            k = int(g.choice([1, 5, 10]))
            queries.append((synth.small_integers(nq, d, -8, 8, seed=1000 + 10 * i + j), k, int(k + g.integers(0, 40))))
        cases.append((X, kw, queries))
    cases.append((synth.gaussian_mixture(4000, 48, 10, seed=seed + 3), dict(S=16, R=32, T1=2, T2=4, seed=9, precision=1),
                  [(synth.gaussian_mixture(64, 48, 10, seed=seed + 4), 10, 32)]))
    return cases


def _oracle_leg(orc, X, kw, queries):
    """The oracle's graph, entry and search results for a request on integer data (exact in
    every form: |x| <= 8 and d * 64 < 2^24)."""
    m = kw.get("metric", 0)
    wids, wd, wdeg, _ = orc.build_graph(X, kw["S"], kw["R"], kw["T1"], kw["T2"], 0.6, kw["seed"], metric=m)
    e = orc.entry(X, m)
    found = [orc.search(wids, wdeg, X, Q, k, beam, e, metric=m)[0] for Q, k, beam in queries]
    return (wids, wd, wdeg), e, found


def test_results_in_the_mix_equal_results_alone(G, orc):
    cases = _mix(1)
    want = [_alone(G, X, kw, q) for X, kw, q in cases]
    # the requests on integer data, alone, are the oracle's builds and searches
    for (X, kw, queries), ((ids, dists, deg), entry, found) in zip(cases[:5], want[:5]):
        (wids, wd, wdeg), went, wfound = _oracle_leg(orc, X, kw, queries)
        assert (ids == wids).all() and (deg == wdeg).all() and entry == went
        assert (dists[wids >= 0] == wd[wids >= 0].astype(np.float32)).all()
        for a, b in zip(found, wfound):
            assert (a == b).all()
    srv = G.Server(slots=3, hbm_budget=4 << 30)
    try:
        builds, searches = [], []
        for ci, (X, kw, queries) in enumerate(cases):  # searches go in right behind their build
            b = srv.submit_build(X, **kw)
            builds.append(b)
            for qi, (Q, k, beam) in enumerate(queries):
                searches.append((ci, qi, srv.submit_search(b, Q, k, beam)))
        for ci, b in enumerate(builds):
            info = srv.wait(b)
            assert info["kind"] == "build" and info["status"] == 0 and info["t_done"] >= info["t_admit"]
            ids, dists, deg, entry = srv.graph(b)
            (wids, wd, wdeg), went, _ = want[ci]
            assert (ids == wids).all() and (deg == wdeg).all() and (dists == wd).all() and entry == went
        for ci, qi, s in searches:
            info = srv.wait(s)
            assert (info["out"] == want[ci][2][qi]).all()
        st = srv.status()
        assert st["running"] == 0 and st["queued"] == 0 and st["indices"] == len(cases)
        assert 0 < st["peak_bytes"] <= 4 << 30
        for b in builds:
            srv.release(b)
        assert srv.status()["bytes_in_use"] == 0
    finally:
        srv.close()


def test_waiting_searches_share_one_launch(G):
    X = synth.small_integers(2000, 32, -8, 8, seed=5)
    kw = dict(S=8, R=16, T1=2, T2=3, seed=1)
    g = G.build(X, **kw)
    srv = G.Server(slots=1, hbm_budget=4 << 30)
    try:
        a = srv.submit_build(X, **kw)
        srv.wait(a)
        big = srv.submit_build(synth.small_integers(150000, 64, -8, 8, seed=6), S=16, R=32, T1=2, T2=4)
        qs = [synth.small_integers(1 + 7 * i, 32, -8, 8, seed=50 + i) for i in range(20)]
        ids = [srv.submit_search(a, Q, 10, 24) for Q in qs]  # queued behind the big build
        infos = [srv.wait(i) for i in ids]
        srv.wait(big)
        assert max(inf["batch"] for inf in infos) > 1
        for Q, inf in zip(qs, infos):
            assert (inf["out"] == g.search(Q, 10, 24)).all()
    finally:
        srv.close()


def test_admission_waits_for_memory(G):
    X = synth.small_integers(20000, 32, -8, 8, seed=7)
    Y = synth.small_integers(20000, 32, -8, 8, seed=8)
    kw = dict(S=8, R=16, T1=2, T2=3, seed=2)
    probe = G.Server(slots=1, hbm_budget=8 << 30)
    try:
        total = probe.wait(probe.submit_build(X, **kw))["bytes"]
        resident = probe.status()["bytes_in_use"]
    finally:
        probe.close()
    assert 0 < resident < total
    srv = G.Server(slots=2, hbm_budget=total + resident - 256)  # one index and one build do not fit
    try:
        a = srv.submit_build(X, **kw)
        b = srv.submit_build(Y, **kw)
        srv.wait(a)
        with pytest.raises(TimeoutError):
            srv.wait(b, timeout=1.0)  # admitted only once index a is released
        assert srv.status()["queued"] == 1
        srv.release(a)
        srv.wait(b, timeout=120.0)
        assert srv.status()["peak_bytes"] <= total + resident - 256
        want = G.build(Y, **kw).to_numpy()
        got = srv.graph(b)
        assert (got[0] == want[0]).all() and (got[2] == want[2]).all()
    finally:
        srv.close()


def test_errors_and_release(G):
    X = synth.small_integers(500, 8, -8, 8, seed=9)
    srv = G.Server(slots=1, hbm_budget=1 << 20)  # 1 MB: too small for any build of X
    try:
        b = srv.submit_build(X, S=4, R=8, T1=1, T2=2)
        with pytest.raises(G.GrnndError) as e:
            srv.wait(b)
        assert e.value.status == G.ENOMEM
        with pytest.raises(G.GrnndError):  # its index failed
            srv.submit_search(b, X[:3], 1, 4)
        with pytest.raises(G.GrnndError):
            srv.submit_search(12345, X[:3], 1, 4)
        with pytest.raises(G.GrnndError):  # k > beam
            srv.submit_search(b, X[:3], 5, 4)
    finally:
        srv.close()
    srv = G.Server(slots=1, hbm_budget=1 << 30)
    try:
        big = srv.submit_build(synth.small_integers(100000, 64, -8, 8, seed=10), S=16, R=32, T1=2, T2=3)
        b = srv.submit_build(X, S=4, R=8, T1=1, T2=2)
        with pytest.raises(G.GrnndError) as e:  # still queued behind the big build
            srv.release(b)
        assert e.value.status == G.EBUSY
        srv.wait(b)
        srv.release(b)
        with pytest.raises(G.GrnndError):
            srv.submit_search(b, X[:3], 1, 4)
        srv.wait(big)
    finally:
        srv.close()


def test_destroy_with_work_in_flight(G):
    srv = G.Server(slots=2, hbm_budget=2 << 30)
    for i in range(4):
        srv.submit_build(synth.small_integers(30000, 32, -8, 8, seed=20 + i), S=8, R=16, T1=2, T2=3)
    time.sleep(0.01)
    srv.close()  # finishes what runs, fails what is queued, frees everything


def test_submissions_from_several_host_threads(G):
    # four host threads submit builds and searches at once (the binding releases the GIL in
    # every call); each result equals the same request run alone
    import threading
    cases = []
    for i in range(8):
        X = synth.small_integers(1500 + 400 * i, 24 + 8 * (i % 3), -8, 8, seed=300 + i)
        Q = synth.small_integers(40, X.shape[1], -8, 8, seed=400 + i)
        kw = dict(S=8, R=16, T1=2, T2=3, seed=i, precision=i % 3)
        g = G.build(X, **kw)
        cases.append((X, Q, kw, g.to_numpy(), g.search(Q, 5, 16)))
    srv = G.Server(slots=3, hbm_budget=4 << 30)
    errors = []

    def worker(idx):
        try:
            for X, Q, kw, want, wq in cases[idx::4]:
                b = srv.submit_build(X, **kw)
                s = srv.submit_search(b, Q, 5, 16)
                srv.wait(b)
                got = srv.graph(b)
                assert (got[0] == want[0]).all() and (got[2] == want[2]).all()
                assert (srv.wait(s)["out"] == wq).all()
                srv.release(b)
        except Exception as e:  # reported below, on the test's thread
            errors.append(e)

    try:
        ts = [threading.Thread(target=worker, args=(i,)) for i in range(4)]
        for t in ts:
            t.start()
        for t in ts:
            t.join()
        assert not errors, errors
        st = srv.status()
        assert st["indices"] == 0 and st["bytes_in_use"] == 0 and st["queued"] == 0
    finally:
        srv.close()
