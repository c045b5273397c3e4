"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Bar: on integer-valued inputs every FP32 distance is exact, so pools, graphs,
entry points, search results and k-NN lists must be bit-identical to the
oracle's (ties broken by id on both sides).  On continuous inputs one join
step must give identical neighbour-id sets except where the oracle flags a
comparison within the FP32 error bound, and every FP32 distance must be within
1e-5 relative of FP64.
"""
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


def to_keys(G, pool):
    return torch.from_numpy(G.encode_keys(pool.ids, pool.dist.astype(np.float32), pool.old).view(np.int64)).cuda()


def from_gpu(G, keys, deg):
    ids, dist, old = G.decode_keys(keys.cpu().numpy().view(np.uint64))
    return ids, dist, old, deg.cpu().numpy()


def assert_pool_equal(G, keys, deg, pool):
    ids, dist, old, dg = from_gpu(G, keys, deg)
    assert (dg == pool.deg).all(), np.nonzero(dg != pool.deg)[0][:10]
    bad = np.nonzero((ids != pool.ids).any(1))[0]
    assert len(bad) == 0, (bad[:5], ids[bad[0]], pool.ids[bad[0]])
    assert (old == pool.old).all()
    m = pool.ids >= 0
    assert (dist[m] == pool.dist[m].astype(np.float32)).all()


def oracle_state(orc, X, S, R, seed, rounds, metric=0, order=0):
    p, _ = orc.init(X, S, R, seed, metric=metric)
    for r in range(rounds):
        p, _, _ = orc.round_(X, p, seed, 1, r + 1, order=order, metric=metric)
    return p


# ---------------------------------------------------------------------------------------
# distances
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("d", [1, 5, 33, 128, 200])
@pytest.mark.parametrize("metric", [0, 1])
def test_pair_dist_exact_on_integers(G, orc, d, metric):
    X = synth.small_integers(400, d, -8, 8, seed=d)
    Xd, _ = G.device_points(X)
    g = np.random.default_rng(1)
    pairs = g.integers(0, 400, size=(3000, 2)).astype(np.int32)
    got = G.pair_dist(Xd, d, torch.from_numpy(pairs), metric).cpu().numpy()
    want = np.array([orc.dist(X[a], X[b], metric) for a, b in pairs])
    assert (got.astype(np.float64) == want).all()


def test_pair_dist_fp32_within_1e5_of_fp64(G, orc):
    X = synth.gaussian_mixture(2000, 128, 20, 10.0, 1.0, seed=0)
    Xd, _ = G.device_points(X)
    pairs = np.random.default_rng(2).integers(0, 2000, size=(4000, 2)).astype(np.int32)
    pairs = pairs[pairs[:, 0] != pairs[:, 1]]
    got = G.pair_dist(Xd, 128, torch.from_numpy(pairs)).cpu().numpy().astype(np.float64)
    want = np.array([orc.dist(X[a], X[b]) for a, b in pairs])
    assert np.max(np.abs(got - want) / want) <= 1e-5


# ---------------------------------------------------------------------------------------
# rnd_init
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("n,d,S,R", [(3000, 33, 16, 32), (700, 8, 64, 64), (2, 3, 1, 2), (65, 5, 64, 64),
                                     (900, 9, 200, 256), (300, 20, 64, 128), (257, 3, 256, 256)])
def test_pool_init_matches_oracle(G, orc, n, d, S, R):
    X = synth.small_integers(n, d, -8, 8, seed=n + d)
    Xd, _ = G.device_points(X)
    keys, deg = G.pool_init(Xd, d, S, R, seed=123)
    pool, _ = orc.init(X, S, R, 123)
    assert_pool_equal(G, keys, deg, pool)


# ---------------------------------------------------------------------------------------
# one round: rnd_join + rev_merge
# ---------------------------------------------------------------------------------------

CASES = [
    # n, d, S, R, order, metric, rounds of history
    (2000, 33, 16, 32, 0, 0, 0),
    (2000, 33, 16, 32, 0, 0, 3),
    (1500, 4, 8, 8, 0, 0, 2),        # many coincident points: ties everywhere
    (1500, 200, 32, 64, 0, 0, 1),    # two dimension chunks, full-width masks
    (1500, 16, 64, 64, 0, 0, 0),     # every pool starts full: 2016 pairs per vertex
    (1200, 12, 16, 32, 1, 0, 2),     # ascending order (Alg 2)
    (1200, 12, 16, 32, 2, 0, 2),     # descending order
    (1200, 12, 16, 32, 0, 1, 2),     # inner product
    (1200, 128, 48, 64, 0, 0, 1),    # pools of 33..64 entries, rows of exactly 128 floats
    (1200, 37, 40, 64, 0, 1, 1),     # pools of 33..64 entries, inner product, ragged rows
    (1200, 11, 40, 64, 2, 0, 2),     # pools of 33..64 entries, descending order
    # wide pools (65..256 entries): multi-word fire and closer masks, the wide merge
    (1000, 12, 80, 96, 0, 0, 1),     # R = 96, pools of every size class
    (800, 10, 128, 128, 0, 0, 0),    # R = 128, every pool starts full
    (700, 9, 200, 256, 0, 0, 1),     # R = 256: four mask words
    (700, 40, 150, 256, 1, 0, 1),    # R = 256, ascending order, two tile chunks of dimensions
    (600, 7, 100, 128, 0, 1, 2),     # R = 128, inner product
    (600, 150, 90, 128, 2, 0, 1),    # R = 128, descending order, FP32 rows longer than 128
]


@pytest.mark.parametrize("n,d,S,R,order,metric,hist", CASES)
def test_join_round_matches_oracle(G, orc, n, d, S, R, order, metric, hist):
    X = synth.small_integers(n, d, -3 if d <= 4 else -8, 3 if d <= 4 else 8, seed=7 * d + R)
    Xd, _ = G.device_points(X)
    seed = 99
    p = oracle_state(orc, X, S, R, seed, hist, metric, order)
    keys, deg = to_keys(G, p), torch.from_numpy(p.deg).cuda()
    for t2 in (hist + 1, hist + 2):
        want, _, st = orc.round_(X, p, seed, 1, t2, order=order, metric=metric)
        stats = torch.zeros(8, dtype=torch.int64, device="cuda")
        keys, deg = G.join_round(Xd, d, keys, deg, seed, 1, t2, order, metric, stats=stats)
        assert_pool_equal(G, keys, deg, want)
        s = stats.cpu().numpy()
        assert s[3] == st[1]          # pairs fired
        assert s[4] == st[2]          # proposals
        assert s[5] == int(((want.old == 0) & (want.ids >= 0)).sum())
        p = want


# ids 26175 and 54119 share the high 32 bits of their visit-order hash at seed 1, round
# (1, 1), vertex 0 (found by searching the oracle's hash); the kernels rank visit orders
# over those bits and must fall back to the full (h, id) order for such a pool
TIE_SEED, TIE_IDS = 1, (26175, 54119)


@pytest.mark.parametrize("m", [12, 30, 50])
def test_join_round_visit_order_tie_in_high_hash_bits(G, orc, m):
    ha, hb = (orc.counter_hash(TIE_SEED, 1, 1, 0, i) for i in TIE_IDS)
    assert ha >> 32 == hb >> 32 and ha != hb
    n, d, R = 60000, 8, 64
    X = synth.small_integers(n, d, -8, 8, seed=m)
    rng = np.random.default_rng(m)
    others = rng.choice(np.setdiff1d(np.arange(1, n), TIE_IDS), m - 2, replace=False)
    ids = np.concatenate([others, TIE_IDS]).astype(np.int64)
    dist = np.array([orc.dist(X[0], X[i]) for i in ids])
    o = np.lexsort((ids, dist))
    p = orc.Pool.empty(n, R)
    p.ids[0, :m], p.dist[0, :m], p.deg[0] = ids[o], dist[o], m
    Xd, _ = G.device_points(X)
    want, _, _ = orc.round_(X, p, TIE_SEED, 1, 1)
    keys, deg = G.join_round(Xd, d, to_keys(G, p), torch.from_numpy(p.deg).cuda(), TIE_SEED, 1, 1)
    assert_pool_equal(G, keys, deg, want)


def test_join_round_skips_old_pairs_exactly(G, orc):
    # the device always skips old x old pairs; the oracle evaluates them: same pools
    X = synth.small_integers(1500, 10, -8, 8, seed=5)
    Xd, _ = G.device_points(X)
    p = oracle_state(orc, X, 16, 32, 3, 4)
    assert p.old.sum() > 0
    want, _, st_full = orc.round_(X, p, 3, 1, 5, skip_old=False)
    _, _, st_skip = orc.round_(X, p, 3, 1, 5, skip_old=True)
    stats = torch.zeros(8, dtype=torch.int64, device="cuda")
    keys, deg = G.join_round(Xd, 10, to_keys(G, p), torch.from_numpy(p.deg).cuda(), 3, 1, 5, stats=stats)
    assert_pool_equal(G, keys, deg, want)
    k = ((p.old == 0) & (p.ids >= 0)).sum(1).astype(np.int64)
    m = p.deg.astype(np.int64)
    assert stats[2].item() == int((k * (m - 1) - k * (k - 1) // 2).sum())  # pairs with a new side
    assert st_skip[0] < st_full[0]


def test_join_round_gaussian_config1(G, orc):
    """10k x 32 mixture: one step from the same state gives the oracle's id sets except
    on vertices the oracle flags as FP32-ambiguous (and the targets they reach)."""
    X = synth.gaussian_mixture(10000, 32, 20, 10.0, 1.0, seed=0)
    Xd, _ = G.device_points(X)
    tol = 2 * (32 + 2) * 2.0**-24 * 2
    p = oracle_state(orc, X, 16, 32, 0, 2)
    want, flags, _ = orc.round_(X, p, 0, 1, 3, tol=tol)
    keys, deg = G.join_round(Xd, 32, to_keys(G, p), torch.from_numpy(p.deg).cuda(), 0, 1, 3)
    ids, dist, old, dg = from_gpu(G, keys, deg)
    unsure = np.zeros(len(X), bool)
    for v in np.nonzero(flags & 1)[0]:
        unsure[v] = True
        unsure[p.ids[v, :p.deg[v]]] = True
    unsure |= (flags & 2) != 0
    assert (flags != 0).mean() < 0.005      # FP32-ambiguous decisions are rare
    assert unsure.mean() < 0.05             # ... and reach few targets
    same = [set(ids[u, :dg[u]]) == set(want.ids[u, :want.deg[u]]) for u in range(len(X)) if not unsure[u]]
    assert all(same)
    m = (ids >= 0) & ~unsure[:, None] & (ids == want.ids)
    rel = np.abs(dist[m].astype(np.float64) - want.dist[m]) / np.maximum(want.dist[m], 1e-30)
    assert rel.max() <= 1e-5


# ---------------------------------------------------------------------------------------
# reverse sampling, final prune
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("rho,R", [(0.0, 32), (0.6, 32), (1.0, 32), (0.6, 128), (1.0, 256)])
def test_reverse_sample_matches_oracle(G, orc, rho, R):
    X = synth.small_integers(3000 if R <= 64 else 800, 9, -8, 8, seed=11)
    p = oracle_state(orc, X, R // 2, R, 5, 6 if R <= 64 else 2)
    want, _ = orc.reverse(p, rho)
    keys, deg = G.reverse_sample(to_keys(G, p), torch.from_numpy(p.deg).cuda(), rho)
    assert_pool_equal(G, keys, deg, want)


@pytest.mark.parametrize("order,R", [(0, 32), (1, 32), (0, 200)])
def test_final_prune_matches_oracle(G, orc, order, R):
    X = synth.small_integers(2500 if R <= 64 else 700, 20, -8, 8, seed=13)
    Xd, _ = G.device_points(X)
    p = oracle_state(orc, X, R // 2, R, 8, 2)
    gids, gd, gdeg, _ = orc.final_prune(X, p, 8, 9, order=order)
    keys, deg = G.final_prune(Xd, 20, to_keys(G, p), torch.from_numpy(p.deg).cuda(), 8, 9, order)
    ids, dist, _, dg = from_gpu(G, keys, deg)
    assert (dg == gdeg).all() and (ids == gids).all()
    m = gids >= 0
    assert (dist[m] == gd[m].astype(np.float32)).all()


# ---------------------------------------------------------------------------------------
# whole build through grnnd_build_ex
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("n,d,S,R,T1,T2,metric,order,final", [
    (3000, 16, 8, 16, 3, 4, 0, 0, True),
    (2000, 7, 12, 32, 2, 5, 0, 0, False),
    (1500, 24, 16, 32, 2, 3, 1, 0, True),
    (1500, 24, 16, 32, 2, 3, 0, 1, True),
])
def test_build_matches_oracle(G, orc, n, d, S, R, T1, T2, metric, order, final):
    X = synth.small_integers(n, d, -8, 8, seed=n + d)
    g = G.build(X, S=S, R=R, T1=T1, T2=T2, rho=0.6, seed=17, metric=metric, order=order, final_prune=final)
    ids, dist, deg = g.to_numpy()
    wids, wd, wdeg, _ = orc.build_graph(X, S, R, T1, T2, 0.6, 17, metric=metric, order=order, final_prune=final)
    assert (deg == wdeg).all()
    assert (ids == wids).all()
    m = wids >= 0
    assert (dist[m] == wd[m].astype(np.float32)).all()
    assert g.entry == orc.entry(X, metric)
    st = g.stats()
    assert st["rounds"] >= 1 and st["pair_distances"] > 0


@pytest.mark.parametrize("R,S,precision,metric", [(96, 48, 0, 0), (128, 100, 1, 0), (256, 64, 0, 1),
                                                   (256, 200, 2, 0), (160, 160, 1, 1)])
def test_build_wide_pools_matches_oracle(G, orc, R, S, precision, metric):
    # pools of up to 256 entries (Sec 3.5's fixed capacity): init, rounds with the wide join
    # and merge, reverse sampling, final prune, search; integer data keeps every form exact
    X, Q = synth.small_integers(1200, 16, -8, 8, seed=R + S, nq=50)
    g = G.build(X, S=S, R=R, T1=2, T2=3, rho=0.6, seed=21, metric=metric, precision=precision)
    ids, dist, deg = g.to_numpy()
    wids, wd, wdeg, _ = orc.build_graph(X, S, R, 2, 3, 0.6, 21, metric=metric)
    assert (deg == wdeg).all() and (ids == wids).all()
    assert (dist[wids >= 0] == wd[wids >= 0].astype(np.float32)).all()
    assert g.stats()["rechecks"] == 0
    want, _, _ = orc.search(wids, wdeg, X, Q, 10, 64, orc.entry(X, metric), metric=metric)
    assert (g.search(Q, 10, 64) == want).all()


def test_build_wide_pools_keep_the_last_pool(G, orc):
    # without the final prune the graph is the last pool: rows of up to R = 256 entries
    X = synth.small_integers(900, 6, -4, 4, seed=3)
    g = G.build(X, S=128, R=256, T1=2, T2=2, seed=2, final_prune=False)
    ids, dist, deg = g.to_numpy()
    wids, wd, wdeg, _ = orc.build_graph(X, 128, 256, 2, 2, 0.6, 2, final_prune=False)
    assert (deg == wdeg).all() and (ids == wids).all()
    assert deg.max() > 64


def test_plain_calls_run_on_the_current_stream(G):
    # grnnd_build / grnnd_search / grnnd_graph_copy take no stream: they run on the calling
    # thread's current stream (here a side stream), with the same results
    import ctypes
    X, Q = synth.small_integers(3000, 16, -8, 8, seed=4, nq=64)
    ref = G.build(X, S=8, R=16, T1=2, T2=3, seed=3)
    want, want_q = ref.to_numpy(), ref.search(Q, 10, 32)
    L = G.lib()
    side = torch.cuda.Stream()
    L.grnnd_set_stream(ctypes.c_void_p(side.cuda_stream))
    try:
        assert L.grnnd_get_stream() == side.cuda_stream
        h = ctypes.c_void_p()
        assert L.grnnd_build(X.ctypes.data_as(ctypes.c_void_p), 3000, 16, 0, 8, 16, 2, 3, 3, ctypes.byref(h)) == G.OK
        g = G._graph_of(h)
        got = g.to_numpy()
        out = np.empty((64, 10), np.int32)
        assert L.grnnd_search(h, Q.ctypes.data_as(ctypes.c_void_p), 64, 10, 32,
                              out.ctypes.data_as(ctypes.c_void_p)) == G.OK
    finally:
        L.grnnd_set_stream(None)
    for a, b in zip(got, want):
        assert (a == b).all()
    assert (out == want_q).all()


def test_build_device_input_equals_host_input(G):
    X = synth.gaussian_mixture(4000, 20, 8, 5.0, 1.0, seed=4)
    a = G.build(X, S=8, R=16, T1=2, T2=3, seed=1).to_numpy()
    b = G.build(torch.from_numpy(X).cuda(), S=8, R=16, T1=2, T2=3, seed=1).to_numpy()
    for x, y in zip(a, b):
        assert (x == y).all()


def test_build_is_deterministic(G):
    X = synth.gaussian_mixture(5000, 32, 10, 10.0, 1.0, seed=9)
    a = G.build(X, S=16, R=32, T1=2, T2=4, seed=3).to_numpy()
    b = G.build(X, S=16, R=32, T1=2, T2=4, seed=3).to_numpy()
    for x, y in zip(a, b):
        assert (x == y).all()


def test_build_degenerate_inputs(G, orc):
    # every point identical: all distances 0, every decision settled by ids
    X = np.ones((300, 6), np.float32)
    g = G.build(X, S=8, R=16, T1=2, T2=2, seed=2)
    ids, dist, deg = g.to_numpy()
    wids, _, wdeg, _ = orc.build_graph(X, 8, 16, 2, 2, 0.6, 2)
    assert (ids == wids).all() and (deg == wdeg).all()
    # the smallest problem: two points
    g2 = G.build(np.array([[0.0], [1.0]], np.float32), S=1, R=2, T1=1, T2=1)
    i2, d2, dg2 = g2.to_numpy()
    assert dg2.tolist() == [1, 1] and i2[0, 0] == 1 and i2[1, 0] == 0 and d2[0, 0] == 1.0


def test_build_rejects_non_finite(G):
    X = np.zeros((50, 4), np.float32)
    X[7, 2] = np.nan
    with pytest.raises(G.GrnndError) as e:
        G.build(X, S=4, R=8)
    assert e.value.status == G.EINVAL


def test_hbm_budget_is_checked_before_allocation(G):
    X = np.zeros((1000, 8), np.float32)
    with pytest.raises(G.GrnndError) as e:
        G.build(X, S=4, R=8, hbm_budget=1000)
    assert e.value.status == G.ENOMEM


# ---------------------------------------------------------------------------------------
# entry, search, k-NN
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("metric", [0, 1])
@pytest.mark.parametrize("case", ["integers", "gauss", "deep", "ties"])
def test_entry_point_matches_oracle(G, orc, metric, case):
    # the FP32 pre-filter must never drop the FP64 nearest point, ties included
    if case == "integers":
        X = synth.small_integers(5000, 13, -8, 8, seed=3)
    elif case == "gauss":
        X = synth.gaussian_mixture(20000, 40, 10, 5.0, 1.0, seed=8)
    elif case == "deep":
        X = synth.deep_like(20000, d=96, seed=9)
    else:  # +-e_k and copies: every point at the same distance from the mean (0)
        E = np.eye(12, dtype=np.float32)
        X = np.concatenate([E, -E, E, -E, 3 * E, -3 * E])
    d = X.shape[1]
    Xd, _ = G.device_points(X)
    assert G.entry_point(Xd, d, metric) == orc.entry(X, metric)


@pytest.mark.parametrize("beam", [10, 32, 64, 200])
def test_search_matches_oracle(G, orc, beam):
    X, Q = synth.small_integers(3000, 12, -8, 8, seed=21, nq=120)
    gids, gd, gdeg, _ = orc.build_graph(X, 8, 16, 2, 3, 0.6, 4)
    e = orc.entry(X)
    want, wdist, _ = orc.search(gids, gdeg, X, Q, 10, beam, e)
    Xd, _ = G.device_points(X)
    Qd, _ = G.device_points(Q)
    ids, dd = G.search_graph(Xd, 12, torch.from_numpy(gids).cuda(), torch.from_numpy(gdeg).cuda(), e, Qd, 10, beam)
    assert (ids.cpu().numpy() == want).all()
    assert (dd.cpu().numpy().astype(np.float64) == wdist).all()


def test_search_api_matches_step_search(G):
    X, Q = synth.gaussian_mixture(6000, 24, 10, 5.0, 1.0, seed=2, nq=200)
    g = G.build(X, S=12, R=24, T1=2, T2=4, seed=5)
    a = g.search(Q, 10, 48)
    ids, _, deg = g.to_numpy()
    Xd, _ = G.device_points(X)
    Qd, _ = G.device_points(Q)
    b, _ = G.search_graph(Xd, 24, torch.from_numpy(ids).cuda(), torch.from_numpy(deg).cuda(), g.entry, Qd, 10, 48)
    assert (a == b.cpu().numpy()).all()
    c = g.search(torch.from_numpy(Q).cuda(), 10, 48)
    assert (c.cpu().numpy() == a).all()


@pytest.mark.parametrize("n,d,k", [(3000, 33, 10), (777, 3, 32), (100, 130, 1)])
def test_brute_knn_matches_oracle(G, orc, n, d, k):
    X, Q = synth.small_integers(n, d, -4, 4, seed=n, nq=70)
    want, wd = orc.brute_knn(X, Q, k)
    Xd, _ = G.device_points(X)
    Qd, _ = G.device_points(Q)
    ids, dd = G.brute_knn(Xd, d, Qd, k)
    assert (ids.cpu().numpy() == want).all()
    assert (dd.cpu().numpy().astype(np.float64) == wd).all()


# ---------------------------------------------------------------------------------------
# BF16 form: tensor-core Gram tiles with an error bound and FP32 re-decisions
# ---------------------------------------------------------------------------------------

def _bf16(X):
    """Round-to-nearest-even float32 -> bfloat16, returned as float32."""
    b = np.ascontiguousarray(X, np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32)


def _bf16_bound(D, ni, nj, ei, ej, d):
    """The per-pair bound that the BF16 form states (include/grnnd.h): arithmetic,
    quantisation and FP32 reference-rounding terms, u = 2^-23."""
    u = 2.0 ** -23
    g = d * u / (1 - d * u)
    si, sj = np.sqrt(ni), np.sqrt(nj)
    ar = (g + 2 * u) * (si + sj) ** 2
    e = ei + ej
    qz = e * (2 * np.sqrt(max(D, 0) + ar) + e)
    return (ar + qz + (d + 3) * u * (max(D, 0) + ar + qz)) * 1.0001


@pytest.mark.parametrize("n,d,S,R,metric", [(3000, 16, 8, 16, 0), (2500, 128, 32, 64, 0), (1800, 40, 16, 32, 1),
                                            (1500, 200, 16, 32, 0), (1800, 40, 32, 64, 1), (2000, 100, 40, 64, 0)])
def test_bf16_build_is_exact_on_integer_data(G, orc, n, d, S, R, metric):
    # integers with d * max|x|^2 < 2^24: every BF16 product and FP32 partial sum is exact,
    # so the BF16 form must return the FP32 form's graph bit for bit (and the oracle's).
    X = synth.small_integers(n, d, -8, 8, seed=d + n)
    a = G.build(X, S=S, R=R, T1=2, T2=4, seed=3, metric=metric, precision=G.FP32).to_numpy()
    gb = G.build(X, S=S, R=R, T1=2, T2=4, seed=3, metric=metric, precision=G.BF16)
    b = gb.to_numpy()
    for x, y in zip(a, b):
        assert (x == y).all()
    assert gb.stats()["rechecks"] == 0
    wids, _, wdeg, _ = orc.build_graph(X, S, R, 2, 4, 0.6, 3, metric=metric)
    assert (b[0] == wids).all() and (b[2] == wdeg).all()


def test_bf16_build_sift_shaped_matches_fp32(G):
    X = synth.sift_like(20000, 0, seed=1)
    a = G.build(X, S=32, R=64, T1=2, T2=5, seed=1, precision=G.FP32).to_numpy()
    b = G.build(X, S=32, R=64, T1=2, T2=5, seed=1, precision=G.BF16).to_numpy()
    for x, y in zip(a, b):
        assert (x == y).all()


def test_bf16_build_continuous_data(G, orc):
    """Gaussian data: BF16 is not exact, so decisions near the bound are re-taken in FP32.
    The graph must satisfy every invariant, its recorded distances must be within the
    stated bound of FP64, and its recall must match the FP32 form's closely."""
    X, Q = synth.gaussian_mixture(6000, 48, 12, 6.0, 1.0, seed=5, nq=300)
    ga = G.build(X, S=16, R=32, T1=3, T2=6, seed=2, precision=G.FP32)
    gb = G.build(X, S=16, R=32, T1=3, T2=6, seed=2, precision=G.BF16)
    ids, dist, deg = gb.to_numpy()
    assert gb.stats()["rechecks"] > 0
    xb = _bf16(X).astype(np.float64)
    nrm = (xb ** 2).sum(1)
    res = np.sqrt(((X.astype(np.float64) - xb) ** 2).sum(1))
    for v in range(0, len(X), 7):
        row = ids[v, :deg[v]]
        assert v not in row and len(set(row.tolist())) == len(row) and (row >= 0).all()
        for j, u in enumerate(row[:8]):
            ref = orc.dist(X[v], X[u])
            bound = _bf16_bound(ref, nrm[v], nrm[u], res[v], res[u], X.shape[1])
            assert abs(dist[v, j] - ref) <= bound
    gt, _ = orc.brute_knn(X, Q, 10)
    ra = orc.recall_at_k(ga.search(Q, 10, 32), gt)
    rb = orc.recall_at_k(gb.search(Q, 10, 32), gt)
    assert rb >= ra - 0.01 and rb > 0.9


# ---------------------------------------------------------------------------------------
# FP8 form: e4m3 Gram tiles with a power-of-two scale per row, the same bound and
# FP32 re-decisions
# ---------------------------------------------------------------------------------------

def _e4m3(a):
    """Round-to-nearest-even float64 -> e4m3 (3 mantissa bits, smallest normal 2^-6,
    subnormal step 2^-9, saturating at 448), returned as float64."""
    a = np.asarray(a, np.float64)
    m = np.abs(a)
    E = np.floor(np.log2(np.where(m > 0, m, 1.0)))
    step = 2.0 ** (np.maximum(E, -6.0) - 3.0)
    q = np.minimum(np.rint(m / step) * step, 448.0)
    return np.sign(a) * np.where(m > 0, q, 0.0)


def _fp8_rows(X):
    """The FP8 form's dequantised rows: per row the scale 2^e with e = E - 8 for
    max|x| = f 2^E, f in [0.5, 1) (e = 0 for a zero row), then x_hat = 2^e e4m3(x 2^-e)."""
    X = np.asarray(X, np.float64)
    amax = np.abs(X).max(1)
    _, E = np.frexp(amax)
    e = np.where(amax > 0, np.clip(E - 8, -126, 127), 0).astype(np.float64)
    sc = 2.0 ** e
    return _e4m3(X / sc[:, None]) * sc[:, None]


def test_e4m3_emulation_pins():
    # the emulation against values fixed by the e4m3 format itself
    assert list(_e4m3([0.0, 1.0, 1.0625, 1.125, 1.1875, 17.0, 448.0, 500.0, -3.3, 2.0 ** -9, 2.0 ** -10 * 1.5])) == \
        [0.0, 1.0, 1.0, 1.125, 1.25, 16.0, 448.0, 448.0, -3.25, 2.0 ** -9, 2.0 ** -9]


@pytest.mark.parametrize("n,d,S,R,metric", [(3000, 16, 8, 16, 0), (2500, 128, 32, 64, 0), (1800, 40, 16, 32, 1),
                                            (1500, 200, 16, 32, 0), (1800, 40, 32, 64, 1), (2000, 100, 40, 64, 0)])
def test_fp8_build_is_exact_on_integer_data(G, orc, n, d, S, R, metric):
    # integers of magnitude <= 16 are exact in e4m3 at any power-of-two scale; with
    # d * max|x|^2 < 2^24 every product and FP32 partial sum is exact, so the FP8 form must
    # return the FP32 form's graph bit for bit (and the oracle's), with no re-decision.
    X = synth.small_integers(n, d, -8, 8, seed=d + n + 1)
    a = G.build(X, S=S, R=R, T1=2, T2=4, seed=3, metric=metric, precision=G.FP32).to_numpy()
    gq = G.build(X, S=S, R=R, T1=2, T2=4, seed=3, metric=metric, precision=G.FP8)
    b = gq.to_numpy()
    for x, y in zip(a, b):
        assert (x == y).all()
    assert gq.stats()["rechecks"] == 0
    wids, _, wdeg, _ = orc.build_graph(X, S, R, 2, 4, 0.6, 3, metric=metric)
    assert (b[0] == wids).all() and (b[2] == wdeg).all()


def test_fp8_exact_mode_needs_full_fp32_accumulation(G):
    # integers in [-16, 16] over d = 1024: dot products reach 2^18 with every unit significant,
    # so an accumulator that kept fewer than 19 significant bits would change distances and the
    # graph; the FP8 form must still equal the FP32 form (its exact mode assumes FP32 sums).
    X = synth.small_integers(1500, 1024, -16, 16, seed=21)
    kw = dict(S=16, R=32, T1=2, T2=3, seed=4)
    a = G.build(X, precision=G.FP32, **kw).to_numpy()
    gq = G.build(X, precision=G.FP8, **kw)
    for x, y in zip(a, gq.to_numpy()):
        assert (x == y).all()
    assert gq.stats()["rechecks"] == 0


@pytest.mark.parametrize("metric", [0, 1])
def test_fp8_build_continuous_data(G, orc, metric):
    """Continuous data: e4m3 rows are far from exact, so many decisions are re-taken in
    FP32.  Invariants hold, every recorded distance is within the stated bound (computed
    from the emulated e4m3 rows) of FP64, and recall stays close to the FP32 form's."""
    if metric == 0:
        X, Q = synth.gaussian_mixture(6000, 48, 12, 6.0, 1.0, seed=5, nq=300)
        kw = dict(S=16, R=32, T1=3, T2=6, seed=2)
    else:
        X, Q = synth.deep_like(6000, 300, d=64, seed=6)
        kw = dict(S=16, R=32, T1=3, T2=6, seed=2, metric=1)
    ga = G.build(X, precision=G.FP32, **kw)
    gq = G.build(X, precision=G.FP8, **kw)
    ids, dist, deg = gq.to_numpy()
    assert gq.stats()["rechecks"] > 0
    xq = _fp8_rows(X)
    nrm = (xq ** 2).sum(1)
    res = np.sqrt(((X.astype(np.float64) - xq) ** 2).sum(1))
    d = X.shape[1]
    for v in range(0, len(X), 7):
        row = ids[v, :deg[v]]
        assert v not in row and len(set(row.tolist())) == len(row) and (row >= 0).all()
        for j, u in enumerate(row[:8]):
            ref = orc.dist(X[v], X[u], metric=metric)
            if metric == 0:
                bound = _bf16_bound(ref, nrm[v], nrm[u], res[v], res[u], d)
            else:
                u_ = 2.0 ** -23
                g = d * u_ / (1 - d * u_)
                si, sj = np.sqrt(nrm[v]), np.sqrt(nrm[u])
                tot = (g + 2 * u_) * si * sj + 2 * u_ * abs(ref) + res[v] * sj + res[u] * si + res[v] * res[u]
                bound = (tot + (d + 3) * u_ * (abs(ref) + si * sj + tot)) * 1.0001
            assert abs(dist[v, j] - ref) <= bound * 1.001 + 1e-30
    gt, _ = orc.brute_knn(X, Q, 10, metric=metric)
    ra = orc.recall_at_k(ga.search(Q, 10, 32), gt)
    rq = orc.recall_at_k(gq.search(Q, 10, 32), gt)
    assert rq >= ra - 0.02 and rq > 0.85


# ---------------------------------------------------------------------------------------
# one step of the BF16 / FP8 forms from an oracle state on continuous data
# ---------------------------------------------------------------------------------------

def _q_rows(X, precision):
    """Dequantised rows of a precision form (emulated in numpy), their squared norms and
    residual norms: the terms the stated error bound is made of."""
    xq = _bf16(X).astype(np.float64) if precision == 1 else _fp8_rows(X)
    return (xq ** 2).sum(1), np.sqrt(((X.astype(np.float64) - xq) ** 2).sum(1))


def _q_bound(metric, D, ni, nj, ei, ej, d):
    """The stated per-pair bound on |tile distance - FP32 distance| (BF16 and FP8 forms)."""
    if metric == 0:
        return _bf16_bound(D, ni, nj, ei, ej, d)
    u = 2.0 ** -23
    g = d * u / (1 - d * u)
    si, sj = np.sqrt(ni), np.sqrt(nj)
    tot = (g + 2 * u) * si * sj + 2 * u * abs(D) + ei * sj + ej * si + ei * ej
    return (tot + (d + 3) * u * (abs(D) + si * sj + tot)) * 1.0001


def _continuous_case(shape):
    if shape == "gauss":  # the 10k x 32 mixture, L2
        return synth.gaussian_mixture(10000, 32, 20, 10.0, 1.0, seed=0), 0, 16, 32
    X = synth.deep_like(8000, d=96, seed=3)  # DEEP-shaped unit vectors, inner product
    return X, 1, 16, 32


@pytest.mark.parametrize("precision", [1, 2])
@pytest.mark.parametrize("shape", ["gauss", "deep"])
def test_precision_prune_matches_oracle_on_continuous_data(G, orc, shape, precision):
    """Every fire decision of the BF16 / FP8 tiles either clears the stated bound or is
    re-taken in FP32, so each vertex's survivors are the oracle's except where the oracle
    itself flags a decision as within FP32 rounding.  The prune-only pass shows the decisions
    alone (no merge): unflagged rows must equal the oracle's bit for bit."""
    X, metric, S, R = _continuous_case(shape)
    n, d = X.shape
    Xd, _ = G.device_points(X)
    qp = G.quantize(Xd, d, precision)
    tol = 2 * (d + 2) * 2.0 ** -24 * 2
    p = oracle_state(orc, X, S, R, 7, 2, metric)
    gids, gd, gdeg, flags = orc.final_prune(X, p, 7, 5, metric=metric, tol=tol)
    keys, deg = G.final_prune(Xd, d, to_keys(G, p), torch.from_numpy(p.deg).cuda(), 7, 5, metric=metric,
                              precision=precision, qpoints=qp)
    ids, dist, _, dg = from_gpu(G, keys, deg)
    ok = flags == 0
    assert ok.mean() > 0.99
    assert (dg[ok] == gdeg[ok]).all()
    assert (ids[ok] == gids[ok]).all()
    m = (gids >= 0) & ok[:, None]
    assert (dist[m] == gd[m].astype(np.float32)).all()  # survivors keep their recorded distances


@pytest.mark.parametrize("precision", [1, 2])
@pytest.mark.parametrize("shape", ["gauss", "deep"])
def test_precision_round_matches_oracle_on_continuous_data(G, orc, shape, precision, record_property):
    """One join round in the BF16 / FP8 forms from an oracle state.  The decisions are the
    oracle's (test above); a redirect records the tile distance, which may differ from FP64
    by the stated bound, so a target's R-entry cut may swap entries whose distances are within
    their bounds of each other.  Every unflagged target must hold the oracle's id set, or a set
    that differs only by such swaps; every recorded distance must be within its bound of FP64."""
    X, metric, S, R = _continuous_case(shape)
    n, d = X.shape
    Xd, _ = G.device_points(X)
    qp = G.quantize(Xd, d, precision)
    nrm, res = _q_rows(X, precision)
    tol = 2 * (d + 2) * 2.0 ** -24 * 2
    p = oracle_state(orc, X, S, R, 7, 2, metric)
    want, flags, _ = orc.round_(X, p, 7, 1, 3, metric=metric, tol=tol)
    keys, deg = G.join_round(Xd, d, to_keys(G, p), torch.from_numpy(p.deg).cuda(), 7, 1, 3, metric=metric,
                             precision=precision, qpoints=qp)
    ids, dist, _, dg = from_gpu(G, keys, deg)
    unsure = np.zeros(n, bool)
    for v in np.nonzero(flags & 1)[0]:  # a flagged prune reaches v and every member of its pool
        unsure[v] = True
        unsure[p.ids[v, :p.deg[v]]] = True
    assert unsure.mean() < 0.5  # most targets are reached by unflagged prunes only

    X64 = X.astype(np.float64)

    def d64(u, xs):  # FP64 distances from u to the ids xs
        xs = np.asarray(xs, np.int64)
        if metric == 0:
            return ((X64[xs] - X64[u]) ** 2).sum(1)
        return 1.0 - X64[xs] @ X64[u]

    def bnd(u, xs, D):
        return np.array([_q_bound(metric, Dk, nrm[u], nrm[x], res[u], res[x], d) for x, Dk in zip(xs, D)])

    exact = swapped = 0
    for u in np.nonzero(~unsure)[0]:
        a = ids[u, :dg[u]]
        b = want.ids[u, :want.deg[u]]
        assert dg[u] == want.deg[u], u  # the same candidates, hence the same count
        ref = d64(u, a)                 # recorded distances within their bound of FP64
        slack = 1e-6 * np.maximum(1.0, np.abs(ref))
        assert (np.abs(dist[u, :dg[u]] - ref) <= bnd(u, a, ref) * 1.001 + slack).all(), u
        if set(a.tolist()) == set(b.tolist()):
            exact += 1
            continue
        swapped += 1
        only_gpu = np.array(sorted(set(a.tolist()) - set(b.tolist())), np.int64)
        only_orc = np.array(sorted(set(b.tolist()) - set(a.tolist())), np.int64)
        dy, dx = d64(u, only_gpu), d64(u, only_orc)
        by, bx = bnd(u, only_gpu, dy), bnd(u, only_orc, dx)
        # every entry only the GPU kept is at most as far as every entry only the oracle kept,
        # up to the two bounds
        assert (dy[:, None] <= dx[None, :] + bx[None, :] + by[:, None] +
                1e-6 * np.maximum(1.0, np.abs(dx))[None, :]).all(), (u, only_gpu, only_orc)
    record_property("exact_targets", exact)
    record_property("swapped_targets", swapped)
    assert exact >= 0.5 * (exact + swapped)


# ---------------------------------------------------------------------------------------
# in-place pool updates (the build's own mode)
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("n,d,S,R,hist", [(2500, 20, 16, 32, 0), (2000, 9, 32, 64, 2), (1500, 150, 48, 64, 1)])
def test_join_round_in_place_matches_oracle(G, orc, n, d, S, R, hist):
    X = synth.small_integers(n, d, -8, 8, seed=n + d)
    Xd, _ = G.device_points(X)
    p = oracle_state(orc, X, S, R, 41, hist)
    keys, deg = to_keys(G, p), torch.from_numpy(p.deg).cuda()
    ws = G.workspace(n, R)
    for t2 in (hist + 1, hist + 2, hist + 3):
        want, _, _ = orc.round_(X, p, 41, 1, t2)
        keys, deg = G.join_round(Xd, d, keys, deg, 41, 1, t2, ws=ws, inplace=True)
        assert_pool_equal(G, keys, deg, want)
        p = want
    want, _ = orc.reverse(p, 0.6)
    keys, deg = G.reverse_sample(keys, deg, 0.6, ws=ws, inplace=True)
    assert_pool_equal(G, keys, deg, want)
    G.workspace_status(ws, n, R)  # no device-side wait gave up


# ---------------------------------------------------------------------------------------
# batched builds: each build of a batch equals the same build alone
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("precision,metric", [("fp32", 0), ("bf16", 0), ("bf16", 1), ("fp32", 1), ("fp8", 0)])
def test_build_batch_equals_single_builds(G, orc, precision, metric):
    sizes = [300, 9, 1000, 57, 2000, 128]
    parts = [synth.small_integers(m, 24, -8, 8, seed=100 + i) for i, m in enumerate(sizes)]
    X = np.concatenate(parts)
    off = np.concatenate([[0], np.cumsum(sizes)])
    prec = {"fp32": G.FP32, "bf16": G.BF16, "fp8": G.FP8}[precision]
    kw = dict(S=8, R=16, T1=2, T2=4, rho=0.6, seed=11, metric=metric, precision=prec)
    gs = G.build_batch(torch.from_numpy(X).cuda(), off, **kw)
    Q = synth.small_integers(50, 24, -8, 8, seed=999)
    for b, part in enumerate(parts):
        one = G.build(torch.from_numpy(part).cuda(), **kw)
        a, o = gs[b].to_numpy(), one.to_numpy()
        assert gs[b].n == len(part) and gs[b].entry == one.entry
        assert (a[2] == o[2]).all() and (a[0] == o[0]).all() and (a[1] == o[1]).all(), b
        qa = gs[b].search(torch.from_numpy(Q).cuda(), 5, 16).cpu().numpy()
        qo = one.search(torch.from_numpy(Q).cuda(), 5, 16).cpu().numpy()
        assert (qa == qo).all()
        # and each build of the batch is the oracle's build of its rows (integer data: every
        # form is exact), with the oracle's entry and search results
        wids, wd, wdeg, _ = orc.build_graph(part, 8, 16, 2, 4, 0.6, 11, metric=metric)
        assert (a[0] == wids).all() and (a[2] == wdeg).all()
        assert (a[1][wids >= 0] == wd[wids >= 0].astype(np.float32)).all()
        went = orc.entry(part, metric)
        assert gs[b].entry == went
        if len(part) > 16:
            wq, _, _ = orc.search(wids, wdeg, part, Q, 5, 16, went, metric=metric)
            assert (qa == wq).all()


def test_build_batch_mixed_data_and_free_order(G):
    # an integer build next to a continuous one (the BF16 form's exact mode is decided over
    # the whole pass); graphs freed in any order keep the others valid
    a = synth.small_integers(700, 40, -8, 8, seed=5)
    b = synth.gaussian_mixture(900, 40, seed=6)
    X = np.concatenate([a, b]).astype(np.float32)
    kw = dict(S=12, R=24, T1=2, T2=5, seed=3, precision=G.BF16)
    gs = G.build_batch(X, [0, 700, 1600], **kw)
    ga, gb = G.build(a, **kw), G.build(b, **kw)
    assert (gs[0].to_numpy()[0] == ga.to_numpy()[0]).all()
    del gs[0]
    import gc
    gc.collect()
    assert (gs[0].to_numpy()[0] == gb.to_numpy()[0]).all()


# ---------------------------------------------------------------------------------------
# join launch shapes (grnnd_tuning) change speed only
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("precision,metric", [("bf16", 0), ("fp32", 0), ("bf16", 1), ("fp8", 1)])
def test_tunings_give_the_same_graph(G, precision, metric):
    X = synth.small_integers(3000, 40, -8, 8, seed=77)
    prec = {"fp32": G.FP32, "bf16": G.BF16, "fp8": G.FP8}[precision]
    kw = dict(S=24, R=48, T1=2, T2=5, seed=2, metric=metric, precision=prec)
    ref = G.build(X, **kw).to_numpy()
    for gm, w, t in [((0, 16, 32), 0, 0), ((0, 0, 32), 1, 2), ((8, 16, 16), 2, 4), ((0, 16, 16), 0, 1),
                     ((0, 0, 0), 0, 0)]:
        got = G.build(X, tuning=G.tuning(gm, w, t), **kw).to_numpy()
        for a, b in zip(got, ref):
            assert (a == b).all(), (gm, w, t)


@pytest.mark.parametrize("precision", ["bf16", "fp8"])
@pytest.mark.parametrize("d", [40, 128, 200, 300])
def test_row_copies_give_the_same_graph(G, precision, d):
    """The warp join stages quantized rows by TMA gather4 copies (four rows per copy, boxes of
    one 128-column chunk plus 16 bytes; out-of-range columns read as zero) or by one bulk copy
    per row: the same rows arrive, so the graphs are equal, on integer data (exact tiles) and
    on Gaussian data (tiles with FP32 re-decisions), with one chunk (d <= 128, the box wider
    than the row for d = 40) and several (d = 200, 300)."""
    prec = {"bf16": G.BF16, "fp8": G.FP8}[precision]
    kw = dict(S=16, R=32, T1=2, T2=4, seed=5, precision=prec)
    for X in (synth.small_integers(3000, d, -8, 8, seed=d), synth.gaussian_mixture(3000, d, 10, seed=d)):
        a = G.build(X, tuning=G.tuning(row_copies=2), **kw).to_numpy()
        b = G.build(X, tuning=G.tuning(row_copies=1), **kw).to_numpy()
        for u, v in zip(a, b):
            assert (u == v).all()


@pytest.mark.parametrize("precision", ["bf16", "fp8"])
def test_build_batch_row_copies_give_the_same_graphs(G, precision):
    """Batched builds stage every build's quantized rows through one tensor map over all of
    them: gather4 and per-row staging give the same graphs, build by build."""
    sizes = [700, 40, 3000, 1200]
    parts = [synth.gaussian_mixture(m, 128, 10, seed=200 + i) for i, m in enumerate(sizes)]
    X = torch.from_numpy(np.concatenate(parts)).cuda()
    off = np.concatenate([[0], np.cumsum(sizes)])
    prec = {"bf16": G.BF16, "fp8": G.FP8}[precision]
    kw = dict(S=12, R=32, T1=2, T2=4, seed=13, precision=prec)
    ga = G.build_batch(X, off, tuning=G.tuning(row_copies=2), **kw)
    gb = G.build_batch(X, off, tuning=G.tuning(row_copies=1), **kw)
    for a, b in zip(ga, gb):
        for u, v in zip(a.to_numpy(), b.to_numpy()):
            assert (u == v).all()


@pytest.mark.parametrize("n,d,R", [(3000, 32, 16), (3001, 30, 6)])
def test_pinned_host_points_and_read_back(G, n, d, R):
    """Points in pinned host memory and a graph read back into pinned host memory: aligned
    buffers move by the library's copy kernel, ragged ones (rows padded to 4 floats, a graph
    whose byte size is not a multiple of 16) by the copy engine.  Either way the graph equals
    the one built from device-resident points and read back through the binding."""
    import ctypes
    import torch
    X = synth.small_integers(n, d, -8, 8, seed=n + d)
    kw = dict(S=min(8, R), R=R, T1=2, T2=3, seed=2)
    wids, _, wdeg = G.build(X, **kw).to_numpy()
    L = G.lib()
    Xh = torch.from_numpy(X).pin_memory()
    ids_h = torch.full((n, R), -7, dtype=torch.int32).pin_memory()
    deg_h = torch.full((n,), -7, dtype=torch.int32).pin_memory()
    p = G.params(**kw)
    h = ctypes.c_void_p()
    G._check(L.grnnd_build_ex(ctypes.c_void_p(Xh.data_ptr()), n, d, ctypes.byref(p), ctypes.byref(h)))
    try:
        G._check(L.grnnd_graph_copy(h, ctypes.c_void_p(ids_h.data_ptr()), None, ctypes.c_void_p(deg_h.data_ptr())))
    finally:
        L.grnnd_free(h)
    assert (ids_h.numpy() == wids).all() and (deg_h.numpy() == wdeg).all()


def test_profile_times_only_the_named_kernels(G):
    """grnnd_profile_begin_only brackets only the named kernels with events; the plain form
    brackets every launch.  The build's result does not depend on either."""
    X = synth.small_integers(2000, 16, -8, 8, seed=4)
    kw = dict(S=8, R=16, T1=2, T2=3, seed=1)
    want = G.build(X, **kw).to_numpy()
    G.profile_begin(only=["select", "rnd_init"])
    got = G.build(X, **kw).to_numpy()
    k = G.profile_end()
    assert set(k) == {"select", "rnd_init"}, k
    assert k["rnd_init"][0] == 1 and k["select"][0] >= 1 and k["select"][1] > 0
    G.profile_begin()
    G.build(X, **kw)
    k = G.profile_end()
    assert {"select", "rnd_init", "prep", "scatter"} <= set(k), k
    for a, b in zip(want, got):
        assert (a == b).all()


def test_autotune_pool_picks_a_capacity_that_reaches_the_target(G, orc):
    """grnnd_autotune_pool measures each candidate R's recall on held-out rows against exact
    k-NN; its choice must reach the target when a candidate does, and its recall must equal
    the recall of the same build measured here (builds are deterministic)."""
    n, nq, d, k, beam = 6000, 200, 32, 10, 32
    X = synth.gaussian_mixture(n + nq, d, 20, 10.0, 1.0, seed=4)
    kw = dict(S=16, T1=3, T2=6, seed=3)
    cands, target = [8, 16, 32], 0.9
    R, rec, ms = G.autotune_pool(X, nq, cands, recall_target=target, k=k, beam=beam, **kw)
    assert R in cands and ms > 0
    Xp, _ = G.device_points(X[:n])
    Qp, _ = G.device_points(X[n:])
    gt = G.brute_knn(Xp, d, Qp, k)[0].cpu().numpy()  # the tuner's own ground truth
    gt64 = orc.brute_knn(X[:n], X[n:], k)[0]
    recalls = {}
    for r in cands:
        g = G.build(X[:n], R=r, **{**kw, "S": min(16, r)})
        found = np.asarray(G.search(g, X[n:], k, beam))
        recalls[r] = orc.recall_at_k(found, gt)
        assert abs(recalls[r] - orc.recall_at_k(found, gt64)) <= 0.005
    assert abs(recalls[R] - rec) < 1e-6, (R, rec, recalls)
    if any(v >= target for v in recalls.values()):
        assert recalls[R] >= target
    else:
        assert recalls[R] == max(recalls.values())


def test_autotune_picks_a_candidate(G):
    X = synth.small_integers(4000, 32, -8, 8, seed=8)
    t = G.autotune(X, S=16, R=32, T1=2, T2=4, precision=G.BF16)
    assert t.ms > 0
    assert list(t.group_max) in ([8, 16, 32], [0, 16, 32], [0, 0, 32], [8, 16, 16], [0, 16, 16])
    assert 0 <= t.warp_ctas_per_sm <= 3 and t.team_ctas_per_sm in (0, 2, 4, 6)
    assert t.row_copies in (0, 1, 2)


# ---------------------------------------------------------------------------------------
# checkpoint / resume: the pool state (keys, degrees) between steps is the whole state of a
# build (randomness is counter-based), so a build stopped after any round, saved to the
# host and resumed in a new workspace ends with the graph of an uninterrupted build
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("stop_after", [1, 5, 9])
def test_resume_from_host_checkpoint_equals_build(G, stop_after):
    n, d, S, R, T1, T2, rho, seed = 3000, 24, 12, 24, 3, 4, 0.6, 17
    X = synth.small_integers(n, d, -8, 8, seed=33)
    want = G.build(X, S=S, R=R, T1=T1, T2=T2, rho=rho, seed=seed)
    wids, wd, wdeg = want.to_numpy()
    Xd, _ = G.device_points(X)
    keys, deg = G.pool_init(Xd, d, S, R, seed)
    ws = G.workspace(n, R)
    rounds = 0
    for t1 in range(1, T1 + 1):
        for t2 in range(1, T2 + 1):
            keys, deg = G.join_round(Xd, d, keys, deg, seed, t1, t2, ws=ws, inplace=True)
            rounds += 1
            if rounds == stop_after:  # checkpoint to the host, drop the device state, resume
                hk, hd = keys.cpu().clone(), deg.cpu().clone()
                del keys, deg, ws
                torch.cuda.synchronize()
                keys, deg = hk.cuda(), hd.cuda()
                ws = G.workspace(n, R)
        if t1 != T1:
            keys, deg = G.reverse_sample(keys, deg, rho, ws=ws, inplace=True)
    G.workspace_status(ws, n, R)
    fk, fdeg = G.final_prune(Xd, d, keys, deg, seed, T1 + 1, ws=ws)
    ids, dd = G.keys_to_graph(fk)
    assert (fdeg.cpu().numpy() == wdeg).all()
    assert (ids.cpu().numpy() == wids).all()
    assert (dd.cpu().numpy()[wids >= 0] == wd[wids >= 0]).all()
    assert G.entry_point(Xd, d) == want.entry


def test_memory_cache_gives_the_same_graphs(G):
    X = synth.small_integers(5000, 40, -8, 8, seed=44)
    kw = dict(S=16, R=32, T1=2, T2=4, seed=5, precision=G.BF16)
    want = G.build(X, **kw).to_numpy()
    try:
        G.set_memory_cache(1 << 30)
        graphs = [G.build(X, **kw) for _ in range(3)]  # later builds reuse the cached memory
        del graphs[0]
        graphs.append(G.build(X, **kw))
        batch = G.build_batch(X, [0, 2000, 5000], **kw)
        for g in graphs:
            for a, b in zip(g.to_numpy(), want):
                assert (a == b).all()
        assert (batch[1].to_numpy()[2] == G.build(X[2000:], **kw).to_numpy()[2]).all()
    finally:
        G.set_memory_cache(0)
    assert (G.build(X, **kw).to_numpy()[0] == want[0]).all()


@pytest.mark.parametrize("precision", ["fp32", "bf16", "fp8"])
def test_build_high_dimension_matches_oracle(G, orc, precision):
    # d = 960 (GIST's dimension): rows staged in eight chunks of 128 dimensions (partial sums
    # carried between chunks in every join kernel; FP32 rows this long use the batched CTA
    # join); integers keep every form exact, so the graph is the oracle's
    X = synth.small_integers(1500, 960, -8, 8, seed=960)
    prec = {"fp32": G.FP32, "bf16": G.BF16, "fp8": G.FP8}[precision]
    g = G.build(X, S=16, R=48, T1=2, T2=3, rho=0.6, seed=5, precision=prec)
    ids, dist, deg = g.to_numpy()
    wids, wd, wdeg, _ = orc.build_graph(X, 16, 48, 2, 3, 0.6, 5)
    assert (deg == wdeg).all() and (ids == wids).all()
    assert (dist[wids >= 0] == wd[wids >= 0].astype(np.float32)).all()
    assert g.stats()["rechecks"] == 0


# ---------------------------------------------------------------------------------------
# failure detection without a fault: a bounded device wait that nothing completes gives up,
# the status channel reports it, and the context stays usable
# ---------------------------------------------------------------------------------------

def test_bounded_wait_gives_up_and_context_stays_usable(G):
    import time
    L = G.lib()
    X = synth.small_integers(600, 8, -8, 8, seed=1)
    before = G.build(X, S=4, R=8, T1=1, T2=2).to_numpy()
    t = time.perf_counter()
    rc = L.grnnd_selftest_bounded_wait(1 << 12, None)
    dt = time.perf_counter() - t
    assert rc == G.ETIMEOUT and b"gave up" in L.grnnd_last_error()
    assert dt < 10.0
    assert L.grnnd_selftest_bounded_wait(0, None) == G.EINVAL
    after = G.build(X, S=4, R=8, T1=1, T2=2).to_numpy()  # later work on the context runs normally
    for a, b in zip(before, after):
        np.testing.assert_array_equal(a, b)
    assert after[2].min() >= 1


@pytest.mark.parametrize("precision", [1, 2])
def test_continuous_builds_repeat_exactly(G, precision):
    """On continuous data the tiles are not exact, so two copies of one id proposed to one
    target can carry different distances (a tile distance and a re-decided FP32 one), and the
    order of a target's proposals in its bucket varies between runs.  The merge's result must
    not depend on that order (an id is old iff some copy is old, whichever copy is kept), so
    repeated builds evaluate the same pairs and return the same graph."""
    X = synth.deep_like(50000, seed=5)
    kw = dict(S=16, R=32, T1=3, T2=10, metric=1, precision=precision)
    first = G.build(X, **kw)
    want, want_stats = first.to_numpy(), first.stats()
    for _ in range(3):
        g = G.build(X, **kw)
        assert g.stats() == want_stats
        for a, b in zip(g.to_numpy(), want):
            np.testing.assert_array_equal(a, b)
