"""Pins for the FP64 oracle against facts fixed outside the oracle itself.

Each test checks the oracle against something it does not compute itself:
hand-derived worked cases of Eq 2, the paper's serial Alg 2 written out
independently, brute-force RNG / k-NN definitions, published SplitMix64
outputs, and dict-based restatements of the merge (C6) and reverse-sampling
(C7) readings.  A plausible slip in the oracle (a dropped bottom-skip, a
swapped close/far, max instead of min in the merge, the wrong end of the pool
in reverse sampling) fails at least one of them.
"""
import os

import numpy as np
import pytest

from paper_2510_02774_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
M64 = 2**64 - 1
G = 0x9E3779B97F4A7C15


def _pts(rows):
    return np.asarray(rows, dtype=np.float32)


def _sqd(X, i, j):
    return float(((X[i].astype(np.float64) - X[j].astype(np.float64)) ** 2).sum())


# --------------------------------------------------------------------------------------
# C9: SplitMix64 against its published reference outputs
# --------------------------------------------------------------------------------------

def test_splitmix64_published_outputs(orc):
    with open(os.path.join(GOLDEN, "splitmix64.txt")) as f:
        lines = [l.split() for l in f if l.strip() and not l.startswith("#")]
    assert lines
    for tok in lines:
        state = int(tok[0], 0)
        want = [int(t, 0) for t in tok[1:]]
        # next() adds the gamma first, so output i is f(state + i * gamma)
        got = [orc.splitmix64((state + i * G) & M64) for i in range(len(want))]
        assert got == want


def test_counter_hash_is_chained_splitmix(orc):
    f = orc.splitmix64
    for args in [(0, 0, 0, 0, 0), (7, 1, 2, 3, 4), (2**63 + 5, 4, 15, 999_999, 123_456)]:
        s, a, b, c, e = args
        assert orc.counter_hash(*args) == f(f(f(f(f(s) ^ a) ^ b) ^ c) ^ e)
    # distinct counters give distinct values (no accidental collapse of an argument)
    vals = {orc.counter_hash(0, t1, t2, v, x) for t1 in range(3) for t2 in range(3)
            for v in range(5) for x in range(5)}
    assert len(vals) == 3 * 3 * 5 * 5


# --------------------------------------------------------------------------------------
# C8: distances
# --------------------------------------------------------------------------------------

def test_distance_definitions(orc):
    x = _pts([1, 2, 3])
    y = _pts([4, 0, -1])
    assert orc.dist(x, y, 0) == 9 + 4 + 16          # squared L2
    assert orc.dist(x, y, 1) == 1.0 - (4 + 0 - 3)    # 1 - <x, y>


# --------------------------------------------------------------------------------------
# Eq 2 / Alg 4: hand-derived worked cases
# --------------------------------------------------------------------------------------

def _prune_case(orc, X, v, cand, perm_ids):
    ids = np.array(cand, np.int32)
    d = np.array([_sqd(X, v, c) for c in cand])
    order = np.argsort(d, kind="stable")  # pools are kept in (dist, id) order
    ids, d = ids[order], d[order]
    perm = np.array([list(ids).index(p) for p in perm_ids], np.int32)
    alive, killer, kd, _, _ = orc.prune(X, ids, d, perm)
    surv = sorted(ids[alive].tolist())
    redirect = {int(ids[i]): (int(ids[killer[i]]), float(kd[i])) for i in range(len(ids)) if not alive[i]}
    return surv, redirect


def test_worked_1d_ascending(orc):
    # v = 0 at x=0; candidates at x = 1, 2, 3; ascending order (Alg 2 special case).
    # (1,2): d=1 < max(1,4) -> 2 -> 1.  (1,3): d=4 < max(1,9) -> 3 -> 1.  (2,3): 2 is bottom.
    X = _pts([[0], [1], [2], [3]])
    surv, red = _prune_case(orc, X, 0, [1, 2, 3], [1, 2, 3])
    assert surv == [1]
    assert red == {2: (1, 1.0), 3: (1, 4.0)}


def test_worked_1d_descending_needs_bottom_skip(orc):
    # Order 3, 2, 1.  (3,2): d=1 < max(9,4) -> close 2, far 3 -> 3 -> 2.
    # (3,1) skipped because 3 is bottom (C4).  (2,1): d=1 < max(4,1) -> 2 -> 1.
    X = _pts([[0], [1], [2], [3]])
    surv, red = _prune_case(orc, X, 0, [1, 2, 3], [3, 2, 1])
    assert surv == [1]
    assert red == {3: (2, 1.0), 2: (1, 1.0)}


def test_worked_2d_both_kept(orc):
    # Eq 1: n1=(1,0), n2=(-1,0): d(n1,n2)=4 is not below max(1,1): both kept.
    X = _pts([[0, 0], [1, 0], [-1, 0]])
    surv, red = _prune_case(orc, X, 0, [1, 2], [1, 2])
    assert surv == [1, 2] and red == {}


def test_worked_fig1_rng_redirect(orc):
    # Sec 2.2 / Fig 1: n2 is closer to n1 than to v, so v-n2 is replaced by n1-n2.
    X = _pts([[0, 0], [2, 0], [3, 1]])  # v, n1, n2: d(v,n1)=4, d(v,n2)=10, d(n1,n2)=2
    for order in ([1, 2], [2, 1]):
        surv, red = _prune_case(orc, X, 0, [1, 2], order)
        assert surv == [1] and red == {2: (1, 2.0)}


def test_worked_fig2_serial_example(orc):
    # Sec 3.1 prose: vertex 1 keeps its closest neighbour 2; vertex 4 is closer to 2
    # than to 1 and is redirected to 2; vertex 5 stays.
    X = _pts([[9, 9], [0, 0], [1, 0], [9, -9], [2, 0.5], [0, -2]])  # ids 0..5, v = 1
    surv, red = _prune_case(orc, X, 1, [2, 4, 5], [2, 5, 4])
    assert surv == [2, 5]
    assert red == {4: (2, 1.25)}


def test_worked_disorder_redirects_to_unseen_node(orc):
    # Sec 3.3: visiting distant candidates first can redirect toward another
    # candidate instead of the nearest one.  v=0 at 0; 2 at 1, 5 at 3, 4 at 3.5.
    X = _pts([[0], [50], [1], [70], [3.5], [3]])
    surv, red = _prune_case(orc, X, 0, [2, 4, 5], [2, 5, 4])  # ascending
    assert surv == [2] and red == {5: (2, 4.0), 4: (2, 6.25)}
    surv, red = _prune_case(orc, X, 0, [2, 4, 5], [4, 5, 2])  # disordered
    # (4,5): 0.25 < max(12.25, 9) -> 4 -> 5;  (4,2) skipped;  (5,2): 4 < max(9,1) -> 5 -> 2
    assert surv == [2] and red == {4: (5, 0.25), 5: (2, 4.0)}


def test_tie_on_distance_breaks_by_id(orc):
    # C5: when d(v,a) == d(v,b) the smaller id is n_close.  Two coincident points
    # at (1,0): d(a,b) = 0 < max(1,1) fires, and id 2 is redirected to id 1.
    X = _pts([[0, 0], [1, 0], [1, 0]])
    surv, red = _prune_case(orc, X, 0, [2, 1], [2, 1])
    assert surv == [1] and red == {2: (1, 0.0)}


# --------------------------------------------------------------------------------------
# Alg 2 (the paper's serial update) as an independent special case of the pair scan
# --------------------------------------------------------------------------------------

def _alg2(X, v, cand, strict):
    """Paper Alg 2 written out: candidates in ascending (dist, id) order, each one
    compared with the accepted list in acceptance order; first hit redirects."""
    cand = sorted(cand, key=lambda c: (_sqd(X, v, c), c))
    acc, red = [], {}
    for n in cand:
        dvn = _sqd(X, v, n)
        hit = None
        for p in acc:
            dnp = _sqd(X, n, p)
            if (dnp < dvn) if strict else (dnp <= dvn):
                hit = p
                break
        if hit is None:
            acc.append(n)
        else:
            red[n] = hit
    return sorted(acc), red


@pytest.mark.parametrize("seed", range(6))
def test_ascending_pair_scan_equals_alg2(orc, seed):
    g = np.random.default_rng(seed)
    X = g.standard_normal((40, 3)).astype(np.float32)
    for v in range(0, 40, 7):
        cand = [int(c) for c in g.choice([i for i in range(40) if i != v], size=int(g.integers(2, 25)), replace=False)]
        ids = np.array(sorted(cand, key=lambda c: (_sqd(X, v, c), c)), np.int32)
        d = np.array([_sqd(X, v, c) for c in ids])
        alive, killer, _, _, _ = orc.prune(X, ids, d, np.arange(len(ids), dtype=np.int32))
        surv = sorted(ids[alive].tolist())
        red = {int(ids[i]): int(ids[killer[i]]) for i in range(len(ids)) if not alive[i]}
        for strict in (True, False):  # continuous data: no exact ties, both forms agree
            a_surv, a_red = _alg2(X, v, cand, strict)
            assert surv == a_surv
            assert red == a_red


# --------------------------------------------------------------------------------------
# Properties of the prune that hold for ANY visit order
# --------------------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(5))
def test_prune_properties_any_order(orc, seed):
    g = np.random.default_rng(100 + seed)
    X = g.standard_normal((60, 4)).astype(np.float32)
    for v in range(0, 60, 5):
        m = int(g.integers(1, 40))
        cand = g.choice([i for i in range(60) if i != v], size=m, replace=False)
        ids = np.array(sorted(cand, key=lambda c: (_sqd(X, v, c), c)), np.int32)
        d = np.array([_sqd(X, v, c) for c in ids])
        perm = g.permutation(m).astype(np.int32)
        alive, killer, kd, _, _ = orc.prune(X, ids, d, perm)
        assert alive[0], "the nearest entry can never be the far side of a pair"
        s = np.nonzero(alive)[0]
        for i in s:  # survivors are pairwise non-firing (each pair was evaluated)
            for j in s:
                if i < j:
                    assert not (_sqd(X, ids[i], ids[j]) < max(d[i], d[j]))
        for f in np.nonzero(~alive)[0]:  # every bottom entry has one valid absorber
            c = killer[f]
            assert c >= 0 and c != f
            assert (d[c], ids[c]) < (d[f], ids[f])
            assert kd[f] == _sqd(X, ids[c], ids[f]) and kd[f] < max(d[c], d[f])


def test_rng_edges_survive_any_order(orc):
    # With the pool equal to every other point, a global RNG edge (v,u) -- no w with
    # max(d(v,w), d(u,w)) < d(v,u) -- can never be pruned, whatever the order.
    g = np.random.default_rng(7)
    n = 30
    X = g.standard_normal((n, 2)).astype(np.float32)
    D = ((X[:, None, :].astype(np.float64) - X[None, :, :]) ** 2).sum(-1)
    for v in range(n):
        rng_nb = [u for u in range(n) if u != v and not any(
            max(D[v, w], D[u, w]) < D[v, u] for w in range(n) if w not in (u, v))]
        assert rng_nb
        cand = [u for u in range(n) if u != v]
        ids = np.array(sorted(cand, key=lambda c: (D[v, c], c)), np.int32)
        dd = np.array([D[v, c] for c in ids])
        for trial in range(4):
            perm = g.permutation(len(ids)).astype(np.int32)
            alive, _, _, _, _ = orc.prune(X, ids, dd, perm)
            surv = set(ids[alive].tolist())
            assert set(rng_nb) <= surv


def _mrng_neighbours(D, v):
    """Brute-force MRNG set of v over every other point (strict lune, ties by id):
    candidates in ascending (d(v,.), id); u is kept iff no kept w has d(w,u) < d(v,u)."""
    n = D.shape[0]
    kept = []
    for u in sorted((u for u in range(n) if u != v), key=lambda u: (D[v, u], u)):
        if not any(D[w, u] < D[v, u] for w in kept):
            kept.append(u)
    return kept


@pytest.mark.parametrize("case", ["gauss", "ties"])
def test_full_pool_ascending_final_prune_is_mrng(orc, case):
    # S = R = n - 1: every pool holds all other points; the ascending (Alg 2) order then
    # makes the prune-only pass keep exactly the brute-force MRNG neighbours of each point.
    if case == "gauss":
        n = 48
        X = np.random.default_rng(31).standard_normal((n, 3)).astype(np.float32)
    else:
        n = 40
        X = synth.small_integers(n, 2, -2, 2, seed=3)  # many equal distances and duplicates
    D = ((X[:, None, :].astype(np.float64) - X[None, :, :]) ** 2).sum(-1)
    pool, _ = orc.init(X, n - 1, n - 1, seed=9)
    assert (pool.deg == n - 1).all()
    gids, gd, gdeg, _ = orc.final_prune(X, pool, seed=9, t1=2, order=1)
    for v in range(n):
        want = _mrng_neighbours(D, v)
        got = gids[v, :gdeg[v]].tolist()
        assert got == want, v
        assert all(gd[v, j] == D[v, u] for j, u in enumerate(got))


def test_visit_order_modes(orc):
    ids = np.array([5, 9, 2, 7], np.int32)
    assert orc.visit_order(0, 1, 1, 3, ids, 1).tolist() == [0, 1, 2, 3]
    assert orc.visit_order(0, 1, 1, 3, ids, 2).tolist() == [3, 2, 1, 0]
    perm = orc.visit_order(11, 2, 5, 3, ids, 0)
    h = [orc.counter_hash(11, 2, 5, 3, int(i)) for i in ids]
    assert perm.tolist() == sorted(range(4), key=lambda i: (h[i], ids[i]))


# --------------------------------------------------------------------------------------
# C6: merge into fixed-capacity pools
# --------------------------------------------------------------------------------------

def _merge_ref(n, R, tgt, ids, dist, old):
    best = {}
    for t, i, dd, o in zip(tgt, ids, dist, old):
        k = (int(t), int(i))
        if k not in best:
            best[k] = [dd, int(o)]
        else:
            best[k][0] = min(best[k][0], dd)
            best[k][1] |= int(o)
    rows = {u: [] for u in range(n)}
    for (t, i), (dd, o) in best.items():
        rows[t].append((dd, i, o))
    return {u: sorted(r)[:R] for u, r in rows.items()}


@pytest.mark.parametrize("seed", range(4))
def test_merge_matches_definition_and_is_order_free(orc, seed):
    g = np.random.default_rng(seed)
    n, R, npr = 12, 5, 300
    tgt = g.integers(0, n, npr)
    ids = g.integers(0, 40, npr)
    dist = (ids * 7 + tgt * 3) % 23 + 0.5   # a function of (target, id): duplicates agree
    old = g.integers(0, 2, npr)
    ref = _merge_ref(n, R, tgt, ids, dist, old)
    for trial in range(3):
        p = g.permutation(npr)
        out = orc.merge(n, R, tgt[p], ids[p], dist[p], old[p])
        for u in range(n):
            got = [(out.dist[u, j], out.ids[u, j], out.old[u, j]) for j in range(out.deg[u])]
            assert got == [(a, b, c) for a, b, c in ref[u]]
            assert (out.ids[u, out.deg[u]:] == -1).all()


def test_merge_keeps_minimum_distance_of_duplicates(orc):
    out = orc.merge(2, 3, [0, 0, 0, 0], [5, 5, 6, 7], [3.0, 1.0, 2.0, 9.0], [1, 0, 0, 0])
    assert out.ids[0, :3].tolist() == [5, 6, 7]
    assert out.dist[0, :3].tolist() == [1.0, 2.0, 9.0]
    assert out.old[0, :3].tolist() == [1, 0, 0]   # old because one copy was old
    assert out.deg.tolist() == [3, 0]


# --------------------------------------------------------------------------------------
# C7: reverse-edge sampling (Sec 3.6)
# --------------------------------------------------------------------------------------

def _pool(rows, R):
    from oracle.oracle import Pool
    n = len(rows)
    p = Pool.empty(n, R)
    for v, r in enumerate(rows):
        for j, (i, dd, o) in enumerate(r):
            p.ids[v, j], p.dist[v, j], p.old[v, j] = i, dd, o
        p.deg[v] = len(r)
    return p


def test_reverse_sampling_hand_case(orc):
    rows = [[(1, 1.0, 0), (2, 4.0, 1)],           # k=2 -> floor(0.6*2)=1: 1 <- 0
            [(0, 1.0, 1)],                         # k=1 -> 0 reverse edges
            [],
            [(0, 9.0, 0), (1, 16.0, 0), (2, 25.0, 0)]]  # k=3 -> floor(1.8)=1: 0 <- 3
    out, _ = orc.reverse(_pool(rows, 3), 0.6)
    assert out.ids[0, :out.deg[0]].tolist() == [1, 2, 3] and out.dist[0, 2] == 9.0
    assert out.old[0, :3].tolist() == [0, 1, 0]
    assert out.ids[1, :out.deg[1]].tolist() == [0] and out.old[1, 0] == 1   # duplicate, old wins
    assert out.deg[2] == 0
    assert out.ids[3, :3].tolist() == [0, 1, 2]
    rows2 = rows[:3] + [[(0, 9.0, 0), (1, 16.0, 0)]]  # k=2 -> floor(1.2)=1: 0 <- 3
    out2, _ = orc.reverse(_pool(rows2, 2), 0.6)   # capacity 2 truncates by (dist, id)
    assert out2.ids[0, :2].tolist() == [1, 2] and out2.deg[0] == 2


def test_reverse_sampling_extremes(orc):
    rows = [[(1, 1.0, 0), (2, 4.0, 0)], [(2, 2.0, 0)], [(0, 4.0, 0)]]
    out0, _ = orc.reverse(_pool(rows, 4), 0.0)  # rho = 0: identity
    assert out0.ids.tolist() == _pool(rows, 4).ids.tolist()
    out1, _ = orc.reverse(_pool(rows, 4), 1.0)  # rho = 1: every reverse edge
    assert sorted(out1.ids[2, :out1.deg[2]].tolist()) == [0, 1]
    assert sorted(out1.ids[0, :out1.deg[0]].tolist()) == [1, 2]
    assert sorted(out1.ids[1, :out1.deg[1]].tolist()) == [0, 2]


# --------------------------------------------------------------------------------------
# Whole build: invariants, determinism, C10 exactness
# --------------------------------------------------------------------------------------

@pytest.fixture(scope="module")
def small_mix():
    return synth.gaussian_mixture(1500, 8, n_components=6, center_range=5.0, sigma=1.0, seed=3, nq=100)


def test_build_invariants(orc, small_mix):
    X, _ = small_mix
    S, R = 8, 16
    gids, gd, gdeg, st = orc.build_graph(X, S, R, 2, 4, 0.6, seed=5)
    n = len(X)
    assert (gdeg <= R).all() and (gdeg >= 1).all()
    for v in range(n):
        row = gids[v, :gdeg[v]]
        assert (row >= 0).all() and v not in row.tolist()
        assert len(set(row.tolist())) == len(row)
        assert (gids[v, gdeg[v]:] == -1).all()
        dv = gd[v, :gdeg[v]]
        for j, u in enumerate(row):
            assert dv[j] == orc.dist(X[v], X[u], 0)   # recorded = recomputed (FP64)
        keys = list(zip(dv.tolist(), row.tolist()))
        assert keys == sorted(keys)
        for a in range(len(row)):                   # C11: kept edges are RNG-consistent
            for b in range(a + 1, len(row)):
                assert not (orc.dist(X[row[a]], X[row[b]], 0) < max(dv[a], dv[b]))
    assert st[0] > 0 and st[1] > 0


def test_build_is_deterministic_and_seeded(orc, small_mix):
    X, _ = small_mix
    a = orc.build_graph(X, 8, 16, 2, 3, 0.6, seed=1)
    b = orc.build_graph(X, 8, 16, 2, 3, 0.6, seed=1)
    c = orc.build_graph(X, 8, 16, 2, 3, 0.6, seed=2)
    assert (a[0] == b[0]).all() and (a[2] == b[2]).all()
    assert not (a[0] == c[0]).all()


def test_skipping_old_pairs_changes_nothing(orc, small_mix):
    # C10: pairs of two old entries never fire, so skipping them is exact.
    X, _ = small_mix
    full = orc.build_graph(X, 8, 16, 2, 4, 0.6, seed=4, skip_old=False)
    skip = orc.build_graph(X, 8, 16, 2, 4, 0.6, seed=4, skip_old=True)
    assert (full[0] == skip[0]).all() and (full[2] == skip[2]).all()
    assert skip[3][0] < full[3][0]  # fewer pair evaluations


def test_round_is_pure_function_of_pool(orc, small_mix):
    X, _ = small_mix
    p, _ = orc.init(X, 8, 16, seed=9)
    a, _, _ = orc.round_(X, p, 9, 1, 1)
    b, _, _ = orc.round_(X, p.copy(), 9, 1, 1)
    assert (a.ids == b.ids).all() and (a.old == b.old).all()
    # init: S distinct ids != v, sorted by (dist, id), all new
    assert (p.deg == 8).all() and (p.old == 0).all()
    for v in range(len(X)):
        row = p.ids[v, :8]
        assert v not in row and len(set(row.tolist())) == 8
        keys = list(zip(p.dist[v, :8].tolist(), row.tolist()))
        assert keys == sorted(keys)
    # every pool entry emits exactly one proposal: sum(deg) proposals
    _, _, st = orc.round_(X, p, 9, 1, 1)
    assert st[2] == p.deg.sum()


def test_init_rejects_bad_sizes(orc):
    X = np.zeros((5, 2), np.float32)
    with pytest.raises(ValueError):
        orc.init(X, 5, 8, 0)      # S > n - 1
    with pytest.raises(ValueError):
        orc.init(X, 4, 3, 0)      # R < S


# --------------------------------------------------------------------------------------
# Sec 2.1 / Sec 4.2: exact k-NN, entry point, candidate-list search
# --------------------------------------------------------------------------------------

def _np_knn(X, Q, k):
    D = ((Q[:, None, :].astype(np.float64) - X[None, :, :].astype(np.float64)) ** 2).sum(-1)
    out = np.zeros((len(Q), k), np.int64)
    for i in range(len(Q)):
        out[i] = np.lexsort((np.arange(len(X)), D[i]))[:k]
    return out


def test_brute_knn_matches_exhaustive(orc):
    X, Q = synth.small_integers(300, 5, -3, 3, seed=2, nq=40)  # many exact ties
    ids, dd = orc.brute_knn(X, Q, 10)
    assert (ids == _np_knn(X, Q, 10)).all()


@pytest.mark.parametrize("metric", [0, 1])
def test_brute_knn_matches_a_second_plain_loop(orc, metric):
    # 2,000 points: every query's k-NN from one distance loop over all points, written out
    # here in FP64, ordered by (dist, id)
    X, Q = synth.small_integers(2000, 16, -4, 4, seed=12, nq=150)
    k = 10
    ids, dd = orc.brute_knn(X, Q, k, metric=metric)
    Xd = X.astype(np.float64)
    for i in range(len(Q)):
        q = Q[i].astype(np.float64)
        dist = np.empty(len(X))
        for u in range(len(X)):
            dist[u] = ((Xd[u] - q) ** 2).sum() if metric == 0 else 1.0 - (Xd[u] * q).sum()
        order = sorted(range(len(X)), key=lambda u: (dist[u], u))[:k]
        assert ids[i].tolist() == order
        assert np.array_equal(dd[i], dist[order])


def test_entry_is_nearest_to_mean(orc):
    X = synth.small_integers(200, 6, -5, 5, seed=4)
    mu = X.astype(np.float64).mean(0)
    D = ((X.astype(np.float64) - mu) ** 2).sum(1)
    assert orc.entry(X) == int(np.argmin(D))


def test_search_on_complete_graph_is_exact(orc):
    X, Q = synth.gaussian_mixture(80, 4, 3, 4.0, 1.0, seed=8, nq=30)
    n = len(X)
    gids = np.array([[u for u in range(n) if u != v] for v in range(n)], np.int32)
    gdeg = np.full(n, n - 1, np.int32)
    ids, dd, _ = orc.search(gids, gdeg, X, Q, 10, 80, orc.entry(X))
    assert (ids == _np_knn(X, Q, 10)).all()


def test_search_results_are_valid(orc, small_mix):
    X, Q = small_mix
    gids, gd, gdeg, _ = orc.build_graph(X, 8, 16, 2, 4, 0.6, seed=5)
    ids, dd, _ = orc.search(gids, gdeg, X, Q, 10, 12, orc.entry(X))
    for i in range(len(Q)):
        assert len(set(ids[i].tolist())) == 10
        keys = list(zip(dd[i].tolist(), ids[i].tolist()))
        assert keys == sorted(keys)
        for j in range(10):
            assert dd[i, j] == orc.dist(Q[i], X[ids[i, j]], 0)


def test_oracle_graph_search_recall(orc, small_mix):
    # Sec 4.2: the GRNND graph supports high-recall candidate-list search.
    X, Q = small_mix
    gids, gd, gdeg, _ = orc.build_graph(X, 8, 16, 2, 4, 0.6, seed=5)
    ids, _, _ = orc.search(gids, gdeg, X, Q, 10, 64, orc.entry(X))
    gt, _ = orc.brute_knn(X, Q, 10)
    assert orc.recall_at_k(ids, gt) >= 0.95


@pytest.mark.parametrize("threads", [1, 2, 7])
@pytest.mark.parametrize("final_prune", [True, False])
def test_threaded_oracle_driver_equals_oracle_build(orc, threads, final_prune):
    # the CPU baseline's multi-threaded driver calls the oracle's own steps over vertex and
    # target ranges: the graph and counters must be orc_build's at any thread count
    X = synth.small_integers(1500, 10, -8, 8, seed=6)
    kw = dict(S=12, R=24, T1=2, T2=3, rho=0.6, seed=5, final_prune=final_prune)
    want = orc.build_graph(X, **kw)
    got = orc.build_graph_mt(X, threads=threads, **kw)
    for a, b in zip(want, got):
        assert np.array_equal(a, b)
