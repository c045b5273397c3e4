"""Parity at the bench workload's full size: the SIFT-shaped set of 1,000,000 points of
dimension 128 (integers in [0, 255]: every FP32 distance is exact), S 32, R 64, T1 4,
T2 15, in the launch configuration bench.py times.  The oracle checks what it can compute
at this size: the whole random initialisation, and the prune of sampled vertices one by one
(pools of up to 32 entries: the warp kernel; of 33..64: the team kernel).  The whole build is
checked through properties that hold at any size and against the FP32 form."""
import numpy as np
import pytest

from paper_2510_02774_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

N, D, S, R, T1, T2, SEED = 1_000_000, 128, 32, 64, 4, 15, 0


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
def orc():
    from oracle import oracle as O
    O.build()
    return O


@pytest.fixture(scope="module")
def X():
    return synth.sift_like(N, 0, seed=SEED)


def _decode(G, keys, deg):
    ids, dist, old = G.decode_keys(keys.cpu().numpy().view(np.uint64))
    return ids, dist, old, deg.cpu().numpy()


def test_init_equals_oracle_at_full_size(G, orc, X):
    Xd, _ = G.device_points(X)
    keys, deg = G.pool_init(Xd, D, S, R, SEED)
    ids, dist, old, dg = _decode(G, keys, deg)
    want, _ = orc.init(X, S, R, SEED)
    assert (dg == want.deg).all() and (ids == want.ids).all()
    assert (dist[ids >= 0].astype(np.float64) == want.dist[ids >= 0]).all()
    assert not old[ids >= 0].any()


@pytest.mark.parametrize("rounds", [0, 1])
def test_prune_of_sampled_vertices_equals_oracle(G, orc, X, rounds):
    # rounds = 0: the init pools (32 entries: warp kernel); rounds = 1: after one round, pools
    # of up to 64 entries (warp and team kernels); the prune pass of t1 = T1 + 1, no redirects
    Xd, _ = G.device_points(X)
    keys, deg = G.pool_init(Xd, D, S, R, SEED)
    ws = G.workspace(N, R)
    for t2 in range(1, rounds + 1):
        keys, deg = G.join_round(Xd, D, keys, deg, SEED, 1, t2, ws=ws, inplace=True)
    ids, dist, old, dg = _decode(G, keys, deg)
    fk, fdeg = G.final_prune(Xd, D, keys, deg, SEED, T1 + 1, ws=ws)
    G.workspace_status(ws, N, R)
    fids, fdist, _, fdg = _decode(G, fk, fdeg)
    rng = np.random.default_rng(5)
    sample = rng.choice(N, 400, replace=False)
    if rounds:  # make sure the large pools (team kernel) are in the sample
        big = np.nonzero(dg > 32)[0]
        assert len(big) > 0
        sample = np.concatenate([sample, rng.choice(big, 400, replace=False)])
    for v in sample:
        m = dg[v]
        row, rd = ids[v, :m], dist[v, :m].astype(np.float64)
        perm = orc.visit_order(SEED, T1 + 1, 0, int(v), row)
        alive, _, _, _, _ = orc.prune(X, row, rd, perm, old=old[v, :m])
        want = row[alive]
        assert fdg[v] == len(want), v
        assert (fids[v, :fdg[v]] == want).all(), v
        assert (fdist[v, :fdg[v]] == dist[v, :m][alive]).all(), v


def test_full_build_bf16_equals_fp32_and_holds_invariants(G, orc, X):
    Xd = torch.from_numpy(X).cuda()
    kw = dict(S=S, R=R, T1=T1, T2=T2, rho=0.6, seed=SEED)
    gb = G.build(Xd, precision=G.BF16, **kw)
    gf = G.build(Xd, precision=G.FP32, **kw)
    ids, dist, deg = gb.to_numpy()
    for a, b in zip(gf.to_numpy(), (ids, dist, deg)):
        assert (a == b).all()
    assert gb.stats()["rechecks"] == 0 and gb.entry == gf.entry == orc.entry(X)
    X64 = X.astype(np.float64)
    for v in np.random.default_rng(6).choice(N, 1000, replace=False):
        m = deg[v]
        row = ids[v, :m]
        assert 1 <= m <= R and (ids[v, m:] == -1).all()
        assert v not in row and len(set(row.tolist())) == m
        d64 = ((X64[row] - X64[v]) ** 2).sum(1)
        assert (dist[v, :m].astype(np.float64) == d64).all()  # exact integers
        assert all((d64[i], row[i]) < (d64[i + 1], row[i + 1]) for i in range(m - 1))  # (dist, id) order
        # the final prune leaves no pair of kept edges that fires (Eq 2)
        P = X64[row]
        dab = ((P[:, None, :] - P[None, :, :]) ** 2).sum(2)
        mx = np.maximum(d64[:, None], d64[None, :])
        iu = np.triu_indices(m, 1)
        assert not (dab[iu] < mx[iu]).any(), v
