"""The prune chain as a fixed point (CPU, against the oracle's sequential prune).

The join kernels do not replay the pair scan of Alg 4 column after column.  Column b of the
scan (pi position b, its pairs (a, b) for a < b taken in order) kills K_b: its live firing
partners before the first closer one f, then b itself (absorbed by f); all of them when no
live firing partner is closer.  Its live partners are the valid positions that no column
c < b killed, so the scan's outcome is the fixed point of
    K_b = rule(fire[b] & valid & ~OR_{c<b} K_c),
which the kernels reach with rounds that apply the rule to every column at once, starting
from K = 0 and stopping at the first round whose K has the prefix it was computed from.
This file restates that iteration in Python and checks it against the oracle's prune on
pools with many distance ties, old entries (pairs of two old entries are not evaluated) and
the oracle's own visit orders: same survivors, same absorbers, at most m rounds."""
import numpy as np
import pytest

from oracle import oracle as O


def _masks(X, v, ids, dist, old, perm, skip_old=True):
    """fire[b] / closer[b] bit a (a < b, pi positions): the pair fires / a is the closer side."""
    m = len(ids)
    P = X[ids[perm]].astype(np.float64)
    D = ((P[:, None, :] - P[None, :, :]) ** 2).sum(-1)
    dv, idp, op = dist[perm], ids[perm], old[perm]
    fire, closer = [0] * m, [0] * m
    for b in range(m):
        for a in range(b):
            if (dv[a], idp[a]) < (dv[b], idp[b]):
                closer[b] |= 1 << a
            if skip_old and op[a] and op[b]:
                continue
            if D[a, b] < max(dv[a], dv[b]):
                fire[b] |= 1 << a
    return fire, closer


def _fixed_point(fire, closer, m):
    """Rounds of the column rule; returns (alive mask, absorber by position, rounds)."""
    valid = (1 << m) - 1
    before = [0] * m
    rounds = 0
    while True:
        rounds += 1
        K, f = [], []
        for b in range(m):
            cand = fire[b] & valid & ~before[b]
            x = cand & closer[b]
            if x:
                fb = (x & -x).bit_length() - 1
                K.append((cand & ((1 << fb) - 1)) | (1 << b))
                f.append(fb)
            else:
                K.append(cand)
                f.append(-1)
        prefix, acc = [], 0
        for b in range(m):
            prefix.append(acc)
            acc |= K[b]
        if prefix == before:
            break
        before = prefix
        assert rounds <= m
    dead = acc
    absorber = [-1] * m
    for b in range(m):
        for a in range(m):
            if a != b and (K[b] >> a) & 1:
                assert absorber[a] == -1  # every entry dies once
                absorber[a] = b
        if f[b] >= 0:
            absorber[b] = f[b]
    return valid & ~dead, absorber, rounds


@pytest.mark.parametrize("d,lo,hi", [(3, -2, 2), (8, -8, 8), (16, 0, 255)])
def test_fixed_point_equals_sequential_prune(d, lo, hi):
    rng = np.random.default_rng(100 + d)
    n = 400
    X = rng.integers(lo, hi + 1, size=(n, d)).astype(np.float32)
    worst = 0
    for trial in range(60):
        v = int(rng.integers(n))
        m = int(rng.integers(2, 65))
        ids = rng.choice(np.delete(np.arange(n), v), m, replace=False).astype(np.int32)
        dist = ((X[ids].astype(np.float64) - X[v]) ** 2).sum(1)
        old = (rng.random(m) < 0.4).astype(np.uint8)
        perm = O.visit_order(7, 1, trial, v, ids)
        fire, closer = _masks(X, v, ids, dist, old, perm)
        alive_p, absorber_p, rounds = _fixed_point(fire, closer, m)
        assert rounds <= m
        worst = max(worst, rounds)
        alive, killer, _, _, _ = O.prune(X, ids, dist, perm, old, skip_old=True)
        for p in range(m):
            s = perm[p]
            assert bool((alive_p >> p) & 1) == bool(alive[s])
            if not alive[s]:
                assert perm[absorber_p[p]] == killer[s]
    assert worst >= 2  # the cases include chains that take more than one round


def test_fixed_point_reaches_the_sequential_worst_case():
    """A chain where each column's outcome depends on the previous one: every round fixes
    one more column, and the iteration still ends within m rounds."""
    m = 12
    # column b fires with b - 1 only; b - 1 is the closer side, so b dies iff b - 1 is alive
    fire = [0] + [1 << (b - 1) for b in range(1, m)]
    closer = [0] + [1 << (b - 1) for b in range(1, m)]
    alive, absorber, rounds = _fixed_point(fire, closer, m)
    want = sum(1 << b for b in range(0, m, 2))  # 0 lives, 1 dies, 2 lives, ...
    assert alive == want
    assert all(absorber[b] == b - 1 for b in range(1, m, 2))
    assert rounds <= m and rounds >= m // 2
