"""The merge's old bits under truncation (CPU, against the oracle's merge).

The device merge of one target (`select`) takes a few proposals one insert at a time, or
many in chunks of 32, and truncates the row to its R smallest keys after every step.  All
bucketed proposals are new; an id is old in the result iff some copy is old, i.e. iff the
target's row held it as old.  When two copies of an id carry different distances (tile
distances and re-decided FP32 ones, outside the exact mode), a truncation can push the
row's old copy out before a nearer copy of the same id arrives, which would then enter as
new.  So in that mode every proposal first takes the old bit its id has in the row.  This
file restates both merge paths in Python and checks them against the oracle's merge: with
that first pass the result always equals the oracle's, and without it some of these
targets end up with a wrong old bit."""
import numpy as np
import pytest

from oracle import oracle as O


def _insert(row, prop, R):
    """One insert into a sorted, id-distinct row of (dist, id, old) keeping the R smallest."""
    d, i, o = prop
    for e, (rd, ri, ro) in enumerate(row):
        if ri == i:
            if (d, i) >= (rd, ri):  # the listed copy is not farther: it stays
                if o:
                    row[e] = (rd, ri, 1)
                return row
            o |= ro  # the nearer copy replaces it
            del row[e]
            break
    row.append((d, i, o))
    row.sort(key=lambda x: (x[0], x[1]))
    return row[:R]


def _merge_chunk(row, chunk, R):
    """Up to 32 proposals at once: one copy per id among them (the nearest, old if any copy
    is), then each against the row (the nearer copy stays, old if either is)."""
    chunk = sorted(chunk, key=lambda x: (x[0], x[1], x[2]))
    best = {}
    for d, i, o in chunk:
        if i in best:
            bd, bi, bo = best[i]
            best[i] = (bd, bi, bo | o)
        else:
            best[i] = (d, i, o)
    out = {ri: (rd, ri, ro) for rd, ri, ro in row}
    for i, (d, _, o) in best.items():
        if i in out:
            rd, _, ro = out[i]
            if (d, i) < (rd, i):
                out[i] = (d, i, o | ro)
            else:
                out[i] = (rd, i, ro | o)
        else:
            out[i] = (d, i, o)
    return sorted(out.values(), key=lambda x: (x[0], x[1]))[:R]


def _device_merge(row, props, R, old_pass):
    held_old = {i for _, i, o in row if o}
    if len(props) <= 4:
        if old_pass:
            props = [(d, i, o | (i in held_old)) for d, i, o in props]
        for p in props:
            row = _insert(list(row), p, R)
        return row
    for c0 in range(0, len(props), 32):
        chunk = props[c0:c0 + 32]
        if old_pass and c0 > 0:
            chunk = [(d, i, o | (i in held_old)) for d, i, o in chunk]
        row = _merge_chunk(row, chunk, R)
    return row


def _oracle_merge(row, props, R):
    allp = list(row) + list(props)
    tgt = np.zeros(len(allp), np.int32)
    ids = np.array([p[1] for p in allp], np.int32)
    dist = np.array([p[0] for p in allp], np.float64)
    old = np.array([p[2] for p in allp], np.uint8)
    pool = O.merge(1, R, tgt, ids, dist, old)
    m = int(pool.deg[0])
    return [(float(pool.dist[0, e]), int(pool.ids[0, e]), int(pool.old[0, e])) for e in range(m)]


def _target(rng, R, c):
    """A full row (some entries old) and c new proposals, some of them nearer copies of the
    row's ids, in a random order."""
    ids = rng.choice(1000, R + c, replace=False)
    row = sorted(((float(rng.integers(10, 200)) + 0.5 * k / R, int(ids[k]), int(rng.random() < 0.6))
                  for k in range(R)), key=lambda x: (x[0], x[1]))
    props = []
    for t in range(c):
        if rng.random() < 0.35:  # a nearer copy of a row entry (a different recorded distance)
            rd, ri, _ = row[int(rng.integers(R))]
            props.append((rd - float(rng.integers(1, 30)) - 0.25, ri, 0))
        else:
            props.append((float(rng.integers(0, 220)) + 0.001 * t, int(ids[R + t]), 0))
    rng.shuffle(props)
    return row, props


@pytest.mark.parametrize("c", [2, 3, 4, 40, 70])
def test_old_pass_makes_the_device_merge_equal_the_oracles(c):
    rng = np.random.default_rng(c)
    R = 16
    deviated = 0
    for _ in range(300):
        row, props = _target(rng, R, c)
        want = _oracle_merge(row, props, R)
        assert _device_merge(row, props, R, old_pass=True) == want
        got = _device_merge(row, props, R, old_pass=False)
        assert [x[:2] for x in got] == [x[:2] for x in want]  # only old bits can differ
        deviated += got != want
    assert deviated > 0  # the truncation really does lose old bits without the pass


def test_exact_copies_need_no_pass():
    """With canonical distances every copy of an id carries the row's distance: a copy can
    only arrive where its row entry was, so the merge is exact without the pass."""
    rng = np.random.default_rng(5)
    R = 16
    for c in (3, 4, 40, 70):
        for _ in range(200):
            row, props = _target(rng, R, c)
            dist_of = {i: d for d, i, _ in row}
            props = [(dist_of.get(i, d), i, o) for d, i, o in props]
            assert _device_merge(row, props, R, old_pass=False) == _oracle_merge(row, props, R)
