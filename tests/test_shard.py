"""Vertex-range sharding of a build (the exchange step of the join), on CPU gloo ranks.

Each rank owns a vertex range, runs the oracle's per-vertex prune (Eq 2, Alg 4) for its own
vertices, sends the proposals to the owners of their targets with shard.exchange, and merges
what it received (C6); the gathered pools must equal the single-process round.  Reverse-edge
sampling (Sec 3.6) goes through the same exchange.
"""
import os
import socket

import numpy as np
import pytest
import torch

from paper_2510_02774_gb300 import shard, synth


def test_owner_ranges_partition_the_vertices():
    for n, world in [(10, 3), (7, 7), (3, 5), (1000, 8), (0, 2)]:
        rs = shard.owner_ranges(n, world)
        assert len(rs) == world and rs[0][0] == 0 and rs[-1][1] == n
        assert all(a[1] == b[0] for a, b in zip(rs, rs[1:]))
        sizes = [hi - lo for lo, hi in rs]
        assert max(sizes) - min(sizes) <= 1
        t = torch.arange(n)
        own = shard.owner_of(t, n, world)
        for r, (lo, hi) in enumerate(rs):
            assert (own[lo:hi] == r).all()


def test_exchange_single_rank_is_identity():
    own = torch.zeros(5, dtype=torch.int64)
    cols = [torch.arange(5), torch.arange(5) * 2.0]
    out = shard.exchange(own, cols, 1)
    assert all(torch.equal(a, b) for a, b in zip(out, cols))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _round_proposals(orc, X, p, vs, seed, t1, t2):
    """Proposals (target, id, dist, old) of the joins of vertices vs: survivors back to v
    as old, bottom entries to their absorber with the pair distance, as new."""
    tgt, ids, dd, old = [], [], [], []
    for v in vs:
        m = int(p.deg[v])
        if m == 0:
            continue
        row_ids, row_d, row_o = p.ids[v][:m], p.dist[v][:m], p.old[v][:m]
        perm = orc.visit_order(seed, t1, t2, v, row_ids)
        alive, killer, kd, _, _ = orc.prune(X, row_ids, row_d, perm, row_o)
        for e in range(m):
            if alive[e]:
                tgt.append(v), ids.append(row_ids[e]), dd.append(row_d[e]), old.append(1)
            else:
                tgt.append(row_ids[killer[e]]), ids.append(row_ids[e]), dd.append(kd[e]), old.append(0)
    return tgt, ids, dd, old


def _reverse_proposals(p, vs, rho):
    """Own rows (kept as they are) and the first floor(rho * deg) entries proposed back."""
    tgt, ids, dd, old = [], [], [], []
    for v in vs:
        m = int(p.deg[v])
        for e in range(m):
            tgt.append(v), ids.append(p.ids[v][e]), dd.append(p.dist[v][e]), old.append(int(p.old[v][e]))
        for e in range(int(np.floor(np.float64(np.float32(rho)) * m))):
            tgt.append(p.ids[v][e]), ids.append(v), dd.append(p.dist[v][e]), old.append(0)
    return tgt, ids, dd, old


def _worker(rank, world, port, q):
    import torch.distributed as dist
    import oracle.oracle as orc
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        n, d, S, R, seed, rho = 400, 8, 8, 16, 5, 0.6
        X = synth.small_integers(n, d, -8, 8, seed=3)
        p, _ = orc.init(X, S, R, seed)
        lo, hi = shard.owner_ranges(n, world)[rank]
        results = []
        for t2 in (1, 2):
            tgt, ids, dd, old = _round_proposals(orc, X, p, range(lo, hi), seed, 1, t2)
            cols = [torch.tensor(ids, dtype=torch.int64), torch.tensor(dd, dtype=torch.float64),
                    torch.tensor(old, dtype=torch.int64), torch.tensor(tgt, dtype=torch.int64)]
            own = shard.owner_of(cols[3], n, world)
            r_ids, r_d, r_old, r_tgt = shard.exchange(own, cols, world)
            assert bool((shard.owner_of(r_tgt, n, world) == rank).all())
            mine = orc.merge(n, R, r_tgt.numpy(), r_ids.numpy(), r_d.numpy(), r_old.numpy())
            want, _, _ = orc.round_(X, p, seed, 1, t2)
            results.append((np.array_equal(mine.ids[lo:hi], want.ids[lo:hi]),
                            np.array_equal(mine.deg[lo:hi], want.deg[lo:hi]),
                            np.array_equal(mine.old[lo:hi], want.old[lo:hi]),
                            np.array_equal(mine.dist[lo:hi], want.dist[lo:hi])))
            p = want
        tgt, ids, dd, old = _reverse_proposals(p, range(lo, hi), rho)
        cols = [torch.tensor(ids, dtype=torch.int64), torch.tensor(dd, dtype=torch.float64),
                torch.tensor(old, dtype=torch.int64), torch.tensor(tgt, dtype=torch.int64)]
        r_ids, r_d, r_old, r_tgt = shard.exchange(shard.owner_of(cols[3], n, world), cols, world)
        mine = orc.merge(n, R, r_tgt.numpy(), r_ids.numpy(), r_d.numpy(), r_old.numpy())
        want, _ = orc.reverse(p, rho)
        results.append((np.array_equal(mine.ids[lo:hi], want.ids[lo:hi]),
                        np.array_equal(mine.deg[lo:hi], want.deg[lo:hi]),
                        np.array_equal(mine.old[lo:hi], want.old[lo:hi]),
                        np.array_equal(mine.dist[lo:hi], want.dist[lo:hi])))
        q.put((rank, results, None))
    except Exception as e:  # reported to the parent
        q.put((rank, None, repr(e)))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_round_and_reverse_equal_single_process(world, orc):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    got = [q.get(timeout=180) for _ in range(world)]
    for pr in procs:
        pr.join(timeout=60)
    for rank, results, err in got:
        assert err is None, (rank, err)
        for step, flags in enumerate(results):
            assert all(flags), (rank, step, flags)


def test_exchange_delivers_every_proposal_to_its_owner():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    world = 3
    procs = [ctx.Process(target=_xchg_worker, args=(r, world, port, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    got = sorted(q.get(timeout=120) for _ in range(world))
    for pr in procs:
        pr.join(timeout=60)
    n = 1000
    sent = []
    for r in range(world):
        g = torch.Generator().manual_seed(r)
        t = torch.randint(0, n, (50 + 37 * r,), generator=g)
        sent += [(int(a), r, i) for i, a in enumerate(t.tolist())]
    for rank, recv, err in got:
        assert err is None, err
        lo, hi = shard.owner_ranges(n, world)[rank]
        want = sorted(s for s in sent if lo <= s[0] < hi)
        assert sorted(recv) == want


def _xchg_worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        n = 1000
        g = torch.Generator().manual_seed(rank)
        t = torch.randint(0, n, (50 + 37 * rank,), generator=g)
        src = torch.full_like(t, rank)
        idx = torch.arange(t.shape[0])
        rt, rs, ri = shard.exchange(shard.owner_of(t, n, world), [t, src, idx], world)
        q.put((rank, list(zip(rt.tolist(), rs.tolist(), ri.tolist())), None))
    except Exception as e:
        q.put((rank, None, repr(e)))
    finally:
        dist.destroy_process_group()
