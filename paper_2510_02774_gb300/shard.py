"""Vertex-range sharding of one build over several ranks: the exchange step of the join.

A build can be split over G ranks that each hold a replica of the points and own the pools
of one contiguous range of vertices.  A round (Alg 4) then has exactly one exchange: every
rank runs the join for the vertices it owns, which proposes each pool entry either back to
its own vertex (a survivor, as old) or to the entry that absorbed it (a redirect, Eq 2),
buckets those proposals by the owner of their target, and sends the buckets in one
all-to-all; every rank then merges what it received into the pools it owns (Sec 3.5, the
merge rule of Alg 6).  Reverse-edge sampling between outer iterations (Sec 3.6) is a second
exchange of the same form, its proposals going from a vertex to the entries it samples.

This module is the host-side partition and exchange.  It moves proposals as plain columns
(tensors of equal length: target, id, distance, old flag, in whatever encoding the caller
uses) and never looks inside them, so the join and the merge on either side can be the
library's kernels on a GPU (NCCL process group) or any other implementation (a gloo group
on CPU).  One proposal of the library's own encoding is 12 bytes (int32 target + uint64
key), so a round moves at most n * R * 12 bytes in total.
"""
from __future__ import annotations

from typing import Sequence

import torch
import torch.distributed as dist


def owner_ranges(n: int, world: int) -> list[tuple[int, int]]:
    """Contiguous, balanced vertex ranges [lo, hi) of the `world` ranks (the first n % world
    ranges hold one vertex more)."""
    if n < 0 or world < 1:
        raise ValueError("need n >= 0 and world >= 1")
    base, extra = divmod(n, world)
    out, lo = [], 0
    for r in range(world):
        hi = lo + base + (1 if r < extra else 0)
        out.append((lo, hi))
        lo = hi
    return out


def owner_of(target: torch.Tensor, n: int, world: int) -> torch.Tensor:
    """Rank that owns each vertex id in `target` under owner_ranges(n, world)."""
    base, extra = divmod(n, world)
    t = target.to(torch.int64)
    split = extra * (base + 1)  # vertices below this id sit in the larger ranges
    big = torch.div(t, base + 1, rounding_mode="floor")
    small = extra + torch.div(t - split, max(base, 1), rounding_mode="floor")
    return torch.where(t < split, big, small)


def bucket_by_owner(owner: torch.Tensor, columns: Sequence[torch.Tensor], world: int):
    """Orders proposals by owner rank (stable) and counts them per rank.

    Returns (the reordered columns, counts[world] as a CPU int64 tensor)."""
    order = torch.argsort(owner, stable=True)
    counts = torch.bincount(owner.to(torch.int64), minlength=world).to(torch.int64).cpu()
    return [c[order] for c in columns], counts


def exchange(owner: torch.Tensor, columns: Sequence[torch.Tensor], world: int, group=None) -> list[torch.Tensor]:
    """The all-to-all of a round: sends proposal j to rank owner[j].

    Every rank calls this with its own proposals; it returns the proposals of all ranks whose
    owner is this rank, in rank order (and, within one sender, in that sender's order)."""
    if any(c.shape[0] != owner.shape[0] for c in columns):
        raise ValueError("every column needs one entry per proposal")
    if world == 1:
        return [c.clone() for c in columns]
    cols, send = bucket_by_owner(owner, columns, world)
    dev = columns[0].device if columns else owner.device
    send_d = send.to(dev)
    recv_d = torch.empty_like(send_d)
    dist.all_to_all_single(recv_d, send_d, group=group)
    recv = recv_d.cpu()
    out = []
    for c in cols:
        r = torch.empty((int(recv.sum()),) + tuple(c.shape[1:]), dtype=c.dtype, device=c.device)
        dist.all_to_all_single(r, c.contiguous(), recv.tolist(), send.tolist(), group=group)
        out.append(r)
    return out
