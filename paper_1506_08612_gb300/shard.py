"""Sharding a scan over processes (one per GPU), host side.

The text is cut into contiguous shards the way Algorithm 1 cuts it into
chunks (Sec. III-A): rank r owns the occurrences that START in
[s_r, e_r) and reads the bytes [s_r, min(e_r + m - 1, n)), i.e. its shard
plus the m - 1 bytes of overlap from its successor, so every occurrence is
found by exactly one rank.  Counts add; positions are concatenated in rank
order, each rank's list shifted by s_r and placed at the exclusive prefix sum
of the counts of the ranks before it.

The per-rank scan is any callable ``engine(text_slice, n_own) -> (count,
positions)`` that returns the occurrences starting before ``n_own`` with
positions relative to the slice; on a GPU it is the library's own find.
"""
from __future__ import annotations

import numpy as np


def shard_range(n: int, world: int, rank: int) -> tuple[int, int]:
    """Starts owned by ``rank``: [s, e).  Shards differ in size by at most
    one byte; the first n % world ranks take the extra byte."""
    if world <= 0 or not 0 <= rank < world or n < 0:
        raise ValueError("bad shard request")
    base, extra = divmod(n, world)
    s = rank * base + min(rank, extra)
    e = s + base + (1 if rank < extra else 0)
    return s, e


def read_range(n: int, world: int, rank: int, m: int) -> tuple[int, int]:
    """Bytes ``rank`` reads: its owned starts plus the m - 1 byte overlap."""
    s, e = shard_range(n, world, rank)
    return s, min(e + m - 1, n) if e > s else e


def local_find(text, m: int, world: int, rank: int, engine):
    """Run ``engine`` on this rank's slice.  Returns (count, global positions)."""
    n = len(text)
    s, e = shard_range(n, world, rank)
    rs, re = read_range(n, world, rank, m)
    if e <= s:
        return 0, np.zeros(0, np.int64)
    c, pos = engine(text[rs:re], e - s)
    pos = np.asarray(pos, dtype=np.int64)
    if len(pos) != c:
        raise RuntimeError("engine returned a truncated position list")
    return int(c), pos + s


def merge(counts, positions):
    """Concatenate per-rank results in rank order (positions at the exclusive
    prefix sums of the counts).  Returns (total, positions)."""
    counts = [int(c) for c in counts]
    offs = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    out = np.empty(int(offs[-1]), np.int64)
    for r, p in enumerate(positions):
        out[offs[r]:offs[r + 1]] = p
    return int(offs[-1]), out


def gather_find(count: int, positions, group=None):
    """All ranks exchange their (count, positions) over ``torch.distributed``
    and return the merged result on every rank.  The exchange is one gather
    of the counts and one of the position lists padded to the longest."""
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group)
    c = torch.tensor([int(count)], dtype=torch.int64)
    cs = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(cs, c, group=group)
    counts = [int(x.item()) for x in cs]
    longest = max(counts) if counts else 0
    mine = torch.zeros(max(longest, 1), dtype=torch.int64)
    mine[:len(positions)] = torch.as_tensor(np.asarray(positions, np.int64))
    ps = [torch.zeros(max(longest, 1), dtype=torch.int64) for _ in range(world)]
    dist.all_gather(ps, mine, group=group)
    return merge(counts, [p[:k].numpy() for p, k in zip(ps, counts)])
