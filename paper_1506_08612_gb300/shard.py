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
positions relative to the slice; on a GPU it is the library's own find, its
positions a device tensor.

The exchange (``gather_find``) runs on the process group's own device: CPU
tensors under gloo, CUDA tensors of the current device under NCCL (which
moves device memory only), so the positions of a GPU find never leave the
device before the merge.
"""
from __future__ import annotations

import numpy as np


def shard_range(n: int, world: int, rank: int, align: int = 1) -> tuple[int, int]:
    """Starts owned by ``rank``: [s, e).  Shards are whole multiples of
    ``align`` bytes (so a device slice keeps the text's alignment) and differ
    by at most one unit; the first ranks take the extra units, the last rank
    the bytes beyond the last whole unit."""
    if world <= 0 or not 0 <= rank < world or n < 0 or align < 1:
        raise ValueError("bad shard request")
    units, tail = divmod(n, align)
    base, extra = divmod(units, world)
    s = (rank * base + min(rank, extra)) * align
    e = s + (base + (1 if rank < extra else 0)) * align
    if rank == world - 1:
        e += tail
    return s, e


def read_range(n: int, world: int, rank: int, m: int, align: int = 1) -> tuple[int, int]:
    """Bytes ``rank`` reads: its owned starts plus the m - 1 byte overlap."""
    s, e = shard_range(n, world, rank, align)
    return s, min(e + m - 1, n) if e > s else e


def local_find(text, m: int, world: int, rank: int, engine, align: int = 1):
    """Run ``engine`` on this rank's slice.  Returns (count, global positions)
    (a numpy array, or a tensor on the engine's device when the engine
    returns one)."""
    n = len(text)
    s, e = shard_range(n, world, rank, align)
    rs, re = read_range(n, world, rank, m, align)
    if e <= s:
        return 0, np.zeros(0, np.int64)
    c, pos = engine(text[rs:re], e - s)
    if not _is_tensor(pos):
        pos = np.asarray(pos, dtype=np.int64)
    if len(pos) != c:
        raise RuntimeError("engine returned a truncated position list")
    return int(c), pos + s


def _is_tensor(x) -> bool:
    try:
        import torch
        return isinstance(x, torch.Tensor)
    except ImportError:          # pragma: no cover
        return False


def exchange_device(group=None):
    """Where ``gather_find`` puts its buffers: the current CUDA device for an
    NCCL group (NCCL moves device memory only), else the CPU."""
    import torch
    import torch.distributed as dist
    if str(dist.get_backend(group)).lower() == "nccl":
        return torch.device("cuda", torch.cuda.current_device())
    return torch.device("cpu")


def merge(counts, positions):
    """Concatenate per-rank results in rank order (positions at the exclusive
    prefix sums of the counts).  Returns (total, positions)."""
    counts = [int(c) for c in counts]
    offs = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    out = np.empty(int(offs[-1]), np.int64)
    for r, p in enumerate(positions):
        out[offs[r]:offs[r + 1]] = p
    return int(offs[-1]), out


def merge_tensors(counts, positions):
    """``merge`` for per-rank position tensors on one device: their
    concatenation in rank order.  Returns (total, positions tensor)."""
    import torch
    counts = [int(c) for c in counts]
    parts = [p[:c] for p, c in zip(positions, counts)]
    if not parts:
        return 0, torch.zeros(0, dtype=torch.int64)
    return sum(counts), torch.cat(parts)


def gather_find(count: int, positions, group=None):
    """All ranks exchange their (count, positions) over ``torch.distributed``
    and return the merged result on every rank: one all-gather of the counts
    and one of the position lists padded to the longest, on the group's
    device (``exchange_device``).  Under gloo the merged positions come back
    as a numpy array; under NCCL as a tensor on the current CUDA device."""
    import torch
    import torch.distributed as dist

    dev = exchange_device(group)
    world = dist.get_world_size(group)
    c = torch.tensor([int(count)], dtype=torch.int64, device=dev)
    cs = [torch.zeros(1, dtype=torch.int64, device=dev) for _ in range(world)]
    dist.all_gather(cs, c, group=group)
    counts = [int(x.item()) for x in cs]
    longest = max(max(counts), 1)
    mine = torch.zeros(longest, dtype=torch.int64, device=dev)
    if int(count):
        src = positions if _is_tensor(positions) else torch.as_tensor(np.asarray(positions, np.int64))
        mine[:int(count)] = src[:int(count)].to(dev)
    ps = [torch.zeros(longest, dtype=torch.int64, device=dev) for _ in range(world)]
    dist.all_gather(ps, mine, group=group)
    total, merged = merge_tensors(counts, ps)
    if dev.type == "cpu":
        return total, merged.numpy()
    return total, merged
