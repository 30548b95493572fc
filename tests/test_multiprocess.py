"""Multi-process host logic on CPU: world_size-2 gloo process groups.

The sharded scan (Algorithm 1's chunking one level up: each rank owns the
starts of its slice and reads m - 1 bytes of overlap) must give exactly the
single-process result; the per-rank engine here is the CPU oracle.  Also
covers bench.py's max-over-ranks timing reduction.
"""
import os
import socket

import numpy as np
import pytest

import oracle
import synth
from paper_1506_08612_gb300 import shard

pytestmark = pytest.mark.timeout(300) if hasattr(pytest.mark, "timeout") else []


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _engine(text_slice, n_own):
    c, pos = oracle.find_brute(np.ascontiguousarray(text_slice), _engine.pat)
    keep = pos < n_own
    return int(keep.sum()), pos[keep]


def _tensor_engine(text_slice, n_own):
    # the engine a GPU rank has: positions come back as a tensor
    import torch
    c, pos = _engine(text_slice, n_own)
    return c, torch.from_numpy(np.ascontiguousarray(pos))


def _worker(rank, world, port, cases, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        res = []
        for n, seed, m, pseed in cases:
            t = synth.genome_text(n, seed, mask_mean=40, n_gap_mean=5000, n_run_mean=300)
            pat = synth.pattern(m, pseed)
            _engine.pat = pat
            c, pos = shard.local_find(t, m, world, rank, _engine)
            total, merged = shard.gather_find(c, pos)
            res.append((total, merged.tolist()))
            # aligned shards and tensor positions: the same merged result
            c2, pos2 = shard.local_find(t, m, world, rank, _tensor_engine, align=64)
            total2, merged2 = shard.gather_find(c2, pos2)
            assert total2 == total and merged2.tolist() == merged.tolist()
        # bench's reduction: the slowest rank's time
        import torch
        tt = torch.tensor([10.0 + rank])
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        res.append(float(tt.item()))
        out.put((rank, res))
    finally:
        dist.destroy_process_group()


CASES = [(50_000, 1, 4, 2), (65_537, 3, 8, 4), (10, 5, 6, 6), (3, 7, 5, 8), (120_001, 9, 33, 10)]


def test_shard_ranges_cover_once():
    for n in (0, 1, 2, 7, 100, 101):
        for world in (1, 2, 3, 8):
            spans = [shard.shard_range(n, world, r) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            for (a, b), (c, d) in zip(spans, spans[1:]):
                assert b == c and a <= b
            for r in range(world):
                s, e = shard.read_range(n, world, r, 5)
                assert s == spans[r][0] and e == (min(spans[r][1] + 4, n) if spans[r][1] > s else s)


def test_aligned_shard_ranges():
    # shards of whole align-byte units (so a device slice keeps the text's
    # alignment), the last one taking the bytes past the last unit
    for n in (0, 1, 4095, 4096, 4097, 3 * 4096 + 5, 10 ** 6 + 7):
        for world in (1, 2, 3, 8):
            for align in (1, 64, 4096):
                spans = [shard.shard_range(n, world, r, align) for r in range(world)]
                assert spans[0][0] == 0 and spans[-1][1] == n
                for (a, b), (c, d) in zip(spans, spans[1:]):
                    assert b == c and a <= b
                assert all(a % align == 0 for a, _ in spans)
                units = [(b - a) // align for a, b in spans[:-1]]
                if units:
                    assert max(units) - min(units) <= 1


def test_exchange_device_follows_the_backend(monkeypatch):
    # NCCL moves device memory only: the exchange buffers live on the
    # current CUDA device for an NCCL group, on the CPU for gloo
    import torch
    import torch.distributed as dist
    monkeypatch.setattr(dist, "get_backend", lambda group=None: "nccl")
    monkeypatch.setattr(torch.cuda, "current_device", lambda: 3)
    assert shard.exchange_device() == torch.device("cuda", 3)
    monkeypatch.setattr(dist, "get_backend", lambda group=None: "gloo")
    assert shard.exchange_device() == torch.device("cpu")


def test_merge_tensors_equals_merge():
    import torch
    rng = np.random.default_rng(5)
    counts = [3, 0, 5, 1]
    parts = [np.sort(rng.integers(0, 10 ** 9, c)) for c in counts]
    padded = [torch.from_numpy(np.concatenate([p, np.full(6 - len(p), -1)]).astype(np.int64)) for p in parts]
    t1, m1 = shard.merge(counts, parts)
    t2, m2 = shard.merge_tensors(counts, padded)
    assert t1 == t2 and np.array_equal(m1, m2.numpy())


def test_sharded_equals_whole_single_process():
    # every world size in one process: local_find per rank + merge
    for n, seed, m, pseed in CASES:
        t = synth.genome_text(n, seed, mask_mean=40, n_gap_mean=5000, n_run_mean=300)
        pat = synth.pattern(m, pseed)
        _engine.pat = pat
        want_c, want_p = oracle.find_brute(t, pat)
        for world in (1, 2, 3, 5, 16):
            for align in (1, 64):
                parts = [shard.local_find(t, m, world, r, _engine, align=align) for r in range(world)]
                c, p = shard.merge([x[0] for x in parts], [x[1] for x in parts])
                assert c == want_c and np.array_equal(p, want_p), (n, m, world, align)


def test_gloo_world2_sharded_find():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, CASES, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=240) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for (n, seed, m, pseed), i in zip(CASES, range(len(CASES))):
        t = synth.genome_text(n, seed, mask_mean=40, n_gap_mean=5000, n_run_mean=300)
        want_c, want_p = oracle.find_brute(t, synth.pattern(m, pseed))
        for r in (0, 1):
            c, p = got[r][i]
            assert c == want_c and p == want_p.tolist(), (n, m, r)
    assert got[0][-1] == got[1][-1] == 11.0
