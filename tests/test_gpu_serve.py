"""The serving loop on the GPU: sequences resident in HBM, a Poisson stream of
count and positions queries, continuous batching over several CUDA streams,
admission by position memory.  Every answer is checked bit-exact against the
oracle, and a sample of queries is run again alone (a fresh server holding
only that query): the answers in the mix and alone are identical."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _setup(sizes=(400_000, 1_500_000, 3_000_003), seed=200):
    import torch
    texts = [synth.genome_text(n, seed + i) for i, n in enumerate(sizes)]
    return texts, [torch.from_numpy(t).cuda() for t in texts]


def _expect(texts, q):
    t = texts[q.seq]
    counts = [oracle.count_brute(t, p) for p in q.patterns]
    pos = [oracle.find_brute(t, p)[1] for p in q.patterns] if q.mode == "positions" else None
    return counts, pos


def _same(a, b):
    assert a.error is None and b.error is None, (a.error, b.error)
    assert a.counts.tolist() == b.counts.tolist()
    if a.mode == "positions":
        assert len(a.positions) == len(b.positions)
        for x, y in zip(a.positions, b.positions):
            assert np.array_equal(x, y)


def test_mixed_trace_matches_oracle_and_alone(gpu):
    from paper_1506_08612_gb300.serve import GpuEngine, Query, Server, latency_summary
    texts, devs = _setup()
    trace = synth.query_trace(80, 4000.0, len(texts), 7, max_patterns=12, m_lo=4, m_hi=14)
    srv = Server(GpuEngine(devs, slots=3, arena_bytes=64 << 20))
    qs = srv.replay(trace)
    assert all(q is not None and q.t_done for q in qs)
    nb = len({q.batch for q in qs})
    assert nb < len(qs)                                # queries shared batches
    for q in qs:
        counts, pos = _expect(texts, q)
        assert q.error is None, q.error
        assert q.counts.tolist() == counts, q.qid
        if q.mode == "positions":
            for a, b in zip(q.positions, pos):
                assert np.array_equal(a, b), q.qid
    # the same queries alone
    solo_srv = Server(GpuEngine(devs, slots=1, arena_bytes=64 << 20))
    for q in qs[::7]:
        s = solo_srv.submit(Query(seq=q.seq, patterns=q.patterns, mode=q.mode))
        solo_srv.run_until_idle()
        _same(q, s)
    st = latency_summary(qs)
    assert st["completed"] == len(qs) and st["p99_ms"] >= st["p50_ms"] > 0


def test_plain_engine_gives_the_same_answers(gpu):
    from paper_1506_08612_gb300.serve import GpuEngine, Server
    texts, devs = _setup((300_000, 800_000), seed=300)
    trace = synth.query_trace(30, 2000.0, len(texts), 11, max_patterns=6, m_lo=4, m_hi=10)
    a = Server(GpuEngine(devs, slots=2, arena_bytes=32 << 20)).replay(trace)
    b = Server(GpuEngine(devs, slots=2, arena_bytes=32 << 20, plain=True),
               max_batch_queries=1).replay(trace)
    for x, y in zip(a, b):
        _same(x, y)


def test_admission_under_a_small_position_arena(gpu):
    import torch
    from paper_1506_08612_gb300.serve import GpuEngine, Query, Server
    t = np.frombuffer((b"ACGTTGCA" * 40_000) + b"N" + (b"A" * 20_000), np.uint8).copy()
    dev = torch.from_numpy(t).cuda()
    # "ACGT" occurs 40,000 times (320,000 bytes of positions); the arena
    # holds 384 KiB, so position batches queue behind one another
    srv = Server(GpuEngine([dev], slots=4, arena_bytes=384 << 10), max_batch_patterns=1)
    qs = [srv.submit(Query(seq=0, patterns=[p], mode="positions"))
          for p in (b"ACGT", b"CGTT", b"GTTG", b"TTGC", b"ACGT")]
    big = srv.submit(Query(seq=0, patterns=[b"AAA"], mode="positions"))    # 19,998 x 8 bytes: fits
    huge = srv.submit(Query(seq=0, patterns=[b"A"], mode="positions"))     # 20,000 + 80,000 starts
    cnt = srv.submit(Query(seq=0, patterns=[b"A"], mode="count"))
    peak = 0
    while not srv.idle():
        srv.step()
        peak = max(peak, srv.arena.used)
    assert peak <= srv.arena.size
    assert srv.stats["mem_stalls"] > 0
    for q in qs + [big]:
        counts, pos = _expect([t], q)
        assert q.error is None and q.counts.tolist() == counts
        assert all(np.array_equal(a, b) for a, b in zip(q.positions, pos))
    assert huge.error is not None and "position arena" in huge.error
    assert cnt.error is None and cnt.counts.tolist() == [oracle.count_brute(t, b"A")]


def test_one_query_larger_than_an_automaton(gpu):
    """A query whose patterns need more trie states than one automaton holds
    (300 patterns of length 56..64) is split over several automata by the
    engine, in the count stage and in the located positions."""
    import torch
    from paper_1506_08612_gb300.batched import MAX_STATES, group_patterns
    from paper_1506_08612_gb300.serve import GpuEngine, Query, Server
    t = synth.genome_text(1_000_003, 330)
    lens = synth.uniform_ints(300, 9, 331) + 56
    pats = [synth.pattern(int(m), 33_000 + i) for i, m in enumerate(lens)]
    for i in range(0, 300, 3):
        synth.plant(t, pats[i], synth.uniform_ints(2, t.size - 64, 332 + i))
    assert len(group_patterns(pats)) >= 2
    assert len({p[:k] for p in pats for k in range(len(p) + 1)}) > MAX_STATES
    srv = Server(GpuEngine([torch.from_numpy(t).cuda()], slots=2, arena_bytes=8 << 20))
    qc = srv.submit(Query(seq=0, patterns=pats, mode="count"))
    qp = srv.submit(Query(seq=0, patterns=pats, mode="positions"))
    srv.run_until_idle()
    want = [oracle.find_brute(t, p) for p in pats]
    for q in (qc, qp):
        assert q.error is None, q.error
        assert q.counts.tolist() == [c for c, _ in want]
    assert sum(c for c, _ in want) >= 150                 # plants may overlap
    for got, (_, pos) in zip(qp.positions, want):
        assert np.array_equal(got, pos)
