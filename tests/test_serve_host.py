"""Host logic of the serving loop (no GPU): the position arena, batching
by sequence, admission by position memory, continuous batching with work in
flight, and answers that match the oracle whether a query runs alone or in
the mix.  The device is replaced by an engine that answers from the oracle
after a few polls."""
import collections

import numpy as np
import pytest

import oracle
import synth
from paper_1506_08612_gb300.batched import MAX_STATES
from paper_1506_08612_gb300.serve import Arena, Query, Server, latency_summary


# ------------------------------------------------------------------ arena

def test_arena_first_fit_and_coalescing():
    a = Arena(4096, align=256)
    x = a.alloc(100)
    y = a.alloc(1000)
    z = a.alloc(256)
    assert x == (0, 256) and y == (256, 1024) and z == (1280, 256)
    assert a.alloc(4096) is None
    a.release(*y)
    assert a.alloc(512) == (256, 512)          # first fit inside the hole
    a.release(256, 512)
    a.release(*x)
    a.release(*z)
    assert a.free == [(0, 4096)] and a.used == 0
    assert a.alloc(4096) == (0, 4096)


def test_arena_random_churn_never_overlaps():
    rng = np.random.default_rng(5)
    a = Arena(1 << 20, align=256)
    live = []
    for _ in range(3000):
        if live and rng.random() < 0.45:
            a.release(*live.pop(int(rng.integers(len(live)))))
        else:
            r = a.alloc(int(rng.integers(1, 40_000)))
            if r is not None:
                live.append(r)
        iv = sorted(live + a.free)
        assert sum(n for _, n in iv) == a.size            # used + free = all
        for (o1, n1), (o2, _) in zip(iv, iv[1:]):
            assert o1 + n1 == o2                          # a partition, no overlap
        assert a.used == sum(n for _, n in live)


# ------------------------------------------------------------------ fake engine

class FakeEngine:
    """Answers from the oracle after ``delay`` polls; records what ran."""

    def __init__(self, texts, slots=2, arena_bytes=1 << 20, delay=2):
        self.texts = texts
        self.nslots = slots
        self.arena_bytes = arena_bytes
        self.delay = delay
        self.launched = []
        self.max_active = 0
        self.active = 0

    def _job(self, kind, slot, seq, patterns, extra=None):
        self.active += 1
        self.max_active = max(self.max_active, self.active)
        self.launched.append((kind, slot, seq, list(patterns), extra))
        return {"polls": 0, "kind": kind, "seq": seq, "patterns": list(patterns), "extra": extra}

    def launch_count(self, slot, seq, patterns):
        assert len({p.upper() for p in patterns}) == len(patterns)
        return self._job("count", slot, seq, patterns)

    def launch_find(self, slot, seq, patterns, counts, region):
        assert region[1] >= 8 * sum(counts)
        return self._job("find", slot, seq, patterns, (list(counts), region))

    def done(self, job):
        job["polls"] += 1
        if job["polls"] > self.delay:
            if not job.get("counted"):
                job["counted"] = True
                self.active -= 1
            return True
        return False

    def count_result(self, job):
        t = self.texts[job["seq"]]
        return np.array([oracle.count_brute(t, p) for p in job["patterns"]], dtype=np.uint64)

    def find_result(self, job):
        t = self.texts[job["seq"]]
        return [oracle.find_brute(t, p)[1] for p in job["patterns"]]


def _texts():
    return [synth.genome_text(20_000 + 3_000 * i, 100 + i, mask_mean=60, n_gap_mean=8_000,
                              n_run_mean=100) for i in range(3)]


def _trace(k=40, seed=3):
    tr = synth.query_trace(k, 1000.0, 3, seed, max_patterns=8, m_lo=3, m_hi=9)
    return tr


def _expect(texts, q):
    t = texts[q.seq]
    counts = [oracle.count_brute(t, p) for p in q.patterns]
    pos = [oracle.find_brute(t, p)[1] for p in q.patterns] if q.mode == "positions" else None
    return counts, pos


def _check(texts, q):
    counts, pos = _expect(texts, q)
    assert q.error is None, q.error
    assert q.counts.tolist() == counts
    if q.mode == "positions":
        assert len(q.positions) == len(q.patterns)
        for a, b in zip(q.positions, pos):
            assert np.array_equal(a, b)
    else:
        assert q.positions is None


def test_every_query_answered_like_alone():
    texts = _texts()
    eng = FakeEngine(texts, slots=3)
    srv = Server(eng)
    qs = [srv.submit(Query(seq=e["seq"], patterns=e["patterns"], mode=e["mode"]))
          for e in _trace()]
    srv.run_until_idle()
    assert len(srv.done) == len(qs)
    for q in qs:
        _check(texts, q)
    # batches hold one sequence each and reuse a pattern shared by two queries
    for kind, slot, seq, pats, _ in eng.launched:
        assert len(set(p.upper() for p in pats)) == len(pats)
    by_batch = collections.defaultdict(set)
    for q in qs:
        by_batch[q.batch].add(q.seq)
    assert all(len(s) == 1 for s in by_batch.values())
    assert len(by_batch) < len(qs)                    # queries were batched together
    assert eng.max_active >= 2                        # stages overlapped on the slots
    # alone: each query in a fresh server gives the same answer
    for q in qs[:10]:
        solo = Server(FakeEngine(texts, slots=1)).submit(
            Query(seq=q.seq, patterns=q.patterns, mode=q.mode))
        s2 = Server(FakeEngine(texts, slots=1))
        s2.submit(solo)
        s2.run_until_idle()
        assert solo.counts.tolist() == q.counts.tolist()
        if q.mode == "positions":
            assert all(np.array_equal(a, b) for a, b in zip(solo.positions, q.positions))


def test_arrivals_while_work_is_in_flight():
    texts = _texts()
    eng = FakeEngine(texts, slots=2, delay=5)
    srv = Server(eng)
    first = srv.submit(Query(seq=0, patterns=[b"ACG"], mode="count"))
    srv.step()
    assert eng.active == 1
    late = srv.submit(Query(seq=1, patterns=[b"CGT", b"A"], mode="positions"))
    srv.step()
    assert eng.active == 2                             # admitted while the first runs
    srv.run_until_idle()
    _check(texts, first)
    _check(texts, late)
    assert first.batch != late.batch


def test_admission_waits_for_position_memory_in_order():
    texts = [np.frombuffer(b"A" * 5000, np.uint8).copy()]
    # each query locates "AAAA" (4997 occurrences = 39,976 bytes): the arena
    # holds one at a time
    eng = FakeEngine(texts, slots=4, arena_bytes=48 * 1024, delay=1)
    srv = Server(eng, max_batch_patterns=1)
    # the four queries of "AAAA" share one batch (one distinct pattern);
    # max_batch_patterns=1 puts "AAAAA" (39,968 bytes) in a second batch,
    # which must wait until the first batch's region is released
    qs = [srv.submit(Query(seq=0, patterns=[b"AAAA"], mode="positions")) for _ in range(4)]
    qs += [srv.submit(Query(seq=0, patterns=[b"AAAAA"], mode="positions"))]
    peak = 0
    while not srv.idle():
        srv.step()
        peak = max(peak, srv.arena.used)
        assert srv.arena.used <= srv.arena.size
    assert peak <= 48 * 1024
    assert srv.stats["mem_stalls"] > 0
    for q in qs:
        _check(texts, q)
    finds = [x for x in eng.launched if x[0] == "find"]
    assert len(finds) == 2
    assert [f[4][1][0] for f in finds] == [0, 0]            # one region live at a time


def test_request_larger_than_the_arena_fails_cleanly():
    texts = [np.frombuffer(b"A" * 5000, np.uint8).copy()]
    srv = Server(FakeEngine(texts, slots=2, arena_bytes=4096))
    big = srv.submit(Query(seq=0, patterns=[b"AA"], mode="positions"))
    small = srv.submit(Query(seq=0, patterns=[b"AA"], mode="count"))
    srv.run_until_idle()
    assert big.error and "position arena" in big.error
    assert small.error is None and small.counts.tolist() == [4999]
    assert srv.stats["rejected_batches"] == 1


def test_batches_respect_the_automaton_state_limit():
    texts = _texts()
    eng = FakeEngine(texts, slots=1)
    srv = Server(eng, max_batch_patterns=100_000)
    for i in range(12):
        pats = [synth.pattern(64, 10_000 * i + j) for j in range(32)]      # 2048 bytes each
        srv.submit(Query(seq=0, patterns=pats, mode="count"))
    srv.run_until_idle()
    counts = [x for x in eng.launched if x[0] == "count"]
    assert len(counts) >= 2
    for _, _, _, pats, _ in counts:
        trie = {bytes(p).upper()[:k] for p in pats for k in range(len(p) + 1)}
        assert len(trie) <= MAX_STATES


def test_replay_and_latency_summary():
    texts = _texts()
    t = [0.0]

    def clock():
        t[0] += 1e-4                                  # a deterministic clock
        return t[0]

    srv = Server(FakeEngine(texts, slots=2), clock=clock)
    trace = _trace(20, seed=9)
    qs = srv.replay(trace, speed=1000.0)
    assert all(q is not None and q.t_done >= q.t_arrive for q in qs)
    s = latency_summary(qs)
    assert s["completed"] == 20 and s["errors"] == 0
    assert 0 < s["p50_ms"] <= s["p99_ms"] <= s["max_ms"]
    for q in qs:
        _check(texts, q)


def test_latency_percentiles_nearest_rank():
    qs = []
    for i in range(100):
        q = Query(seq=0, patterns=[b"A"], t_arrive=0.0)
        q.t_done = (i + 1) * 1e-3
        qs.append(q)
    s = latency_summary(qs)
    assert s["p50_ms"] == pytest.approx(50.0) and s["p99_ms"] == pytest.approx(99.0)
    assert s["max_ms"] == pytest.approx(100.0)


def test_malformed_queries_complete_with_an_error():
    from paper_1506_08612_gb300.serve import query_error
    texts = _texts()
    eng = FakeEngine(texts, slots=2)
    eng.nseq = len(texts)
    srv = Server(eng)
    bad = [Query(seq=0, patterns=[b"ACGN"]), Query(seq=0, patterns=[b""]),
           Query(seq=0, patterns=["A" * 65]), Query(seq=0, patterns=[]),
           Query(seq=3, patterns=[b"ACG"]), Query(seq=-1, patterns=[b"ACG"]),
           Query(seq=0, patterns=[b"ACG"], mode="regex"), Query(seq=0, patterns=["ACGÄ"])]
    good = Query(seq=1, patterns=["acgT", b"A" * 64], mode="positions")
    qs = [srv.submit(q) for q in bad[:4]] + [srv.submit(good)] + [srv.submit(q) for q in bad[4:]]
    assert all(q.error and q.t_done >= q.t_arrive for q in bad)
    assert srv.stats["rejected_queries"] == len(bad)
    srv.run_until_idle()
    _check(texts, good)
    assert all(x[3] != [b"ACGN"] for x in eng.launched)      # nothing malformed reached the engine
    assert len(srv.done) == len(qs)
    assert query_error(good, 2) is None
    assert "no sequence 1" in query_error(good, 1)
    assert query_error(good) is None                          # engine without a sequence count
    s = latency_summary(qs)
    assert s["completed"] == 1 and s["errors"] == len(bad)
