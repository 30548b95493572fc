"""Parity at the workloads' full sizes, in the launch configurations the
benchmark times (library defaults for one pattern, the autotuned batched
launch for many).

* Genome-scale single pattern: the 3.2e9-byte genome-like text (seed 2) and
  the five patterns m = 4, 8, 16, 32, 64 (seeds 3..7): counts and every
  position against the oracle's window compare, which finishes in seconds
  per pattern at this size.
* Batched: the six sequences (0.2 .. 3.2 GB, seeds 10..15) x 256 patterns of
  length uniform in [4, 64] (seed 16) in one graph-captured launch; every
  one of the 1536 (sequence, pattern) counts against the oracle's set
  compare (each window start compared with all 256 patterns).
* 6-mer census: 1e9 bytes (seed 20), all 4096 6-mers in one batched launch,
  against the oracle's census and the invariant sum = valid windows.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

GENOME_N = 3_200_000_000
BATCH_SIZES = (200_000_000, 1_000_000_000, 2_400_000_000, 2_400_000_000, 2_700_000_000,
               3_200_000_000)


@pytest.fixture(autouse=True)
def _tune_cache(tmp_path, monkeypatch):
    from paper_1506_08612_gb300 import autotune
    monkeypatch.setenv("DNADFA_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    monkeypatch.delenv("DNADFA_CONFIG", raising=False)
    autotune.reset_memory_cache()
    yield
    autotune.reset_memory_cache()


def _dev(a):
    import torch
    return torch.from_numpy(a).cuda()


def test_genome_scale_single_pattern_all_positions(gpu):
    import torch
    from concurrent.futures import ThreadPoolExecutor
    text = synth.genome_text(GENOME_N, 2)
    td = _dev(text)
    pats = [synth.pattern(m, seed) for m, seed in zip((4, 8, 16, 32, 64), (3, 4, 5, 6, 7))]
    with ThreadPoolExecutor(len(pats)) as ex:      # independent window compares
        wants = list(ex.map(lambda p: oracle.find_brute(text, p), pats))
    for pat, (want_c, want_p) in zip(pats, wants):
        m = len(pat)
        c, pos = gpu.find(td, pat)
        assert c == want_c, (m, c, want_c)
        assert np.array_equal(pos.cpu().numpy(), want_p), m
        del pos
    del td
    torch.cuda.empty_cache()


def test_batched_six_sequences_every_pair(gpu):
    import torch
    lens = synth.uniform_ints(256, 61, 16) + 4
    pats = [synth.pattern(int(m), 16 * 100_000 + i) for i, m in enumerate(lens)]
    texts, devs = [], []
    for i, n in enumerate(BATCH_SIZES):
        t = synth.genome_text(n, 10 + i)
        texts.append(t)
        devs.append(_dev(t))
    b = gpu.BatchedCount(devs, pats, cfg="auto")
    b.run()
    got = b.result()
    b.close()
    del devs
    torch.cuda.empty_cache()
    # all 6 x 256 counts, bit for bit
    want = oracle.count_set(texts, pats)
    assert got.shape == want.shape == (len(BATCH_SIZES), len(pats))
    bad = np.argwhere(got != want)
    assert bad.size == 0, [(int(i), int(j), int(got[i, j]), int(want[i, j])) for i, j in bad[:10]]
    assert (want.sum(axis=1) > 0).all()


def test_kmer_census_1GB(gpu):
    import itertools
    text = synth.genome_text(1_000_000_000, 20)
    pats = ["".join(s) for s in itertools.product("ACGT", repeat=6)]
    b = gpu.BatchedCount([_dev(text)], pats, cfg="auto")
    b.run()
    got = b.result()[0]
    want = oracle.kmer_census(text, 6)
    assert np.array_equal(got, want)
    assert int(got.sum()) == oracle.valid_windows(text, 6)


def test_serving_full_size_300_queries(gpu):
    # the serving workload's six resident sequences (11.9e9 bytes): a Poisson
    # trace of 300 count and positions queries (1-8 patterns of length
    # 7..40 each), every answer checked against the oracle's set compare
    # (all patterns asked of one sequence in one pass over it)
    import torch

    from paper_1506_08612_gb300.serve import GpuEngine, Server
    texts, devs = [], []
    for i, n in enumerate(BATCH_SIZES):
        t = synth.genome_text(n, 10 + i)
        texts.append(t)
        devs.append(_dev(t))
    trace = synth.query_trace(300, 200.0, len(texts), 31, max_patterns=8, m_lo=7, m_hi=40)
    for i, e in enumerate(trace[:6]):
        e["seq"] = i
    srv = Server(GpuEngine(devs, slots=4, arena_bytes=2 << 30))
    qs = srv.replay(trace)
    del devs, srv
    torch.cuda.empty_cache()
    assert len(qs) == 300
    for sq in range(len(texts)):
        mine = [q for q in qs if q.seq == sq]
        pats = sorted({p for q in mine for p in q.patterns})
        if not pats:
            continue
        wc, wp = oracle.find_set(texts[sq], pats)
        idx = {p: k for k, p in enumerate(pats)}
        for q in mine:
            assert q.error is None, q.error
            for j, p in enumerate(q.patterns):
                assert int(q.counts[j]) == int(wc[idx[p]]), (q.qid, j)
                if q.mode == "positions":
                    assert np.array_equal(q.positions[j], wp[idx[p]]), (q.qid, j)
