"""Batched, graph-captured, autotuned count (many patterns x many sequences
in one persistent launch) against the CPU oracle, bit-exact.

The batched workload is six genome-like sequences x 256 patterns of length
uniform in [4, 64]; here the sequences are the same recipe at 1/1000 of the
sizes (0.2 .. 3.2 MB), so the oracle's one-by-one window compare finishes in
seconds while every sequence still spans many tiles and ends ragged.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

SIZES_GB = (0.2, 1.0, 2.4, 2.4, 2.7, 3.2)


@pytest.fixture(autouse=True)
def _tune_cache(tmp_path, monkeypatch):
    from paper_1506_08612_gb300 import autotune
    monkeypatch.setenv("DNADFA_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    monkeypatch.delenv("DNADFA_CONFIG", raising=False)
    autotune.reset_memory_cache()
    yield
    autotune.reset_memory_cache()


def batch_patterns(k=256, seed=16):
    lens = synth.uniform_ints(k, 61, seed) + 4
    return [synth.pattern(int(m), seed * 100_000 + i) for i, m in enumerate(lens)]


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_six_sequences_256_patterns_autotuned_graph(gpu):
    texts = [synth.genome_text(int(g * 1e6) + 7 * i, 10 + i) for i, g in enumerate(SIZES_GB)]
    pats = batch_patterns()
    # plant a few occurrences of the long patterns so they are not all zero
    for i, t in enumerate(texts):
        for j in range(0, len(pats), 16):
            at = synth.uniform_ints(2, len(t) - len(pats[j]), 77 * i + j)
            synth.plant(t, pats[j], at)
    b = gpu.BatchedCount([_dev(t) for t in texts], pats, cfg="auto")
    assert b.graph is not None and b.launches == 1
    b.run()
    got = b.result()
    want = oracle.multi_count(texts, pats)
    assert np.array_equal(got, want), np.argwhere(got != want)[:5]
    assert (want[:, ::16] > 0).all()
    # replay twice more: same answer
    for _ in range(2):
        b.run()
        assert np.array_equal(b.result(), want)


def test_graph_replay_sees_new_text_contents(gpu):
    import torch
    texts = [synth.genome_text(500_003, 31), synth.genome_text(200_001, 32)]
    pats = [synth.pattern(m, 300 + m) for m in (4, 6, 9, 20)]
    dts = [_dev(t) for t in texts]
    b = gpu.BatchedCount(dts, pats, cfg=None)
    b.run()
    assert np.array_equal(b.result(), oracle.multi_count(texts, pats))
    new = [synth.genome_text(t.size, 40 + i) for i, t in enumerate(texts)]
    for d, t in zip(dts, new):
        d.copy_(torch.from_numpy(t))
    b.run()
    assert np.array_equal(b.result(), oracle.multi_count(new, pats))
    # writes still queued on the caller's stream (behind a ~10 ms spin)
    # when run() is called are seen by the batch's own stream
    src = [_dev(t) for t in texts]
    torch.cuda.synchronize()
    torch.cuda._sleep(20_000_000)
    for d, s in zip(dts, src):
        d.copy_(s, non_blocking=True)
    b.run()
    assert np.array_equal(b.result(), oracle.multi_count(texts, pats))


def test_many_sequences_and_split_automata(gpu):
    # 70 sequences (two launches of <= 64) x 300 patterns of length 56..64
    # (more trie states than one automaton holds: two automata)
    texts = [synth.genome_text(3_000 + 97 * i, 500 + i, mask_mean=40, n_gap_mean=5_000,
                               n_run_mean=50) for i in range(70)]
    lens = synth.uniform_ints(300, 9, 5) + 56
    pats = [synth.pattern(int(m), 9000 + i) for i, m in enumerate(lens)]
    pats[:6] = [b"ACGT", b"CG", b"A", b"TTTT", b"GATTACA", b"ACGT"]
    for i, t in enumerate(texts):
        p = pats[6 + (i % 290)]
        synth.plant(t, p, [i * 3 % (len(t) - len(p))])
    b = gpu.BatchedCount([_dev(t) for t in texts], pats, cfg=dict(threads=128, chunk=256))
    assert len(b.groups) == 2 and len(b.seq_groups) == 2 and b.launches == 4
    b.run()
    got = b.result()
    assert np.array_equal(got, oracle.multi_count(texts, pats))
    assert got[:, 6:].sum() >= 70


def test_empty_and_short_sequences(gpu):
    import torch
    texts = [np.zeros(0, np.uint8), np.frombuffer(b"ACG", np.uint8).copy(),
             np.frombuffer(b"acgtNacgt", np.uint8).copy()]
    pats = [b"ACGT", b"ACG", b"CGT", b"T"]
    dts = [torch.from_numpy(t).cuda() if t.size else torch.empty(0, dtype=torch.uint8, device="cuda")
           for t in texts]
    b = gpu.BatchedCount(dts, pats, cfg=None)
    b.run()
    got = b.result()
    assert np.array_equal(got, oracle.multi_count(texts, pats))
    assert got.tolist() == [[0, 0, 0, 0], [0, 1, 0, 0], [2, 2, 2, 2]]


def test_single_pattern_autotune_and_cache(gpu):
    import json
    import os

    from paper_1506_08612_gb300 import autotune
    n = 40_000_000
    t = synth.genome_text(n, 51)
    pat = synth.pattern(12, 5100)
    synth.plant(t, pat, synth.uniform_ints(50, n - 12, 52))
    td = _dev(t)
    tab = gpu.dfa_build(pat)
    cfg = autotune.tune_single(td, tab, reps=2)
    assert cfg in autotune.single_candidates(12)
    assert gpu.count(td, tab, cfg=cfg) == oracle.count_brute(t, pat)
    c, pos = gpu.find(td, tab, cfg=cfg)
    assert np.array_equal(pos.cpu().numpy(), oracle.find_brute(t, pat)[1])
    # a second call is answered from the cache file
    path = os.environ["DNADFA_AUTOTUNE_CACHE"]
    key = autotune.single_key(autotune.device_name(), n, 12)
    assert json.load(open(path))[key]["cfg"] == cfg
    autotune.reset_memory_cache()
    assert autotune.tune_single(td, tab) == cfg


def test_class_patterns_batched_and_split(gpu):
    """Class patterns in the graph-captured batch: a set too large for one
    automaton (four patterns of 6144 states each) is split into groups, one
    launch each, and every count matches the oracle."""
    pats = ["A" + "N" * 11 + "T", "C" + "N" * 11 + "G", "G" + "N" * 11 + "A", "T" + "N" * 11 + "C",
            "ACGT", "R" * 5] + [c for c, _ in synth.class_pattern_pairs(5, 43)]
    texts = [synth.genome_text(n, 750 + i) for i, n in enumerate((700_001, 1_300_003, 33))]
    b = gpu.BatchedCount([_dev(t) for t in texts], pats, cfg=None, classes=True)
    assert len(b.groups) >= 5 and b.graph is not None
    b.run()
    assert np.array_equal(b.result(), oracle.multi_count_class(texts, pats))
