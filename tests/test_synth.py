"""The seeded input generators: determinism and the workload shapes."""
import numpy as np

import synth


def test_deterministic_and_seeded():
    a = synth.genome_text(100_000, 2)
    b = synth.genome_text(100_000, 2)
    c = synth.genome_text(100_000, 3)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    # a prefix of a longer text is the shorter text (counter-mode draws)
    assert np.array_equal(synth.uniform_text(1000, 0), synth.uniform_text(5000, 0)[:1000])
    assert synth.pattern(8, 1) == synth.pattern(8, 1)
    assert set(synth.pattern(64, 5)) <= set(b"ACGT")


def test_genome_composition():
    t = synth.genome_text(20_000_000, 2)
    vals, cnt = np.unique(t, return_counts=True)
    frac = dict(zip(bytes(vals).decode(), cnt / t.size))
    nfrac = frac.get("N", 0.0)
    lower = sum(frac.get(c, 0.0) for c in "acgt")
    gc = sum(frac.get(c, 0.0) for c in "CGcg") / (1 - nfrac)
    assert set(frac) <= set("ACGTacgtN")
    assert 0.40 < gc < 0.42
    assert 0.44 < lower / (1 - nfrac) < 0.56
    assert 0.01 < nfrac < 0.12          # 5% expected; few blocks in 20 MB


def test_uniform_composition():
    t = synth.uniform_text(1_000_000, 0)
    _, cnt = np.unique(t, return_counts=True)
    assert len(cnt) == 4 and (abs(cnt / t.size - 0.25) < 0.005).all()


def test_geometric_means():
    for mean in (300, 5000):
        xs = [synth.geometric(9, 1, k, mean) for k in range(40000)]
        assert min(xs) >= 1
        assert abs(np.mean(xs) / mean - 1) < 0.03


def test_plant():
    t = synth.genome_text(10_000, 4, n_gap_mean=0)
    synth.plant(t, b"ACGTACGTACGTACGT", [0, 100, 9990])
    assert t[100:116].tobytes().upper() == b"ACGTACGTACGTACGT"
    assert t[:16].tobytes().upper() == b"ACGTACGTACGTACGT"
