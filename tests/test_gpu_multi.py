"""Multi-pattern automaton and batched count (through the C ABI) against the
CPU oracle: the automaton state by state against the oracle's own
multi-pattern table (the Table I construction, Sec. III-B), counts
bit-exact against brute force per pattern, the 6-mer census against the
oracle's census."""
import itertools

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

CODE = {"A": 0, "C": 1, "T": 2, "G": 3}      # (c >> 1) & 3


def _dev(arr):
    import torch
    return torch.from_numpy(np.ascontiguousarray(arr)).cuda()


def _walk(nxt, s):
    q = 0
    for ch in s:
        q = nxt[q, CODE[ch]]
    return q


PATTERN_SETS = [
    ["ACG", "ACT", "CTA", "TGA"],                       # Table I's caption
    ["A", "AA", "AAA", "AAAA"],                         # nested repeats
    ["ACGT", "CGTA", "GTAC", "TACG", "ACGT"],           # rotations + a duplicate
    ["GATTACA", "ATTA", "TTAC", "TA", "CAGATTACA"],
]


@pytest.mark.parametrize("pats", PATTERN_SETS + [None])
def test_automaton_matches_oracle_table(gpu, pats):
    if pats is None:
        pats = [synth.pattern(int(m), 40 + i).decode()
                for i, m in enumerate(synth.uniform_ints(40, 12, 7) + 1)]
    t = gpu.MultiTable(pats)
    nxt, nout = t.export()
    stt, _, names = oracle.stt_ascii(pats)
    idx = {nm: q for q, nm in enumerate(names)}
    prefixes = {p[:k] for p in pats for k in range(len(p) + 1)}
    assert t.states() == len(prefixes) == len(names)
    for w in prefixes:
        q = _walk(nxt, w)
        for ch in "ACGT":
            target = names[stt[idx[w], ord(ch)]]       # the oracle's transition
            assert nxt[q, CODE[ch]] == _walk(nxt, target), (w, ch)
            assert stt[idx[w], ord(ch.lower())] == stt[idx[w], ord(ch)]
        # patterns (with multiplicity) that end in state w: those that are a suffix of w
        assert nout[q] == sum(1 for p in pats if w.endswith(p)), w


def _check(gpu, texts, pats, cfg=None):
    got = gpu.multi_count([_dev(t) for t in texts], pats, cfg=cfg)
    want = oracle.multi_count(texts, pats)
    assert np.array_equal(got, want), (cfg, np.argwhere(got != want)[:5])
    return want


@pytest.mark.parametrize("cfg", [None, dict(threads=128, chunk=16), dict(threads=256, chunk=48),
                                 dict(threads=512, chunk=1024), dict(threads=128, chunk=4096)])
def test_counts_uneven_lengths_and_sequences(gpu, cfg):
    sizes = [0, 1, 5, 4099, 100_003, 257_000]
    texts = [synth.genome_text(n, 60 + i, mask_mean=50, n_gap_mean=20_000, n_run_mean=400)
             for i, n in enumerate(sizes)]
    lens = synth.uniform_ints(48, 61, 9) + 4                     # 4..64
    pats = [synth.pattern(int(m), 500 + i) for i, m in enumerate(lens)]
    pats += [pats[3][:5], pats[3], pats[7][2:11], b"AAAA", b"ACGTACGT", b"CGCG"]
    rng = np.random.default_rng(3)
    for i, t in enumerate(texts[3:]):
        for j, p in enumerate(pats):
            if len(t) > len(p) + 1:
                at = synth.uniform_ints(3, len(t) - len(p), 1000 * i + j)
                for a in at:
                    t[a:a + len(p)] = np.frombuffer(p, np.uint8)
    assert _check(gpu, texts, pats, cfg).sum() > 0


def test_borders_every_chunk(gpu):
    # occurrences of several lengths planted across every chunk border
    chunk = 64
    n = 256 * chunk * 3 + 33
    t = synth.genome_text(n, 5, n_gap_mean=0)
    pats = [synth.pattern(m, 700 + m) for m in (4, 9, 17, 33, 64)]
    for b in range(chunk, n - 70, chunk):
        p = pats[(b // chunk) % len(pats)]
        off = (b // chunk) % len(p)
        st = max(0, b - off)
        t[st:st + len(p)] = np.frombuffer(p, np.uint8)
    _check(gpu, [t], pats, dict(threads=256, chunk=chunk))
    _check(gpu, [t[1:]], pats, dict(threads=128, chunk=chunk))       # unaligned text


def test_kmer_census_4096(gpu):
    k = 6
    n = 16_000_000
    t = synth.genome_text(n, 20)
    pats = ["".join(s) for s in itertools.product("ACGT", repeat=k)]   # lexicographic = census order
    got = gpu.multi_count([_dev(t)], pats)[0]
    want = oracle.kmer_census(t, k)
    assert np.array_equal(got, want)
    assert int(got.sum()) == oracle.valid_windows(t, k)


def test_graph_captured_launch(gpu):
    import torch
    texts = [synth.genome_text(n, 80 + i) for i, n in enumerate((300_000, 1_000_000, 50_000))]
    pats = [synth.pattern(m, 900 + m) for m in (4, 5, 6, 8, 12)]
    want = oracle.multi_count(texts, pats).astype(np.int64).ravel()
    dt = [_dev(t) for t in texts]
    tab = gpu.MultiTable(pats)
    out = torch.zeros(len(texts) * len(pats), dtype=torch.int64, device="cuda")
    s = torch.cuda.Stream()
    gpu.dfa_multi_count(dt, tab, out, stream=s)                     # first call outside capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        gpu.dfa_multi_count(dt, tab, out, stream=s)
    for _ in range(3):
        out.fill_(-1)
        g.replay()
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), want)
