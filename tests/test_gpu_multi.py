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


def test_multi_locate_sorted_positions(gpu):
    # every pattern's sorted start positions from one walk of the automaton:
    # patterns of several lengths (a duplicate, nested ones), copies planted
    # across chunk borders and in the overlap, an unaligned text
    import torch
    n = 3_000_011
    t = synth.genome_text(n, 410, mask_mean=80, n_gap_mean=200_000, n_run_mean=3_000)
    lens = synth.uniform_ints(40, 40, 411) + 7                      # 7..46
    pats = [synth.pattern(int(m), 4200 + i) for i, m in enumerate(lens)]
    pats += [pats[5], pats[9][:8], pats[9][:12], b"GATTACAGATTACA"]
    for i, p in enumerate(pats):
        at = synth.uniform_ints(30, n - len(p), 4300 + i)
        at = np.concatenate([at, [1024 * k - len(p) // 2 for k in range(1, 40, 7)]])
        synth.plant(t, p, at)
    for text, td in ((t, _dev(t)), (t[3:], _dev(t)[3:])):
        mt = gpu.MultiTable(pats)
        counts = gpu.multi_count([td], mt)[0]
        assert counts.max() <= gpu.DFA_LOCATE_MAX
        total = int(counts.sum())
        pos = torch.full((total,), -1, dtype=torch.int64, device="cuda")
        work = torch.empty(gpu.dfa_multi_locate_work_bytes(len(pats)), dtype=torch.uint8, device="cuda")
        gpu.dfa_multi_locate(td, mt, counts, pos, work)
        assert gpu.dfa_multi_locate_status(work, len(pats)) == gpu.DFA_OK
        got = pos.cpu().numpy()
        o = 0
        for p, c in zip(pats, counts):
            want_c, want_p = oracle.find_brute(text, p)
            assert int(c) == want_c
            assert np.array_equal(got[o:o + want_c], want_p), p
            o += want_c


def test_multi_locate_rejects_and_reports(gpu):
    import torch
    t = synth.genome_text(500_000, 412)
    td = _dev(t)
    pats = [b"ACGTACGT", b"TTGACCA"]
    mt = gpu.MultiTable(pats)
    counts = gpu.multi_count([td], mt)[0]
    work = torch.empty(gpu.dfa_multi_locate_work_bytes(2), dtype=torch.uint8, device="cuda")
    pos = torch.empty(int(counts.sum()) + 8, dtype=torch.int64, device="cuda")
    with pytest.raises(gpu.DfaError):                       # a count above the bound
        gpu.dfa_multi_locate(td, mt, [gpu.DFA_LOCATE_MAX + 1, 0], pos, work)
    with pytest.raises(gpu.DfaError):                       # positions buffer too small
        gpu.dfa_multi_locate(td, mt, counts, pos[:1], work)
    # counts that do not belong to the text: the segments do not fill exactly
    wrong = [int(counts[0]) + 1, int(counts[1])]
    gpu.dfa_multi_locate(td, mt, wrong, pos, work)
    assert gpu.dfa_multi_locate_status(work, 2) == gpu.DFA_EINVAL


def test_count_with_the_largest_automaton(gpu):
    """An automaton of exactly 16384 states (the last state number, 16383,
    makes the largest transition entry, 4 * 16383 + 1) counts every pattern
    exactly, the deepest states included."""
    from test_multi_host import patterns_with_trie_states
    pats = patterns_with_trie_states(16384, 72_000)
    mt = gpu.MultiTable(pats)
    assert mt.states() == 16384
    texts = [synth.genome_text(2_000_003, 720), synth.genome_text(700_001, 721)]
    for i, t in enumerate(texts):
        for j in range(i, len(pats), 5):
            synth.plant(t, pats[j], synth.uniform_ints(1, t.size - 64, 7200 + 10 * j + i))
    counts = torch_zeros(len(texts) * len(pats))
    gpu.dfa_multi_count([_dev(t) for t in texts], mt, counts)
    want = oracle.multi_count(texts, pats)
    got = counts.cpu().numpy().astype(np.uint64).reshape(want.shape)
    assert np.array_equal(got, want), np.argwhere(got != want)[:5]
    assert (want > 0).sum() >= len(pats) // 5


def torch_zeros(n):
    import torch
    return torch.zeros(n, dtype=torch.int64, device="cuda")


CLASS_PATTERNS = ["R", "[AC]A", "NN", "GATTACA", "gaWtaca", "[ACT]TCGGAGC", "GCCTAAG[ACG]",
                  "ACGTRYSWKMBDHVN", "A" + "N" * 6 + "T", "[ac][gt][ac][gt][ac][gt]"]


def test_class_patterns_count_and_locate(gpu):
    """Character-class patterns through the multi-pattern kernels: counts of
    every (sequence, pattern) and the sorted positions of the sparse ones,
    bit-exact against the oracle's window compare, over sequences of several
    tiles with ragged ends, soft-masked runs and N blocks."""
    pairs = synth.class_pattern_pairs(9, 41)
    pats = CLASS_PATTERNS + [c.decode() for c, _ in pairs]
    texts = [synth.genome_text(n, 730 + i, mask_mean=80, n_gap_mean=40_000, n_run_mean=500)
             for i, n in enumerate((1_000_003, 262_147, 50_001, 5))]
    for i, t in enumerate(texts[:3]):
        for j, (c, exp) in enumerate(pairs):
            synth.plant(t, exp[j % 3], synth.uniform_ints(3, t.size - 8, 7300 + 10 * j + i))
    mt = gpu.MultiTable(pats, classes=True)
    assert mt.lengths == [len(oracle.class_sets(p)) for p in pats]
    import torch
    counts = torch.zeros(len(texts) * len(pats), dtype=torch.int64, device="cuda")
    gpu.dfa_multi_count([_dev(t) for t in texts], mt, counts)
    want = oracle.multi_count_class(texts, pats)
    got = counts.cpu().numpy().astype(np.uint64).reshape(want.shape)
    assert np.array_equal(got, want), np.argwhere(got != want)[:5]
    assert (want[:3, len(CLASS_PATTERNS):] > 0).all()          # every planted class pattern found
    # N^64 counts every window of 64 bases (it multiplies the states of any
    # automaton it joins, so it has its own)
    m64 = gpu.MultiTable(["N" * 64, "nnnn"], classes=True)
    c64 = torch.zeros(len(texts) * 2, dtype=torch.int64, device="cuda")
    gpu.dfa_multi_count([_dev(t) for t in texts], m64, c64)
    w64 = oracle.multi_count_class(texts, ["N" * 64, "nnnn"])
    assert np.array_equal(c64.cpu().numpy().astype(np.uint64).reshape(w64.shape), w64)
    assert w64[0, 0] > 0 and w64[3, 0] == 0
    # positions of the patterns with at most DFA_LOCATE_MAX occurrences
    t = texts[0]
    sparse = [p for p, c in zip(pats, want[0]) if 0 < c <= gpu.DFA_LOCATE_MAX]
    assert len(sparse) >= 15
    ms = gpu.MultiTable(sparse, classes=True)
    c0 = [int(oracle.find_class_brute(t, p)[0]) for p in sparse]
    pos = torch.empty(sum(c0), dtype=torch.int64, device="cuda")
    work = torch.empty(gpu.dfa_multi_locate_work_bytes(len(sparse)), dtype=torch.uint8, device="cuda")
    gpu.dfa_multi_locate(_dev(t), ms, c0, pos, work)
    assert gpu.dfa_multi_locate_status(work, len(sparse)) == gpu.DFA_OK
    h, o = pos.cpu().numpy(), 0
    for p, c in zip(sparse, c0):
        assert np.array_equal(h[o:o + c], oracle.find_class_brute(t, p)[1]), p
        o += c


def test_multi_count_convenience_with_classes(gpu):
    t = synth.genome_text(300_007, 745)
    pats = ["R[AC]NT", "gattaca", "W" * 6]
    got = gpu.multi_count([_dev(t)], pats, classes=True)
    assert np.array_equal(got, oracle.multi_count_class([t], pats))


def test_class_automaton_counts_the_sum_of_its_expansions(gpu):
    """A class pattern counts what its plain expansions count together, on a
    full-tile text: the class automaton against the single-pattern kernels."""
    import torch
    t = synth.genome_text(20_000_017, 740)
    td = _dev(t)
    for c, exp in synth.class_pattern_pairs(4, 42):
        mt = gpu.MultiTable([c], classes=True)
        out = torch.zeros(1, dtype=torch.int64, device="cuda")
        gpu.dfa_multi_count([td], mt, out)
        assert int(out.item()) == sum(gpu.count(td, e) for e in exp), c


@pytest.mark.parametrize("layout", [1, 2, 3, 4, 5])
def test_table_layouts_agree(gpu, layout):
    """The table as one shared copy (layout 1), as 32 per-lane copies
    (layout 2, conflict-free lookups) and as one copy with 2, 4 or 8 counter
    copies a state (layouts 3-5, 512 and 1024 threads) count the same,
    bit-exact against the oracle, for plain and class automata and every
    block size the layout takes."""
    import torch
    texts = [synth.genome_text(n, 760 + i, mask_mean=60, n_gap_mean=30_000, n_run_mean=300)
             for i, n in enumerate((2_000_003, 333_331, 17))]
    sets = [([p.encode() for p in PATTERN_SETS[3]], False),
            ([c.decode() for c, _ in synth.class_pattern_pairs(9, 44)], True),
            (["R", "[AC]A", "NN", "gaWtaca", "ACGTRYSWKMBDHVN"], True)]
    for pats, cls in sets:
        mt = gpu.MultiTable(pats, classes=cls)
        want = oracle.multi_count_class(texts, pats) if cls else oracle.multi_count(texts, pats)
        for threads in (128, 256, 512, 1024) if layout < 3 else (512, 1024):
            out = torch.zeros(len(texts) * len(pats), dtype=torch.int64, device="cuda")
            gpu.dfa_multi_count([_dev(t) for t in texts], mt, out,
                                cfg=dict(layout=layout, threads=threads, chunk=256))
            got = out.cpu().numpy().astype(np.uint64).reshape(want.shape)
            assert np.array_equal(got, want), (pats[:2], threads, np.argwhere(got != want)[:3])


def test_per_lane_copies_refused_when_too_large(gpu):
    import torch
    mt = gpu.MultiTable(["".join(x) for x in itertools.product("ACGT", repeat=6)])   # 5461 states
    out = torch.zeros(4096, dtype=torch.int64, device="cuda")
    with pytest.raises(gpu.DfaError):
        gpu.dfa_multi_count([_dev(synth.genome_text(10_000, 3))], mt, out, cfg=dict(layout=2))
    gpu.dfa_multi_count([_dev(synth.genome_text(10_000, 3))], mt, out, cfg=dict(layout=1))
    assert int(out.sum().item()) == oracle.valid_windows(synth.genome_text(10_000, 3), 6)
    # counter copies: 8 a state beside this table fit one CTA of 1024 threads;
    # at 256 threads the kernel has none
    gpu.dfa_multi_count([_dev(synth.genome_text(10_000, 3))], mt, out, cfg=dict(layout=5, threads=1024))
    assert int(out.sum().item()) == oracle.valid_windows(synth.genome_text(10_000, 3), 6)
    with pytest.raises(gpu.DfaError):
        gpu.dfa_multi_count([_dev(synth.genome_text(10_000, 3))], mt, out, cfg=dict(layout=3, threads=256))
