"""Pins of the CPU oracle to facts outside itself (no GPU).

Each group below checks the oracle against something the paper or the
mathematics fixes — printed values, closed forms, textbook algorithms,
library routines, invariants — chosen so that a dropped term, an off-by-one
or a transposed operand in ``oracle.c`` fails at least one of them.
"""
import itertools
import os
import re

import numpy as np
import pytest

import oracle
import synth
from conftest import GOLDEN

BASES = b"ACGT"


def _golden_lines(name):
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                yield line


# --------------------------------------------------------------------------
# fixed facts of the problem statement (Sec. II-A)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("line", list(_golden_lines("fixed_facts.txt")))
def test_fixed_facts(line):
    text, pat, cnt, pos = line.split()
    expect = [] if pos == "-" else [int(x) for x in pos.split(",")]
    c, p = oracle.find_brute(text.encode(), pat.encode())
    assert c == int(cnt) and list(p) == expect
    d = oracle.dfa_delta(pat.encode())
    c2, p2 = oracle.dfa_scan(text.encode(), d, len(pat))
    assert c2 == int(cnt) and list(p2) == expect


# --------------------------------------------------------------------------
# closed forms
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n,m", [(1, 1), (6, 4), (100, 1), (100, 7), (1000, 64), (63, 64)])
def test_homopolymer_closed_form(n, m):
    c, p = oracle.find_brute(b"A" * n, b"A" * m)
    assert c == max(0, n - m + 1)
    assert list(p) == list(range(max(0, n - m + 1)))


@pytest.mark.parametrize("pat,r", [(b"AAAC", 10), (b"ACGT", 7), (b"GATTACA", 5), (b"C", 9)])
def test_border_free_repeat(pat, r):
    # a pattern with no proper border occurs in P^r exactly at the multiples of m
    c, p = oracle.find_brute(pat * r, pat)
    assert c == r and list(p) == [i * len(pat) for i in range(r)]


@pytest.mark.parametrize("k,r", [(1, 10), (2, 10), (3, 4), (5, 5)])
def test_periodic_repeat(k, r):
    # (AC)^k inside (AC)^r occurs at every even offset 0, 2, .., 2(r-k)
    c, p = oracle.find_brute(b"AC" * r, b"AC" * k)
    assert c == r - k + 1 and list(p) == list(range(0, 2 * (r - k) + 1, 2))


def test_no_bases_no_matches():
    for t in (b"N" * 50, b"n" * 50, b"\n" * 9, bytes(range(256)) * 2):
        for pat in (b"A", b"T", b"ACGT", b"AAA"):
            # only the 8 base bytes can match; bytes(range(256)) holds each of
            # A and a twice per copy and no run of two bases
            want = t.upper().count(pat) if len(pat) == 1 else 0
            assert oracle.count_brute(t, pat) == want


def test_empty_and_short_texts():
    assert oracle.find_brute(b"", b"A")[0] == 0
    assert oracle.find_brute(b"ACG", b"ACGT")[0] == 0
    assert oracle.find_brute(b"ACGT", b"ACGT")[0] == 1


def test_invalid_patterns_rejected():
    for bad in (b"", b"ACGN", b"AC-T", b"\x00"):
        with pytest.raises(oracle.OracleError):
            oracle.find_brute(b"ACGT", bad)


def test_expected_count_uniform_text():
    # E[count] of a fixed non-self-overlapping 6-mer in uniform text is
    # (n - 5) / 4^6, variance ~ the mean; allow 6 standard deviations.
    n = 4_000_000
    t = synth.uniform_text(n, seed=123)
    for pat in (b"ACGTTG", b"GATTAC"):
        mu = (n - 5) / 4096
        assert abs(oracle.count_brute(t, pat) - mu) < 6 * mu ** 0.5


# --------------------------------------------------------------------------
# agreement with a library routine: the regex engine (overlapping look-ahead)
# --------------------------------------------------------------------------

def _regex_find(text: bytes, pat: bytes):
    folded = bytes(text).upper()            # ASCII-only upper-casing
    return [mt.start() for mt in re.finditer(b"(?=" + re.escape(pat.upper()) + b")", folded)]


def test_exhaustive_tiny_texts_vs_regex():
    alphabet = b"ACGTNa"
    pats = [b"A", b"C", b"AA", b"AC", b"CA", b"AAA", b"ACA", b"TGT"]
    for L in range(0, 7):
        for tup in itertools.product(alphabet, repeat=L):
            t = bytes(tup)
            for pat in pats:
                c, p = oracle.find_brute(t, pat)
                r = _regex_find(t, pat)
                assert c == len(r) and list(p) == r, (t, pat)


def test_random_texts_vs_regex():
    for seed in range(20):
        t = synth.random_text(3000, seed, b"ACGTacgtNn\n")
        for m in range(1, 13):
            pat = synth.pattern(m, 1000 + seed * 13 + m)
            c, p = oracle.find_brute(t, pat)
            r = _regex_find(t.tobytes(), pat)
            assert c == len(r) and list(p) == r


# --------------------------------------------------------------------------
# the automaton: definitional table vs the Knuth-Morris-Pratt construction
# --------------------------------------------------------------------------

def _kmp_delta(pat: bytes) -> np.ndarray:
    """Automaton from the KMP prefix function (an independent construction):
    delta(q, a) = q+1 if q < m and P[q] = a, else delta(pi[q-1], a) (q > 0),
    else 0."""
    m = len(pat)
    pi = [0] * m
    k = 0
    for i in range(1, m):
        while k and pat[i] != pat[k]:
            k = pi[k - 1]
        if pat[i] == pat[k]:
            k += 1
        pi[i] = k
    d = np.zeros((m + 1, 4), dtype=np.int32)
    for q in range(m + 1):
        for b, a in enumerate(BASES):
            if q < m and pat[q] == a:
                d[q, b] = q + 1
            elif q == 0:
                d[q, b] = 0
            else:
                d[q, b] = d[pi[q - 1], b]
    return d


def test_delta_equals_kmp_exhaustive_m_le_6():
    for m in range(1, 7):
        for tup in itertools.product(BASES, repeat=m):
            pat = bytes(tup)
            assert np.array_equal(oracle.dfa_delta(pat), _kmp_delta(pat)), pat


def test_delta_equals_kmp_random_long():
    for m in (7, 13, 31, 32, 64, 100):
        for s in range(5):
            pat = synth.pattern(m, 77 + 7 * m + s)
            assert np.array_equal(oracle.dfa_delta(pat), _kmp_delta(pat))


def test_delta_structure():
    pat = b"GATTACA"
    d = oracle.dfa_delta(pat)
    m = len(pat)
    for q in range(m):                       # forward edges
        assert d[q, BASES.index(pat[q])] == q + 1
    assert (d <= np.arange(m + 1)[:, None] + 1).all()
    assert (d[0] == [1 if a == pat[0] else 0 for a in BASES]).all()
    hom = oracle.dfa_delta(b"AAAA")
    assert hom[4, 0] == 4 and (hom[:, 1:] == 0).all()
    assert oracle.dfa_delta(b"acgt").tolist() == oracle.dfa_delta(b"ACGT").tolist()


def test_dfa_scan_equals_brute_random():
    for seed in range(10):
        t = synth.genome_text(20000, seed, mask_mean=40, n_gap_mean=900, n_run_mean=60)
        for m in (1, 2, 3, 4, 5, 8, 12, 16):
            pat = synth.pattern(m, 5000 + seed * 31 + m)
            d = oracle.dfa_delta(pat)
            c1, p1 = oracle.find_brute(t, pat)
            c2, p2 = oracle.dfa_scan(t, d, m)
            assert c1 == c2 and np.array_equal(p1, p2)


# --------------------------------------------------------------------------
# Table I (Sec. III-B): the sparse ASCII STT layout and values
# --------------------------------------------------------------------------

def test_table_I_sparse_stt():
    lines = list(_golden_lines("table_I.txt"))
    cols = [int(x) for x in lines[0].split()[1:]]
    assert cols == [ord("A"), ord("C"), ord("G"), ord("T")]
    rows, corrections = {}, {}
    final_from = None
    for ln in lines[1:]:
        if ln.startswith("final_from"):
            final_from = int(ln.split()[1])
            continue
        head, _, fix = ln.partition("!")
        parts = head.split()
        q, name, vals = int(parts[0]), parts[1], [int(x) for x in parts[2:6]]
        rows[q] = ("" if name == "e" else name.upper(), vals)
        if fix.strip():
            col, change = fix.strip().split("=")
            printed, corrected = (int(x) for x in change.split("->"))
            corrections[(q, "ACGT".index(col))] = (printed, corrected)
    names_paper = {q: rows[q][0] for q in rows}
    stt, f, names = oracle.stt_ascii(["acg", "act", "cta", "t"], [True, True, True, False])
    assert sorted(names) == sorted(names_paper.values())
    assert names.index("ACG") >= f and f == final_from   # finals numbered last
    ours = {nm: q for q, nm in enumerate(names)}
    for q, (nm, vals) in rows.items():
        row = stt[ours[nm]]
        for j, c in enumerate(cols):
            want = vals[j]
            if (q, j) in corrections:
                printed, corrected = corrections[(q, j)]
                assert printed == want
                want = corrected
            assert names[row[c]] == names_paper[want], (nm, "ACGT"[j])
            assert row[c + 32] == row[c]                   # lower-case column
        others = [c for c in range(256) if c not in cols and c - 32 not in cols]
        assert (row[others] == 0).all()                    # every other column -> q0


def test_stt_single_pattern_matches_delta():
    for pat in (b"ACGT", b"AAAA", b"GATTACA", synth.pattern(20, 9)):
        stt, f, names = oracle.stt_ascii([pat])
        d = oracle.dfa_delta(pat)
        m = len(pat)
        assert f == m and len(names) == m + 1
        # single pattern: prefix numbering is the prefix length
        assert [len(nm) for nm in names] == list(range(m + 1))
        assert np.array_equal(stt[:, list(BASES)], d)


# --------------------------------------------------------------------------
# Algorithm 1 (Sec. III-A): decomposition with m-1 overlap
# --------------------------------------------------------------------------

def test_fig2b_lane_starts():
    for ln in _golden_lines("fig2b_lanes.txt"):
        n, p, v, ch, starts = ln.split()
        assert oracle.alg1_lane_starts(int(n), int(p), int(v), int(ch)) == \
            [int(x) for x in starts.split(",")]


@pytest.mark.parametrize("p,v", [(1, 1), (1, 4), (3, 1), (4, 4), (7, 3), (60, 16), (240, 16),
                                 (5000, 1), (2, 5000)])
def test_alg1_equals_brute(p, v):
    t = synth.genome_text(30011, 5, mask_mean=50, n_gap_mean=3000, n_run_mean=100)
    for m in (1, 2, 4, 8, 13, 16, 33, 64):
        pat = synth.pattern(m, 900 + m)
        c1, p1 = oracle.find_brute(t, pat)
        c2, p2, _ = oracle.alg1_scan(t, oracle.dfa_delta(pat), m, p, v)
        assert c1 == c2 and np.array_equal(p1, p2), (m, p, v)


def test_alg1_dense_matches_cross_every_border():
    t = b"A" * 4099
    for m in (1, 3, 4, 17):
        for p, v in ((1, 1), (4, 4), (16, 8), (1000, 3)):
            c, pos, _ = oracle.alg1_scan(t, oracle.dfa_delta(b"A" * m), m, p, v)
            assert c == 4099 - m + 1 and list(pos) == list(range(4099 - m + 1))


def test_alg1_overlap_cost():
    # each of the P non-empty pieces except the last re-scans m-1 bytes of
    # its successor: steps = n + (P - 1)(m - 1) when every piece ends at
    # least m - 1 bytes before n.
    n = 1 << 16
    t = synth.uniform_text(n, 3)
    for m, p, v in ((8, 4, 4), (64, 16, 16), (2, 240, 16), (33, 7, 3)):
        pat = synth.pattern(m, 4)
        _, _, steps = oracle.alg1_scan(t, oracle.dfa_delta(pat), m, p, v, want_positions=False)
        assert steps == n + (p * v - 1) * (m - 1)


# --------------------------------------------------------------------------
# metamorphic relations
# --------------------------------------------------------------------------

COMP = bytes.maketrans(b"ACGTacgt", b"TGCAtgca")


def _genome(seed, n=50000):
    return synth.genome_text(n, seed, mask_mean=30, n_gap_mean=5000, n_run_mean=200).tobytes()


@pytest.mark.parametrize("seed", range(4))
def test_metamorphic(seed):
    t = _genome(seed)
    n = len(t)
    flip = synth.uniform_ints(n, 2, seed, stream=3).astype(bool)
    arr = np.frombuffer(t, dtype=np.uint8).copy()
    letters = np.isin(arr, np.frombuffer(b"ACGTacgt", np.uint8))
    arr[flip & letters] ^= 0x20
    t_case = arr.tobytes()
    for m in (1, 3, 4, 6, 9):
        pat = synth.pattern(m, 300 + seed * 10 + m)
        c, p = oracle.find_brute(t, pat)
        # case of the text does not matter
        assert np.array_equal(oracle.find_brute(t_case, pat)[1], p)
        # complementing text and pattern keeps every occurrence
        assert np.array_equal(oracle.find_brute(t.translate(COMP), pat.translate(COMP))[1], p)
        # reversing text and pattern mirrors the positions
        cr, pr = oracle.find_brute(t[::-1], pat[::-1])
        assert cr == c and sorted(n - m - int(i) for i in pr) == list(p)
        # an N between two texts separates them
        half = n // 2
        c1, p1 = oracle.find_brute(t[:half], pat)
        c2, p2 = oracle.find_brute(t[half:], pat)
        cj, pj = oracle.find_brute(t[:half] + b"N" + t[half:], pat)
        assert cj == c1 + c2
        assert list(pj) == list(p1) + [int(x) + half + 1 for x in p2]


# --------------------------------------------------------------------------
# k-mer census
# --------------------------------------------------------------------------

def _de_bruijn(k: int) -> bytes:
    """Linear de Bruijn sequence B(4, k) (Fredricksen-Kessler-Maiorana
    construction): every k-mer over ACGT occurs exactly once."""
    a = [0] * (k + 1)
    seq = []

    def db(t, p):
        if t > k:
            if k % p == 0:
                seq.extend(a[1:p + 1])
        else:
            a[t] = a[t - p]
            db(t + 1, p)
            for j in range(a[t - p] + 1, 4):
                a[t] = j
                db(t + 1, t)
    db(1, 1)
    seq = seq + seq[: k - 1]
    return bytes(BASES[i] for i in seq)


@pytest.mark.parametrize("k", [1, 2, 3, 4, 6])
def test_census_de_bruijn(k):
    h = oracle.kmer_census(_de_bruijn(k), k)
    assert (h == 1).all()


def test_census_invariants():
    t = _genome(11, 200000)
    for k in (1, 2, 4, 6):
        h = oracle.kmer_census(t, k)
        assert int(h.sum()) == oracle.valid_windows(t, k)
    h6 = oracle.kmer_census(t, 6)
    for s in range(30):
        pat = synth.pattern(6, 40 + s)
        code = 0
        for ch in pat:
            code = code * 4 + BASES.index(ch)
        assert int(h6[code]) == oracle.count_brute(t, pat)


def test_valid_windows_closed_form():
    # runs of bases of lengths L_i separated by N: sum max(0, L_i - k + 1)
    runs = [0, 1, 5, 6, 7, 100, 3]
    t = b"N".join(b"A" * L for L in runs)
    for k in (1, 3, 6, 7):
        assert oracle.valid_windows(t, k) == sum(max(0, L - k + 1) for L in runs)


# --------------------------------------------------------------------------
# planted occurrences of long patterns
# --------------------------------------------------------------------------

def test_planted_long_patterns_found():
    n = 1 << 20
    t = synth.genome_text(n, 8)
    for m in (16, 32, 64):
        pat = synth.pattern(m, 50 + m)
        pos = np.unique(synth.uniform_ints(200, n - m, 60 + m) // (2 * m) * (2 * m))
        synth.plant(t, pat, pos)
        c, p = oracle.find_brute(t, pat)
        assert set(pos.tolist()) <= set(p.tolist())
        assert c == oracle.dfa_scan(t, oracle.dfa_delta(pat), m)[0]


def test_multi_count_equals_census_and_definition():
    # two separately written oracle routines agree: the per-pattern brute
    # force over all 4^k k-mers (lexicographic) and the census by codes
    import itertools
    t = synth.genome_text(60_000, 4, mask_mean=30, n_gap_mean=3000, n_run_mean=100)
    k = 4
    pats = ["".join(s) for s in itertools.product("ACGT", repeat=k)]
    mc = oracle.multi_count([t], pats)[0]
    assert np.array_equal(mc, oracle.kmer_census(t, k))
    assert int(mc.sum()) == oracle.valid_windows(t, k)
    # empty text, and a text per pattern set with nested patterns
    assert oracle.multi_count([np.zeros(0, np.uint8)], ["A"]).tolist() == [[0]]
    aa = np.frombuffer(b"AAAAAA", np.uint8).copy()
    assert oracle.multi_count([aa], ["A", "AA", "AAAA"]).tolist() == [[6, 5, 3]]


# --------------------------------------------------------------------------
# the definition for a set of patterns (trie descent per window start)
# --------------------------------------------------------------------------

SET_PATS = [b"A", b"C", b"AA", b"AC", b"CA", b"AAA", b"ACA", b"TGT", b"AC", b"ACAT"]


def test_find_set_exhaustive_tiny_texts_vs_regex():
    # every text of length <= 6 over {A,C,G,T,N,a}: each pattern of a set with
    # shared prefixes, nested patterns and a duplicate, against the regex
    # engine's overlapping look-ahead (a library routine)
    alphabet = b"ACGTNa"
    for L in range(0, 7):
        for tup in itertools.product(alphabet, repeat=L):
            t = bytes(tup)
            c, pos = oracle.find_set(t, SET_PATS, threads=1)
            for pat, cc, pp in zip(SET_PATS, c, pos):
                r = _regex_find(t, pat)
                assert int(cc) == len(r) and list(pp) == r, (t, pat)


@pytest.mark.parametrize("threads", [1, 3, 8])
def test_find_set_random_texts_vs_regex(threads):
    for seed in range(6):
        t = synth.random_text(4000, 300 + seed, b"ACGTacgtNn\n")
        pats = [synth.pattern(m, 2000 + seed * 17 + m) for m in range(1, 13)]
        pats += [pats[3][:2], pats[5], pats[7].lower()]       # a prefix, a duplicate, lower case
        c, pos = oracle.find_set(t, pats, threads=threads)
        for pat, cc, pp in zip(pats, c, pos):
            r = _regex_find(t.tobytes(), pat)
            assert int(cc) == len(r) and list(pp) == r, (seed, pat)


@pytest.mark.parametrize("k", [1, 2, 3, 5])
def test_find_set_de_bruijn_all_kmers_once(k):
    # B(4, k) holds every k-mer exactly once, at a position fixed by the
    # sequence; lower case matches too
    seq = _de_bruijn(k)
    pats = ["".join(x) for x in itertools.product("ACGT", repeat=k)]
    for text in (seq, seq.lower()):
        c, pos = oracle.find_set(text, pats, threads=4)
        assert (c == 1).all()
        assert [int(p[0]) for p in pos] == [text.upper().find(q.encode()) for q in pats]


def test_find_set_sum_is_valid_windows_and_homopolymer():
    # over all 4^k k-mers the counts add up to the windows of k bases
    # (computed from run lengths), and A, AA, ..., A^j on A^n give n - j + 1
    t = synth.genome_text(80_000, 9, mask_mean=30, n_gap_mean=3000, n_run_mean=100)
    for k in (2, 4):
        pats = ["".join(x) for x in itertools.product("ACGT", repeat=k)]
        c, _ = oracle.find_set(t, pats, positions=False, threads=5)
        assert int(c.sum()) == oracle.valid_windows(t, k)
    n = 40
    hp = b"A" * n
    c, pos = oracle.find_set(hp, [b"A" * j for j in range(1, 12)], threads=3)
    assert [int(x) for x in c] == [n - j + 1 for j in range(1, 12)]
    assert all(list(p) == list(range(n - j + 1)) for j, p in zip(range(1, 12), pos))
    assert oracle.find_set(b"", [b"A"])[0].tolist() == [0]
    with pytest.raises(oracle.OracleError):
        oracle.find_set(b"ACGT", [b"ACNT"])


# --------------------------------------------------------------------------
# character-class patterns (the class cells of Table III, Sec. IV)
# --------------------------------------------------------------------------

BASE_COMP = {"A": "T", "C": "G", "G": "C", "T": "A"}


def test_iupac_table_structure():
    """The IUPAC nucleotide codes by their structure: each base stands for
    itself; the six two-base codes are the six pairs of bases, each once;
    B, D, H, V are 'not A', 'not C', 'not G', 'not T'; N is any base; the
    chemical names fix the pairs (puRine A/G, pYrimidine C/T, Strong C/G,
    Weak A/T, Keto G/T, aMino A/C); complementing a code's set gives the set
    of its complementary code (R-Y, K-M, B-V, D-H; S, W, N map to
    themselves)."""
    T = oracle.IUPAC
    assert len(T) == 15
    for b in "ACGT":
        assert T[b] == b
    pairs = sorted(v for v in T.values() if len(v) == 2)
    assert pairs == sorted("".join(c) for c in itertools.combinations("ACGT", 2))
    for code, missing in zip("BDHV", "ACGT"):
        assert T[code] == "".join(sorted(set("ACGT") - {missing}))
    assert T["N"] == "ACGT"
    assert (T["R"], T["Y"], T["S"], T["W"], T["K"], T["M"]) == ("AG", "CT", "CG", "AT", "GT", "AC")
    comp_code = dict(zip("ACGTRYKMBVDHSWN", "TGCAYRMKVBHDSWN"))
    for k, v in T.items():
        assert "".join(sorted(BASE_COMP[b] for b in v)) == T[comp_code[k]], k


CLASS_FACTS = [
    ("ACGTNacgtn", "R", [0, 2, 5, 7]),
    ("AAACA", "[AC]A", [0, 1, 3]),
    ("ACgtNa", "N", [0, 1, 2, 3, 5]),
    ("ACNGT", "NN", [0, 3]),
    ("ACGT", "[ACGT][acgt]", [0, 1, 2]),
    ("GATTACA", "GAW", [0]),
    ("TTTT", "[AG]", []),
    ("ACG", "NNNN", []),
    ("aCgT", "mS", [0, 1]),
    ("CATTAG", "(c|t)A", [0, 3]),
    ("ACGTT", "(a|c)(g|c)(t|r)", [0, 1]),
]


@pytest.mark.parametrize("text,pat,pos", CLASS_FACTS)
def test_class_fixed_facts(text, pat, pos):
    c, p = oracle.find_class_brute(text.encode(), pat)
    assert c == len(pos) and list(p) == pos


def _class_regex(sets):
    return b"(?=" + b"".join(b"[" + s.encode() + s.lower().encode() + b"]" for s in sets) + b")"


def test_class_patterns_vs_regex_and_expansions():
    """Against Python's regular expressions (a character class per
    position, overlapping matches by look-ahead), and against the plain
    brute force: a class pattern's occurrences are the disjoint union of its
    expansions' occurrences (distinct strings of one length never start at
    the same position)."""
    rng = np.random.default_rng(11)
    syms = list("ACGTRYSWKMBDHVNacgtrn")
    for seed in range(12):
        t = synth.random_text(4000, 60 + seed, b"ACGTacgtNn")
        for _ in range(6):
            m = int(rng.integers(1, 7))
            pat = "".join(str(rng.choice(syms)) if rng.random() < 0.7
                          else "[" + "".join(rng.choice(list("ACGTR"), size=2)) + "]" for _ in range(m))
            c, p = oracle.find_class_brute(t, pat)
            r = [mt.start() for mt in re.finditer(_class_regex(oracle.class_sets(pat)), t.tobytes())]
            assert c == len(r) and list(p) == r, pat
            exp = oracle.class_expansions(pat)
            if len(exp) <= 256:
                assert sum(oracle.count_brute(t, e) for e in exp) == c, pat
                union = sorted(itertools.chain.from_iterable(oracle.find_brute(t, e)[1].tolist() for e in exp))
                assert union == list(p), pat


def test_single_base_classes_are_plain_patterns():
    for seed in range(6):
        t = synth.random_text(5000, 80 + seed, b"ACGTacgtN")
        for m in (1, 3, 8, 20):
            pat = synth.pattern(m, 800 + seed * 7 + m)
            mixed = "".join(ch if i % 2 else "[" + ch + "]" for i, ch in enumerate(pat.decode().lower()))
            c, p = oracle.find_class_brute(t, mixed)
            c2, p2 = oracle.find_brute(t, pat)
            assert c == c2 and np.array_equal(p, p2)


def test_groups_equal_brackets():
    """The paper's notation (a group of single symbols separated by |)
    allows the same bases as the bracket set of those symbols."""
    for g, br in [("(c|g|w)", "[CGW]"), ("(a|c)", "[AC]"), ("(r|y)", "[RY]"), ("(n)", "[N]"),
                  ("(a|A)", "[A]")]:
        assert oracle.class_sets(g + "TT" + g) == oracle.class_sets(br + "TT" + br)


@pytest.mark.parametrize("bad", ["", "[", "[]", "[AX]", "AZ", "A]", "[A[C]]", "N" * 65, "AC-GT", "U",
                                 "()", "(c|)", "(|c)", "(cg)", "(c|g", "(c|gt)", "(c||g)"])
def test_class_syntax_errors(bad):
    with pytest.raises(ValueError):
        oracle.class_sets(bad)
