"""The multi-pattern automaton built on the host through the C ABI
(dfa_multi_build_host, no device needed), state by state against the
oracle's failure-less automaton (Sec. III-B, the corrected Table I), plus
the host-side size queries and limits."""
import pytest

import oracle
import synth

CODE = {"A": 0, "C": 1, "T": 2, "G": 3}      # (c >> 1) & 3


def _walk(nxt, s):
    q = 0
    for ch in s:
        q = nxt[q, CODE[ch]]
    return q


@pytest.mark.parametrize("pats", [
    ["ACG", "ACT", "CTA", "TGA"],                         # Table I's caption
    ["acg", "ACT", "cta"],                                # Table I's printed states, mixed case
    ["A", "AA", "AAA", "AAAA"],
    ["GATTACA", "ATTA", "TTAC", "TA", "CAGATTACA", "GATTACA"],
    None,
])
def test_host_automaton_matches_oracle(pats):
    import paper_1506_08612_gb300 as dd
    if pats is None:
        pats = [synth.pattern(int(m), 90 + i).decode()
                for i, m in enumerate(synth.uniform_ints(60, 20, 9) + 1)]
    t = dd.MultiTable(pats, device=False)
    nxt, nout = t.export()
    stt, _, names = oracle.stt_ascii(pats)
    idx = {nm: q for q, nm in enumerate(names)}
    up = [p.upper() for p in pats]
    prefixes = {p[:k] for p in up for k in range(len(p) + 1)}
    assert t.states() == len(prefixes) == len(names)
    for w in prefixes:
        q = _walk(nxt, w)
        for ch in "ACGT":
            assert nxt[q, CODE[ch]] == _walk(nxt, names[stt[idx[w], ord(ch)]]), (w, ch)
        assert nout[q] == sum(1 for p in up if w.endswith(p)), w
    # the device image: transitions, offsets, ids, lengths, spans, 16-byte parts
    assert t.image_bytes() % 16 == 0 and t.image_bytes() >= t.states() * 8
    assert t.smem_bytes() == ((t.states() * 8 + 15) // 16) * 16 + 4 * t.states()


def test_host_limits_and_sizes():
    import paper_1506_08612_gb300 as dd
    with pytest.raises(dd.DfaError):
        dd.MultiTable(["ACGN"], device=False)              # not a base
    with pytest.raises(dd.DfaError):
        dd.MultiTable(["A" * 65], device=False)            # longer than DFA_MAX_M
    many = [synth.pattern(64, 7000 + i) for i in range(300)]   # more than 16383 trie states
    with pytest.raises(dd.DfaError):
        dd.MultiTable(many, device=False)
    assert dd._lib.dfa_table_bytes(0) == -1 and dd._lib.dfa_table_bytes(65) == -1
    assert dd._lib.dfa_table_bytes(4) == 5 * 512 + 32 + 2 * 5 * 256 + (8 + 5) * 256
    assert dd.dfa_multi_locate_work_bytes(3) == 3 * 16 + 16 + 16
    assert dd.dfa_multi_locate_work_bytes(0) == -1
    # a table not attached to device memory is refused by the device calls
    t = dd.MultiTable(["ACGT"], device=False)
    assert dd._lib.dfa_multi_attach(t.handle, None, 1 << 20, None) == dd.DFA_EINVAL


def patterns_with_trie_states(states: int, seed: int):
    """Patterns (length <= 64) whose trie has exactly ``states`` states, the
    root included: random 64-mers while they fit, then one pattern that
    leaves an existing one after a shared prefix to add the remainder."""
    from paper_1506_08612_gb300.batched import new_prefixes
    seen, pats, i = {b""}, [], 0
    while True:
        p = synth.pattern(64, seed + i)
        i += 1
        add = new_prefixes(seen, p)
        if len(seen) + len(add) > states:
            break
        pats.append(p)
        seen.update(add)
    r = states - len(seen)
    if r:
        base = pats[-1]
        k = 64 - r                                  # shared prefix; base[k] is replaced
        alt = next(c for c in b"ACGT" if c != base[k])
        p = base[:k] + bytes([alt]) + base[k + 1:]
        assert len(new_prefixes(seen, p)) == r
        pats.append(p)
        seen.update(new_prefixes(seen, p))
    assert len(seen) == states
    return pats


def test_state_limit_is_exact():
    """16384 states (numbers 0..16383, 4 * 16383 + 1 < 2^16) build; one more
    state is refused, and the batch grouping agrees with the library."""
    import paper_1506_08612_gb300 as dd
    from paper_1506_08612_gb300.batched import MAX_STATES, group_patterns
    assert MAX_STATES == 16384
    full = patterns_with_trie_states(16384, 71_000)
    t = dd.MultiTable(full, device=False)
    assert t.states() == 16384 and len(group_patterns(full)) == 1
    over = patterns_with_trie_states(16385, 71_000)
    with pytest.raises(dd.DfaError, match="16384 states"):
        dd.MultiTable(over, device=False)
    assert len(group_patterns(over)) == 2


# ------------------------------------------------------------ class patterns

def _host_walk_total(nxt, nout, text) -> int:
    """Occurrences of all the automaton's patterns in ``text``, walked
    byte by byte on the host: a base takes its code's transition and adds
    the state's output count, any other byte goes back to the root."""
    q, c = 0, 0
    for b in bytes(text):
        if b in b"ACGTacgt":
            q = nxt[q, (b >> 1) & 3]
            c += int(nout[q])
        else:
            q = 0
    return c


@pytest.mark.parametrize("seed", range(4))
def test_class_builder_on_plain_patterns_is_the_trie_automaton(seed):
    """For patterns of single bases the subset construction finds the trie's
    states in the trie's breadth-first order: equal tables and sizes."""
    import paper_1506_08612_gb300 as dd
    pats = [synth.pattern(int(m), 3000 * seed + i) for i, m in enumerate(synth.uniform_ints(150, 24, seed) + 1)]
    pats[:4] = [b"ACG", b"ACT", b"CTA", b"acg"]
    a = dd.MultiTable(pats, device=False)
    b = dd.MultiTable(pats, device=False, classes=True)
    assert a.states() == b.states() and a.image_bytes() == b.image_bytes()
    for x, y in zip(a.export(), b.export()):
        assert (x == y).all()
    assert b.lengths == [len(p) for p in pats]


def test_class_automaton_walk_equals_oracle():
    """Each class pattern's automaton, walked on the host, counts what the
    oracle's window compare finds; the automaton of all of them together
    counts the sum."""
    import numpy as np

    import paper_1506_08612_gb300 as dd
    rng = np.random.default_rng(5)
    syms = list("ACGTRYSWKMBDHVN")
    pats = []
    for i in range(24):
        m = int(rng.integers(1, 9))
        pats.append("".join(str(rng.choice(syms)) if rng.random() < 0.6
                            else "[" + "".join(rng.choice(list("ACGT"), size=2)) + "]" for _ in range(m)))
    pats[:3] = ["R", "[AC]A", "nNn"]
    texts = [synth.random_text(3000, 70 + k, b"ACGTacgtNn") for k in range(3)]
    for p in pats:
        t = dd.MultiTable([p], device=False, classes=True)
        assert t.lengths == [len(oracle.class_sets(p))]
        nxt, nout = t.export()
        for tx in texts:
            assert _host_walk_total(nxt, nout, tx) == oracle.find_class_brute(tx, p)[0], p
    allt = dd.MultiTable(pats, device=False, classes=True)
    nxt, nout = allt.export()
    for tx in texts:
        assert _host_walk_total(nxt, nout, tx) == sum(oracle.find_class_brute(tx, p)[0] for p in pats)


def test_class_builder_limits_and_syntax():
    import paper_1506_08612_gb300 as dd
    for bad in ["", "[", "[]", "[AX]", "AZ", "A]", "[A[C]]", "N" * 65, "U",
                "()", "(c|)", "(|c)", "(cg)", "(c|g", "(c|gt)", "(c||g)"]:
        with pytest.raises(dd.DfaError):
            dd.MultiTable([bad], device=False, classes=True)
    # remembering where each of the last 16 A's was takes more than 16384 states
    with pytest.raises(dd.DfaError, match="16384 states"):
        dd.MultiTable(["A" + "N" * 16 + "T"], device=False, classes=True)
    # N^64 alone: the root and one state per number of bases read, 1..64
    assert dd.MultiTable(["N" * 64], device=False, classes=True).states() == 65
    # with [acgt] and RY: after k >= 2 bases the last one is a purine (RY cannot
    # have just ended), or a pyrimidine after a purine (it has), or after a
    # pyrimidine; after one base, purine or not: 1 + 2 + 63 * 3 states
    t = dd.MultiTable(["N" * 64, "[acgt]", "ry"], device=False, classes=True)
    assert t.lengths == [64, 1, 2] and t.mmax == 64
    assert t.states() == 1 + 2 + 63 * 3


def test_group_notation_builds_the_bracket_automaton():
    """The paper's group notation, (a|g|y) say, and the bracket [AGY] give the
    same automaton."""
    import paper_1506_08612_gb300 as dd
    for g, br in [(["(a|g|y)AC", "GG(a|c)T(r|y)"], ["[AGY]AC", "GG[AC]T[RY]"]),
                  (["(n)(a|t)"], ["N[AT]"])]:
        a = dd.MultiTable(g, device=False, classes=True)
        b = dd.MultiTable(br, device=False, classes=True)
        assert a.states() == b.states() and a.lengths == b.lengths
        for x, y in zip(a.export(), b.export()):
            assert (x == y).all()


def test_class_automaton_exhaustive_tiny_texts():
    """Every text of length <= 6 over {A, C, G, T, N, a}: the class
    automaton's host walk counts what the oracle's window compare finds, per
    pattern and for the patterns together."""
    import itertools

    import paper_1506_08612_gb300 as dd
    pats = ["R", "(a|c)A", "NN", "[AG]Y", "WaS", "ANT", "(r|y)(r|y)(r|y)"]
    singles = []
    for p in pats:
        singles.append(dd.MultiTable([p], device=False, classes=True).export())
    together = dd.MultiTable(pats, device=False, classes=True).export()
    for L in range(0, 7):
        for tup in itertools.product(b"ACGTNa", repeat=L):
            t = bytes(tup)
            want = [oracle.find_class_brute(t, p)[0] for p in pats]
            for (nxt, nout), w in zip(singles, want):
                assert _host_walk_total(nxt, nout, t) == w, (t, w)
            assert _host_walk_total(*together, t) == sum(want)
