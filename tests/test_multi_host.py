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
