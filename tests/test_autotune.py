"""Host logic of the autotuner and of the batched launch (no GPU): cache
keys, candidate grids within the kernels' documented limits, selection with
a fake timer, the JSON cache round trip, the forced configuration, and the
split of large pattern sets into automata that fit."""
import json

import pytest

from paper_1506_08612_gb300 import autotune
from paper_1506_08612_gb300.batched import MAX_STATES, group_patterns


@pytest.fixture
def cache(tmp_path, monkeypatch):
    p = tmp_path / "sub" / "tune.json"
    monkeypatch.setenv("DNADFA_AUTOTUNE_CACHE", str(p))
    monkeypatch.delenv("DNADFA_CONFIG", raising=False)
    autotune.reset_memory_cache()
    yield p
    autotune.reset_memory_cache()


def test_keys_bucket_sizes():
    a = autotune.single_key("GB300x152", 3_200_000_000, 8)
    b = autotune.single_key("GB300x152", 3_000_000_000, 8)
    c = autotune.single_key("GB300x152", 1_000_000_000, 8)
    assert a == b != c
    assert autotune.single_key("GB300x152", 3_200_000_000, 9) != a
    k1 = autotune.multi_key("d", 11_900_000_000, 256, 64, 8000)
    k2 = autotune.multi_key("d", 11_900_000_000, 300, 60, 8100)
    k3 = autotune.multi_key("d", 11_900_000_000, 4096, 6, 5461)
    assert k1 == k2 != k3


def test_candidates_respect_kernel_limits():
    for mmax in (1, 6, 8, 33, 64):
        cands = autotune.multi_candidates(mmax)
        assert cands
        for c in cands:
            assert c["threads"] in (128, 256, 512, 1024)
            assert c["chunk"] % 16 == 0 and 16 <= c["chunk"] <= 32768
            assert c["chunk"] >= 4 * (mmax - 1)       # overlap at most a quarter of a chunk
            # counter copies only where the kernel has them
            assert c["layout"] < 3 or c["threads"] in (512, 1024)
        # every table layout of the multi-pattern count is timed
        assert {c["layout"] for c in cands} == {1, 2, 3, 4, 5}
        one = {(c["threads"], c["chunk"]) for c in cands if c["layout"] == 1}
        assert one == {(c["threads"], c["chunk"]) for c in cands if c["layout"] == 2}
        assert {(c["threads"], c["chunk"]) for c in cands if c["layout"] == 5} == \
            {(t, ch) for t, ch in one if t in (512, 1024)}
    for m in (4, 7, 8, 64):
        lays = set()
        for c in autotune.single_candidates(m):
            assert c["loader"] == 2
            ch = c.get("chunk", 0)
            assert ch == 0 or (ch % 64 == 0 and 128 <= ch <= 64 * 63)
            assert c["layout"] in (0, 1, 3, 4)
            assert not (c["layout"] in (3, 4) and m < 8)
            lays.add(c["layout"])
        assert lays == ({0, 1} if m < 8 else {0, 1, 3, 4})


def test_select_best_with_fake_timer():
    calls = []

    def timer(cfg):
        calls.append(cfg["chunk"])
        if cfg["chunk"] == 512:
            raise ValueError("rejected by the kernel")
        return {256: 3.0, 1024: 1.0, 2048: 2.0}[cfg["chunk"]]

    cands = [{"chunk": c} for c in (256, 512, 1024, 2048)]
    best, ms = autotune.select_best(cands, timer, reps=3)
    assert best == {"chunk": 1024} and ms == 1.0
    assert calls.count(1024) == 4                       # one warm-up + three timed
    with pytest.raises(ValueError):
        autotune.select_best([{"chunk": 512}], timer)


def test_select_best_uses_the_median():
    seq = iter([9.0, 1.0, 50.0, 2.0,       # a: warm-up, then 1, 50, 2 -> median 2
                9.0, 3.0, 3.0, 3.0])       # b: median 3
    best, ms = autotune.select_best([{"x": "a"}, {"x": "b"}], lambda c: next(seq), reps=3)
    assert best == {"x": "a"} and ms == 2.0


def test_cache_round_trip(cache):
    k = autotune.multi_key("dev", 1 << 30, 256, 64, 8000)
    assert autotune.lookup(k) is None
    autotune.remember(k, {"threads": 256, "chunk": 1024}, 1.25, 12)
    assert autotune.lookup(k) == {"threads": 256, "chunk": 1024}
    autotune.reset_memory_cache()                      # re-read from the file
    assert autotune.lookup(k) == {"threads": 256, "chunk": 1024}
    d = json.loads(cache.read_text())
    assert d[k]["ms"] == 1.25 and d[k]["candidates"] == 12


def test_corrupt_cache_is_ignored(cache):
    cache.parent.mkdir(parents=True, exist_ok=True)
    cache.write_text("{not json")
    assert autotune.lookup("x") is None
    autotune.remember("x", {"chunk": 64}, 1.0, 1)
    assert json.loads(cache.read_text())["x"]["cfg"] == {"chunk": 64}


def test_keys_carry_the_kernel_version_and_operation():
    k = autotune.multi_key("d", 1 << 30, 256, 64, 8000)
    assert autotune.KERNEL_VERSION in k
    assert autotune.single_key("d", 1 << 30, 8, "find") != autotune.single_key("d", 1 << 30, 8, "count")


def test_forced_single_pattern_fields_do_not_reach_the_multi_count(monkeypatch):
    # a single-pattern layout (3, 4) or loader forced for every call must not
    # make the multi-pattern count refuse its launches
    monkeypatch.setenv("DNADFA_CONFIG", '{"layout": 4, "loader": 2, "chunk": 768}')
    assert autotune.forced_config() == {"layout": 4, "loader": 2, "chunk": 768}
    assert autotune.forced_config("multi") == {"chunk": 768}
    monkeypatch.setenv("DNADFA_CONFIG", '{"layout": 2, "threads": 256}')
    assert autotune.forced_config("multi") == {"layout": 2, "threads": 256}
    # the multi-pattern count's own layouts (counter copies) under their own key
    monkeypatch.setenv("DNADFA_CONFIG", '{"layout": 4, "multi_layout": 5, "threads": 1024}')
    assert autotune.forced_config("multi") == {"layout": 5, "threads": 1024}
    assert autotune.forced_config() == {"layout": 4, "threads": 1024}


def test_forced_config(monkeypatch):
    monkeypatch.setenv("DNADFA_CONFIG", '{"threads": 128, "chunk": 512}')
    assert autotune.forced_config() == {"threads": 128, "chunk": 512}
    monkeypatch.setenv("DNADFA_CONFIG", '{"bogus": 1}')
    with pytest.raises(ValueError):
        autotune.forced_config()
    monkeypatch.delenv("DNADFA_CONFIG")
    assert autotune.forced_config() is None


def _trie_states(pats):
    bs = [p.encode() if isinstance(p, str) else bytes(p) for p in pats]
    return len({p.upper()[:k] for p in bs for k in range(len(p) + 1)})


def test_group_patterns_fits_the_automaton_limits():
    import itertools
    import synth
    pats = [synth.pattern(64, 50 + i) for i in range(300)] + [b"ACGT"] * 10
    groups = group_patterns(pats)
    assert [i for g in groups for i in g] == list(range(len(pats)))
    for g in groups:
        assert _trie_states([pats[i] for i in g]) <= MAX_STATES
    assert len(groups) == 2
    assert group_patterns([b"ACG"] * 5, max_pat=2) == [[0, 1], [2, 3], [4]]
    # shared prefixes cost nothing: 300 copies of one pattern, one group;
    # all 4096 6-mers share their prefixes (5461 states), one group
    assert group_patterns([b"A" * 64] * 300) == [list(range(300))]
    kmers = ["".join(x) for x in itertools.product("ACGT", repeat=6)]
    assert group_patterns(kmers) == [list(range(4096))]
    assert _trie_states(kmers) == 5461
    assert group_patterns(["acgt", "ACGA"], max_states=6) == [[0, 1]]      # case folded
    assert group_patterns(["acgt", "ACGA"], max_states=5) == [[0], [1]]


def test_select_best_stops_at_a_device_error():
    """A rejected configuration is skipped; a CUDA error is not retried with
    the remaining candidates."""
    import paper_1506_08612_gb300 as dd
    seen = []

    def timer(cfg):
        seen.append(cfg["x"])
        if cfg["x"] == "einval":
            raise dd.DfaError(dd.DFA_EINVAL, "dfa_count")
        if cfg["x"] == "cuda":
            raise dd.DfaError(dd.DFA_ECUDA, "dfa_count")
        return 1.0

    best, _ = autotune.select_best([{"x": "einval"}, {"x": "ok"}], timer, reps=1)
    assert best == {"x": "ok"}
    seen.clear()
    with pytest.raises(dd.DfaError) as ei:
        autotune.select_best([{"x": "cuda"}, {"x": "ok"}], timer, reps=1)
    assert ei.value.code == dd.DFA_ECUDA and seen == ["cuda"]
    with pytest.raises(RuntimeError):
        autotune.select_best([{"x": "ok2"}], lambda c: (_ for _ in ()).throw(RuntimeError("CUDA error")))
