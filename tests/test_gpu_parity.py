"""Parity of the CUDA scan (through the C ABI) with the CPU oracle.

Counts and positions are integers: the bar is bit-exact equality.
Every input is seeded and synthetic (``synth``).
"""
import os

import numpy as np
import pytest

import oracle
import synth
from conftest import GOLDEN

pytestmark = pytest.mark.gpu

CONFIGS = [
    None,
    # direct-load kernel (loader 1)
    dict(loader=1, layout=1, threads=128, chunk=16),
    dict(loader=1, layout=1, threads=256, chunk=48),
    dict(loader=1, layout=1, threads=512, chunk=256),
    dict(loader=1, layout=2, threads=256, chunk=64),
    dict(loader=1, layout=2, threads=128, chunk=1008),
    # TMA-staged persistent kernel (loader 2): chunk = 64 x stages per tile
    dict(loader=2, layout=1, chunk=128),
    dict(loader=2, layout=1, chunk=384),
    dict(loader=2, layout=2, chunk=192),
    dict(loader=2, layout=1, chunk=1280),
    # relaxed walks with exact replays (loader 2): states only (layout 3),
    # states with accept flags (layout 4; layout 3 beyond m = 31)
    dict(loader=2, layout=3, chunk=128),
    dict(loader=2, layout=3, chunk=1280),
    dict(loader=2, layout=4, chunk=128),
    dict(loader=2, layout=4, chunk=1280),
]


def _dev(gpu, arr):
    import torch
    return torch.from_numpy(np.ascontiguousarray(arr)).cuda()


def _find(gpu, text_dev, pat, cfg=None, cap=None):
    c, p = gpu.find(text_dev, pat, cap=cap, cfg=cfg)
    return c, p.cpu().numpy()


def _check(gpu, text_np, pat, cfg=None, text_dev=None):
    if text_dev is None:
        text_dev = _dev(gpu, text_np)
    want_c, want_p = oracle.find_brute(text_np, pat)
    c, p = _find(gpu, text_dev, pat, cfg)
    assert c == want_c, (len(pat), cfg, c, want_c)
    assert np.array_equal(p, want_p), (len(pat), cfg)
    assert gpu.count(text_dev, pat, cfg=cfg) == want_c
    return want_c


def _lines(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


def test_fixed_facts(gpu):
    for text, pat, cnt, pos in _lines("fixed_facts.txt"):
        t = np.frombuffer(text.encode(), dtype=np.uint8).copy()
        c, p = _find(gpu, _dev(gpu, t), pat.encode())
        assert c == int(cnt)
        assert list(p) == ([] if pos == "-" else [int(x) for x in pos.split(",")])


def test_export_stt_is_paper_table(gpu):
    for pat in (b"ACGT", b"AAAA", b"GATTACA", synth.pattern(64, 3)):
        stt, f, _ = oracle.stt_ascii([pat])
        t = gpu.dfa_build(pat)
        assert np.array_equal(gpu.dfa_export_stt(t).astype(np.int32), stt)
        assert f == len(pat)


@pytest.mark.parametrize("cfg", CONFIGS)
def test_random_genome_all_lengths(gpu, cfg):
    # several tiles plus a ragged tail under every configuration
    n = 300_007
    t = synth.genome_text(n, 21, mask_mean=60, n_gap_mean=20_000, n_run_mean=700)
    td = _dev(gpu, t)
    for m in list(range(1, 17)) + [31, 32, 33, 47, 63, 64]:
        _check(gpu, t, synth.pattern(m, 100 + m), cfg, td)


@pytest.mark.parametrize("cfg", CONFIGS[:4] + CONFIGS[6:])
def test_planted_long_patterns(gpu, cfg):
    n = 1 << 20
    t = synth.genome_text(n, 8)
    rng_pos = synth.uniform_ints(400, n - 64, 31)
    for m in (16, 32, 64):
        pat = synth.pattern(m, 40 + m)
        tt = t.copy()
        pos = np.unique(rng_pos // (2 * m) * (2 * m))
        synth.plant(tt, pat, pos)
        assert _check(gpu, tt, pat, cfg) >= len(pos)


@pytest.mark.parametrize("cfg,chunk", [(dict(loader=1, layout=1, threads=128, chunk=64), 64),
                                       (dict(loader=2, layout=1, chunk=128), 128),
                                       (dict(loader=2, layout=2, chunk=64 * 3), 192),
                                       (dict(loader=2, layout=3, chunk=128), 128),
                                       (dict(loader=2, layout=4, chunk=128), 128)])
def test_border_plants(gpu, cfg, chunk):
    # occurrences planted at +-m around every chunk / tile border
    n = 256 * chunk * 6 + 77
    for m in (5, 16, 33, 64):
        t = synth.genome_text(n, 3, n_gap_mean=0)
        pat = synth.pattern(m, 7 * m)
        borders = np.arange(0, n, chunk)
        pos = np.unique(np.clip(np.concatenate([borders - m + 1, borders - 1, borders,
                                                borders - m // 2]), 0, n - m))
        pos = pos[np.concatenate([[True], np.diff(pos) >= m])]  # keep them disjoint
        synth.plant(t, pat, pos)
        assert _check(gpu, t, pat, cfg) >= len(pos)


def test_edge_cases(gpu):
    import torch
    # empty text, shorter than the pattern, exactly the pattern
    empty = torch.empty(0, dtype=torch.uint8, device="cuda")
    assert gpu.find(empty, b"ACGT")[0] == 0 and gpu.count(empty, b"ACGT") == 0
    for n in range(0, 40):
        t = synth.uniform_text(n, n)
        for m in (1, 3, 8, 17):
            _check(gpu, t, synth.pattern(m, m + 5))
    _check(gpu, np.frombuffer(b"ACGT", np.uint8).copy(), b"ACGT")
    # no bases at all, every byte value
    _check(gpu, np.full(100_000, ord("N"), np.uint8), b"A")
    allbytes = np.tile(np.arange(256, dtype=np.uint8), 500)
    for pat in (b"A", b"C", b"T", b"G", b"AB"[:1]):
        _check(gpu, allbytes, pat)
    # lower case only
    _check(gpu, np.frombuffer(b"acgt" * 10000, np.uint8).copy(), b"GTAC")


def test_dense_matches_overflow_and_truncation(gpu):
    # every position matches: exercises the per-thread staging overflow path
    n = 200_003
    t = np.full(n, ord("A"), np.uint8)
    for cfg in (None, dict(loader=1, layout=1, threads=128, chunk=1024),
                dict(loader=1, layout=2, threads=256, chunk=512), dict(loader=2, chunk=128),
                dict(loader=2, layout=2, chunk=768), dict(loader=2, layout=3, chunk=256)):
        for m in (1, 4, 64):
            _check(gpu, t, b"A" * m, cfg)
    # cap smaller than the count: exact count, first cap positions, ETRUNC
    import torch
    td = _dev(gpu, t)
    tab = gpu.dfa_build(b"AAAA")
    cap = 1000
    pos = torch.full((cap,), -1, dtype=torch.int64, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    ws = torch.empty(gpu.dfa_find_workspace_bytes(n), dtype=torch.uint8, device="cuda")
    gpu.dfa_find(td, tab, pos, cnt, ws)
    rc, c = gpu.dfa_find_status(ws, cnt, cap)
    assert rc == gpu.DFA_ETRUNC and c == n - 3
    assert pos.cpu().numpy().tolist() == list(range(cap))


def test_misaligned_text(gpu):
    t = synth.genome_text(100_000, 5, mask_mean=50)
    td = _dev(gpu, t)
    for off in (1, 3, 8, 15):
        sub = t[off:]
        for m in (4, 8, 33):
            pat = synth.pattern(m, 60 + m + off)
            want_c, want_p = oracle.find_brute(sub, pat)
            c, p = _find(gpu, td[off:], pat)
            assert c == want_c and np.array_equal(p, want_p)


def test_config1_uniform_16MiB_m8(gpu):
    """The 16 MiB uniform text, m = 8, full positions."""
    n = 16 * 1024 * 1024
    t = synth.uniform_text(n, 0)
    pat = synth.pattern(8, 1)
    c = _check(gpu, t, pat)
    assert 100 < c < 500          # ~256 expected


def test_host_buffer_path(gpu):
    import torch
    n = 5_000_000
    t = synth.genome_text(n, 9)
    ht = torch.from_numpy(t).pin_memory()
    for m in (4, 8, 16):
        pat = synth.pattern(m, 90 + m)
        want_c, want_p = oracle.find_brute(t, pat)
        tab = gpu.dfa_build(pat)
        for seg in (1 << 20, (1 << 20) + 16 * 1000 + 7, 1 << 23):
            cap = want_c + 10
            hp = torch.zeros(cap, dtype=torch.int64)
            stage = torch.empty(gpu.dfa_host_stage_bytes(seg, cap), dtype=torch.uint8, device="cuda")
            rc, c = gpu.dfa_find_host(ht, tab, hp, stage, seg)
            assert rc == gpu.DFA_OK and c == want_c
            assert np.array_equal(hp[:c].numpy(), want_p)


def test_host_buffer_path_many_patterns(gpu):
    # one copy of each segment serves every pattern; occurrences of the long
    # patterns planted across segment borders, small caps truncate
    import torch
    n = 6_000_011
    t = synth.genome_text(n, 19)
    pats = [synth.pattern(m, 190 + m) for m in (4, 7, 8, 16, 33, 64)]
    for p in pats[3:]:
        at = [k * (1 << 20) - len(p) // 2 for k in range(1, 6)] + list(synth.uniform_ints(40, n - len(p), len(p)))
        synth.plant(t, p, at)
    ht = torch.from_numpy(t).pin_memory()
    want = [oracle.find_brute(t, p) for p in pats]
    tabs = [gpu.dfa_build(p) for p in pats]
    for seg in (1 << 20, (1 << 20) + 16 * 1000 + 7):
        caps = [c + 3 for c, _ in want]
        hps = [torch.full((c,), -1, dtype=torch.int64) for c in caps]
        stage = torch.empty(gpu.dfa_host_stage_bytes_multi(seg, caps), dtype=torch.uint8, device="cuda")
        rc, cs = gpu.dfa_find_host_multi(ht, tabs, hps, stage, seg)
        assert rc == gpu.DFA_OK
        for (wc, wp), c, hp in zip(want, cs, hps):
            assert c == wc and np.array_equal(hp[:c].numpy(), wp)
    # truncation: the counts stay exact, the first cap positions are valid
    caps = [max(c // 2, 1) for c, _ in want]
    hps = [torch.zeros(c, dtype=torch.int64) for c in caps]
    stage = torch.empty(gpu.dfa_host_stage_bytes_multi(1 << 20, caps), dtype=torch.uint8, device="cuda")
    rc, cs = gpu.dfa_find_host_multi(ht, tabs, hps, stage, 1 << 20)
    assert rc == gpu.DFA_ETRUNC
    for (wc, wp), c, hp, cap in zip(want, cs, hps, caps):
        assert c == wc and np.array_equal(hp.numpy()[:min(c, cap)], wp[:cap])


def test_find_batched(gpu):
    # several patterns over one device text through one call and one
    # workspace; one pattern's buffer is too small (truncated, count exact)
    import torch
    n = 2_000_003
    t = synth.genome_text(n, 29)
    pats = [synth.pattern(m, 290 + m) for m in (3, 4, 8, 16, 64)]
    for p in pats[3:]:
        synth.plant(t, p, synth.uniform_ints(25, n - len(p), len(p)))
    td = _dev(gpu, t)
    want = [oracle.find_brute(t, p) for p in pats]
    tabs = [gpu.dfa_build(p) for p in pats]
    caps = [c + 2 for c, _ in want]
    caps[1] = want[1][0] // 3
    pos = [torch.full((c,), -1, dtype=torch.int64, device="cuda") for c in caps]
    cnt = torch.zeros(len(pats), dtype=torch.int64, device="cuda")
    ws = torch.empty(gpu.dfa_find_workspace_bytes(n), dtype=torch.uint8, device="cuda")
    gpu.dfa_find_batched(td, tabs, pos, cnt, ws)
    got = cnt.cpu().numpy()
    for i, ((wc, wp), cap) in enumerate(zip(want, caps)):
        assert got[i] == wc, i
        k = min(wc, cap)
        assert np.array_equal(pos[i][:k].cpu().numpy(), wp[:k]), i


def test_tables_in_caller_memory(gpu):
    # dfa_build_into / dfa_multi_build_host + dfa_multi_attach: the tables
    # land in caller-owned device memory (copied on a stream) and give the
    # same results as the library-allocated ones
    import torch
    t = synth.genome_text(1_000_003, 33)
    td = _dev(gpu, t)
    s = torch.cuda.Stream()
    for m in (1, 4, 9, 31, 64):
        pat = synth.pattern(m, 330 + m)
        buf = torch.empty(gpu.dfa_table_bytes(m) + 256, dtype=torch.uint8, device="cuda")
        with torch.cuda.stream(s):
            tab = gpu.Table(pat, into=buf[256:], stream=s)
            cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
            gpu.dfa_count(td, tab, cnt, stream=s)
        s.synchronize()
        assert int(cnt.item()) == oracle.count_brute(t, pat), m
        tab.free()
    with pytest.raises(gpu.DfaError):
        gpu.Table(b"ACGT", into=torch.empty(16, dtype=torch.uint8, device="cuda"))       # too small
    pats = [synth.pattern(m, 340 + m) for m in (3, 5, 8, 12)]
    mt = gpu.MultiTable(pats, device=False)
    with pytest.raises(gpu.DfaError):
        gpu.dfa_multi_count([td], mt, torch.zeros(4, dtype=torch.int64, device="cuda"))  # not attached yet
    img = torch.empty(mt.image_bytes(), dtype=torch.uint8, device="cuda")
    mt.attach(img, stream=s)
    out = torch.zeros(len(pats), dtype=torch.int64, device="cuda")
    with torch.cuda.stream(s):
        gpu.dfa_multi_count([td], mt, out, stream=s)
    s.synchronize()
    assert np.array_equal(out.cpu().numpy().astype(np.uint64), oracle.multi_count([t], pats)[0])


def test_streams_and_concurrency(gpu):
    import torch
    t = synth.genome_text(2_000_000, 13)
    td = _dev(gpu, t)
    pats = [synth.pattern(m, 500 + m) for m in (4, 6, 8, 12)]
    want = [oracle.find_brute(t, p) for p in pats]
    streams = [torch.cuda.Stream() for _ in pats]
    outs = []
    for p, s in zip(pats, streams):
        with torch.cuda.stream(s):
            tab = gpu.dfa_build(p)
            cap = 200_000
            pos = torch.empty(cap, dtype=torch.int64, device="cuda")
            cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
            ws = torch.empty(gpu.dfa_find_workspace_bytes(td.numel()), dtype=torch.uint8, device="cuda")
            gpu.dfa_find(td, tab, pos, cnt, ws)
            outs.append((tab, pos, cnt, ws, s))
    for (tab, pos, cnt, ws, s), (wc, wp) in zip(outs, want):
        rc, c = gpu.dfa_find_status(ws, cnt, pos.numel(), stream=s)
        assert rc == gpu.DFA_OK and c == wc
        assert np.array_equal(pos[:c].cpu().numpy(), wp)


def _same_code_nonbases(code):
    """Bytes that are not bases but share a base's 2-bit code (c >> 1) & 3."""
    return [c for c in range(256) if (c >> 1) & 3 == code and c not in b"ACGTacgt"]


@pytest.mark.parametrize("cfg", [None, dict(loader=2, layout=3, chunk=128), dict(loader=2, layout=4, chunk=256),
                                 dict(loader=2, layout=1, chunk=128)])
def test_relaxed_walk_decoys(gpu, cfg):
    # copies of P with one byte swapped for a non-base of the same code: a walk
    # that reads codes only sees P there, the exact walk must not; placed
    # across every stage (64 B) and row border, plus true copies beside them
    chunk = 256 if cfg is None else cfg["chunk"]
    n = 512 * chunk * 3 + 4099
    for m in (8, 12, 19, 20, 31, 33, 64):
        t = synth.genome_text(n, 40 + m, n_gap_mean=0)
        pat = synth.pattern(m, 900 + m)
        codes = [(c >> 1) & 3 for c in pat]
        rnd = synth.uniform_ints(4 * (n // 64), 1 << 30, 70 + m)
        k = 0
        step = 64 * ((3 * m + 3 + 63) // 64)       # decoy and true copy never overwrite the next ones
        for b in range(64, n - 3 * m - 3, step):
            st = b - int(rnd[k] % (m + 1)) if b >= m + 1 else b
            k += 1
            if st < 0 or st + m > n:
                continue
            dec = bytearray(pat)
            j = int(rnd[k] % m); k += 1
            alts = _same_code_nonbases(codes[j])
            dec[j] = alts[int(rnd[k] % len(alts))]; k += 1
            if rnd[k] & 1:
                dec = bytearray(bytes(dec).lower())
            k += 1
            t[st:st + m] = np.frombuffer(bytes(dec), np.uint8)
            if (b // step) % 5 == 0:
                t[st + m + 3:st + 2 * m + 3] = np.frombuffer(pat, np.uint8)
        assert _check(gpu, t, pat, cfg) > 0


@pytest.mark.parametrize("cfg", [None, dict(loader=2, layout=1, chunk=128), dict(loader=2, layout=1, chunk=1280)])
def test_dense_relaxed_decoys(gpu, cfg):
    # short (dense) patterns walk by codes alone and test only the stages
    # that accepted: decoys (one byte swapped for a non-base of the same code)
    # ending in every stage and row, true copies right after a non-base that
    # sits in the 8 bytes before a stage, and non-bases in a row's last bytes
    # before its overlap
    chunk = 128 if cfg is None else cfg["chunk"]
    n = 512 * chunk * 3 + 4099
    for m in (1, 2, 3, 4, 5, 6):
        t = synth.genome_text(n, 140 + m, n_gap_mean=0)
        pat = synth.pattern(m, 1900 + m)
        codes = [(c >> 1) & 3 for c in pat]
        rnd = synth.uniform_ints(6 * (n // 64) + 10, 1 << 30, 170 + m)
        k = 0
        for b in range(64, n - 80, 64):
            kind = int(rnd[k] % 3); k += 1
            if kind == 0:                              # a decoy ending near the border
                st = b - int(rnd[k] % (m + 2)); k += 1
                dec = bytearray(pat)
                j = int(rnd[k] % m); k += 1
                alts = _same_code_nonbases(codes[j])
                dec[j] = alts[int(rnd[k] % len(alts))]; k += 1
                t[st:st + m] = np.frombuffer(bytes(dec), np.uint8)
            elif kind == 1:                            # a non-base shortly before a true copy
                d = 1 + int(rnd[k] % 8); k += 1
                t[b:b + m] = np.frombuffer(pat, np.uint8)
                t[b - d] = _same_code_nonbases(int(rnd[k] % 4))[0]; k += 1
            else:                                      # a true copy across the border
                st = b - int(rnd[k] % m) if m > 1 else b; k += 1
                t[st:st + m] = np.frombuffer(pat, np.uint8)
        assert _check(gpu, t, pat, cfg) > 0


@pytest.mark.parametrize("cfg", [None, dict(loader=2, layout=4, chunk=128), dict(loader=2, layout=4, chunk=1280),
                                 dict(loader=2, layout=3, chunk=640)])
def test_staged_find_borders(gpu, cfg):
    # the staged two-pass find records each row's exact accepts in its count
    # pass and copies them in the third: copies at row starts, across every
    # 64-byte stage border, ending in a row's overlap, several in one row, in
    # the ragged last rows
    chunk = 1280 if cfg is None else cfg["chunk"]
    n = 512 * chunk * 2 + 7 * chunk + 77
    for m in (8, 12, 33, 64):
        t = synth.genome_text(n, 240 + m, n_gap_mean=30_000, n_run_mean=200)
        pat = synth.pattern(m, 2400 + m)
        rnd = synth.uniform_ints(n // 64 + 8, 1 << 30, 250 + m)
        at = []
        for k, b in enumerate(range(0, n - m - 1, 64 * 3)):
            r = int(rnd[k] % 4)
            st = b if r == 0 else b - int(rnd[k] >> 2) % m if r == 1 else b - m + 1 if r == 2 else b + 5
            if 0 <= st <= n - m:
                at.append(st)
        for row_end in range(chunk, n, chunk * 37):        # ending in the overlap
            at.append(row_end - m // 2)
        at += [n - m, n - m - 70]                          # the ragged end
        synth.plant(t, pat, sorted(set(at)))
        assert _check(gpu, t, pat, cfg) > 0


@pytest.mark.parametrize("chunk", [128, 640, 1280])
def test_staged_row_end_offsets(gpu, chunk):
    # rows holding 0..11 occurrences in turn (the relaxed layout stages 8 a
    # row: rows with more are walked again by the third pass), some ending in
    # the row's overlap, rows spilling into their successors
    cfg = dict(loader=2, layout=4, chunk=chunk)
    n = 512 * chunk * 2 + 3 * chunk + 41
    for m in (8, 13, 40):
        t = synth.genome_text(n, 260 + m, n_gap_mean=0)
        pat = synth.pattern(m, 2600 + m)
        at = []
        for row in range(n // chunk):
            k = row % 12
            gap = max(m + 1, (chunk - m) // max(k, 1))
            for j in range(k):
                st = row * chunk + j * gap
                if j == k - 1 and row % 3 == 0:
                    st = row * chunk + chunk - m // 2          # ends in the overlap
                if st + m <= n:
                    at.append(st)
        synth.plant(t, pat, sorted(set(at)))
        assert _check(gpu, t, pat, cfg) > 0


@pytest.mark.parametrize("chunk", [128, 960, 1024])
def test_staged_dense_rows_past_their_slots(gpu, chunk):
    # layout 1 stages up to 16 end offsets a row: rows holding 0..23 true
    # copies of a short pattern in turn (rows above 16 are walked again by
    # the third pass), each copy preceded by a non-base at a varying
    # distance, and decoys (one byte swapped for a non-base of the same code)
    # between them
    cfg = dict(loader=2, layout=1, chunk=chunk)
    n = 512 * chunk * 2 + 5 * chunk + 19
    for m in (3, 5, 8):
        t = synth.genome_text(n, 270 + m, n_gap_mean=0)
        pat = synth.pattern(m, 2700 + m)
        codes = [(c >> 1) & 3 for c in pat]
        rnd = synth.uniform_ints(4 * (n // chunk) * 24 + 8, 1 << 30, 280 + m)
        k = 0
        for row in range(n // chunk):
            want = row % 24
            gap = max(2 * m + 2, (chunk - m) // max(want, 1))
            for j in range(want):
                st = row * chunk + j * gap
                if st + m > n:
                    break
                t[st:st + m] = np.frombuffer(pat, np.uint8)
                d = 1 + int(rnd[k] % 8); k += 1
                if st - d >= 0 and j % 3 == 1:
                    t[st - d] = _same_code_nonbases(int(rnd[k] % 4))[0]; k += 1
                ds = st + m + 1
                if j % 4 == 2 and ds + m <= min(n, row * chunk + (j + 1) * gap):
                    dec = bytearray(pat)
                    q = int(rnd[k] % m); k += 1
                    dec[q] = _same_code_nonbases(codes[q])[0]
                    t[ds:ds + m] = np.frombuffer(bytes(dec), np.uint8)
        assert _check(gpu, t, pat, cfg) > 0


def test_dense_patterns_on_nonbase_runs(gpu):
    # N reads as G by its code: dense patterns of G's meet runs of N
    n = 1_000_003
    t = synth.genome_text(n, 78, n_gap_mean=2_000, n_run_mean=300)
    for pat in (b"G", b"GG", b"GGGG", b"GGGGGG", b"AGGGG", b"GGGGT", b"CGG"):
        for cfg in (None, dict(loader=2, layout=1, chunk=128), dict(loader=2, layout=1, chunk=640)):
            _check(gpu, t, pat, cfg)


def test_relaxed_walk_nonbase_runs(gpu):
    # runs of N read as runs of G by codes alone: a pattern of G's makes the
    # relaxed walk flag every run, the exact walk counts nothing inside them
    n = 2_000_003
    t = synth.genome_text(n, 77, n_gap_mean=3_000, n_run_mean=500)
    for pat in (b"GGGGGGGG", b"G" * 20, b"G" * 40, b"ACGGGGGGGGGT"):
        for cfg in (None, dict(loader=2, layout=4, chunk=128), dict(loader=2, layout=3, chunk=1280)):
            _check(gpu, t, pat, cfg)


def test_unaligned_workspace_rejected(gpu):
    # the workspace holds u64 words and 16-byte aligned parts: a pointer off
    # a 16-byte boundary is refused before anything runs
    import torch
    n = 1_000_003
    td = _dev(gpu, synth.genome_text(n, 33))
    tab = gpu.dfa_build(b"ACGTA")
    W = gpu.dfa_find_workspace_bytes(n)
    buf = torch.empty(W + 16, dtype=torch.uint8, device="cuda")
    pos = torch.empty(1 << 16, dtype=torch.int64, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    with pytest.raises(gpu.DfaError) as e:
        gpu.dfa_find(td, tab, pos, cnt, buf[8:8 + W])
    assert e.value.code == gpu.DFA_EINVAL
    gpu.dfa_find(td, tab, pos, cnt, buf[16:16 + W])
    rc, c = gpu.dfa_find_status(buf[16:16 + W], cnt, pos.numel())
    assert rc == gpu.DFA_OK and c == oracle.count_brute(synth.genome_text(n, 33), b"ACGTA")


@pytest.mark.parametrize("layout", [1, 3, 4])
def test_single_pass_find_with_small_workspace(gpu, layout):
    # a workspace with room for the tile words only (no per-row counts) takes
    # the single-pass find; both forms must give the same exact result
    import torch
    n = 3_000_017
    t = synth.genome_text(n, 31)
    td = _dev(gpu, t)
    cfg = dict(loader=2, layout=layout, chunk=128)
    ntiles = -(-n // (512 * 128))
    for m in ((1, 2, 4, 6, 8, 9) if layout == 1 else (8, 13, 24, 31)):
        pat = synth.pattern(m, 300 + m)
        pos_idx = synth.uniform_ints(300, n - m, 5 + m)
        synth.plant(t, pat, np.unique(pos_idx // m * m))
        td = _dev(gpu, t)
        want_c, want_p = oracle.find_brute(t, pat)
        tab = gpu.dfa_build(pat)
        for ws_bytes in (8 * (2 + ntiles), gpu.dfa_find_workspace_bytes(n, cfg)):
            cap = want_c + 5
            pos = torch.full((cap,), -1, dtype=torch.int64, device="cuda")
            cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
            ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
            gpu.dfa_find(td, tab, pos, cnt, ws, cfg=cfg)
            rc, c = gpu.dfa_find_status(ws, cnt, cap)
            assert rc == gpu.DFA_OK and c == want_c, (m, ws_bytes, c, want_c)
            assert np.array_equal(pos[:c].cpu().numpy(), want_p)


def test_repeated_launches_identical(gpu):
    # the same find many times on a text larger than L2: every result equal
    # (a race between a ring slot's reload and its readers would show here)
    import torch
    n = 400_000_000
    t = synth.genome_text(n, 2)
    td = _dev(gpu, t)
    for m, seed in ((4, 3), (8, 4), (16, 5)):
        pat = synth.pattern(m, seed)
        want_c = oracle.count_brute(t, pat)
        tab = gpu.dfa_build(pat)
        cap = want_c + 16
        pos = torch.empty(cap, dtype=torch.int64, device="cuda")
        cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
        ws = torch.empty(gpu.dfa_find_workspace_bytes(n), dtype=torch.uint8, device="cuda")
        ref = None
        for _ in range(12):
            gpu.dfa_find(td, tab, pos, cnt, ws)
            rc, c = gpu.dfa_find_status(ws, cnt, cap)
            assert rc == gpu.DFA_OK and c == want_c, (m, c, want_c)
            cur = pos[:c].clone()
            if ref is None:
                ref = cur
            else:
                assert torch.equal(cur, ref), m
            out = torch.zeros(1, dtype=torch.int64, device="cuda")
            gpu.dfa_count(td, tab, out)
            assert int(out.item()) == want_c


def test_sharded_find_with_library_engine(gpu):
    # the multi-process decomposition run rank by rank on one GPU (no rank
    # waits on another): each slice scanned by the library, results merged
    from paper_1506_08612_gb300 import shard
    n = 3_000_001
    t = synth.genome_text(n, 17)
    td = _dev(gpu, t)
    for m, pseed in ((4, 1), (9, 2), (40, 3)):
        pat = synth.pattern(m, pseed)
        t2 = t.copy()
        synth.plant(t2, pat, np.arange(0, n - m, 99_991))
        td = _dev(gpu, t2)

        def engine(sl, n_own):
            c, p = gpu.find(sl, pat)
            p = p.cpu().numpy()
            keep = p < n_own
            return int(keep.sum()), p[keep]

        want_c, want_p = oracle.find_brute(t2, pat)
        for world in (2, 3, 7):
            parts = [shard.local_find(td, m, world, r, engine) for r in range(world)]
            c, p = shard.merge([x[0] for x in parts], [x[1] for x in parts])
            assert c == want_c and np.array_equal(p, want_p), (m, world)


def test_autotuned_find_and_count(gpu, tmp_path, monkeypatch):
    # cfg="auto": the autotuner times the TMA layouts x row lengths on the
    # call itself (find or count) and caches the winner; results stay exact
    from paper_1506_08612_gb300 import autotune
    monkeypatch.setenv("DNADFA_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    monkeypatch.delenv("DNADFA_CONFIG", raising=False)
    autotune.reset_memory_cache()
    n = 20_000_003
    t = synth.genome_text(n, 35)
    td = _dev(gpu, t)
    for m, seed in ((4, 3501), (12, 3502)):
        pat = synth.pattern(m, seed)
        want_c, want_p = oracle.find_brute(t, pat)
        c, p = gpu.find(td, pat, cfg="auto")
        assert c == want_c and np.array_equal(p.cpu().numpy(), want_p)
        assert gpu.count(td, pat, cfg="auto") == want_c
    cached = autotune._load_cache()
    assert any(k.startswith("single-find|") for k in cached)
    assert any(k.startswith("single-count|") for k in cached)
    autotune.reset_memory_cache()


def test_bench_shard_mode_single_rank(gpu):
    # bench.py --shard at world size 1: the slice is the whole text and the
    # merged counts equal a whole-text count (the bench asserts it); the
    # counts it prints equal the oracle's
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    n = 40_000_000
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--shard", "--n", str(n),
                          "--steps", "2", "--warmup", "1"], stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                         text=True, cwd=root, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads([ln for ln in out.stdout.splitlines() if ln.startswith("{")][-1])
    assert line["scaling"] == "strong" and line["config"]["parallelism"].startswith("shard x1")
    text = synth.genome_text(n, 2)
    want = [oracle.count_brute(text, synth.pattern(m, s)) for m, s in zip((4, 8, 16, 32, 64), (3, 4, 5, 6, 7))]
    assert line["counts"] == want
