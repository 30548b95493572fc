"""dfa_find_noalloc: dfa_find with the library's static device workspace.

This entry point serves callers that may not allocate device memory (a
process whose memory a framework's pool already holds, a latency-bound
stream on which cudaMalloc/cudaFree would synchronise the device, a plug-in
handed only its buffers).  Every call shares one workspace array that keeps
the previous call's contents, so the checks run two calls in a row and
compare each, bit for bit, with the oracle's window compare and with
dfa_find on a caller-owned workspace.  The static array holds tile
descriptors only, so this entry point always takes the single-pass ordered
find; one case plants occurrences across every 64-byte border (every stage,
row and tile border) of a pattern long enough for the relaxed walk.

The file name makes pytest collect it last; it passes both alone in a fresh
process and after the other tests.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _with_workspace(gpu, td, table, cap, cfg):
    import torch
    pos = torch.full((cap,), -1, dtype=torch.int64, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    ws = torch.empty(gpu.dfa_find_workspace_bytes(td.numel(), cfg), dtype=torch.uint8,
                     device="cuda")
    gpu.dfa_find(td, table, pos, cnt, ws, cfg=cfg)
    rc, c = gpu.dfa_find_status(ws, cnt, cap)
    assert rc == gpu.DFA_OK, rc
    return c, pos[:c].cpu().numpy()


def _without_workspace(gpu, td, table, cap, cfg):
    import torch
    pos = torch.full((cap,), -1, dtype=torch.int64, device="cuda")
    cnt = torch.full((1,), 12345, dtype=torch.int64, device="cuda")  # overwritten
    gpu.dfa_find_noalloc(td, table, pos, cnt, cfg=cfg)
    torch.cuda.synchronize()
    c = int(cnt.item()) & (2**64 - 1)
    assert not c & gpu.DFA_COUNT_FAILED
    assert c <= cap
    return c, pos[:c].cpu().numpy()


# (text bytes, text seed, pattern length, pattern seed, config); the first
# case is the longest, so it leaves published descriptors over every tile the
# later calls use, and one not cleared would surface as a wrong look-back
# offset
CASES = [
    (24_000_011, 5, 8, 61, None),
    (3_000_017, 6, 12, 62, None),
    (2_000_003, 7, 5, 63, dict(loader=1, layout=1, threads=256, chunk=64)),
    (1_000_033, 8, 33, 64, dict(loader=2, layout=3, chunk=128)),
]


def _text(gpu, n, seed, pat):
    import torch
    t = synth.genome_text(n, seed)
    pos = np.unique(synth.uniform_ints(2_000, n - len(pat), seed + 1000) // len(pat) * len(pat))
    synth.plant(t, pat, pos)
    return t, torch.from_numpy(t).cuda()


def test_matches_oracle_and_dfa_find_on_consecutive_calls(gpu):
    for n, seed, m, pseed, cfg in CASES:
        pat = synth.pattern(m, pseed)
        host, td = _text(gpu, n, seed, pat)
        table = gpu.dfa_build(pat)
        want_c, want_p = oracle.find_brute(host, pat)
        ws_c, ws_p = _with_workspace(gpu, td, table, 1 << 20, cfg)
        assert want_c > 0
        assert ws_c == want_c and np.array_equal(ws_p, want_p), (n, m, cfg)
        got_c, got_p = _without_workspace(gpu, td, table, 1 << 20, cfg)
        assert got_c == want_c, (n, m, cfg)
        assert np.array_equal(got_p, want_p), (n, m, cfg)
        # the same input again right after: identical result
        again_c, again_p = _without_workspace(gpu, td, table, 1 << 20, cfg)
        assert again_c == want_c and np.array_equal(again_p, want_p)


def test_occurrences_across_every_64_byte_border(gpu):
    # tiles, rows and TMA stages all start at multiples of 64 bytes: an
    # occurrence of a 12-mer straddles every such border at a different
    # depth d = 1 .. 11, plus one starting exactly on a border, in a text with
    # N blocks and soft-masked runs; the default launch (relaxed walk)
    import torch
    m, n = 12, 3_000_017
    pat = synth.pattern(m, 65)
    host = synth.genome_text(n, 10)
    starts = np.arange(64, n - 64, 64, dtype=np.int64)
    depth = starts // 64 % m                               # 0 .. m - 1 bytes before the border
    pos = starts - depth
    synth.plant(host, pat, pos)
    want_c, want_p = oracle.find_brute(host, pat)
    assert set(pos.tolist()) <= set(want_p.tolist())
    td = torch.from_numpy(host).cuda()
    table = gpu.dfa_build(pat)
    for _ in range(2):
        got_c, got_p = _without_workspace(gpu, td, table, want_c + 16, None)
        assert got_c == want_c and np.array_equal(got_p, want_p)


def test_truncation_and_empty_text(gpu):
    import torch
    pat = synth.pattern(4, 71)
    table = gpu.dfa_build(pat)
    host, td = _text(gpu, 5_000_000, 9, pat)
    want_c, want_p = oracle.find_brute(host, pat)
    cap = want_c // 3
    pos = torch.full((cap,), -1, dtype=torch.int64, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    gpu.dfa_find_noalloc(td, table, pos, cnt)
    assert int(cnt.item()) == want_c
    assert np.array_equal(pos.cpu().numpy(), want_p[:cap])
    empty = torch.empty(0, dtype=torch.uint8, device="cuda")
    cnt.fill_(7)
    gpu.dfa_find_noalloc(empty, table, None, cnt)
    assert int(cnt.item()) == 0


def test_rejects_text_beyond_the_static_workspace(gpu):
    import torch
    # 2 KiB tiles (128 threads x 16 bytes): 65536 tiles fit, 65537 do not.
    # The text buffer is real and covers n, so nothing would read past it.
    cfg = dict(loader=1, layout=1, threads=128, chunk=16)
    n = 128 * 16 * 65536 + 1
    td = torch.full((n,), ord("A"), dtype=torch.uint8, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    table = gpu.dfa_build(b"ACGT")
    with pytest.raises(gpu.DfaError) as e:
        gpu.dfa_find_noalloc(td, table, None, cnt, cfg=cfg)
    assert e.value.code == gpu.DFA_EWORKSPACE
    assert "65536" in str(e.value)
    # one tile fewer fits, and the count is exact (no ACGT in a run of A)
    gpu.dfa_find_noalloc(td[: n - 1], table, None, cnt, cfg=cfg)
    assert int(cnt.item()) == 0
