"""Failure detection without a GPU fault: a device-side wait that nothing
satisfies gives up after its bound, records the failure in the workspace's
status word, and the host reads DFA_ETIMEOUT; the device stays usable.  The
wait is the ordered compaction's look-back of dfa_find, run on a zeroed
workspace (no predecessor tile ever publishes), through the library's
diagnostic entry point."""
import time

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def test_lookback_wait_gives_up_and_reports(gpu):
    import torch
    tile = 5
    ws = torch.zeros(8 * (2 + tile + 1), dtype=torch.uint8, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    t0 = time.perf_counter()
    gpu.dfa_debug_wait_timeout(ws, tile)
    rc, _ = gpu.dfa_find_status(ws, cnt, 0)
    dt = time.perf_counter() - t0
    assert rc == gpu.DFA_ETIMEOUT
    assert 0.3 < dt < 60, dt
    # the context is still usable: a normal find afterwards is exact
    t = synth.genome_text(300_001, 91)
    td = torch.from_numpy(t).cuda()
    c, pos = gpu.find(td, b"ACGTA")
    want_c, want_p = oracle.find_brute(t, b"ACGTA")
    assert c == want_c and np.array_equal(pos.cpu().numpy(), want_p)


def test_lookback_wait_ends_when_a_predecessor_publishes(gpu):
    import torch
    tile = 5
    ws = torch.zeros(8 * (2 + tile + 1), dtype=torch.uint8, device="cuda")
    words = ws.view(torch.int64)
    # tiles 0..3 published aggregates (flag 1 in bits 62..63), tile 4 an
    # inclusive prefix of 7 (flag 2): the warp reads them all at once
    for j in range(tile - 1):
        words[2 + j] = (1 << 62) + 1
    words[2 + tile - 1] = -(2 ** 63) + 7
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    t0 = time.perf_counter()
    gpu.dfa_debug_wait_timeout(ws, tile)
    rc, _ = gpu.dfa_find_status(ws, cnt, 0)
    assert rc == gpu.DFA_OK
    assert time.perf_counter() - t0 < 5
    d = int(words[2 + tile].item()) & (2 ** 64 - 1)
    assert d >> 62 == 2 and d & ((1 << 62) - 1) == 8     # its own prefix: 7 + its total 1


def test_rejects_a_workspace_too_small(gpu):
    import torch
    ws = torch.zeros(8 * 4, dtype=torch.uint8, device="cuda")
    with pytest.raises(gpu.DfaError) as e:
        gpu.dfa_debug_wait_timeout(ws, 5)
    assert e.value.code == gpu.DFA_EINVAL
