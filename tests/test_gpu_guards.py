"""Every device write stays inside its buffer: positions, counts and
workspaces are views into larger buffers filled with a sentinel, and after
the calls the guard bands around them are unchanged (a stand-in for a
memory checker, which is not available here)."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

SENT = -0x5A5A5A5A5A5A5A5B
G = 64                                            # guard elements each side


def _guarded(n, dtype, fill, torch):
    buf = torch.full((n + 2 * G,), fill, dtype=dtype, device="cuda")
    return buf, buf[G:G + n]


def _intact(buf, n, fill):
    h = buf.cpu().numpy()
    return bool((h[:G] == fill).all() and (h[G + n:] == fill).all())


@pytest.mark.parametrize("m,planted", [(4, 0), (6, 0), (8, 300), (12, 300), (40, 200)])
def test_find_writes_inside_its_buffers(gpu, m, planted):
    import torch
    n = 5_000_011
    t = synth.genome_text(n, 600 + m)
    pat = synth.pattern(m, 6000 + m)
    if planted:
        synth.plant(t, pat, synth.uniform_ints(planted, n - m, 6100 + m))
    td = torch.from_numpy(t).cuda()
    want_c, want_p = oracle.find_brute(t, pat)
    tab = gpu.dfa_build(pat)
    W = gpu.dfa_find_workspace_bytes(n)
    for cap in (want_c, max(want_c // 3, 1)):
        pbuf, pos = _guarded(cap, torch.int64, SENT, torch)
        cbuf, cnt = _guarded(1, torch.int64, SENT, torch)
        wbuf = torch.full((W + 2 * 256,), 0xAB, dtype=torch.uint8, device="cuda")
        ws = wbuf[256:256 + W]
        gpu.dfa_find(td, tab, pos, cnt, ws)
        rc, c = gpu.dfa_find_status(ws, cnt, cap)
        assert c == want_c and rc == (gpu.DFA_OK if cap >= want_c else gpu.DFA_ETRUNC)
        k = min(cap, want_c)
        assert np.array_equal(pos[:k].cpu().numpy(), want_p[:k])
        assert _intact(pbuf, cap, SENT) and _intact(cbuf, 1, SENT)
        w = wbuf.cpu().numpy()
        assert (w[:256] == 0xAB).all() and (w[256 + W:] == 0xAB).all()
        # the count alone
        cbuf2, cnt2 = _guarded(1, torch.int64, SENT, torch)
        gpu.dfa_count(td, tab, cnt2)
        assert int(cnt2.item()) == want_c and _intact(cbuf2, 1, SENT)


def test_multi_outputs_write_inside_their_buffers(gpu):
    import torch
    texts = [synth.genome_text(n, 620 + i) for i, n in enumerate((700_001, 1_300_003))]
    pats = [synth.pattern(m, 6200 + m) for m in (7, 9, 13, 21)]
    dts = [torch.from_numpy(t).cuda() for t in texts]
    mt = gpu.MultiTable(pats)
    cbuf, counts = _guarded(len(texts) * len(pats), torch.int64, SENT, torch)
    gpu.dfa_multi_count(dts, mt, counts)
    want = oracle.multi_count(texts, pats)
    assert np.array_equal(counts.cpu().numpy().astype(np.uint64).reshape(want.shape), want)
    assert _intact(cbuf, counts.numel(), SENT)
    # locate on the first text
    c0 = [int(x) for x in want[0]]
    total = sum(c0)
    pbuf, pos = _guarded(total, torch.int64, SENT, torch)
    wb = gpu.dfa_multi_locate_work_bytes(len(pats))
    wbuf = torch.full((wb + 2 * 256,), 0xAB, dtype=torch.uint8, device="cuda")
    gpu.dfa_multi_locate(dts[0], mt, c0, pos, wbuf[256:256 + wb])
    assert gpu.dfa_multi_locate_status(wbuf[256:256 + wb], len(pats)) == gpu.DFA_OK
    assert _intact(pbuf, total, SENT)
    w = wbuf.cpu().numpy()
    assert (w[:256] == 0xAB).all() and (w[256 + wb:] == 0xAB).all()
    got, o = pos.cpu().numpy(), 0
    for p, c in zip(pats, c0):
        assert np.array_equal(got[o:o + c], oracle.find_brute(texts[0], p)[1])
        o += c


def test_binding_rejects_misfit_device_buffers(gpu):
    """Device tensors the library would misread or overrun (a narrower
    element type, a strided view, a count buffer too short) are refused in
    Python, before any launch; a well-formed call after them still counts."""
    import torch
    t = synth.genome_text(100_003, 630)
    pat = synth.pattern(6, 6300)
    td = torch.from_numpy(t).cuda()
    tab = gpu.dfa_build(pat)
    ws = torch.empty(gpu.dfa_find_workspace_bytes(td.numel()), dtype=torch.uint8, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    with pytest.raises(TypeError, match="torch.int64"):
        gpu.dfa_find(td, tab, torch.empty(64, dtype=torch.int32, device="cuda"), cnt, ws)
    with pytest.raises(TypeError, match="torch.uint8"):
        gpu.dfa_count(td.to(torch.int16), tab, cnt)
    with pytest.raises(ValueError, match="contiguous"):
        gpu.dfa_count(td[::2], tab, cnt)
    with pytest.raises(ValueError, match="at least 1"):
        gpu.dfa_count(td, tab, cnt[:0])
    with pytest.raises(ValueError, match="outside"):
        gpu.dfa_find(td, tab, None, cnt, ws, n=td.numel() + 1)
    mt = gpu.MultiTable([pat, synth.pattern(9, 6301)])
    with pytest.raises(ValueError, match="at least 4"):
        gpu.dfa_multi_count([td, td], mt, torch.zeros(3, dtype=torch.int64, device="cuda"))
    gpu.dfa_count(td, tab, cnt)
    assert int(cnt.item()) == oracle.count_brute(t, pat)
