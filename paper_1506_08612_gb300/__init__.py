"""GB300-native finite-automaton DNA pattern scan (Memeti & Pllana 2015).

Thin Python binding over the C ABI of ``include/dnadfa.h`` (``libdnadfa.so``,
built in place from ``csrc/``).  Every step of the scan runs in the library's
CUDA kernels; this module only marshals arguments: PyTorch tensors supply
device memory and the current CUDA stream.  The names follow the C ABI:

* ``dfa_build(pattern) -> Table`` / ``dfa_free(table)``
* ``dfa_count(text, table, count)`` — count occurrences (overlaps included)
* ``dfa_find(text, table, positions, count, workspace)`` — count and sorted
  start positions, single pass
* ``dfa_find_status(workspace, count, cap)`` — device-side outcome
* ``dfa_find_host(...)`` — host buffers in, host buffers out (copies inside)
* ``MultiTable(patterns)`` / ``dfa_multi_count(texts, table, counts)`` — the
  multi-pattern automaton and one batched count over many sequences
* ``dfa_find_noalloc(text, table, positions, count)`` — ``dfa_find`` with the
  library's static device workspace, for callers that may not allocate

plus ``find``/``count`` conveniences that allocate their outputs with torch.
There is no CPU fallback: importing this package fails if the CUDA library
cannot be built or loaded.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _native
from ._native import (DFA_COUNT_FAILED, DFA_ECUDA, DFA_EINVAL, DFA_ENOMEM, DFA_ETIMEOUT,
                      DFA_ETRUNC, DFA_EWORKSPACE, DFA_LOCATE_MAX, DFA_MAX_M, DFA_OK, LIBRARY_PATH,
                      dfa_config)

_lib = _native.lib

__all__ = ["Table", "DfaError", "dfa_build", "dfa_free", "dfa_export_stt", "dfa_count",
           "dfa_find", "dfa_find_workspace_bytes", "dfa_table_bytes", "dfa_find_status", "dfa_host_stage_bytes",
           "dfa_find_host", "dfa_find_host_multi", "dfa_find_batched", "dfa_debug_wait_timeout", "dfa_host_stage_bytes_multi", "dfa_find_noalloc", "MultiTable", "dfa_multi_count", "multi_count", "dfa_multi_locate",
           "dfa_multi_locate_work_bytes", "dfa_multi_locate_status",
           "dfa_strerror", "dfa_config", "find", "count", "LIBRARY_PATH",
           "DFA_OK", "DFA_EINVAL", "DFA_ETRUNC", "DFA_ETIMEOUT", "DFA_ECUDA", "DFA_EWORKSPACE",
           "DFA_ENOMEM", "DFA_MAX_M"]


class DfaError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        msg = f"{what}: {dfa_strerror(code)} (code {code})" if what else dfa_strerror(code)
        if code == DFA_ECUDA:
            msg += f" [{_lib.dfa_last_error().decode(errors='replace')}]"
        super().__init__(msg)


def dfa_strerror(code: int) -> str:
    return _lib.dfa_strerror(int(code)).decode()


def _check(rc: int, what: str) -> int:
    if rc != DFA_OK:
        raise DfaError(rc, what)
    return rc


def _cfg(cfg):
    if cfg is None:
        return None
    if isinstance(cfg, dict):
        cfg = dfa_config(**{k: int(v) for k, v in cfg.items()})
    return ctypes.byref(cfg)


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _ptr(t) -> ctypes.c_void_p:
    return ctypes.c_void_p(t.data_ptr() if t is not None else 0)


def _nbytes(t) -> int:
    return int(t.numel() * t.element_size())


def _desc(t) -> str:
    if not hasattr(t, "device"):
        return type(t).__name__
    return f"{t.dtype} on {t.device}" + ("" if t.is_contiguous() else ", not contiguous")


def _dev(t, what: str, dtype=None, numel: int = 0):
    """Checks a device-buffer argument: a contiguous CUDA tensor on the
    current CUDA device (the library launches there), of ``dtype`` when
    given, with at least ``numel`` elements.  The library reads and writes
    such buffers as flat arrays at ``data_ptr()``, so a strided view, a host
    tensor or a narrower element type would be misread or overrun."""
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{what}: expected a CUDA tensor, got {_desc(t)}")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{what}: expected {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{what}: expected a contiguous tensor")
    if t.device.index != torch.cuda.current_device():
        raise ValueError(f"{what}: tensor on {t.device}, current device is cuda:{torch.cuda.current_device()}")
    if t.numel() < numel:
        raise ValueError(f"{what}: {t.numel()} elements, at least {numel} needed")
    return t


def _host(t, what: str, dtype):
    """Checks a host-buffer argument: a contiguous CPU tensor of ``dtype``."""
    import torch
    if not isinstance(t, torch.Tensor) or t.device.type != "cpu":
        raise ValueError(f"{what}: expected a CPU tensor, got {_desc(t)}")
    if t.dtype != dtype:
        raise TypeError(f"{what}: expected {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{what}: expected a contiguous tensor")
    return t


def _u8():
    import torch
    return torch.uint8


def _i64():
    import torch
    return torch.int64


class Table:
    """Automaton of one pattern (library-owned host + device tables)."""

    def __init__(self, pattern, into=None, stream=None):
        """``into``: optional device uint8 tensor of at least
        ``dfa_table_bytes(m)`` bytes that receives the tables (dfa_build_into,
        copy enqueued on ``stream``); the caller keeps it alive while the
        table is in use."""
        if isinstance(pattern, str):
            pattern = pattern.encode("ascii")
        pattern = bytes(pattern)
        h = ctypes.c_void_p()
        if into is None:
            _check(_lib.dfa_build(pattern, len(pattern), ctypes.byref(h)), "dfa_build")
        else:
            _dev(into, "Table(into=)")
            _check(_lib.dfa_build_into(pattern, len(pattern), _ptr(into),
                                       _nbytes(into), _stream(stream),
                                       ctypes.byref(h)), "dfa_build_into")
        self._h = h
        self._into = into
        self.pattern = pattern.upper()
        self.m = len(pattern)

    @property
    def handle(self) -> ctypes.c_void_p:
        if self._h is None:
            raise ValueError("table already freed")
        return self._h

    def free(self):
        if getattr(self, "_h", None) is not None:
            _lib.dfa_free(self._h)
            self._h = None

    def __del__(self):  # pragma: no cover - interpreter shutdown order
        try:
            self.free()
        except Exception:
            pass


def dfa_build(pattern) -> Table:
    return Table(pattern)


def dfa_free(table: Table) -> None:
    table.free()


def dfa_table_bytes(m: int) -> int:
    return int(_lib.dfa_table_bytes(int(m)))


def dfa_export_stt(table: Table) -> np.ndarray:
    """The paper's sparse ASCII STT, (m+1, 256) uint8 (Sec. III-B, Table I)."""
    out = np.zeros((table.m + 1) * 256, dtype=np.uint8)
    _check(_lib.dfa_export_stt(table.handle, out.ctypes.data_as(ctypes.c_void_p), out.size),
           "dfa_export_stt")
    return out.reshape(table.m + 1, 256)


def dfa_count(text, table: Table, count, cfg=None, stream=None) -> None:
    """Enqueue a count; ``count`` is a 1-element int64 device tensor."""
    _dev(text, "dfa_count text", _u8())
    _dev(count, "dfa_count count", _i64(), 1)
    _check(_lib.dfa_count(_ptr(text), int(text.numel()), table.handle, _ptr(count), _cfg(cfg),
                          _stream(stream)), "dfa_count")


def dfa_find_workspace_bytes(n: int, cfg=None) -> int:
    return int(_lib.dfa_find_workspace_bytes(int(n), _cfg(cfg)))


def dfa_find(text, table: Table, positions, count, workspace, cfg=None, stream=None,
             n: int | None = None) -> None:
    """Enqueue count + sorted start positions (int64 device tensor, capacity =
    its length) into ``count`` (1-element int64 device tensor)."""
    _dev(text, "dfa_find text", _u8())
    if positions is not None:
        _dev(positions, "dfa_find positions", _i64())
    _dev(count, "dfa_find count", _i64(), 1)
    _dev(workspace, "dfa_find workspace")
    cap = int(positions.numel()) if positions is not None else 0
    nbytes = int(text.numel()) if n is None else int(n)
    if not 0 <= nbytes <= text.numel():
        raise ValueError(f"dfa_find: n={nbytes} outside [0, {text.numel()}]")
    _check(_lib.dfa_find(_ptr(text), nbytes, table.handle, _ptr(positions), cap, _ptr(count),
                         _ptr(workspace), _nbytes(workspace),
                         _cfg(cfg), _stream(stream)), "dfa_find")


def dfa_find_status(workspace, count, cap: int, stream=None):
    """Synchronise and return (return code, count)."""
    _dev(workspace, "dfa_find_status workspace")
    _dev(count, "dfa_find_status count", _i64(), 1)
    h = ctypes.c_uint64(0)
    rc = _lib.dfa_find_status(_ptr(workspace), _ptr(count), int(cap), ctypes.byref(h),
                              _stream(stream))
    return rc, int(h.value)


def dfa_find_noalloc(text, table: Table, positions, count, cfg=None, stream=None) -> None:
    """Enqueue dfa_find with the library's static device workspace: for
    callers that may not allocate device memory.  A bounded wait that gave up
    sets bit 63 of ``count``; calls that may overlap on the GPU race on the
    shared workspace."""
    _dev(text, "dfa_find_noalloc text", _u8())
    if positions is not None:
        _dev(positions, "dfa_find_noalloc positions", _i64())
    _dev(count, "dfa_find_noalloc count", _i64(), 1)
    cap = int(positions.numel()) if positions is not None else 0
    rc = _lib.dfa_find_noalloc(_ptr(text), int(text.numel()), table.handle, _ptr(positions), cap,
                               _ptr(count), _cfg(cfg), _stream(stream))
    if rc != DFA_OK:
        err = DfaError(rc, "dfa_find_noalloc")
        if rc != DFA_ECUDA and _lib.dfa_last_error():
            err.args = (f"{err.args[0]} [{_lib.dfa_last_error().decode(errors='replace')}]",)
        raise err


def dfa_debug_wait_timeout(workspace, tile: int, stream=None) -> None:
    """Enqueue the look-back wait of ``tile`` on ``workspace`` (failure
    detection test: on a zeroed workspace the wait gives up and
    dfa_find_status reports DFA_ETIMEOUT)."""
    _dev(workspace, "dfa_debug_wait_timeout workspace")
    _check(_lib.dfa_debug_wait_timeout(_ptr(workspace), _nbytes(workspace),
                                       int(tile), _stream(stream)), "dfa_debug_wait_timeout")


def dfa_host_stage_bytes(seg: int, cap: int) -> int:
    return int(_lib.dfa_host_stage_bytes(int(seg), int(cap)))


def dfa_find_host(h_text, table: Table, h_positions, stage, seg: int, stream=None):
    """Host buffers in and out: ``h_text`` a CPU uint8 tensor (pinned for full
    copy bandwidth), ``h_positions`` a CPU int64 tensor (or None), ``stage``
    a device uint8 tensor of dfa_host_stage_bytes(seg, cap) bytes.
    Returns (return code, count)."""
    _host(h_text, "dfa_find_host h_text", _u8())
    if h_positions is not None:
        _host(h_positions, "dfa_find_host h_positions", _i64())
    _dev(stage, "dfa_find_host stage")
    cap = int(h_positions.numel()) if h_positions is not None else 0
    h = ctypes.c_uint64(0)
    rc = _lib.dfa_find_host(_ptr(h_text), int(h_text.numel()), table.handle, _ptr(h_positions), cap,
                            ctypes.byref(h), _ptr(stage), _nbytes(stage), int(seg),
                            _stream(stream))
    if rc not in (DFA_OK, DFA_ETRUNC):
        raise DfaError(rc, "dfa_find_host")
    return rc, int(h.value)


def dfa_find_batched(text, tables, positions, counts, workspace, cfg=None, stream=None) -> None:
    """Enqueue the finds of several patterns over one device text:
    ``positions`` a list of int64 device tensors (capacity = length, or
    None), ``counts`` an int64 device tensor of len(tables)."""
    k = len(tables)
    _dev(text, "dfa_find_batched text", _u8())
    if len(positions) != k:
        raise ValueError(f"dfa_find_batched: {len(positions)} position buffers for {k} tables")
    for p in positions:
        if p is not None:
            _dev(p, "dfa_find_batched positions", _i64())
    _dev(counts, "dfa_find_batched counts", _i64(), k)
    _dev(workspace, "dfa_find_batched workspace")
    th = (ctypes.c_void_p * k)(*[t.handle.value for t in tables])
    ph = (ctypes.c_void_p * k)(*[p.data_ptr() if p is not None and p.numel() else 0 for p in positions])
    cp = (ctypes.c_int64 * k)(*[int(p.numel()) if p is not None else 0 for p in positions])
    _check(_lib.dfa_find_batched(_ptr(text), int(text.numel()), th, k, ph, cp, _ptr(counts), _ptr(workspace),
                                 _nbytes(workspace), _cfg(cfg), _stream(stream)),
           "dfa_find_batched")


def dfa_host_stage_bytes_multi(seg: int, caps) -> int:
    c = (ctypes.c_int64 * len(caps))(*[int(x) for x in caps])
    return int(_lib.dfa_host_stage_bytes_multi(int(seg), c, len(caps)))


def dfa_find_host_multi(h_text, tables, h_positions, stage, seg: int, stream=None):
    """Several patterns over one host text, each segment copied once:
    ``h_positions`` a list of CPU int64 tensors (or None), one per table.
    Returns (return code, list of counts)."""
    k = len(tables)
    _host(h_text, "dfa_find_host_multi h_text", _u8())
    if len(h_positions) != k:
        raise ValueError(f"dfa_find_host_multi: {len(h_positions)} position buffers for {k} tables")
    for p in h_positions:
        if p is not None:
            _host(p, "dfa_find_host_multi h_positions", _i64())
    _dev(stage, "dfa_find_host_multi stage")
    caps = [int(p.numel()) if p is not None else 0 for p in h_positions]
    th = (ctypes.c_void_p * k)(*[t.handle.value for t in tables])
    ph = (ctypes.c_void_p * k)(*[p.data_ptr() if p is not None and p.numel() else 0 for p in h_positions])
    cp = (ctypes.c_int64 * k)(*caps)
    hc = (ctypes.c_uint64 * k)()
    rc = _lib.dfa_find_host_multi(_ptr(h_text), int(h_text.numel()), th, k, ph, cp, hc, _ptr(stage),
                                  _nbytes(stage), int(seg), _stream(stream))
    if rc not in (DFA_OK, DFA_ETRUNC):
        raise DfaError(rc, "dfa_find_host_multi")
    return rc, [int(x) for x in hc]


# ------------------------------------------------------- many patterns

class MultiTable:
    """Owns a dfa_multi (multi-pattern automaton); frees it on close/del."""

    def __init__(self, patterns, device: bool = True, classes: bool = False):
        """device=False builds the host automaton only (dfa_multi_build_host);
        ``attach`` then copies it into caller-owned device memory.
        classes=True reads the patterns as character-class patterns (IUPAC
        codes and bracket sets, dfa_multi_build_class)."""
        pats = [p.encode() if isinstance(p, str) else bytes(p) for p in patterns]
        self.patterns = pats
        self.classes = bool(classes)
        arr = (ctypes.c_char_p * len(pats))(*pats)
        lens = (ctypes.c_int32 * len(pats))(*[len(p) for p in pats])
        h = ctypes.c_void_p()
        if classes:
            fn = _lib.dfa_multi_build_class if device else _lib.dfa_multi_build_class_host
        else:
            fn = _lib.dfa_multi_build if device else _lib.dfa_multi_build_host
        rc = fn(arr, lens, len(pats), ctypes.byref(h))
        if rc != DFA_OK:
            msg = _lib.dfa_last_error().decode(errors="replace")
            raise DfaError(rc, f"{fn.__name__} [{msg}]")
        self._h = h
        self._into = None
        self.npat = len(pats)
        self.lengths = [int(_lib.dfa_multi_pattern_length(h, i)) for i in range(len(pats))]
        self.mmax = max(self.lengths)

    @property
    def handle(self) -> ctypes.c_void_p:
        if self._h is None:
            raise ValueError("multi table already freed")
        return self._h

    def states(self) -> int:
        return int(_lib.dfa_multi_states(self.handle))

    def export(self):
        """(next[states, 4] over codes A0 C1 T2 G3, outputs[states])."""
        ns = self.states()
        nxt = np.zeros(ns * 4, dtype=np.int32)
        nout = np.zeros(ns, dtype=np.int32)
        _check(_lib.dfa_multi_export(self.handle, nxt.ctypes.data_as(ctypes.c_void_p),
                                     nout.ctypes.data_as(ctypes.c_void_p), ns), "dfa_multi_export")
        return nxt.reshape(ns, 4), nout

    def smem_bytes(self) -> int:
        return int(_lib.dfa_multi_smem_bytes(self.handle))

    def image_bytes(self) -> int:
        return int(_lib.dfa_multi_image_bytes(self.handle))

    def attach(self, into, stream=None) -> None:
        """Copy the automaton into ``into`` (device uint8 tensor of at least
        image_bytes(), kept alive by the caller) on ``stream``."""
        _dev(into, "MultiTable.attach into")
        _check(_lib.dfa_multi_attach(self.handle, _ptr(into), _nbytes(into),
                                     _stream(stream)), "dfa_multi_attach")
        self._into = into

    def free(self):
        if getattr(self, "_h", None) is not None:
            _lib.dfa_multi_free(self._h)
            self._h = None

    def __del__(self):  # pragma: no cover - interpreter shutdown order
        try:
            self.free()
        except Exception:
            pass


def dfa_multi_count(texts, table: MultiTable, counts, cfg=None, stream=None) -> None:
    """Enqueue per-(sequence, pattern) counts of every pattern in every text
    (device uint8 tensors) into ``counts`` (device int64 tensor of
    len(texts) * npat, row-major by sequence)."""
    ns = len(texts)
    for t in texts:
        _dev(t, "dfa_multi_count text", _u8())
    _dev(counts, "dfa_multi_count counts", _i64(), ns * table.npat)
    ptrs = (ctypes.c_void_p * ns)(*[t.data_ptr() if t.numel() else 0 for t in texts])
    lens = (ctypes.c_int64 * ns)(*[int(t.numel()) for t in texts])
    _check(_lib.dfa_multi_count(ptrs, lens, ns, table.handle, _ptr(counts), _cfg(cfg),
                                _stream(stream)), "dfa_multi_count")


def dfa_multi_locate_work_bytes(npat: int) -> int:
    return int(_lib.dfa_multi_locate_work_bytes(int(npat)))


def dfa_multi_locate(text, table: MultiTable, counts, positions, workspace, stream=None) -> None:
    """Enqueue the sorted positions of every pattern of ``table`` in ``text``
    into ``positions`` (int64 device tensor, pattern p's segment at the sum
    of the counts before it); ``counts``: the exact per-pattern counts (host
    sequence), each at most DFA_LOCATE_MAX."""
    _dev(text, "dfa_multi_locate text", _u8())
    if positions is not None:
        _dev(positions, "dfa_multi_locate positions", _i64())
    _dev(workspace, "dfa_multi_locate workspace")
    if len(counts) != table.npat:
        raise ValueError(f"dfa_multi_locate: {len(counts)} counts for {table.npat} patterns")
    hc = (ctypes.c_uint64 * table.npat)(*[int(c) for c in counts])
    rc = _lib.dfa_multi_locate(_ptr(text), int(text.numel()), table.handle, hc, _ptr(positions),
                               int(positions.numel()) if positions is not None else 0, _ptr(workspace),
                               _nbytes(workspace), _stream(stream))
    if rc != DFA_OK:
        raise DfaError(rc, f"dfa_multi_locate [{_lib.dfa_last_error().decode(errors='replace')}]")


def dfa_multi_locate_status(workspace, npat: int, stream=None) -> int:
    _dev(workspace, "dfa_multi_locate_status workspace")
    return int(_lib.dfa_multi_locate_status(_ptr(workspace), int(npat), _stream(stream)))


def multi_count(texts, patterns, cfg=None, classes: bool = False) -> np.ndarray:
    """Synchronous batched count: returns uint64[len(texts), len(patterns)].
    classes: the patterns are character-class patterns."""
    import torch
    t = patterns if isinstance(patterns, MultiTable) else MultiTable(patterns, classes=classes)
    dev = texts[0].device
    out = torch.zeros(len(texts) * t.npat, dtype=torch.int64, device=dev)
    dfa_multi_count(texts, t, out, cfg=cfg)
    return out.cpu().numpy().astype(np.uint64).reshape(len(texts), t.npat)


# ----------------------------------------------------------- conveniences

def _as_table(p):
    return p if isinstance(p, Table) else Table(p)


def count(text, pattern, cfg=None) -> int:
    """Synchronous count on the current stream (allocates its output).
    cfg: None (library defaults), a dfa_config dict, or "auto" (the
    autotuner's layout and row length for this pattern and text size)."""
    import torch
    t = _as_table(pattern)
    if isinstance(cfg, str) and cfg == "auto":
        from . import autotune
        cfg = autotune.tune_single(text, t, op="count")
    out = torch.zeros(1, dtype=torch.int64, device=text.device)
    dfa_count(text, t, out, cfg=cfg)
    v = int(out.item()) & (2**64 - 1)
    if v & DFA_COUNT_FAILED:
        raise DfaError(DFA_ETIMEOUT, "dfa_count")
    return v


def find(text, pattern, cap: int | None = None, cfg=None):
    """Synchronous find: returns (count, int64 positions tensor on device).
    With cap=None the buffer grows until every position fits.  cfg as for
    ``count`` ("auto" tunes on dfa_find itself)."""
    import torch
    t = _as_table(pattern)
    if isinstance(cfg, str) and cfg == "auto":
        from . import autotune
        cfg = autotune.tune_single(text, t, op="find")
    dev = text.device
    if cap is None:
        cap = max(1024, text.numel() // 4096)
    while True:
        pos = torch.empty(max(int(cap), 1), dtype=torch.int64, device=dev)
        cnt = torch.zeros(1, dtype=torch.int64, device=dev)
        ws = torch.empty(dfa_find_workspace_bytes(text.numel(), cfg), dtype=torch.uint8, device=dev)
        dfa_find(text, t, pos[:cap], cnt, ws, cfg=cfg)
        rc, c = dfa_find_status(ws, cnt, cap)
        if rc == DFA_OK:
            return c, pos[:c]
        if rc == DFA_ETRUNC:
            cap = c
            continue
        raise DfaError(rc, "dfa_find")


from .batched import BatchedCount  # noqa: E402  (needs the names above)

__all__ += ["BatchedCount"]
