"""Launch-configuration autotuner for the scan kernels.

The paper tunes one knob by hand, the number of OpenMP threads and their
affinity (Sec. IV, Table IV).  On the GPU the knobs are the chunk length C
(bytes one thread walks per tile, each chunk carrying the m-1 byte overlap of
Algorithm 1), the threads per CTA, and, for one pattern, the table layout.
This module times a small set of candidates with CUDA events on a sample of
the caller's own text and remembers the fastest per key:

* key = (kind, kernel version, device name and SM count, log2 bucket of the
  text bytes, pattern bucket), where the pattern bucket is the pattern length
  for one pattern and (log2 of the pattern count, m_max bucket, log2 of the
  automaton states) for the multi-pattern automaton; the version tag changes
  whenever the kernels' candidate space does, so entries timed on earlier
  kernels miss and are tuned again;
* cache = a JSON file (``DNADFA_AUTOTUNE_CACHE``, default
  ``~/.cache/dnadfa/autotune.json``), read once and rewritten atomically
  after each new entry;
* ``DNADFA_CONFIG`` (a JSON object of dfa_config fields) forces one
  configuration for every call and skips tuning; the multi-pattern tuner
  keeps only the fields dfa_multi_count reads (threads, chunk, ctas_per_sm,
  and its table layout: ``multi_layout`` 0..5, or ``layout`` when it is
  0..2, a value the two counts read alike).

Candidates: the multi-pattern count varies threads x chunk x table layout
(one shared copy; one copy per lane where the automaton is small enough;
one table copy with 2, 4 or 8 copies of each state's counter at 512 or
1024 threads: the library refuses what does not fit, and a refused
candidate is skipped); one pattern varies the table layout x row length of
the TMA kernel, timed on the call it will serve (dfa_count or dfa_find).

Timing and selection are separate from the GPU so that the host logic runs
(and is tested) without one: ``select_best`` takes any timing callable.
"""
from __future__ import annotations

import json
import math
import os
import tempfile
import threading

# Candidate grids.  Multi-pattern count: threads per CTA in {128, 256, 512}
# (the kernel's instantiations) x chunk bytes; the chunk must stay well above
# m_max - 1 so the overlap re-scan (Algorithm 1) stays a small fraction.
MULTI_THREADS = (128, 256, 512, 1024)
MULTI_CHUNKS = (256, 512, 1024, 2048, 4096)
# one shared table copy / 32 per-lane copies / one table copy with 2, 4, 8
# counter copies a state (at 512 and 1024 threads)
MULTI_LAYOUTS = (1, 2, 3, 4, 5)
MULTI_COPY_THREADS = (512, 1024)
# One pattern, TMA loader: chunk bytes per row (multiples of 64) x layout
# (0 = library default for m, 1 = four-step table with accept counts,
# 3 = four-step states with exact replays, 4 = relaxed walk on the flagged
# four-step table; 3 and 4 from m = 8 on).
SINGLE_CHUNKS = (0, 512, 768, 960, 1024, 1280)
SINGLE_LAYOUTS = (0, 1, 3, 4)
# Bumped when a kernel or its candidate space changes.
KERNEL_VERSION = "v4"

_lock = threading.Lock()
_cache: dict | None = None


def cache_path() -> str:
    p = os.environ.get("DNADFA_AUTOTUNE_CACHE")
    if p:
        return p
    return os.path.join(os.path.expanduser("~"), ".cache", "dnadfa", "autotune.json")


def _load_cache() -> dict:
    global _cache
    if _cache is None:
        try:
            with open(cache_path()) as f:
                d = json.load(f)
            _cache = d if isinstance(d, dict) else {}
        except (OSError, ValueError):
            _cache = {}
    return _cache


def _store_cache() -> None:
    path = cache_path()
    d = os.path.dirname(path)
    try:
        os.makedirs(d, exist_ok=True)
        fd, tmp = tempfile.mkstemp(dir=d, prefix=".autotune")
        with os.fdopen(fd, "w") as f:
            json.dump(_cache, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except OSError:
        pass                         # a read-only home keeps the in-memory cache only


def reset_memory_cache() -> None:
    """Forget the in-memory copy (the file is re-read on the next lookup)."""
    global _cache
    with _lock:
        _cache = None


def forced_config(kind: str = "single") -> dict | None:
    """The configuration DNADFA_CONFIG forces, or None.  For the
    multi-pattern count (kind "multi") only the fields it reads are kept: a
    single-pattern layout (3, 4) or a loader would make it refuse the call."""
    s = os.environ.get("DNADFA_CONFIG")
    if not s:
        return None
    d = json.loads(s)
    if not isinstance(d, dict):
        raise ValueError("DNADFA_CONFIG must be a JSON object")
    allowed = {"layout", "threads", "chunk", "loader", "ctas_per_sm", "multi_layout"}
    bad = set(d) - allowed
    if bad:
        raise ValueError(f"DNADFA_CONFIG: unknown fields {sorted(bad)}")
    out = {k: int(v) for k, v in d.items()}
    multi_layout = out.pop("multi_layout", None)
    if kind == "multi":
        out.pop("loader", None)
        if multi_layout is not None:
            out["layout"] = multi_layout
        elif out.get("layout", 0) not in (0, 1, 2):
            out.pop("layout")
    return out


def _log2_bucket(x: int) -> int:
    return int(math.floor(math.log2(x))) if x > 0 else 0


def single_key(device: str, n: int, m: int, op: str = "count") -> str:
    return f"single-{op}|{KERNEL_VERSION}|{device}|n2^{_log2_bucket(n)}|m{m}"


def multi_key(device: str, total_bytes: int, npat: int, mmax: int, states: int) -> str:
    mb = 8 if mmax <= 8 else 16 if mmax <= 16 else 32 if mmax <= 32 else 64
    return (f"multi|{KERNEL_VERSION}|{device}|n2^{_log2_bucket(total_bytes)}|p2^{_log2_bucket(npat)}"
            f"|mmax{mb}|s2^{_log2_bucket(states)}")


def lookup(key: str) -> dict | None:
    with _lock:
        v = _load_cache().get(key)
    return dict(v["cfg"]) if isinstance(v, dict) and "cfg" in v else None


def remember(key: str, cfg: dict, ms: float, candidates: int) -> None:
    with _lock:
        c = _load_cache()
        c[key] = {"cfg": dict(cfg), "ms": round(float(ms), 5), "candidates": int(candidates)}
        _store_cache()


def multi_candidates(mmax: int) -> list[dict]:
    out = []
    for lay in MULTI_LAYOUTS:
        for t in MULTI_THREADS:
            if lay >= 3 and t not in MULTI_COPY_THREADS:
                continue
            for c in MULTI_CHUNKS:
                if c >= 4 * max(mmax - 1, 1):
                    out.append({"threads": t, "chunk": c, "layout": lay})
    return out


def single_candidates(m: int) -> list[dict]:
    out = []
    for lay in SINGLE_LAYOUTS:
        if lay in (3, 4) and m < 8:
            continue
        for c in SINGLE_CHUNKS:
            d = {"layout": lay, "loader": 2}
            if c:
                d["chunk"] = c
            out.append(d)
    return out


def _rejected(e: Exception) -> bool:
    """True for a candidate the library refuses before launching (an
    argument it does not take, memory it cannot get); False for a failure
    that may have left the device unusable (a CUDA error), which must not be
    retried with the next candidate."""
    code = getattr(e, "code", None)
    if code is not None:
        from ._native import DFA_EINVAL, DFA_ENOMEM, DFA_EWORKSPACE
        return code in (DFA_EINVAL, DFA_ENOMEM, DFA_EWORKSPACE)
    return isinstance(e, ValueError)


def select_best(candidates, time_ms, reps: int = 3):
    """Time every candidate ``reps`` times with ``time_ms(cfg) -> ms`` (the
    first call of each is a warm-up) and return (best cfg, its median ms).
    Candidates the library rejects are skipped (if all are, the last
    rejection is raised); any other error is raised at once."""
    best, best_ms, err = None, float("inf"), None
    for cfg in candidates:
        try:
            time_ms(cfg)
            ts = sorted(time_ms(cfg) for _ in range(max(reps, 1)))
        except Exception as e:
            if not _rejected(e):
                raise
            err = e
            continue
        med = ts[len(ts) // 2]
        if med < best_ms:
            best, best_ms = cfg, med
    if best is None:
        raise err if err is not None else ValueError("no candidates")
    return best, best_ms


# ------------------------------------------------------------ GPU timing

def device_name(dev=None) -> str:
    import torch
    d = torch.cuda.current_device() if dev is None else dev
    p = torch.cuda.get_device_properties(d)
    return f"{p.name.replace(' ', '_')}x{p.multi_processor_count}"


def _event_timer(launch, stream):
    import torch

    def run(cfg):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        launch(cfg)
        b.record(stream)
        b.synchronize()
        return a.elapsed_time(b)
    return run


def _sample(texts, budget: int):
    """Prefixes of the texts holding about ``budget`` bytes in all, each
    text keeping its share of the total (so the sample has the batch's mix
    of sequence sizes)."""
    total = sum(int(t.numel()) for t in texts)
    if total <= budget:
        return list(texts)
    f = budget / total
    return [t[: max(int(t.numel() * f) // 64 * 64, min(int(t.numel()), 64))] for t in texts]


def tune_multi(texts, table, sample_bytes: int = 1 << 30, reps: int = 3, stream=None,
               retune: bool = False) -> dict:
    """Best (threads, chunk) for dfa_multi_count on these texts and this
    automaton, from the cache or by timing candidates on a sample."""
    import torch

    from . import dfa_multi_count
    forced = forced_config("multi")
    if forced is not None:
        return forced
    total = sum(int(t.numel()) for t in texts)
    key = multi_key(device_name(), total, table.npat, table.mmax, table.states())
    if not retune:
        hit = lookup(key)
        if hit is not None:
            return hit
    stream = stream or torch.cuda.current_stream()
    sample = _sample(texts, sample_bytes)
    out = torch.zeros(len(texts) * table.npat, dtype=torch.int64, device=texts[0].device)
    timer = _event_timer(lambda cfg: dfa_multi_count(sample, table, out, cfg=cfg, stream=stream),
                         stream)
    cands = multi_candidates(table.mmax)
    best, ms = select_best(cands, timer, reps)
    remember(key, best, ms, len(cands))
    return best


def tune_single(text, table, reps: int = 3, stream=None, retune: bool = False,
                sample_bytes: int = 1 << 30, op: str = "count") -> dict:
    """Best (layout, chunk) of the TMA kernel for one pattern on this text,
    timed on ``op``: "count" (dfa_count) or "find" (dfa_find, count and
    sorted positions, with a workspace of its own)."""
    import torch

    from . import dfa_count, dfa_find, dfa_find_workspace_bytes
    forced = forced_config()
    if forced is not None:
        return forced
    if op not in ("count", "find"):
        raise ValueError(f"tune_single: op {op!r}")
    n = int(text.numel())
    key = single_key(device_name(), n, table.m, op)
    if not retune:
        hit = lookup(key)
        if hit is not None:
            return hit
    stream = stream or torch.cuda.current_stream()
    sample = text[: min(n, sample_bytes) // 64 * 64] if n > sample_bytes else text
    out = torch.zeros(1, dtype=torch.int64, device=text.device)
    if op == "count":
        timer = _event_timer(lambda cfg: dfa_count(sample, table, out, cfg=cfg, stream=stream), stream)
    else:
        cap = [1 << 16]
        pos = [torch.empty(cap[0], dtype=torch.int64, device=text.device)]
        ws = [torch.empty(0, dtype=torch.uint8, device=text.device)]

        def launch(cfg):
            need = dfa_find_workspace_bytes(int(sample.numel()), cfg)
            if need < 0:
                raise ValueError("configuration refused")
            if ws[0].numel() < need:
                ws[0] = torch.empty(need, dtype=torch.uint8, device=text.device)
            dfa_find(sample, table, pos[0], out, ws[0], cfg=cfg, stream=stream)
        timer = _event_timer(launch, stream)
        # size the position buffer once (a truncated find writes only cap)
        launch(None)
        stream.synchronize()
        c = int(out.item())
        if c > cap[0]:
            pos[0] = torch.empty(c, dtype=torch.int64, device=text.device)
    cands = single_candidates(table.m)
    best, ms = select_best(cands, timer, reps)
    remember(key, best, ms, len(cands))
    return best
