"""Serving loop: genomes resident in HBM, pattern queries arriving over time.

The paper scans one genome per program run and advises keeping the data on
the coprocessor (Sec. II-B).  A server keeps every sequence resident on the
GPU and answers queries {sequence, patterns, mode} as they arrive:

* **Continuous batching.**  Each scheduler iteration takes the arrivals,
  polls the work in flight (CUDA events, never a blocking wait) and, while
  a stream slot is free, forms a batch from the waiting queries of one
  sequence (the oldest query's sequence, then every other waiting query on
  it, up to ``max_batch_patterns`` distinct patterns).  Batches on different
  slots run on different CUDA streams, so new work overlaps with work
  already on the device.
* **Count stage.**  The batch's distinct patterns become one multi-pattern
  failure-less automaton (Sec. III-B) and one persistent launch counts them
  all over the sequence.  Count-mode queries are answered from it.
* **Admission by position memory.**  A positions-mode query needs 8 bytes
  per occurrence.  After the count stage those sizes are exact; the batch's
  positions are admitted when they fit in the position arena (a fixed
  device buffer, first-fit), in arrival order, and wait otherwise.  A request
  larger than the whole arena fails with an error instead of waiting forever.
* **Find stage.**  The distinct positions patterns with at most
  DFA_LOCATE_MAX occurrences are located together: one walk of their
  multi-pattern automaton writes each occurrence into its pattern's segment
  of the admitted region and each segment is sorted on the device
  (dfa_multi_locate); every other one by the single-pattern find (exact
  count as capacity).  The region is copied back in one transfer.

The GPU work sits behind an engine interface (``GpuEngine``) so the
scheduler's policy can run against a stand-in engine on the CPU.
"""
from __future__ import annotations

import collections
import threading
import time
from dataclasses import dataclass, field

import numpy as np

from . import DFA_MAX_M
from .batched import MAX_STATES, group_patterns


# ------------------------------------------------------------------ queries

@dataclass
class Query:
    seq: int
    patterns: list
    mode: str = "count"                  # "count" | "positions"
    t_arrive: float = 0.0                # perf_counter seconds
    qid: int = -1
    t_done: float = 0.0
    counts: np.ndarray | None = None     # uint64[len(patterns)]
    positions: list | None = None        # per pattern, sorted int64 start positions
    error: str | None = None
    batch: int = -1                      # id of the batch that served it
    _keys: set | None = field(default=None, repr=False, compare=False)
    _prefixes: set | None = field(default=None, repr=False, compare=False)

    @property
    def latency(self) -> float:
        return self.t_done - self.t_arrive


def _key(p) -> bytes:
    b = p.encode() if isinstance(p, str) else bytes(p)
    return b.upper()


_LETTERS = frozenset(b"ACGTacgt")


def query_error(q: Query, nseq: int | None = None) -> str | None:
    """Why the query cannot be served (None if it can): an unknown mode or
    sequence, no patterns, or a pattern that is not 1 to DFA_MAX_M letters
    of {A,C,G,T} (either case), the alphabet of Sec. III-A."""
    if q.mode not in ("count", "positions"):
        return f"unknown mode {q.mode!r}"
    if nseq is not None and not (isinstance(q.seq, (int, np.integer)) and 0 <= q.seq < nseq):
        return f"no sequence {q.seq!r} (the server holds {nseq})"
    if not q.patterns:
        return "no patterns"
    for p in q.patterns:
        try:
            b = p.encode("ascii") if isinstance(p, str) else bytes(p)
        except (UnicodeEncodeError, TypeError, ValueError):
            return f"pattern {p!r} is not a byte string of ACGT letters"
        if not 1 <= len(b) <= DFA_MAX_M or not _LETTERS.issuperset(b):
            return f"pattern {b[:80]!r}: 1 to {DFA_MAX_M} letters of ACGT expected"
    return None


# ------------------------------------------------------------------ arena

class Arena:
    """First-fit allocator over [0, size) with coalescing of free blocks.
    Offsets and sizes are multiples of ``align`` bytes."""

    def __init__(self, size: int, align: int = 256):
        self.size = int(size) // align * align
        self.align = align
        self.free = [(0, self.size)]          # sorted (offset, length)
        self.used = 0

    def alloc(self, nbytes: int):
        n = max(self.align, (int(nbytes) + self.align - 1) // self.align * self.align)
        for i, (off, ln) in enumerate(self.free):
            if ln >= n:
                if ln == n:
                    self.free.pop(i)
                else:
                    self.free[i] = (off + n, ln - n)
                self.used += n
                return off, n
        return None

    def release(self, off: int, n: int) -> None:
        self.used -= n
        fl = self.free
        lo, hi = 0, len(fl)
        while lo < hi:
            mid = (lo + hi) // 2
            if fl[mid][0] < off:
                lo = mid + 1
            else:
                hi = mid
        fl.insert(lo, (off, n))
        # coalesce with the next, then the previous block
        if lo + 1 < len(fl) and fl[lo][0] + fl[lo][1] == fl[lo + 1][0]:
            fl[lo] = (fl[lo][0], fl[lo][1] + fl[lo + 1][1])
            fl.pop(lo + 1)
        if lo > 0 and fl[lo - 1][0] + fl[lo - 1][1] == fl[lo][0]:
            fl[lo - 1] = (fl[lo - 1][0], fl[lo - 1][1] + fl[lo][1])
            fl.pop(lo)


# ------------------------------------------------------------------ batches

@dataclass
class Batch:
    bid: int
    seq: int
    queries: list
    patterns: list                        # distinct upper-case patterns
    index: dict                           # pattern -> column
    state: str = "count"                  # count -> (wait_mem -> find) -> done
    job: object = None
    counts: np.ndarray | None = None
    find_patterns: list = field(default_factory=list)
    region: tuple | None = None           # (offset, bytes) in the position arena


def host_automata(dd, patterns):
    """(groups, host automata) for ``patterns``: one automaton over all of
    them when the library takes the set (the batches are formed to fit),
    else one per group of group_patterns (a single query too large for one
    automaton)."""
    try:
        return [list(range(len(patterns)))], [dd.MultiTable(patterns, device=False)]
    except dd.DfaError as e:
        if e.code != dd.DFA_EINVAL or len(patterns) < 2:
            raise
    groups = group_patterns(patterns)
    return groups, [dd.MultiTable([patterns[i] for i in g], device=False) for g in groups]


class GpuEngine:
    """The device side of the server: resident sequences, stream slots, the
    position arena, and the two stages as non-blocking jobs."""

    def __init__(self, sequences, slots: int = 4, arena_bytes: int = 8 << 30,
                 table_bytes: int = 64 << 20, device=None, plain: bool = False, locate: bool | None = None):
        """plain=True counts and locates with one single-pattern launch per
        pattern instead of the multi-pattern automaton (the unbatched form,
        for comparison); locate (default: not plain) locates the patterns
        with few occurrences together in one walk."""
        import torch

        import paper_1506_08612_gb300 as dd
        self.dd = dd
        self.torch = torch
        self.seqs = list(sequences)
        self.device = device or self.seqs[0].device
        self.nslots = slots
        self.nseq = len(self.seqs)
        self.streams = [torch.cuda.Stream(self.device) for _ in range(slots)]
        nmax = max(int(s.numel()) for s in self.seqs)
        self.ws = [torch.empty(dd.dfa_find_workspace_bytes(nmax), dtype=torch.uint8, device=self.device)
                   for _ in range(slots)]
        self.tab = [torch.empty(table_bytes, dtype=torch.uint8, device=self.device) for _ in range(slots)]
        self.arena_bytes = int(arena_bytes)
        self.arena = torch.empty(self.arena_bytes // 8, dtype=torch.int64, device=self.device)
        self.plain = plain
        self.locate = (not plain) if locate is None else bool(locate)
        # the slots' streams are non-blocking: the sequences' contents must be
        # on the device before the first batch reads them
        torch.cuda.current_stream(self.device).synchronize()

    # -- count stage: one multi-pattern launch over the batch's sequence
    def launch_count(self, slot: int, seq: int, patterns):
        dd, torch = self.dd, self.torch
        st = self.streams[slot]
        if self.plain:
            return self._launch_count_plain(slot, seq, patterns)
        # one automaton per group of patterns within its limits (a batch is
        # formed to need one; a single query may need several)
        groups, mts = host_automata(dd, patterns)
        sizes = [(mt.image_bytes() + 255) // 256 * 256 for mt in mts]
        if sum(sizes) > self.tab[slot].numel():
            self.tab[slot] = torch.empty(sum(sizes), dtype=torch.uint8, device=self.device)
        with torch.cuda.stream(st):
            out = torch.empty(len(patterns), dtype=torch.int64, device=self.device)
            toff = 0
            for g, mt, sz in zip(groups, mts, sizes):
                mt.attach(self.tab[slot][toff:toff + sz], stream=st)
                dd.dfa_multi_count([self.seqs[seq]], mt, out[g[0]:g[-1] + 1], stream=st)
                toff += sz
            host = torch.empty(len(patterns), dtype=torch.int64, pin_memory=True)
            host.copy_(out, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(st)
        return {"ev": ev, "host": host, "keep": (mts, out)}

    def _launch_count_plain(self, slot, seq, patterns):
        dd, torch = self.dd, self.torch
        st = self.streams[slot]
        need = sum((dd.dfa_table_bytes(len(p)) + 255) // 256 * 256 for p in patterns)
        if need > self.tab[slot].numel():
            self.tab[slot] = torch.empty(need, dtype=torch.uint8, device=self.device)
        tabs = []
        with torch.cuda.stream(st):
            out = torch.empty(len(patterns), dtype=torch.int64, device=self.device)
            toff = 0
            for i, p in enumerate(patterns):
                tb = dd.dfa_table_bytes(len(p))
                t = dd.Table(p, into=self.tab[slot][toff:toff + tb], stream=st)
                toff += (tb + 255) // 256 * 256
                tabs.append(t)
                dd.dfa_count(self.seqs[seq], t, out[i:i + 1], stream=st)
            host = torch.empty(len(patterns), dtype=torch.int64, pin_memory=True)
            host.copy_(out, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(st)
        return {"ev": ev, "host": host, "keep": (tabs, out)}

    # -- find stage: positions of the batch's positions patterns into the
    #    admitted arena region, then one copy of the region to the host.
    #    Patterns with at most DFA_LOCATE_MAX occurrences are located
    #    together in one walk of their multi-pattern automaton (each
    #    pattern's segment sorted on the device); the others by the
    #    single-pattern find, one each.
    def launch_find(self, slot: int, seq: int, patterns, counts, region):
        dd, torch = self.dd, self.torch
        st = self.streams[slot]
        off, nbytes = region
        base = off // 8
        counts = [int(c) for c in counts]
        sparse = [i for i, c in enumerate(counts) if 0 < c <= dd.DFA_LOCATE_MAX] if self.locate else []
        sset = set(sparse)
        dense = [i for i, c in enumerate(counts) if c and i not in sset]
        order = sparse + dense                         # layout of the region
        sgroups, mts = host_automata(dd, [patterns[i] for i in sparse]) if sparse else ([], [])
        sgroups = [[sparse[j] for j in g] for g in sgroups]
        msizes = [(mt.image_bytes() + 255) // 256 * 256 for mt in mts]
        mt_bytes = sum(msizes)
        need = mt_bytes + sum((dd.dfa_table_bytes(len(patterns[i])) + 255) // 256 * 256 for i in dense)
        if need > self.tab[slot].numel():
            self.tab[slot] = torch.empty(need, dtype=torch.uint8, device=self.device)
        text = self.seqs[seq]
        total = sum(counts)
        tabs = []
        with torch.cuda.stream(st):
            cnt = torch.zeros(max(len(patterns), 1), dtype=torch.int64, device=self.device)
            poff = base
            toff = 0
            for g, mt, sz in zip(sgroups, mts, msizes):
                mt.attach(self.tab[slot][toff:toff + sz], stream=st)
                toff += sz
                work = torch.empty(dd.dfa_multi_locate_work_bytes(len(g)), dtype=torch.uint8,
                                   device=self.device)
                ns = sum(counts[i] for i in g)
                dd.dfa_multi_locate(text, mt, [counts[i] for i in g], self.arena[poff:poff + ns], work,
                                    stream=st)
                poff += ns
                tabs.append((mt, work))
            for i in dense:
                p, c = patterns[i], counts[i]
                tb = dd.dfa_table_bytes(len(p))
                t = dd.Table(p, into=self.tab[slot][toff:toff + tb], stream=st)
                toff += (tb + 255) // 256 * 256
                tabs.append(t)
                dd.dfa_find(text, t, self.arena[poff:poff + c], cnt[i:i + 1], self.ws[slot], stream=st)
                poff += c
            host = torch.empty(max(total, 1), dtype=torch.int64, pin_memory=True)
            host[:total].copy_(self.arena[base:base + total], non_blocking=True)
            hcnt = torch.empty(cnt.numel(), dtype=torch.int64, pin_memory=True)
            hcnt.copy_(cnt, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(st)
        return {"ev": ev, "host": host, "hcnt": hcnt, "keep": tabs, "counts": counts, "order": order,
                "dense": dense}

    @staticmethod
    def done(job) -> bool:
        return job["ev"].query()

    @staticmethod
    def count_result(job) -> np.ndarray:
        return job["host"].numpy().astype(np.uint64)

    @staticmethod
    def find_result(job):
        counts = job["counts"]
        got = job["hcnt"].numpy()
        for i in job["dense"]:
            if int(got[i]) != counts[i]:
                raise RuntimeError("find counts differ from the count stage")
        # views into the batch's pinned buffer (no second copy); the buffer
        # lives as long as any of them
        h = job["host"].numpy()
        out = [np.zeros(0, np.int64) for _ in counts]
        o = 0
        for i in job["order"]:
            out[i] = h[o:o + counts[i]]
            o += counts[i]
        for t in job["keep"]:
            if isinstance(t, tuple):
                t[0].free()
            else:
                t.free()
        return out


class Server:
    """Continuous-batching scheduler over an engine (see module doc)."""

    def __init__(self, engine, max_batch_patterns: int = 2048, clock=time.perf_counter,
                 max_batch_queries: int = 1 << 30):
        self.engine = engine
        self.clock = clock
        self.max_batch_patterns = max_batch_patterns
        self.max_batch_queries = max_batch_queries
        self.arena = Arena(engine.arena_bytes)
        self.free_slots = collections.deque(range(engine.nslots))
        self.waiting = {}                      # sequence -> FIFO of queries not yet in a batch
        self.n_waiting = 0
        self.mem_wait = collections.deque()   # batches waiting for position memory
        self.find_ready = collections.deque() # admitted batches waiting for a slot
        self.active = []                       # (batch, slot) with a job in flight
        self.done = []
        self._lock = threading.Lock()
        self._inbox = collections.deque()
        self._next_q = 0
        self._next_b = 0
        self.stats = collections.Counter()

    # -- public API
    def submit(self, q: Query) -> Query:
        """Queue a query; one that cannot be served completes at once with
        ``error`` set (see query_error)."""
        err = query_error(q, getattr(self.engine, "nseq", None))
        with self._lock:
            if q.qid < 0:
                q.qid = self._next_q
            self._next_q = max(self._next_q, q.qid + 1)
            if not q.t_arrive:
                q.t_arrive = self.clock()
            if err is None:
                self._inbox.append(q)
            else:
                q.error = err
                q.t_done = self.clock()
                self.done.append(q)
                self.stats["rejected_queries"] += 1
        return q

    def idle(self) -> bool:
        return not (self._inbox or self.n_waiting or self.mem_wait or self.find_ready or self.active)

    def step(self) -> int:
        """One scheduler iteration; returns how many state changes it made."""
        moved = 0
        with self._lock:
            while self._inbox:
                q = self._inbox.popleft()
                self.waiting.setdefault(q.seq, collections.deque()).append(q)
                self.n_waiting += 1
                moved += 1
        moved += self._poll()
        moved += self._admit()
        moved += self._launch_finds()
        moved += self._launch_counts()
        return moved

    def run_until_idle(self, poll_s: float = 0.0):
        while not self.idle():
            if not self.step() and poll_s:
                time.sleep(poll_s)

    def replay(self, trace, speed: float = 1.0, poll_s: float = 0.0):
        """Open-loop replay of a trace (dicts with t, seq, patterns, mode):
        each query arrives at its scheduled time, the latency is measured from
        that time.  Returns the completed queries in arrival order."""
        t0 = self.clock()
        order = sorted(range(len(trace)), key=lambda i: trace[i]["t"])
        qs = [None] * len(trace)
        k = 0
        while k < len(order) or not self.idle():
            now = self.clock()
            while k < len(order) and t0 + trace[order[k]]["t"] / speed <= now:
                e = trace[order[k]]
                qs[order[k]] = self.submit(Query(seq=e["seq"], patterns=list(e["patterns"]),
                                                 mode=e["mode"], t_arrive=t0 + e["t"] / speed,
                                                 qid=order[k]))
                k += 1
            if not self.step() and poll_s:
                time.sleep(poll_s)
        return qs

    # -- internals
    def _finish(self, q: Query, now: float):
        q.t_done = now
        self.done.append(q)

    def _poll(self) -> int:
        moved = 0
        still = []
        for b, slot in self.active:
            if not self.engine.done(b.job):
                still.append((b, slot))
                continue
            moved += 1
            self.free_slots.append(slot)
            now = self.clock()
            if b.state == "count":
                b.counts = self.engine.count_result(b.job)
                b.job = None
                need = set()
                for q in b.queries:
                    q.counts = np.array([b.counts[b.index[_key(p)]] for p in q.patterns], dtype=np.uint64)
                    if q.mode == "count":
                        self._finish(q, now)
                    else:
                        need.update(_key(p) for p in q.patterns)
                if need:
                    b.find_patterns = sorted(need, key=lambda k: b.index[k])
                    b.state = "wait_mem"
                    self.mem_wait.append(b)
                else:
                    b.state = "done"
                    self.stats["batches"] += 1
            else:                                   # find stage done
                pos = self.engine.find_result(b.job)
                b.job = None
                self.arena.release(*b.region)
                got = dict(zip(b.find_patterns, pos))
                for q in b.queries:
                    if q.mode == "positions" and q.error is None:
                        q.positions = [got[_key(p)] for p in q.patterns]
                        self._finish(q, now)
                b.state = "done"
                self.stats["batches"] += 1
        self.active = still
        return moved

    def _admit(self) -> int:
        moved = 0
        while self.mem_wait:
            b = self.mem_wait[0]
            nbytes = 8 * sum(int(b.counts[b.index[k]]) for k in b.find_patterns)
            if nbytes > self.arena.size:
                self.mem_wait.popleft()
                now = self.clock()
                for q in b.queries:
                    if q.mode == "positions":
                        q.error = (f"positions need {nbytes} bytes, more than the {self.arena.size}-byte"
                                   " position arena")
                        self._finish(q, now)
                self.stats["rejected_batches"] += 1
                moved += 1
                continue
            r = self.arena.alloc(max(nbytes, 8))
            if r is None:
                self.stats["mem_stalls"] += 1
                break                               # arrival order: wait for memory
            b.region = r
            self.mem_wait.popleft()
            self.find_ready.append(b)
            moved += 1
        return moved

    def _launch_finds(self) -> int:
        moved = 0
        while self.find_ready and self.free_slots:
            b = self.find_ready.popleft()
            slot = self.free_slots.popleft()
            counts = [int(b.counts[b.index[k]]) for k in b.find_patterns]
            b.job = self.engine.launch_find(slot, b.seq, b.find_patterns, counts, b.region)
            b.state = "find"
            self.active.append((b, slot))
            moved += 1
        return moved

    @staticmethod
    def _query_keys(q):
        """The query's distinct case-folded patterns and every prefix of
        them (its trie states), computed once."""
        if q._keys is None:
            keys = {_key(p) for p in q.patterns}
            q._keys = keys
            q._prefixes = {k[:i] for k in keys for i in range(len(k) + 1)}
        return q._keys, q._prefixes

    def _launch_counts(self) -> int:
        moved = 0
        while self.n_waiting and self.free_slots:
            # the sequence whose oldest waiting query arrived first, then its
            # queries in arrival order while the automaton's limits allow
            seq = min((d[0].t_arrive, sq) for sq, d in self.waiting.items() if d)[1]
            queue = self.waiting[seq]
            take = []
            index = {}
            prefixes = {b""}                        # the trie's states: distinct prefixes
            while queue:
                q = queue[0]
                keys, pfx = self._query_keys(q)
                new = keys - index.keys()
                grow = len(pfx - prefixes)
                if take and (len(index) + len(new) > self.max_batch_patterns
                             or len(prefixes) + grow > MAX_STATES
                             or len(take) >= self.max_batch_queries):
                    break
                for p in q.patterns:
                    k = _key(p)
                    if k not in index:
                        index[k] = len(index)
                prefixes |= pfx
                take.append(queue.popleft())
            self.n_waiting -= len(take)
            b = Batch(bid=self._next_b, seq=seq, queries=take, patterns=list(index), index=index)
            self._next_b += 1
            for q in take:
                q.batch = b.bid
            slot = self.free_slots.popleft()
            b.job = self.engine.launch_count(slot, seq, b.patterns)
            self.active.append((b, slot))
            self.stats["queries_batched"] += len(take)
            moved += 1
        return moved


def latency_summary(queries) -> dict:
    """Throughput and latency percentiles of completed queries."""
    ok = [q for q in queries if q is not None and q.t_done and q.error is None]
    if not ok:
        return {"completed": 0}
    lat = np.sort(np.array([q.latency for q in ok]))
    span = max(q.t_done for q in ok) - min(q.t_arrive for q in ok)

    def pct(p):
        return float(lat[min(len(lat) - 1, int(np.ceil(p / 100.0 * len(lat))) - 1)])

    return {"completed": len(ok), "errors": sum(1 for q in queries if q is not None and q.error),
            "qps": len(ok) / span if span > 0 else float("inf"),
            "p50_ms": pct(50) * 1e3, "p99_ms": pct(99) * 1e3, "max_ms": float(lat[-1]) * 1e3,
            "mean_ms": float(lat.mean()) * 1e3}
