"""Many patterns over many sequences in one persistent, graph-captured launch.

The paper scans one genome per program run.  Here a batch of patterns of
uneven length over sequences of uneven size is counted in one persistent
kernel launch per automaton: the patterns become one failure-less
multi-pattern automaton (Sec. III-B), each CTA takes tiles of (sequence,
offset) in turn, and every thread walks its chunk plus the m_max - 1 byte
overlap of Algorithm 1.  The launch is captured once in a CUDA graph and
replayed, so a repeated batch costs one graph launch on the host.

Pattern sets whose automaton would exceed the kernel's limits (8192 patterns,
16384 states) are split into groups, one automaton and one launch each,
all inside the same graph; more than 64 sequences are split the same way.
The chunk length and threads per CTA come from the autotuner unless given.
"""
from __future__ import annotations

import numpy as np

from . import DFA_EINVAL, DfaError, MultiTable, autotune, dfa_multi_count

MAX_SEQ_PER_LAUNCH = 64
MAX_PAT_PER_TABLE = 8192
MAX_STATES = 16384                 # trie states, the root included


def new_prefixes(prefixes: set, pattern) -> list:
    """Prefixes of ``pattern`` (case folded) not yet in ``prefixes``: the
    trie states it would add to an automaton holding those prefixes."""
    p = (pattern.encode() if isinstance(pattern, str) else bytes(pattern)).upper()
    out = []
    for k in range(len(p), 0, -1):
        q = p[:k]
        if q in prefixes:
            break
        out.append(q)
    return out


def group_patterns(patterns, max_states: int = MAX_STATES, max_pat: int = MAX_PAT_PER_TABLE):
    """Split pattern indices into consecutive groups whose automaton fits:
    a group's trie has one state per distinct prefix (the empty one
    included), counted exactly as patterns are added."""
    groups, cur, seen = [], [], {b""}
    for i, p in enumerate(patterns):
        add = new_prefixes(seen, p)
        if cur and (len(seen) + len(add) > max_states or len(cur) >= max_pat):
            groups.append(cur)
            cur, seen = [], {b""}
            add = new_prefixes(seen, p)
        cur.append(i)
        seen.update(add)
    if cur:
        groups.append(cur)
    return groups


def class_groups(patterns, lo: int = 0, hi: int | None = None) -> list:
    """Consecutive index groups of character-class patterns whose automata
    the library takes: the whole range if it does, else each half in turn
    (a class automaton's size is known only once it is built)."""
    hi = len(patterns) if hi is None else hi
    try:
        MultiTable(patterns[lo:hi], device=False, classes=True).free()
        return [list(range(lo, hi))]
    except DfaError as e:
        if e.code != DFA_EINVAL or hi - lo < 2:
            raise
    mid = (lo + hi) // 2
    return class_groups(patterns, lo, mid) + class_groups(patterns, mid, hi)


class BatchedCount:
    """Counts of every pattern in every sequence (overlaps included).

    texts: device uint8 tensors (kept referenced; their contents may change
    between runs, their storage may not).  patterns: bytes/str.  cfg:
    "auto" (autotuner), None (library default) or a dfa_config dict.
    classes: read the patterns as character-class patterns (IUPAC codes,
    bracket sets; dfa_multi_build_class).
    ``run()`` enqueues the whole batch on ``stream`` (one graph replay when
    captured), after the work already enqueued on the caller's current
    stream (writes into the texts, for instance); ``result()`` waits and
    returns uint64[nseq, npat].
    """

    def __init__(self, texts, patterns, cfg="auto", stream=None, capture: bool = True,
                 classes: bool = False):
        import torch

        if not texts:
            raise ValueError("no sequences")
        self.texts = list(texts)
        self.device = self.texts[0].device
        self.patterns = [p.encode() if isinstance(p, str) else bytes(p) for p in patterns]
        if not self.patterns:
            raise ValueError("no patterns")
        self.stream = stream if stream is not None else torch.cuda.Stream(self.device)
        self.groups = class_groups(self.patterns) if classes else group_patterns(self.patterns)
        self.tables = [MultiTable([self.patterns[i] for i in g], classes=classes) for g in self.groups]
        self.seq_groups = [list(range(i, min(i + MAX_SEQ_PER_LAUNCH, len(self.texts))))
                           for i in range(0, len(self.texts), MAX_SEQ_PER_LAUNCH)]
        self.out = [[torch.zeros(len(sg) * t.npat, dtype=torch.int64, device=self.device)
                     for t in self.tables] for sg in self.seq_groups]
        # the outputs were zeroed, and the texts written, on the caller's
        # stream; ``stream`` is a separate (non-blocking) stream
        self.stream.wait_stream(torch.cuda.current_stream(self.device))
        if cfg == "auto":
            with torch.cuda.stream(self.stream):
                self.cfgs = [autotune.tune_multi(self.texts, t, stream=self.stream)
                             for t in self.tables]
        else:
            self.cfgs = [cfg] * len(self.tables)
        self.launches = len(self.tables) * len(self.seq_groups)
        self.graph = None
        # first run eagerly: loads the kernel and sets its shared-memory limit
        # outside any capture
        self._enqueue()
        self.stream.synchronize()
        if capture:
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=self.stream):
                self._enqueue()
            self.graph = g

    def _enqueue(self):
        for si, sg in enumerate(self.seq_groups):
            seqs = [self.texts[i] for i in sg]
            for ti, t in enumerate(self.tables):
                dfa_multi_count(seqs, t, self.out[si][ti], cfg=self.cfgs[ti], stream=self.stream)

    def run(self):
        """Enqueue the batch (asynchronous), ordered after the work already
        enqueued on the caller's current stream."""
        import torch
        self.stream.wait_stream(torch.cuda.current_stream(self.device))
        if self.graph is not None:
            with torch.cuda.stream(self.stream):
                self.graph.replay()
        else:
            self._enqueue()

    def result(self) -> np.ndarray:
        """Wait for the last run and return uint64[nseq, npat]."""
        self.stream.synchronize()
        res = np.zeros((len(self.texts), len(self.patterns)), dtype=np.uint64)
        for si, sg in enumerate(self.seq_groups):
            for ti, g in enumerate(self.groups):
                block = self.out[si][ti].cpu().numpy().astype(np.uint64).reshape(len(sg), len(g))
                res[np.ix_(sg, g)] = block
        return res

    def close(self):
        self.stream.synchronize()
        self.graph = None
        for t in self.tables:
            t.free()
        self.tables = []
