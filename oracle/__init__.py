"""CPU oracle for the finite-automaton DNA pattern scan — TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg (and its ``--impl reference`` arm) may import this package.  The product
path (``paper_1506_08612_gb300``) never imports it, and the two share no code.

The arithmetic lives in ``oracle.c`` (plain C, compiled here with gcc); this
module only marshals numpy arrays.  Functions:

* ``find_brute(text, pattern)`` — the result by its definition (Sec. II-A):
  every window compared; returns ``(count, positions)``.
* ``dfa_delta(pattern)`` — the string-matching automaton's transition function
  built from its definition (Sec. II-A).
* ``dfa_scan(text, delta, m)`` — sequential automaton walk.
* ``alg1_scan(text, delta, m, p, v)`` — Algorithm 1's decomposition (Sec. III-A).
* ``stt_ascii(strings, finals)`` — sparse 256-column STT (Sec. III-B, Table I).
* ``kmer_census(text, k)`` and ``valid_windows(text, k)``.
* ``find_set(text, patterns)`` and ``count_set(texts, patterns)`` — the
  definition for a set of patterns: each window start compared with every
  pattern, the comparisons of patterns sharing a prefix done once (a trie
  descent per start; no failure links), threaded over contiguous ranges.
* ``class_sets(pattern)``, ``class_expansions(pattern)`` and
  ``find_class_brute(text, pattern)`` — character-class patterns (the class
  cells of Table III, Sec. IV) by their definition, in numpy.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``_build/liboracle.so`` (OpenMP when available)."""
    src = os.path.join(_HERE, "oracle.c")
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(src):
        return _SO
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _SO + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", src, "-o", tmp]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       stdout=subprocess.PIPE, stderr=subprocess.PIPE)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True)
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        u8p = ctypes.POINTER(ctypes.c_uint8)
        i32p = ctypes.POINTER(ctypes.c_int32)
        i64p = ctypes.POINTER(ctypes.c_int64)
        u64p = ctypes.POINTER(ctypes.c_uint64)
        i64, i32 = ctypes.c_int64, ctypes.c_int32
        lib.oracle_find_brute.argtypes = [u8p, i64, u8p, i32, i64p, i64]
        lib.oracle_find_brute.restype = i64
        lib.oracle_dfa_delta.argtypes = [u8p, i32, i32p]
        lib.oracle_dfa_delta.restype = ctypes.c_int
        lib.oracle_dfa_scan.argtypes = [u8p, i64, i32p, i32, i64p, i64]
        lib.oracle_dfa_scan.restype = i64
        lib.oracle_alg1_lane_starts.argtypes = [i64, i64, i64, i64, i64p]
        lib.oracle_alg1_lane_starts.restype = ctypes.c_int
        lib.oracle_alg1_scan.argtypes = [u8p, i64, i32p, i32, i64, i64, i32, i64p, i64, i64p]
        lib.oracle_alg1_scan.restype = i64
        lib.oracle_stt_ascii.argtypes = [u8p, i32p, i32p, i32, i32p, i32, i32p, i32p, i32p]
        lib.oracle_stt_ascii.restype = i32
        lib.oracle_kmer_census.argtypes = [u8p, i64, i32, u64p]
        lib.oracle_kmer_census.restype = ctypes.c_int
        lib.oracle_valid_windows.argtypes = [u8p, i64, i32]
        lib.oracle_valid_windows.restype = i64
        lib.oracle_find_set.argtypes = [u8p, i64, u8p, i32p, i32, u64p, i64p, i64p, i32]
        lib.oracle_find_set.restype = ctypes.c_int
        lib.oracle_num_threads.argtypes = []
        lib.oracle_num_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _bytes(x) -> np.ndarray:
    if isinstance(x, (bytes, bytearray)):
        return np.frombuffer(bytes(x), dtype=np.uint8).copy()
    if isinstance(x, str):
        return np.frombuffer(x.encode("ascii"), dtype=np.uint8).copy()
    a = np.ascontiguousarray(x, dtype=np.uint8)
    return a


def _p(a: np.ndarray, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


class OracleError(ValueError):
    pass


def find_brute(text, pattern, cap: int | None = None):
    """(count, sorted int64 start positions) of every occurrence, by definition."""
    t = _bytes(text)
    p = _bytes(pattern)
    lib = _load()
    n = int(t.size)
    if cap is None:
        cnt = lib.oracle_find_brute(_p(t, ctypes.c_uint8), n, _p(p, ctypes.c_uint8), int(p.size),
                                    None, 0)
        if cnt < 0:
            raise OracleError("invalid pattern")
        cap = cnt
    pos = np.empty(max(int(cap), 1), dtype=np.int64)
    cnt = lib.oracle_find_brute(_p(t, ctypes.c_uint8), n, _p(p, ctypes.c_uint8), int(p.size),
                                _p(pos, ctypes.c_int64), int(cap))
    if cnt < 0:
        raise OracleError("invalid pattern")
    return int(cnt), pos[: min(int(cnt), int(cap))].copy()


def count_brute(text, pattern) -> int:
    t = _bytes(text)
    p = _bytes(pattern)
    cnt = _load().oracle_find_brute(_p(t, ctypes.c_uint8), int(t.size), _p(p, ctypes.c_uint8),
                                    int(p.size), None, 0)
    if cnt < 0:
        raise OracleError("invalid pattern")
    return int(cnt)


def dfa_delta(pattern) -> np.ndarray:
    """delta as an (m+1, 4) int32 array, columns A, C, G, T."""
    p = _bytes(pattern)
    m = int(p.size)
    d = np.zeros((m + 1) * 4, dtype=np.int32)
    if m < 1 or _load().oracle_dfa_delta(_p(p, ctypes.c_uint8), m, _p(d, ctypes.c_int32)) != 0:
        raise OracleError("invalid pattern")
    return d.reshape(m + 1, 4)


def dfa_scan(text, delta: np.ndarray, m: int, cap: int | None = None):
    t = _bytes(text)
    d = np.ascontiguousarray(delta, dtype=np.int32).ravel()
    lib = _load()
    if cap is None:
        cap = lib.oracle_dfa_scan(_p(t, ctypes.c_uint8), int(t.size), _p(d, ctypes.c_int32), m,
                                  None, 0)
    pos = np.empty(max(int(cap), 1), dtype=np.int64)
    cnt = lib.oracle_dfa_scan(_p(t, ctypes.c_uint8), int(t.size), _p(d, ctypes.c_int32), m,
                              _p(pos, ctypes.c_int64), int(cap))
    return int(cnt), pos[: min(int(cnt), int(cap))].copy()


def alg1_lane_starts(n: int, p: int, v: int, chunk: int = 0) -> list[int]:
    out = np.zeros(v, dtype=np.int64)
    if _load().oracle_alg1_lane_starts(n, p, v, chunk, _p(out, ctypes.c_int64)) != 0:
        raise OracleError("invalid arguments")
    return [int(x) for x in out]


def alg1_scan(text, delta: np.ndarray, m: int, p: int, v: int, nthreads: int = 1,
              want_positions: bool = True):
    """Algorithm 1: returns (count, positions or None, automaton steps)."""
    t = _bytes(text)
    d = np.ascontiguousarray(delta, dtype=np.int32).ravel()
    lib = _load()
    steps = ctypes.c_int64(0)
    if not want_positions:
        cnt = lib.oracle_alg1_scan(_p(t, ctypes.c_uint8), int(t.size), _p(d, ctypes.c_int32), m,
                                   p, v, nthreads, None, 0, ctypes.byref(steps))
        return int(cnt), None, int(steps.value)
    cnt = lib.oracle_alg1_scan(_p(t, ctypes.c_uint8), int(t.size), _p(d, ctypes.c_int32), m,
                               p, v, nthreads, None, 0, None)
    if cnt < 0:
        raise OracleError("invalid arguments")
    pos = np.empty(max(int(cnt), 1), dtype=np.int64)
    cnt = lib.oracle_alg1_scan(_p(t, ctypes.c_uint8), int(t.size), _p(d, ctypes.c_int32), m,
                               p, v, nthreads, _p(pos, ctypes.c_int64), int(cnt),
                               ctypes.byref(steps))
    return int(cnt), pos[: int(cnt)].copy(), int(steps.value)


def stt_ascii(strings, finals=None):
    """Sparse ASCII STT of the failure-less automaton of ``strings``.

    Returns (stt[int32 states x 256], f, state_strings) where state_strings[q]
    is the (upper-case) string of state q.
    """
    strs = [s.encode() if isinstance(s, str) else bytes(s) for s in strings]
    if finals is None:
        finals = [True] * len(strs)
    buf = np.frombuffer(b"".join(strs), dtype=np.uint8).copy()
    lens = np.array([len(s) for s in strs], dtype=np.int32)
    fin = np.array([1 if f else 0 for f in finals], dtype=np.int32)
    cap = int(lens.sum()) + 1
    stt = np.zeros(cap * 256, dtype=np.int32)
    src = np.zeros(cap, dtype=np.int32)
    ln = np.zeros(cap, dtype=np.int32)
    f = ctypes.c_int32(0)
    ns = _load().oracle_stt_ascii(_p(buf, ctypes.c_uint8), _p(lens, ctypes.c_int32),
                                  _p(fin, ctypes.c_int32), len(strs), _p(stt, ctypes.c_int32), cap,
                                  ctypes.byref(f), _p(src, ctypes.c_int32), _p(ln, ctypes.c_int32))
    if ns < 0:
        raise OracleError("invalid strings")
    upper = [s.upper() for s in strs]
    names = [upper[src[q]][: ln[q]].decode() for q in range(ns)]
    return stt[: ns * 256].reshape(ns, 256).copy(), int(f.value), names


def kmer_census(text, k: int) -> np.ndarray:
    t = _bytes(text)
    h = np.zeros(4 ** k, dtype=np.uint64)
    if _load().oracle_kmer_census(_p(t, ctypes.c_uint8), int(t.size), k, _p(h, ctypes.c_uint64)) != 0:
        raise OracleError("invalid k")
    return h


def valid_windows(text, k: int) -> int:
    t = _bytes(text)
    return int(_load().oracle_valid_windows(_p(t, ctypes.c_uint8), int(t.size), k))


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def multi_count(texts, patterns, threads: int | None = None) -> np.ndarray:
    """Counts of every pattern (overlaps included) in every text, by the
    definition (Sec. II-A, one brute-force window compare per pattern):
    uint64[len(texts), len(patterns)].  The independent (text, pattern)
    compares run on ``threads`` host threads (default: all cores); each is
    the same single-threaded C loop."""
    from concurrent.futures import ThreadPoolExecutor
    out = np.zeros((len(texts), len(patterns)), dtype=np.uint64)
    ts = [_bytes(t) for t in texts]
    jobs = [(i, j) for i in range(len(ts)) for j in range(len(patterns))]
    with ThreadPoolExecutor(max_workers=threads or os.cpu_count() or 1) as ex:
        for (i, j), c in zip(jobs, ex.map(lambda ij: count_brute(ts[ij[0]], patterns[ij[1]]), jobs)):
            out[i, j] = c
    return out


def _pattern_block(patterns):
    ps = [p.encode() if isinstance(p, str) else bytes(p) for p in patterns]
    if not ps:
        raise OracleError("no patterns")
    buf = np.frombuffer(b"".join(ps), dtype=np.uint8).copy()
    lens = np.array([len(p) for p in ps], dtype=np.int32)
    return buf, lens


def find_set(text, patterns, positions: bool = True, threads: int | None = None):
    """(uint64 counts[len(patterns)], list of sorted int64 position arrays or
    None) of every pattern of a set in one text, by the definition (every
    window start compared with every pattern; Sec. II-A)."""
    t = _bytes(text)
    buf, lens = _pattern_block(patterns)
    lib = _load()
    nt = int(threads or num_threads())
    counts = np.zeros(lens.size, dtype=np.uint64)
    if lib.oracle_find_set(_p(t, ctypes.c_uint8), int(t.size), _p(buf, ctypes.c_uint8),
                           _p(lens, ctypes.c_int32), int(lens.size), _p(counts, ctypes.c_uint64),
                           None, None, nt) != 0:
        raise OracleError("invalid pattern")
    if not positions:
        return counts, None
    off = np.zeros(lens.size, dtype=np.int64)
    off[1:] = np.cumsum(counts.astype(np.int64))[:-1]
    pos = np.empty(max(int(counts.sum()), 1), dtype=np.int64)
    again = np.zeros_like(counts)
    if lib.oracle_find_set(_p(t, ctypes.c_uint8), int(t.size), _p(buf, ctypes.c_uint8),
                           _p(lens, ctypes.c_int32), int(lens.size), _p(again, ctypes.c_uint64),
                           _p(pos, ctypes.c_int64), _p(off, ctypes.c_int64), nt) != 0:
        raise OracleError("invalid pattern")
    return counts, [pos[o:o + int(c)].copy() for o, c in zip(off, counts)]


def count_set(texts, patterns, threads: int | None = None) -> np.ndarray:
    """uint64[len(texts), len(patterns)]: find_set's counts of every pattern
    in every text."""
    return np.stack([find_set(t, patterns, positions=False, threads=threads)[0] for t in texts])


# ------------------------------------------------------------ class patterns
#
# A class pattern allows a set of bases at each position (the class cells of
# the paper's Table III, Sec. IV).  Symbols are the IUPAC nucleotide codes
# (a base stands for itself); a bracket joins the sets of the symbols inside,
# and so does the paper's group of single symbols separated by "|".

IUPAC = {"A": "A", "C": "C", "G": "G", "T": "T",
         "R": "AG", "Y": "CT", "S": "CG", "W": "AT", "K": "GT", "M": "AC",
         "B": "CGT", "D": "AGT", "H": "ACT", "V": "ACG", "N": "ACGT"}


def class_sets(pattern) -> list[str]:
    """The bases (upper case, sorted) each position of a class pattern
    allows; ValueError for an empty pattern, an unknown symbol, an empty or
    unclosed bracket, or more than 64 positions."""
    s = pattern.decode("ascii") if isinstance(pattern, (bytes, bytearray)) else str(pattern)
    out, i = [], 0
    while i < len(s):
        if s[i] == "[":
            j = s.find("]", i + 1)
            if j < 0 or j == i + 1:
                raise ValueError(f"bad bracket in {s!r}")
            members = set()
            for ch in s[i + 1:j]:
                if ch.upper() not in IUPAC:
                    raise ValueError(f"bad symbol {ch!r} in {s!r}")
                members |= set(IUPAC[ch.upper()])
            out.append("".join(sorted(members)))
            i = j + 1
        elif s[i] == "(":
            # the paper's notation for a class: single symbols separated by |
            j = s.find(")", i + 1)
            if j < 0:
                raise ValueError(f"unclosed group in {s!r}")
            members = set()
            for alt in s[i + 1:j].split("|"):
                if len(alt) != 1 or alt.upper() not in IUPAC:
                    raise ValueError(f"bad alternative {alt!r} in {s!r}")
                members |= set(IUPAC[alt.upper()])
            out.append("".join(sorted(members)))
            i = j + 1
        else:
            if s[i].upper() not in IUPAC:
                raise ValueError(f"bad symbol {s[i]!r} in {s!r}")
            out.append(IUPAC[s[i].upper()])
            i += 1
    if not out or len(out) > 64:
        raise ValueError(f"{len(out)} positions in {s!r}")
    return out


def class_expansions(pattern) -> list[bytes]:
    """Every plain pattern the class pattern stands for."""
    import itertools
    return [("".join(t)).encode() for t in itertools.product(*class_sets(pattern))]


def find_class_brute(text, pattern):
    """Every window compared (the definition): an occurrence at i iff each
    byte T[i + j] is a base, either case, in the set of position j.  Returns
    ``(count, sorted start positions)``."""
    t = _bytes(text)
    sets = class_sets(pattern)
    m, n = len(sets), t.size
    if n < m:
        return 0, np.zeros(0, np.int64)
    ok = np.ones(n - m + 1, dtype=bool)
    for j, bases in enumerate(sets):
        allowed = np.zeros(256, dtype=bool)
        for b in bases:
            allowed[ord(b)] = allowed[ord(b.lower())] = True
        ok &= allowed[t[j:n - m + 1 + j]]
    pos = np.flatnonzero(ok).astype(np.int64)
    return int(pos.size), pos


def multi_count_class(texts, patterns) -> np.ndarray:
    """uint64[len(texts), len(patterns)]: find_class_brute counts."""
    out = np.zeros((len(texts), len(patterns)), dtype=np.uint64)
    for i, t in enumerate(texts):
        for j, p in enumerate(patterns):
            out[i, j] = find_class_brute(t, p)[0]
    return out
