"""Seeded synthetic DNA inputs (texts, patterns, planted occurrences).

The one module that feeds both the CPU oracle and the CUDA path.  It draws
random numbers and lays out bytes; it holds none of the scan's arithmetic.
Generators run in C (``synth.c``, built in place with gcc) so that multi-GB
genome-like texts take seconds; every output is a pure function of its seed.

Recipes (stand-ins for the paper's GenBank genomes, Table II, and its 8-mer
patterns, Table III):

* ``uniform_text(n, seed)``: i.i.d. uniform A/C/G/T.
* ``genome_text(n, seed)``: GC 0.41, ~50% soft-masked lower case in geometric
  runs of mean 300, ~5% ``N`` in blocks of geometric mean 50 kb.
* ``pattern(m, seed)``: uniform upper-case A/C/G/T.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libsynth.so")

_lib = None


def build(force: bool = False) -> str:
    """Compile ``synth.c`` into ``_build/libsynth.so`` (OpenMP when available)."""
    src = os.path.join(_HERE, "synth.c")
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
        i64p = ctypes.POINTER(ctypes.c_int64)
        lib.synth_uniform.argtypes = [u8p, ctypes.c_int64, ctypes.c_uint64]
        lib.synth_pattern.argtypes = [u8p, ctypes.c_int32, ctypes.c_uint64]
        lib.synth_genome.argtypes = [u8p, ctypes.c_int64, ctypes.c_uint64, ctypes.c_int32,
                                     ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64]
        lib.synth_plant.argtypes = [u8p, ctypes.c_int64, u8p, ctypes.c_int32, i64p,
                                    ctypes.c_int64, ctypes.c_int32]
        lib.synth_uniform_ints.argtypes = [i64p, ctypes.c_int64, ctypes.c_int64,
                                           ctypes.c_uint64, ctypes.c_uint64]
        lib.synth_draw.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64]
        lib.synth_draw.restype = ctypes.c_uint64
        lib.synth_geometric.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                        ctypes.c_uint64]
        lib.synth_geometric.restype = ctypes.c_int64
        _lib = lib
    return _lib


def _u8(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


def _i64(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def empty_text(n: int, out: np.ndarray | None = None) -> np.ndarray:
    if out is None:
        return np.empty(int(n), dtype=np.uint8)
    assert out.dtype == np.uint8 and out.flags.c_contiguous and out.size >= n
    return out[:n]


def uniform_text(n: int, seed: int, out: np.ndarray | None = None) -> np.ndarray:
    """i.i.d. uniform upper-case A/C/G/T text of n bytes."""
    t = empty_text(n, out)
    if n:
        _load().synth_uniform(_u8(t), int(n), int(seed) & (2**64 - 1))
    return t


def genome_text(n: int, seed: int, *, gc: bool = True, mask_mean: int = 300,
                n_gap_mean: int = 950_000, n_run_mean: int = 50_000,
                out: np.ndarray | None = None) -> np.ndarray:
    """Genome-like text: GC 0.41, soft-masked runs, N blocks (see module doc).

    ``mask_mean=0`` disables soft-masking and ``n_gap_mean=0`` the N blocks.
    """
    t = empty_text(n, out)
    if n:
        _load().synth_genome(_u8(t), int(n), int(seed) & (2**64 - 1), 1 if gc else 0,
                             int(mask_mean), int(n_gap_mean), int(n_run_mean))
    return t


def pattern(m: int, seed: int) -> bytes:
    """Uniform upper-case A/C/G/T pattern of length m."""
    p = np.empty(int(m), dtype=np.uint8)
    if m:
        _load().synth_pattern(_u8(p), int(m), int(seed) & (2**64 - 1))
    return p.tobytes()


def uniform_ints(k: int, bound: int, seed: int, stream: int = 7) -> np.ndarray:
    """k seeded uniform integers in [0, bound)."""
    out = np.empty(int(k), dtype=np.int64)
    if k:
        _load().synth_uniform_ints(_i64(out), int(k), int(bound), int(seed) & (2**64 - 1),
                                   int(stream))
    return out


def plant(text: np.ndarray, pat: bytes, positions, keep_case: bool = True) -> np.ndarray:
    """Overwrite ``text`` in place with ``pat`` at each position (skipping
    positions that would run past the end)."""
    pos = np.ascontiguousarray(np.asarray(positions, dtype=np.int64))
    p = np.frombuffer(pat, dtype=np.uint8).copy()
    _load().synth_plant(_u8(text), int(text.size), _u8(p), len(pat), _i64(pos),
                        int(pos.size), 1 if keep_case else 0)
    return text


def draw(seed: int, stream: int, k: int) -> int:
    return int(_load().synth_draw(int(seed) & (2**64 - 1), int(stream), int(k)))


def geometric(seed: int, stream: int, k: int, mean: int) -> int:
    return int(_load().synth_geometric(int(seed) & (2**64 - 1), int(stream), int(k), int(mean)))


def random_text(n: int, seed: int, alphabet: bytes = b"ACGT") -> np.ndarray:
    """Seeded text over an arbitrary byte alphabet (for edge-case tests)."""
    idx = uniform_ints(n, len(alphabet), seed, stream=11)
    return np.frombuffer(alphabet, dtype=np.uint8)[idx].copy()


if __name__ == "__main__":  # pragma: no cover
    build(force="--force" in sys.argv)
    print(_SO)


def query_trace(k: int, rate: float, nseq: int, seed: int, max_patterns: int = 64,
                m_lo: int = 4, m_hi: int = 64) -> list[dict]:
    """k seeded pattern queries with Poisson arrivals at ``rate`` per second:
    each {"t": arrival offset in s, "seq": uniform in [0, nseq), "patterns":
    1..max_patterns uniform patterns of length uniform in [m_lo, m_hi],
    "mode": "count" or "positions" with probability 1/2}.  Inter-arrival gaps
    are -ln(U)/rate with U uniform in (0, 1]."""
    import math
    gaps = uniform_ints(k, 1 << 53, seed, stream=11)
    seqs = uniform_ints(k, nseq, seed, stream=12)
    npats = uniform_ints(k, max_patterns, seed, stream=13) + 1
    modes = uniform_ints(k, 2, seed, stream=14)
    out, t = [], 0.0
    for i in range(k):
        t += -math.log((int(gaps[i]) + 1) / float(1 << 53)) / rate
        lens = uniform_ints(int(npats[i]), m_hi - m_lo + 1, seed * 1_000_003 + i, stream=15) + m_lo
        pats = [pattern(int(m), (seed << 24) + (i << 7) + j) for j, m in enumerate(lens)]
        out.append({"t": t, "seq": int(seqs[i]), "patterns": pats,
                    "mode": "positions" if modes[i] else "count"})
    return out


_RC = bytes.maketrans(b"ACGT", b"TGCA")


def class_pattern_pairs(npairs: int, seed: int, m: int = 8) -> list:
    """Seeded character-class patterns shaped like the class cells of the
    paper's Table III (Sec. IV): a uniform m-mer with one position widened to
    the three bases other than its own ("[CGT]" where the m-mer has A), then
    the reverse complement of that pattern (the widened set complemented),
    so 2 * npairs patterns.  Returns (class pattern, its plain expansions)
    pairs; the expansions are the m-mers the class pattern stands for."""
    out = []
    for i in range(npairs):
        w = pattern(m, seed * 1000 + i)
        j = int(uniform_ints(1, m, seed * 1000 + i, stream=11)[0])
        others = bytes(b for b in b"ACGT" if b != w[j])
        exp = [w[:j] + bytes([b]) + w[j + 1:] for b in others]
        cls = w[:j] + b"[" + others + b"]" + w[j + 1:]
        out.append((cls, exp))
        rexp = [e.translate(_RC)[::-1] for e in exp]
        k = m - 1 - j
        rw = w.translate(_RC)[::-1]
        rothers = bytes(sorted(others.translate(_RC)))
        out.append((rw[:k] + b"[" + rothers + b"]" + rw[k + 1:], rexp))
    return out
