// Many patterns over many sequences in one launch: the multi-pattern
// failure-less automaton of Sec. III-B (one automaton for a set of patterns,
// the failure transitions folded into the table so every step is a single
// lookup) and a persistent batched count over up to kMultiMaxSeq sequences.
//
// Automaton: the trie of the patterns over the 2-bit base codes; states are
// numbered in breadth-first order, root 0.  For a state u and code a,
// delta(u, a) is the trie child if there is one, else delta(fail(u), a)
// (the root loops to itself), where fail(v) is the longest proper suffix of
// v's string that is a trie state.  out(v), the patterns ending at v, is v's
// own patterns followed by out(fail(v)).  A device entry holds 4 * next | 1
// when out(next) is not empty, so the next lookup index is the entry with
// its low two bits replaced by the code.
//
// Walk: Algorithm 1 with patterns of several lengths.  A thread owns the
// starts of its chunk [s, e), walks from q0 at s through
// min(e + m_max - 1, n) and keeps pattern p's occurrence ending at j iff it
// starts before e, i.e. j - m_p + 1 < e; every byte outside ACGTacgt sends
// the walk back to q0 (Sec. III-B).  Inside the chunk every occurrence is
// owned, so a step into a state with outputs adds one to that state's
// shared-memory counter; in the overlap the lengths decide (out of line).
// When the CTA moves to another sequence, and at its end, each state's count
// goes to every pattern of its output list in the global per-(sequence,
// pattern) counts.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <array>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <unordered_map>
#include <vector>

#include "dnadfa_internal.h"

using namespace dnadfa;

struct dfa_multi {
    int32_t npat = 0, nstates = 0, mmax = 0;
    std::vector<uint8_t> mlen;          // pattern lengths
    std::vector<uint16_t> delta;        // nstates * 4
    std::vector<uint32_t> out_off;      // nstates + 1
    std::vector<uint16_t> out_ids;      // concatenated output lists
    int device = 0;
    void* d_mem = nullptr;
    int32_t delta_bytes = 0, off_bytes = 0, ids_bytes = 0, mlen_bytes = 0, span_bytes = 0;
    bool owns_mem = true;               // false: d_mem is the caller's (dfa_multi_attach)
    std::vector<uint8_t> img;           // device image, kept until the table is freed
};

namespace {

constexpr int kMultiMaxSeq = 64;
constexpr int kMultiMaxStates = 16383;   // largest state number: 4 * 16383 + 1 fits the u16 entry (16384 states)
constexpr int kMultiMaxPat = 8192;       // per-CTA counters: 32 KiB
// Shared memory per SM that the per-lane table copies may take: the copies
// (4 * 32 * 4 bytes a state) are used when the CTAs of 1024 threads fit in it.
constexpr int64_t kRepSmemPerSm = 200 * 1024;

int round16(int64_t b) { return (int)((b + 15) & ~(int64_t)15); }

struct MultiArgs {
    const uint8_t* text[kMultiMaxSeq];
    int64_t n[kMultiMaxSeq];
    int64_t tile0[kMultiMaxSeq + 1];     // first tile of each sequence; tile0[nseq] = all tiles
    int32_t nseq, npat, mmax, chunk;
    int32_t nstates;
    int32_t delta_bytes;                 // the part copied to shared memory
    const uint8_t* tab;                  // device image: [delta][off][ids][mlen][span]
    const uint32_t* off;                 // output list of state q: ids[off[q] .. off[q+1])
    const uint16_t* ids;
    const uint8_t* mlen;                 // pattern lengths
    const uint8_t* span;                 // per state: shortest and longest output length
    unsigned long long* counts;         // [nseq][npat]
};

// 32 bytes of text (one sector) per load.
__device__ __forceinline__ void ldg32m(const uint8_t* p, uint4& a, uint4& b)
{
    asm volatile("ld.global.nc.L1::no_allocate.v8.u32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(a.x), "=r"(a.y), "=r"(a.z), "=r"(a.w), "=r"(b.x), "=r"(b.y), "=r"(b.z), "=r"(b.w)
                 : "l"(p));
}

// Per byte of x: zero iff the byte is a base (A C G T a c g t).
__device__ __forceinline__ uint32_t word_bad_m(uint32_t x)
{
    uint32_t t = (x >> 2) & ~(x >> 1) & 0x01010101u;
    return ((x ^ (t * 0x11u)) & 0xD9D9D9D9u) ^ 0x41414141u;
}

// Shared-memory view of one CTA: the transition table and one counter per
// automaton state (occurrences of every pattern the state outputs, at owned
// starts); the launch arguments for the rare out-of-line paths.
struct LocateArgs;

struct MultiTab {
    const uint16_t* delta;   // 4 * state + code -> 4 * next | (out(next) not empty)
    const uint32_t* rep;     // per-lane copies: entry i of lane l at rep[32 * i + l]
    uint32_t lane;           // threadIdx.x % 32
    uint32_t* hs;            // this lane's per-state counters: with 2^CG copies a
                             // state, copy g = lane % 2^CG of state q at hs[q << CG]
    const MultiArgs* args;
    unsigned long long* row; // this sequence's per-pattern global counts
    const LocateArgs* loc;   // dfa_multi_locate: where occurrences go
    int64_t s0;              // dfa_multi_locate: text offset of the chunk
};

// dfa_multi_locate: one text, every occurrence written to its pattern's
// segment of pos (base[p] .. base[p] + count[p]) at a slot taken from
// cursor[p]; status bit 0 when a pattern meets more than count[p].
struct LocateArgs {
    const uint8_t* text;
    int64_t n;
    int64_t ntiles;
    int32_t npat, mmax, chunk, nstates;
    int32_t delta_bytes;
    const uint8_t* tab;
    const uint32_t* off;
    const uint16_t* ids;
    const uint8_t* mlen;
    const unsigned long long* base;
    const unsigned long long* count;
    unsigned int* cursor;
    unsigned long long* status;
    int64_t* pos;
};

// Every owned output of state st ending at chunk offset j (owned: inside the
// chunk, or in the overlap d = j - own + 1 bytes past it with m_p > d).
__device__ __noinline__ void locate_out(const LocateArgs* a, uint32_t st, uint32_t j, uint32_t own, int64_t s0)
{
    const uint32_t k1 = __ldg(a->off + st + 1);
    for (uint32_t k = __ldg(a->off + st); k < k1; k++) {
        const uint32_t p = __ldg(a->ids + k);
        const uint32_t m = __ldg(a->mlen + p);
        if (j >= own && m <= j - own + 1u) continue;
        const unsigned int slot = atomicAdd(a->cursor + p, 1u);
        if (slot < __ldg(a->count + p))
            a->pos[__ldg(a->base + p) + slot] = s0 + (int64_t)j - (int64_t)m + 1;
        else
            atomicOr(a->status, 1ull);
    }
}

// A flagged step in the overlap, d = (end offset) - own + 1 >= 1 bytes past
// the chunk: an output of length m_p started before the chunk's end (is
// owned) iff m_p > d.  All of the state's outputs owned: its counter; some:
// those patterns one by one in global memory.
template <int CG>
__device__ __noinline__ void emit_overlap(const MultiArgs* a, uint32_t* hs, unsigned long long* row, uint32_t st,
                                          uint32_t d)
{
    const uint32_t shortest = __ldg(a->span + 2 * st), longest = __ldg(a->span + 2 * st + 1);
    if (longest <= d) return;
    if (shortest > d) {
        atomicAdd(hs + (st << CG), 1u);
        return;
    }
    const uint32_t k1 = __ldg(a->off + st + 1);
    for (uint32_t k = __ldg(a->off + st); k < k1; k++) {
        const uint32_t p = __ldg(a->ids + k);
        if (__ldg(a->mlen + p) > d) atomicAdd(row + p, 1ull);
    }
}

// Output flag set on entry e ending at offset j: owned (CHECK false, or
// j < own) adds one to the state's counter; a locate writes the positions.
template <bool CHECK, bool LOC = false, int CG = 0>
__device__ __forceinline__ void emit(const MultiTab& M, uint32_t e, uint32_t j, uint32_t own)
{
    if (LOC)
        locate_out(M.loc, e >> 2, j, own, M.s0);
    else if (!CHECK || j < own)
        atomicAdd(M.hs + ((e >> 2) << CG), 1u);
    else
        emit_overlap<CG>(M.args, M.hs, M.row, e >> 2, j - own + 1u);
}

// An owned step's output without a branch: the add to the state's counter
// is predicated on the entry's output flag (most steps of a sparse output
// set have none, but some lane of a warp usually does, so a branch would
// send the whole warp through the add).
template <int CG>
__device__ __forceinline__ void emit_owned(const MultiTab& M, uint32_t e)
{
    // one counter a state: a flagged entry is 4 * next + 1, so e - 1 is the
    // byte offset of next's counter
    const uint32_t hs_sa = (uint32_t)__cvta_generic_to_shared(M.hs);
    const uint32_t addr = CG == 0 ? e + (hs_sa - 1u) : hs_sa + (((e >> 2) << CG) << 2);
    asm volatile("{\n\t.reg .pred p;\n\t.reg .b32 f;\n\tand.b32 f, %1, 1;\n\tsetp.ne.u32 p, f, 0;\n\t"
                 "@p red.shared.add.u32 [%0], 1;\n\t}"
                 ::"r"(addr), "r"(e) : "memory");
}

// Four bases of a word w, byte k ending at offset j + k: four dependent
// lookups; owned outputs by predicated adds, the others behind one test of
// the output flags.
// One table lookup.  REP: the lane's own copy of the entry; the 32 copies
// of an entry sit in the 32 banks, so a warp's 32 lookups never conflict.
template <bool REP>
__device__ __forceinline__ uint32_t lookup(const MultiTab& M, uint32_t idx)
{
    if (REP) return M.rep[(idx << 5) | M.lane];
    return M.delta[idx];
}

template <bool CHECK, bool LOC = false, bool REP = false, int CG = 0>
__device__ __forceinline__ void word_bases(const MultiTab& M, uint32_t& ent, uint32_t w, uint32_t j, uint32_t own)
{
    const uint32_t c = (w >> 1) & 0x03030303u;
    const uint32_t e0 = lookup<REP>(M, (ent & ~3u) | (c & 3u));
    const uint32_t e1 = lookup<REP>(M, (e0 & ~3u) | ((c >> 8) & 3u));
    const uint32_t e2 = lookup<REP>(M, (e1 & ~3u) | ((c >> 16) & 3u));
    const uint32_t e3 = lookup<REP>(M, (e2 & ~3u) | (c >> 24));
    ent = e3;
    if (!CHECK && !LOC) {
        emit_owned<CG>(M, e0);
        emit_owned<CG>(M, e1);
        emit_owned<CG>(M, e2);
        emit_owned<CG>(M, e3);
    } else if ((e0 | e1 | e2 | e3) & 1u) {
        if (e0 & 1u) emit<CHECK, LOC, CG>(M, e0, j, own);
        if (e1 & 1u) emit<CHECK, LOC, CG>(M, e1, j + 1, own);
        if (e2 & 1u) emit<CHECK, LOC, CG>(M, e2, j + 2, own);
        if (e3 & 1u) emit<CHECK, LOC, CG>(M, e3, j + 3, own);
    }
}

// One byte, any value: a non-base sends the walk back to q0 (Sec. III-B:
// columns outside the alphabet lead to q0).
template <bool LOC = false, bool REP = false, int CG = 0>
__device__ __forceinline__ void byte_any(const MultiTab& M, uint32_t& ent, uint32_t b, uint32_t j, uint32_t own)
{
    const uint32_t t = (b >> 2) & ~(b >> 1) & 1u;
    if (((b ^ (t * 0x11u)) & 0xD9u) == 0x41u) {
        ent = lookup<REP>(M, (ent & ~3u) | ((b >> 1) & 3u));
        if (ent & 1u) emit<true, LOC, CG>(M, ent, j, own);
    } else {
        ent = 0u;
    }
}

// A word holding bases and non-bases, byte by byte.
template <bool LOC = false, bool REP = false, int CG = 0>
__device__ __forceinline__ uint32_t word_mixed(const MultiTab& M, uint32_t ent, uint32_t w, uint32_t j, uint32_t own)
{
#pragma unroll 1
    for (int k = 0; k < 4; k++) byte_any<LOC, REP, CG>(M, ent, (w >> (8 * k)) & 0xFFu, j + k, own);
    return ent;
}

template <bool CHECK, bool LOC = false, bool REP = false, int CG = 0>
__device__ __forceinline__ void word_any(const MultiTab& M, uint32_t& ent, uint32_t w, uint32_t j, uint32_t own)
{
    const uint32_t bad = word_bad_m(w);
    if (bad == 0u) {
        word_bases<CHECK, LOC, REP, CG>(M, ent, w, j, own);
    } else if (((bad - 0x01010101u) & ~bad & 0x80808080u) == 0u) {
        ent = 0u;                                   // four non-bases (an N block)
    } else {
        ent = word_mixed<LOC, REP, CG>(M, ent, w, j, own);
    }
}

template <bool CHECK, bool LOC = false, bool REP = false, int CG = 0>
__device__ __forceinline__ void vec_any(const MultiTab& M, uint32_t& ent, uint4 v, uint32_t j, uint32_t own)
{
    // one base test for the 16 bytes: all bases (nearly every block) take
    // the four words without a branch between them (not with the per-lane
    // table copies, whose walk it left short of registers)
    if (!REP && (word_bad_m(v.x) | word_bad_m(v.y) | word_bad_m(v.z) | word_bad_m(v.w)) == 0u) {
        word_bases<CHECK, LOC, REP, CG>(M, ent, v.x, j, own);
        word_bases<CHECK, LOC, REP, CG>(M, ent, v.y, j + 4, own);
        word_bases<CHECK, LOC, REP, CG>(M, ent, v.z, j + 8, own);
        word_bases<CHECK, LOC, REP, CG>(M, ent, v.w, j + 12, own);
        return;
    }
    word_any<CHECK, LOC, REP, CG>(M, ent, v.x, j, own);
    word_any<CHECK, LOC, REP, CG>(M, ent, v.y, j + 4, own);
    word_any<CHECK, LOC, REP, CG>(M, ent, v.z, j + 8, own);
    word_any<CHECK, LOC, REP, CG>(M, ent, v.w, j + 12, own);
}

// REP: the table as 32 per-lane copies (4 bytes an entry) instead of one
// (2 bytes an entry), for automata small enough (kMultiRepStates).
// CG: 2^CG copies of each state's counter, lane l adding to copy l % 2^CG
// (the lanes' atomics of a dense output then spread over more banks).
template <int THREADS, bool REP, int CG = 0>
__global__ void __launch_bounds__(THREADS, 1024 / THREADS) k_multi_count(const __grid_constant__ MultiArgs a)
{
    extern __shared__ __align__(16) uint8_t msm[];
    int64_t table_bytes;
    if (REP) {
        const uint16_t* src = reinterpret_cast<const uint16_t*>(a.tab);
        uint32_t* dst = reinterpret_cast<uint32_t*>(msm);
        const int nrep = a.nstates * 4 * 32;
        for (int i = threadIdx.x; i < nrep; i += THREADS) dst[i] = src[i >> 5];
        table_bytes = (int64_t)nrep * 4;
    } else {
        const uint4* src = reinterpret_cast<const uint4*>(a.tab);
        uint4* dst = reinterpret_cast<uint4*>(msm);
        for (int i = threadIdx.x; i < (a.delta_bytes >> 4); i += THREADS) dst[i] = src[i];
        table_bytes = a.delta_bytes;
    }
    MultiTab M;
    M.delta = reinterpret_cast<const uint16_t*>(msm);
    M.rep = reinterpret_cast<const uint32_t*>(msm);
    M.lane = threadIdx.x & 31u;
    uint32_t* const hs0 = reinterpret_cast<uint32_t*>(msm + table_bytes);
    M.hs = hs0 + (M.lane & ((1u << CG) - 1u));
    M.args = &a;
    for (int q = threadIdx.x; q < (a.nstates << CG); q += THREADS) hs0[q] = 0u;
    __syncthreads();

    // the per-state counters go to the per-pattern counts of sequence sq:
    // each pattern of a state's (failure-closed) output list gets its count
    auto flush = [&](int sq) {
        __syncthreads();
        unsigned long long* row = a.counts + (int64_t)sq * a.npat;
        for (int q = threadIdx.x; q < a.nstates; q += THREADS) {
            uint32_t* const hq = hs0 + ((uint32_t)q << CG);
            uint32_t v = 0u;
#pragma unroll
            for (int g = 0; g < (1 << CG); g++) {
                v += hq[g];
                hq[g] = 0u;
            }
            if (v) {
                const uint32_t k1 = __ldg(a.off + q + 1);
                for (uint32_t k = __ldg(a.off + q); k < k1; k++)
                    atomicAdd(row + __ldg(a.ids + k), (unsigned long long)v);
            }
        }
        __syncthreads();
    };

    const int64_t C = a.chunk;
    const int64_t tb = (int64_t)THREADS * C;
    const int64_t total = a.tile0[a.nseq];
    int cur = -1;
    for (int64_t t = blockIdx.x; t < total; t += gridDim.x) {
        int sq = 0;
        while (sq + 1 < a.nseq && a.tile0[sq + 1] <= t) sq++;
        if (sq != cur) {
            if (cur >= 0) flush(cur);
            cur = sq;
            M.row = a.counts + (int64_t)sq * a.npat;
        }
        const int64_t n = a.n[sq];
        const uint8_t* text = a.text[sq];
        const int64_t s = (t - a.tile0[sq]) * tb + (int64_t)threadIdx.x * C;
        if (s >= n) continue;
        const int64_t e = min(s + C, n);
        const int64_t hi = min(e + (int64_t)a.mmax - 1, n);
        const uint32_t own = (uint32_t)(e - s);
        const uint32_t len = (uint32_t)(hi - s);
        const uint8_t* base = text + s;
        uint32_t ent = 0u;
        uint32_t j = 0;
        if ((((uintptr_t)base) & 15u) == 0) {
            if ((((uintptr_t)base) & 31u) != 0 && len >= 16) {
                vec_any<true, false, REP, CG>(M, ent, *reinterpret_cast<const uint4*>(base), 0u, own);
                j = 16;
            }
            // owned 32-byte blocks, the next one in flight while one is walked
            const uint32_t nb = j < own ? (own - j) >> 5 : 0u;
            if (nb) {
                uint4 a0, a1;
                ldg32m(base + j, a0, a1);
#pragma unroll 1
                for (uint32_t g = 0; g < nb; g++) {
                    const uint4 c0 = a0, c1 = a1;
                    if (g + 1 < nb) ldg32m(base + j + 32 * (g + 1), a0, a1);
                    const uint32_t jj = j + 32u * g;
                    vec_any<false, false, REP, CG>(M, ent, c0, jj, own);
                    vec_any<false, false, REP, CG>(M, ent, c1, jj + 16, own);
                }
                j += nb << 5;
            }
            // the rest of the chunk and its overlap, 16 bytes at a time
            for (; j + 16 <= len; j += 16)
                vec_any<true, false, REP, CG>(M, ent, *reinterpret_cast<const uint4*>(base + j), j, own);
        }
        for (; j < len; j++) byte_any<false, REP, CG>(M, ent, base[j], j, own);
    }
    if (cur >= 0) flush(cur);
}

// dfa_multi_locate, pass 1: the walk of k_multi_count over one text, each
// owned occurrence written to its pattern's segment (in no particular order
// within it).
template <int THREADS>
__global__ void __launch_bounds__(THREADS, 1024 / THREADS) k_multi_locate(const __grid_constant__ LocateArgs a)
{
    extern __shared__ __align__(16) uint8_t msm[];
    {
        const uint4* src = reinterpret_cast<const uint4*>(a.tab);
        uint4* dst = reinterpret_cast<uint4*>(msm);
        for (int i = threadIdx.x; i < (a.delta_bytes >> 4); i += THREADS) dst[i] = src[i];
    }
    MultiTab M;
    M.delta = reinterpret_cast<const uint16_t*>(msm);
    M.rep = nullptr;
    M.lane = threadIdx.x & 31u;
    M.hs = nullptr;
    M.args = nullptr;
    M.row = nullptr;
    M.loc = &a;
    __syncthreads();
    const int64_t C = a.chunk;
    const int64_t tb = (int64_t)THREADS * C;
    for (int64_t t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
        const int64_t s = t * tb + (int64_t)threadIdx.x * C;
        if (s >= a.n) continue;
        const int64_t e = min(s + C, a.n);
        const int64_t hi = min(e + (int64_t)a.mmax - 1, a.n);
        const uint32_t own = (uint32_t)(e - s);
        const uint32_t len = (uint32_t)(hi - s);
        const uint8_t* base = a.text + s;
        M.s0 = s;
        uint32_t ent = 0u;
        uint32_t j = 0;
        if ((((uintptr_t)base) & 15u) == 0) {
            for (; j + 16 <= own; j += 16)
                vec_any<false, true>(M, ent, *reinterpret_cast<const uint4*>(base + j), j, own);
            for (; j + 16 <= len; j += 16)
                vec_any<true, true>(M, ent, *reinterpret_cast<const uint4*>(base + j), j, own);
        }
        for (; j < len; j++) byte_any<true>(M, ent, base[j], j, own);
    }
}

// dfa_multi_locate, pass 2: one CTA per pattern sorts its segment (at most
// DFA_LOCATE_MAX positions) in shared memory, bitonically; a segment whose
// slots were not all filled, or overfilled, sets status bit 1.
__global__ void __launch_bounds__(512) k_sort_segments(int64_t* pos, const unsigned long long* base,
                                                       const unsigned long long* count, const unsigned int* cursor,
                                                       unsigned long long* status)
{
    __shared__ long long sv[DFA_LOCATE_MAX];
    const int p = blockIdx.x;
    const int64_t b = (int64_t)base[p];
    const int c = (int)count[p];
    if (threadIdx.x == 0 && cursor[p] != (unsigned int)c) atomicOr(status, 2ull);
    if (c <= 1) return;
    int L = 1;
    while (L < c) L <<= 1;
    for (int i = threadIdx.x; i < L; i += 512) sv[i] = i < c ? pos[b + i] : LLONG_MAX;
    __syncthreads();
    for (int k = 2; k <= L; k <<= 1) {
        for (int jj = k >> 1; jj > 0; jj >>= 1) {
            for (int i = threadIdx.x; i < L; i += 512) {
                const int ixj = i ^ jj;
                if (ixj > i) {
                    const long long x = sv[i], y = sv[ixj];
                    if ((x > y) == ((i & k) == 0)) {
                        sv[i] = y;
                        sv[ixj] = x;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int i = threadIdx.x; i < c; i += 512) pos[b + i] = sv[i];
}

typedef void (*MultiFn)(const MultiArgs);

// The instantiation for threads, the per-lane table copies (rep) or 2^cg
// counter copies (one table copy; cg > 0 only at 512 and 1024 threads,
// where the copies fit beside the table), else null.
MultiFn pick_multi(int threads, bool rep, int cg)
{
    if (rep) {
        if (threads == 128) return k_multi_count<128, true>;
        if (threads == 256) return k_multi_count<256, true>;
        if (threads == 512) return k_multi_count<512, true>;
        if (threads == 1024) return k_multi_count<1024, true>;
        return nullptr;
    }
    if (cg == 0) {
        if (threads == 128) return k_multi_count<128, false>;
        if (threads == 256) return k_multi_count<256, false>;
        if (threads == 512) return k_multi_count<512, false>;
        if (threads == 1024) return k_multi_count<1024, false>;
        return nullptr;
    }
    if (threads == 512) return cg == 1 ? k_multi_count<512, false, 1> : cg == 2 ? k_multi_count<512, false, 2>
                                                                              : k_multi_count<512, false, 3>;
    if (threads == 1024) return cg == 1 ? k_multi_count<1024, false, 1> : cg == 2 ? k_multi_count<1024, false, 2>
                                                                                : k_multi_count<1024, false, 3>;
    return nullptr;
}

int multi_fail(const char* what, cudaError_t err)
{
    char buf[256];
    snprintf(buf, sizeof(buf), "%s: %s", what, cudaGetErrorString(err));
    return set_last_error(DFA_ECUDA, buf);
}

// The table of an automaton whose states are numbered breadth first from
// the root 0: next[s][a] is the state after code a, outs[s] the patterns an
// occurrence of which ends on entering s (each pattern at most once).
int make_multi(int32_t npat, const int32_t* lengths, const std::vector<std::array<int32_t, 4>>& next,
               const std::vector<std::vector<uint16_t>>& outs, dfa_multi** out)
{
    const int S = (int)next.size();
    dfa_multi* t = new (std::nothrow) dfa_multi();
    if (!t) return DFA_ENOMEM;
    t->npat = npat;
    t->nstates = S;
    t->mlen.resize(npat);
    for (int p = 0; p < npat; p++) {
        t->mlen[p] = (uint8_t)lengths[p];
        t->mmax = std::max<int32_t>(t->mmax, lengths[p]);
    }
    t->delta.resize((size_t)S * 4);
    t->out_off.assign(S + 1, 0);
    for (int i = 0; i < S; i++) {
        for (int a = 0; a < 4; a++) {
            const int v = next[i][a];
            t->delta[(size_t)i * 4 + a] = (uint16_t)(4 * v + (outs[v].empty() ? 0 : 1));
        }
        t->out_off[i + 1] = t->out_off[i] + (uint32_t)outs[i].size();
        t->out_ids.insert(t->out_ids.end(), outs[i].begin(), outs[i].end());
    }
    // device image: [delta][out_off][out_ids][mlen], 16-byte aligned parts
    // span[q]: the shortest and longest length among the state's outputs
    std::vector<uint8_t> span((size_t)S * 2, 0);
    for (int i = 0; i < S; i++) {
        uint32_t lo = 255, hi = 0;
        for (uint32_t k = t->out_off[i]; k < t->out_off[i + 1]; k++) {
            lo = std::min<uint32_t>(lo, t->mlen[t->out_ids[k]]);
            hi = std::max<uint32_t>(hi, t->mlen[t->out_ids[k]]);
        }
        span[2 * i] = (uint8_t)(hi ? lo : 0);
        span[2 * i + 1] = (uint8_t)hi;
    }
    t->delta_bytes = round16((int64_t)S * 4 * 2);
    t->off_bytes = round16((int64_t)(S + 1) * 4);
    t->ids_bytes = round16((int64_t)std::max<size_t>(t->out_ids.size(), 1) * 2);
    t->mlen_bytes = round16(npat);
    t->span_bytes = round16((int64_t)S * 2);
    const size_t bytes =
        (size_t)t->delta_bytes + t->off_bytes + t->ids_bytes + t->mlen_bytes + t->span_bytes;
    std::vector<uint8_t>& img = t->img;
    img.assign(bytes, 0);
    uint8_t* q = img.data();
    memcpy(q, t->delta.data(), t->delta.size() * 2);
    q += t->delta_bytes;
    memcpy(q, t->out_off.data(), t->out_off.size() * 4);
    q += t->off_bytes;
    if (!t->out_ids.empty()) memcpy(q, t->out_ids.data(), t->out_ids.size() * 2);
    q += t->ids_bytes;
    memcpy(q, t->mlen.data(), npat);
    q += t->mlen_bytes;
    memcpy(q, span.data(), span.size());
    t->owns_mem = false;
    *out = t;
    return DFA_OK;
}

// ------------------------------------------------------------ class patterns
//
// A class pattern allows a set of bases at each position (the character
// classes of the paper's Table III cells, Sec. IV).  Symbols: a base, an
// IUPAC nucleotide code (R = A/G, Y = C/T, S = C/G, W = A/T, K = G/T,
// M = A/C, B = not A, D = not C, H = not G, V = not T, N = any), either case,
// a bracket set of those, "[CGT]", or the paper's alternation of single
// symbols, "(a|g)".  The text side is unchanged: a text
// byte outside ACGTacgt matches no position.

// Mask over base codes (bit base_code: A 0, C 1, T 2, G 3) of one symbol; 0
// if the byte is not a symbol.
uint32_t symbol_mask(uint32_t c)
{
    constexpr uint32_t A = 1u, C = 2u, T = 4u, G = 8u;
    switch (c | 0x20u) {
    case 'a': return A;
    case 'c': return C;
    case 'g': return G;
    case 't': return T;
    case 'r': return A | G;
    case 'y': return C | T;
    case 's': return C | G;
    case 'w': return A | T;
    case 'k': return G | T;
    case 'm': return A | C;
    case 'b': return C | G | T;
    case 'd': return A | G | T;
    case 'h': return A | C | T;
    case 'v': return A | C | G;
    case 'n': return A | C | G | T;
    default: return 0u;
    }
}

// The per-position masks of a class pattern of len bytes; DFA_EINVAL for an
// empty pattern, an unknown byte, an empty or unclosed bracket or group, a
// group alternative longer than one symbol, or more than DFA_MAX_M
// positions.
int parse_class(const char* s, int32_t len, std::vector<uint8_t>& masks)
{
    masks.clear();
    for (int32_t i = 0; i < len; i++) {
        uint32_t mk = 0u;
        if (s[i] == '[') {
            int32_t j = i + 1;
            for (; j < len && s[j] != ']'; j++) {
                const uint32_t b = symbol_mask((uint8_t)s[j]);
                if (!b) return DFA_EINVAL;
                mk |= b;
            }
            if (j >= len || j == i + 1) return DFA_EINVAL;
            i = j;
        } else if (s[i] == '(') {
            // the paper's notation: an alternation of single symbols, (a|g)
            int32_t j = i + 1;
            bool want_symbol = true;
            for (; j < len && s[j] != ')'; j++) {
                if (want_symbol) {
                    const uint32_t b = symbol_mask((uint8_t)s[j]);
                    if (!b) return DFA_EINVAL;
                    mk |= b;
                } else if (s[j] != '|') {
                    return DFA_EINVAL;
                }
                want_symbol = !want_symbol;
            }
            if (j >= len || want_symbol) return DFA_EINVAL;   // unclosed, empty or ending in '|'
            i = j;
        } else {
            mk = symbol_mask((uint8_t)s[i]);
            if (!mk) return DFA_EINVAL;
        }
        if ((int)masks.size() >= DFA_MAX_M) return DFA_EINVAL;
        masks.push_back((uint8_t)mk);
    }
    return masks.empty() ? DFA_EINVAL : DFA_OK;
}

// The automaton of class patterns by the subset construction.  A state is
// the set of pairs (p, k), k = 1..m_p, such that the last k bytes read match
// the first k positions of pattern p (pair index pos0[p] + k - 1); the root
// is the empty set, which every non-base leads back to.  Code a maps a set to
// the (p, k + 1) of its pairs whose position k allows a, plus (p, 1) for
// every p whose first position allows a; a state outputs each p with
// (p, m_p) in its set.  States are numbered in the order found, breadth
// first.  For patterns of single bases each set is that of one trie node
// (the pattern prefixes that are suffixes of the node's string), found in
// the trie's breadth-first order, so the tables equal the trie
// construction's (up to the order within output lists).
int build_class_automaton(const std::vector<std::vector<uint8_t>>& cls, std::vector<std::array<int32_t, 4>>& next,
                          std::vector<std::vector<uint16_t>>& outs)
{
    const int npat = (int)cls.size();
    std::vector<uint32_t> pos0(npat + 1, 0u);
    for (int p = 0; p < npat; p++) pos0[p + 1] = pos0[p] + (uint32_t)cls[p].size();
    const uint32_t L = pos0[npat];
    std::vector<uint16_t> pat_of(L);
    std::vector<uint8_t> allow_next(L), final_pair(L);   // mask of position k (none at k = m_p)
    std::array<std::vector<uint32_t>, 4> first;
    for (int p = 0; p < npat; p++) {
        const uint32_t m = (uint32_t)cls[p].size();
        for (uint32_t k = 1; k <= m; k++) {
            const uint32_t x = pos0[p] + k - 1;
            pat_of[x] = (uint16_t)p;
            allow_next[x] = k < m ? cls[p][k] : 0u;
            final_pair[x] = k == m;
        }
        for (int a = 0; a < 4; a++)
            if ((cls[p][0] >> a) & 1u) first[a].push_back(pos0[p]);
    }
    // sets keyed by the bytes of their sorted pair indices
    std::unordered_map<std::string, int32_t> id;
    std::vector<const std::string*> sets;
    auto intern = [&](std::string&& key, int32_t& sid) -> bool {
        auto it = id.find(key);
        if (it != id.end()) {
            sid = it->second;
            return true;
        }
        if ((int)sets.size() > kMultiMaxStates) return false;
        auto r = id.emplace(std::move(key), (int32_t)sets.size());
        sid = r.first->second;
        sets.push_back(&r.first->first);
        return true;
    };
    int32_t root;
    intern(std::string(), root);
    std::vector<uint32_t> cur, adv, nxt;
    for (size_t h = 0; h < sets.size(); h++) {
        const std::string& key = *sets[h];
        cur.resize(key.size() / 4);
        if (!cur.empty()) memcpy(cur.data(), key.data(), key.size());
        std::vector<uint16_t> o;
        for (uint32_t x : cur)
            if (final_pair[x]) o.push_back(pat_of[x]);
        outs.push_back(std::move(o));
        std::array<int32_t, 4> nx;
        for (int a = 0; a < 4; a++) {
            adv.clear();
            for (uint32_t x : cur)
                if ((allow_next[x] >> a) & 1u) adv.push_back(x + 1);
            nxt.resize(adv.size() + first[a].size());
            std::merge(adv.begin(), adv.end(), first[a].begin(), first[a].end(), nxt.begin());
            std::string k2;
            if (!nxt.empty()) k2.assign(reinterpret_cast<const char*>(nxt.data()), nxt.size() * 4);
            if (!intern(std::move(k2), nx[a]))
                return set_last_error(DFA_EINVAL, "dfa_multi_build_class: the automaton needs more than 16384 states");
        }
        next.push_back(nx);
    }
    return DFA_OK;
}

// Copies a host-built automaton to a new allocation on the current device.
int upload_multi(dfa_multi* t, const char* what, dfa_multi** out)
{
    const size_t bytes = t->img.size();
    cudaError_t err;
    if ((err = cudaGetDevice(&t->device)) != cudaSuccess || (err = cudaMalloc(&t->d_mem, bytes)) != cudaSuccess) {
        t->d_mem = nullptr;
        delete t;
        return multi_fail(what, err);
    }
    t->owns_mem = true;
    if ((err = cudaMemcpy(t->d_mem, t->img.data(), bytes, cudaMemcpyHostToDevice)) != cudaSuccess) {
        cudaFree(t->d_mem);
        delete t;
        return multi_fail(what, err);
    }
    *out = t;
    return DFA_OK;
}

}  // namespace

extern "C" {

int dfa_multi_build_host(const char* const* patterns, const int32_t* lengths, int32_t npat, dfa_multi** out)
{
    if (!patterns || !lengths || !out || npat < 1 || npat > kMultiMaxPat) return DFA_EINVAL;
    *out = nullptr;
    // trie
    std::vector<std::array<int32_t, 4>> child(1, {-1, -1, -1, -1});
    std::vector<std::vector<uint16_t>> own(1);
    for (int p = 0; p < npat; p++) {
        const int m = lengths[p];
        if (m < 1 || m > DFA_MAX_M || !patterns[p]) return DFA_EINVAL;
        int u = 0;
        for (int j = 0; j < m; j++) {
            const uint32_t c = (uint8_t)patterns[p][j];
            if (!code_valid(c)) return DFA_EINVAL;
            const int a = (int)base_code(c);
            if (child[u][a] < 0) {
                if ((int)child.size() > kMultiMaxStates)
                    return set_last_error(DFA_EINVAL, "dfa_multi_build: the automaton needs more than 16384 states");
                child[u][a] = (int32_t)child.size();
                child.push_back({-1, -1, -1, -1});
                own.emplace_back();
            }
            u = child[u][a];
        }
        own[u].push_back((uint16_t)p);
    }
    const int S = (int)child.size();
    // breadth-first order, failure links, full transitions, output closure
    std::vector<int32_t> order, fail(S, 0), num(S, -1);
    std::vector<std::array<int32_t, 4>> delta(S);
    std::vector<std::vector<uint16_t>> outs(S);
    order.reserve(S);
    order.push_back(0);
    for (size_t h = 0; h < order.size(); h++) {
        const int u = order[h];
        outs[u] = own[u];
        if (u) outs[u].insert(outs[u].end(), outs[fail[u]].begin(), outs[fail[u]].end());
        for (int a = 0; a < 4; a++) {
            const int v = child[u][a];
            if (v >= 0) {
                fail[v] = u ? delta[fail[u]][a] : 0;
                delta[u][a] = v;
                order.push_back(v);
            } else {
                delta[u][a] = u ? delta[fail[u]][a] : 0;
            }
        }
    }
    for (int i = 0; i < S; i++) num[order[i]] = i;      // states numbered breadth first
    std::vector<std::array<int32_t, 4>> next(S);
    std::vector<std::vector<uint16_t>> bouts(S);
    for (int i = 0; i < S; i++) {
        const int u = order[i];
        for (int a = 0; a < 4; a++) next[i][a] = num[delta[u][a]];
        bouts[i] = std::move(outs[u]);
    }
    return make_multi(npat, lengths, next, bouts, out);
}

int dfa_multi_build(const char* const* patterns, const int32_t* lengths, int32_t npat, dfa_multi** out)
{
    if (!out) return DFA_EINVAL;
    dfa_multi* t = nullptr;
    int rc = dfa_multi_build_host(patterns, lengths, npat, &t);
    if (rc) return rc;
    return upload_multi(t, "dfa_multi_build", out);
}

int dfa_multi_build_class_host(const char* const* patterns, const int32_t* lengths, int32_t npat, dfa_multi** out)
{
    if (!patterns || !lengths || !out || npat < 1 || npat > kMultiMaxPat) return DFA_EINVAL;
    *out = nullptr;
    try {
        std::vector<std::vector<uint8_t>> cls(npat);
        std::vector<int32_t> m(npat);
        for (int p = 0; p < npat; p++) {
            if (!patterns[p] || lengths[p] < 1 || parse_class(patterns[p], lengths[p], cls[p]) != DFA_OK) {
                char buf[96];
                snprintf(buf, sizeof(buf), "dfa_multi_build_class: pattern %d is not a class pattern", p);
                return set_last_error(DFA_EINVAL, buf);
            }
            m[p] = (int32_t)cls[p].size();
        }
        std::vector<std::array<int32_t, 4>> next;
        std::vector<std::vector<uint16_t>> outs;
        const int rc = build_class_automaton(cls, next, outs);
        if (rc) return rc;
        return make_multi(npat, m.data(), next, outs, out);
    } catch (const std::bad_alloc&) {
        return DFA_ENOMEM;
    }
}

int dfa_multi_build_class(const char* const* patterns, const int32_t* lengths, int32_t npat, dfa_multi** out)
{
    if (!out) return DFA_EINVAL;
    dfa_multi* t = nullptr;
    int rc = dfa_multi_build_class_host(patterns, lengths, npat, &t);
    if (rc) return rc;
    return upload_multi(t, "dfa_multi_build_class", out);
}

int32_t dfa_multi_pattern_length(const dfa_multi* t, int32_t p)
{
    return t && p >= 0 && p < t->npat ? (int32_t)t->mlen[p] : -1;
}

int64_t dfa_multi_image_bytes(const dfa_multi* t) { return t ? (int64_t)t->img.size() : -1; }

int dfa_multi_attach(dfa_multi* t, void* d_mem, int64_t bytes, void* stream)
{
    if (!t || t->d_mem || !d_mem || (reinterpret_cast<uintptr_t>(d_mem) & 15u) ||
        bytes < (int64_t)t->img.size())
        return DFA_EINVAL;
    cudaError_t err;
    if ((err = cudaGetDevice(&t->device)) != cudaSuccess ||
        (err = cudaMemcpyAsync(d_mem, t->img.data(), t->img.size(), cudaMemcpyHostToDevice,
                               static_cast<cudaStream_t>(stream))) != cudaSuccess)
        return multi_fail("dfa_multi_attach", err);
    t->d_mem = d_mem;
    t->owns_mem = false;
    return DFA_OK;
}

void dfa_multi_free(dfa_multi* t)
{
    if (!t) return;
    if (t->d_mem && t->owns_mem) cudaFree(t->d_mem);
    delete t;
}

int32_t dfa_multi_states(const dfa_multi* t) { return t ? t->nstates : -1; }

int dfa_multi_export(const dfa_multi* t, int32_t* h_next, int32_t* h_nout, int64_t cap_states)
{
    if (!t || cap_states < t->nstates) return DFA_EINVAL;
    for (int i = 0; i < t->nstates; i++) {
        for (int a = 0; a < 4; a++)
            if (h_next) h_next[(size_t)i * 4 + a] = t->delta[(size_t)i * 4 + a] >> 2;
        if (h_nout) h_nout[i] = (int32_t)(t->out_off[i + 1] - t->out_off[i]);
    }
    return DFA_OK;
}

int64_t dfa_multi_smem_bytes(const dfa_multi* t)
{
    if (!t) return -1;
    return (int64_t)t->delta_bytes + (int64_t)t->nstates * 4;
}

int dfa_multi_count(const uint8_t* const* d_texts, const int64_t* lengths, int32_t nseq, const dfa_multi* t,
                    uint64_t* d_counts, const dfa_config* cfg, void* stream)
{
    if (!t || !d_counts || !d_texts || !lengths || nseq < 1 || nseq > kMultiMaxSeq) return DFA_EINVAL;
    if (!t->d_mem) return set_last_error(DFA_EINVAL, "dfa_multi_count: the automaton has no device copy (dfa_multi_attach)");
    const int threads = cfg && cfg->threads ? cfg->threads : 256;
    const int chunk = cfg && cfg->chunk ? cfg->chunk : 1024;
    if (threads != 128 && threads != 256 && threads != 512 && threads != 1024) return DFA_EINVAL;
    if (chunk < 16 || chunk > 32768 || (chunk & 15)) return DFA_EINVAL;
    // table layout: 1 = one shared copy, 2 = 32 per-lane copies, 3..5 = one
    // shared copy and 2, 4 or 8 copies of each state's counter (lane l adds
    // to copy l % copies: the lanes' atomics of a dense output spread over
    // more banks; 512 or 1024 threads), 0 = the per-lane copies when the SM
    // still holds 1024 threads' worth of CTAs, else layout 1
    const int layout = cfg ? cfg->layout : 0;
    if (layout < 0 || layout > 5) return DFA_EINVAL;
    const int64_t rep_smem = (int64_t)t->nstates * (4 * 32 * 4 + 4);
    const bool rep = layout == 2 || (layout == 0 && rep_smem * (1024 / threads) <= kRepSmemPerSm);
    const int cg = layout >= 3 ? layout - 2 : 0;
    int dev;
    cudaError_t err;
    if ((err = cudaGetDevice(&dev)) != cudaSuccess) return multi_fail("dfa_multi_count", err);
    if (dev != t->device) return DFA_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    MultiArgs a;
    memset(&a, 0, sizeof(a));
    const int64_t tb = (int64_t)threads * chunk;
    a.tile0[0] = 0;
    for (int i = 0; i < nseq; i++) {
        if (lengths[i] < 0 || (lengths[i] > 0 && !d_texts[i])) return DFA_EINVAL;
        a.text[i] = d_texts[i];
        a.n[i] = lengths[i];
        a.tile0[i + 1] = a.tile0[i] + (lengths[i] + tb - 1) / tb;
    }
    a.nseq = nseq;
    a.npat = t->npat;
    a.mmax = t->mmax;
    a.chunk = chunk;
    a.delta_bytes = t->delta_bytes;
    a.nstates = t->nstates;
    a.tab = static_cast<const uint8_t*>(t->d_mem);
    a.off = reinterpret_cast<const uint32_t*>(a.tab + t->delta_bytes);
    a.ids = reinterpret_cast<const uint16_t*>(a.tab + t->delta_bytes + t->off_bytes);
    a.mlen = a.tab + t->delta_bytes + t->off_bytes + t->ids_bytes;
    a.span = a.mlen + t->mlen_bytes;
    a.counts = reinterpret_cast<unsigned long long*>(d_counts);
    if ((err = cudaMemsetAsync(d_counts, 0, (size_t)nseq * t->npat * 8, st)) != cudaSuccess)
        return multi_fail("dfa_multi_count", err);
    if (a.tile0[nseq] == 0) return DFA_OK;
    MultiFn fn = pick_multi(threads, rep, cg);
    if (!fn) return set_last_error(DFA_EINVAL, "dfa_multi_count: counter copies need 512 or 1024 threads");
    const int64_t smem64 = rep ? rep_smem : (int64_t)t->delta_bytes + ((int64_t)t->nstates << cg) * 4;
    const int smem = (int)std::min<int64_t>(smem64, INT_MAX);
    int optin = 0, sms = 0;
    if ((err = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess ||
        (err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return multi_fail("dfa_multi_count", err);
    if (smem > optin) return set_last_error(DFA_EINVAL, "dfa_multi_count: the automaton does not fit in shared memory");
    if ((err = cudaFuncSetAttribute((const void*)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) != cudaSuccess)
        return multi_fail("dfa_multi_count", err);
    int occ = 0;
    if ((err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, (const void*)fn, threads, smem)) != cudaSuccess)
        return multi_fail("dfa_multi_count", err);
    if (occ <= 0) return set_last_error(DFA_ECUDA, "dfa_multi_count: kernel does not fit on an SM");
    if (cfg && cfg->ctas_per_sm) occ = std::min(occ, (int)cfg->ctas_per_sm);
    const int64_t grid = std::min<int64_t>(a.tile0[nseq], (int64_t)occ * sms);
    fn<<<(unsigned)grid, threads, smem, st>>>(a);
    if ((err = cudaGetLastError()) != cudaSuccess) return multi_fail("dfa_multi_count", err);
    return DFA_OK;
}

int64_t dfa_multi_locate_work_bytes(int32_t npat)
{
    if (npat < 1 || npat > kMultiMaxPat) return -1;
    return (int64_t)npat * 8 * 2 + (((int64_t)npat * 4 + 15) & ~(int64_t)15) + 16;
}

int dfa_multi_locate(const uint8_t* d_text, int64_t n, const dfa_multi* t, const uint64_t* h_counts, int64_t* d_pos,
                     int64_t cap, void* d_work, int64_t work_bytes, void* stream)
{
    if (!t || !h_counts || !d_work || n < 0 || (n > 0 && !d_text) || cap < 0) return DFA_EINVAL;
    if (!t->d_mem)
        return set_last_error(DFA_EINVAL, "dfa_multi_locate: the automaton has no device copy (dfa_multi_attach)");
    if (work_bytes < dfa_multi_locate_work_bytes(t->npat)) return DFA_EWORKSPACE;
    const int npat = t->npat;
    std::vector<unsigned long long> host((size_t)npat * 2);
    unsigned long long total = 0;
    for (int p = 0; p < npat; p++) {
        if (h_counts[p] > (uint64_t)DFA_LOCATE_MAX)
            return set_last_error(DFA_EINVAL, "dfa_multi_locate: a count above DFA_LOCATE_MAX");
        host[p] = total;
        host[(size_t)npat + p] = h_counts[p];
        total += h_counts[p];
    }
    if ((int64_t)total > cap || (total > 0 && !d_pos)) return DFA_EINVAL;
    int dev;
    cudaError_t err;
    if ((err = cudaGetDevice(&dev)) != cudaSuccess) return multi_fail("dfa_multi_locate", err);
    if (dev != t->device) return DFA_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned long long* w = static_cast<unsigned long long*>(d_work);
    unsigned int* cursor = reinterpret_cast<unsigned int*>(w + 2 * npat);
    unsigned long long* status =
        reinterpret_cast<unsigned long long*>(reinterpret_cast<uint8_t*>(cursor) + (((int64_t)npat * 4 + 15) & ~15));
    // the pageable source is staged before the call returns
    if ((err = cudaMemcpyAsync(w, host.data(), host.size() * 8, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (err = cudaMemsetAsync(cursor, 0, (size_t)npat * 4, st)) != cudaSuccess ||
        (err = cudaMemsetAsync(status, 0, 8, st)) != cudaSuccess)
        return multi_fail("dfa_multi_locate", err);
    const int threads = 256, chunk = 1024;
    LocateArgs a;
    memset(&a, 0, sizeof(a));
    a.text = d_text;
    a.n = n;
    a.ntiles = (n + (int64_t)threads * chunk - 1) / ((int64_t)threads * chunk);
    a.npat = npat;
    a.mmax = t->mmax;
    a.chunk = chunk;
    a.nstates = t->nstates;
    a.delta_bytes = t->delta_bytes;
    a.tab = static_cast<const uint8_t*>(t->d_mem);
    a.off = reinterpret_cast<const uint32_t*>(a.tab + t->delta_bytes);
    a.ids = reinterpret_cast<const uint16_t*>(a.tab + t->delta_bytes + t->off_bytes);
    a.mlen = a.tab + t->delta_bytes + t->off_bytes + t->ids_bytes;
    a.base = w;
    a.count = w + npat;
    a.cursor = cursor;
    a.status = status;
    a.pos = d_pos;
    if (a.ntiles > 0 && total > 0) {
        int optin = 0, sms = 0, occ = 0;
        const int smem = t->delta_bytes;
        if ((err = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess ||
            (err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
            return multi_fail("dfa_multi_locate", err);
        if (smem > optin) return set_last_error(DFA_EINVAL, "dfa_multi_locate: the automaton does not fit in shared memory");
        if ((err = cudaFuncSetAttribute((const void*)k_multi_locate<256>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        smem)) != cudaSuccess ||
            (err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, (const void*)k_multi_locate<256>, threads,
                                                                 smem)) != cudaSuccess)
            return multi_fail("dfa_multi_locate", err);
        if (occ <= 0) return set_last_error(DFA_ECUDA, "dfa_multi_locate: kernel does not fit on an SM");
        const int64_t grid = std::min<int64_t>(a.ntiles, (int64_t)occ * sms);
        k_multi_locate<256><<<(unsigned)grid, threads, smem, st>>>(a);
        if ((err = cudaGetLastError()) != cudaSuccess) return multi_fail("dfa_multi_locate", err);
    }
    k_sort_segments<<<npat, 512, 0, st>>>(d_pos, w, w + npat, cursor, status);
    if ((err = cudaGetLastError()) != cudaSuccess) return multi_fail("dfa_multi_locate", err);
    return DFA_OK;
}

int dfa_multi_locate_status(const void* d_work, int32_t npat, void* stream)
{
    if (!d_work || npat < 1 || npat > kMultiMaxPat) return DFA_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const uint8_t* st_addr =
        static_cast<const uint8_t*>(d_work) + (int64_t)npat * 16 + (((int64_t)npat * 4 + 15) & ~(int64_t)15);
    unsigned long long v = 0;
    cudaError_t err;
    if ((err = cudaStreamSynchronize(st)) != cudaSuccess ||
        (err = cudaMemcpy(&v, st_addr, 8, cudaMemcpyDeviceToHost)) != cudaSuccess)
        return multi_fail("dfa_multi_locate_status", err);
    return v ? DFA_EINVAL : DFA_OK;
}

}  // extern "C"
