// Finite-automaton DNA pattern scan for GB300 (sm_103a): kernels and C ABI.
//
// The walk is the one of Algorithm 1 (Memeti & Pllana 2015, Sec. III-A):
// the text is cut into per-thread chunks, each thread walks its chunk from
// q0 and carries on m-1 bytes into its successor's chunk (Fig. 2a), so every
// occurrence is found by exactly the thread whose chunk holds its start.
// GPU-first choices (the paper's Xeon Phi design is prior art):
//   * a warp's 32 lanes play the role of the paper's SIMD lanes (Fig. 2b),
//     each lane walking its own contiguous chunk;
//   * the transition table lives in shared memory; the default layout is a
//     four-step composite table over 2-bit base codes, so one lookup
//     advances the automaton by four bytes; the paper's sparse 256-column
//     STT (Sec. III-B, Table I) is kept as a selectable layout;
//   * the default kernel (k_scan_tma) is persistent, one CTA per SM: tiles
//     of 512 rows x C bytes, each walker warp streaming its 32 rows through
//     a ring of TMA boxes (64 bytes x 32 rows) in shared memory; unaligned
//     or short texts take 16-byte vector loads (k_count / k_find);
//   * bytes outside A/C/G/T/a/c/g/t reset the walk to q0 (Sec. III-B).  The
//     walk reads bytes through their 2-bit codes alone (a non-base read as
//     the base of its code never hides an occurrence) and the exact test
//     runs only where that walk accepted: for short patterns the stage is
//     tested with the 8 bytes before it, for patterns of 8 and more the
//     flagged stages are walked again exactly at the end of the tile;
//   * counts are reduced by warp shuffles, then one atomic per CTA;
//   * positions are written in text order.  Patterns of 8 and more: a count
//     pass leaving per-row counts and stage masks, a scan of the tile totals,
//     and an exact re-walk of the masked bytes of the rows that accepted.
//     Shorter patterns: one pass in which tiles are taken in order from an
//     atomic ticket, a CTA learns its tile's global offset by decoupled
//     look-back over its predecessors' published sums, and writes its
//     positions there.  Every wait is bounded and reports DFA_ETIMEOUT
//     instead of hanging.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <type_traits>

#include "dnadfa_internal.h"

using namespace dnadfa;

namespace {

constexpr int kLayoutK4 = 1;
constexpr int kLayoutStt = 2;
constexpr int kLayoutK4S = 3;     // four-step table of states only (u8)
constexpr int kLayoutK4F = 4;     // four-step states with accept flag (u8), m >= kOptMinM
constexpr int kOptMinM = 8;       // default: layout 4 (relaxed walk + exact replay) from here on
constexpr int kSlots = 16;                  // staged positions per thread per tile
constexpr unsigned long long kFlagAgg = 1ull << 62;
constexpr unsigned long long kFlagPre = 2ull << 62;
constexpr unsigned long long kValMask = kFlagAgg - 1;
constexpr unsigned kSpinLimit = 1u << 21;   // ~2 s with the back-off below
constexpr int kWorkHeader = 2;              // [0] ticket, [1] status

struct ScanArgs {
    const uint8_t* text;
    int64_t n;            // readable bytes
    int64_t n_own;        // occurrences must start before n_own (<= n)
    int64_t chunk;        // bytes per thread per tile, multiple of 16
    int64_t ntiles;
    const uint8_t* tab;   // device table allocation
    int32_t m;
    int32_t k4_bytes, d1_bytes, stt_bytes, k4s_bytes, k4f_bytes;
    int32_t aligned;      // text is 16-byte aligned
    unsigned long long* count;
    int64_t* pos;
    int64_t cap;
    int64_t pos_base;                     // added to every position written
    const unsigned long long* base_in;    // running total of earlier segments (or null)
    unsigned long long* work;             // [ticket, status, desc[ntiles]]
};

// Tables in shared memory, as 32-bit shared-window addresses.
struct SmemTab {
    uint32_t k4;    // (m+1)*256 u16
    uint32_t d1;    // (m+1)*4 u8
    uint32_t stt;   // (m+1)*256 u8
    uint32_t k4s;   // (m+1)*256 u8
    uint32_t m;
    uint32_t sh;    // k4s: a group of four steps can accept only from a state with (q >> sh) != 0
    uint32_t force; // k4s: 1 when m <= 4 (any state, even q0, may accept within four steps)
    uint32_t fl;    // k4f: the accept flag (smallest power of two above m)
};

// Dynamic shared memory of every kernel here.  Each kernel puts its layout's
// main table (k4, k4s or stt) at offset 0, so a lookup is one load whose base
// the compiler folds into the instruction.
extern __shared__ __align__(1024) uint8_t g_smem[];

__device__ __forceinline__ uint32_t lds_u8(uint32_t addr)
{
    uint32_t v;
    asm("ld.shared.u8 %0, [%1];" : "=r"(v) : "r"(addr));
    return v;
}

// main-table lookups at offset 0 of dynamic shared memory
__device__ __forceinline__ uint32_t tab16(uint32_t idx)
{
    return reinterpret_cast<const uint16_t*>(g_smem)[idx];
}

__device__ __forceinline__ uint32_t tab8(uint32_t idx)
{
    return g_smem[idx];
}

// ---------------------------------------------------------------- helpers

__device__ __forceinline__ uint4 ldg16(const uint4* p)
{
    uint4 v;
    asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
}

__device__ __forceinline__ void st_release(unsigned long long* p, unsigned long long v)
{
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long* p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Zero iff all four bytes of x are bases (A C G T a c g t), see code_valid.
__device__ __forceinline__ uint32_t word_bad(uint32_t x)
{
    uint32_t t = (x >> 2) & ~(x >> 1) & 0x01010101u;
    return ((x ^ (t * 0x11u)) & 0xD9D9D9D9u) ^ 0x41414141u;
}

// Four automaton steps on the four bases of x, from the state in byte 0 of e.
// (x & 0x06060606) holds the 2-bit codes at bits 8k+1; the multiply gathers
// them, first byte lowest, into bits 24..31 without carries; byte_perm forms
// the table index (state << 8) | code4.
// The u16 table sits at shared offset 0, or at shared address k4 in layout 4
// (behind its flagged table, used there by the exact replays only).
template <int LAYOUT = kLayoutK4>
__device__ __forceinline__ uint32_t k4_next(uint32_t k4, uint32_t e, uint32_t x)
{
    uint32_t code = (x & 0x06060606u) * 0x00820820u;
    uint32_t idx = __byte_perm(code, e, 0x7743u);
    if (LAYOUT == kLayoutK4F) {
        uint32_t v;
        asm("ld.shared.u16 %0, [%1];" : "=r"(v) : "r"(k4 + idx * 2u));
        return v;
    }
    return tab16(idx);
}

// One automaton step on one raw byte (any byte value).
__device__ __forceinline__ uint32_t byte_next(uint32_t d1, uint32_t q, uint32_t c)
{
    uint32_t t = (c >> 2) & ~(c >> 1) & 1u;
    bool ok = ((c ^ (t * 0x11u)) & 0xD9u) == 0x41u;
    uint32_t nq = lds_u8(d1 + q * 4u + ((c >> 1) & 3u));
    return ok ? nq : 0u;
}

// Bits i (i < 4) of an accept mask whose end offset r + i is below lim.
__device__ __forceinline__ uint32_t lim_mask(uint32_t r, uint32_t lim)
{
    if (lim <= r) return 0u;
    uint32_t d = lim - r;
    return d >= 4 ? 0xFu : ((1u << d) - 1u);
}

// ---------------------------------------------------------------- sinks

struct CountSink {
    static constexpr bool kRecord = false;
    __device__ __forceinline__ void put(uint32_t) {}
};

// Stages end offsets (relative to the chunk start) in shared memory,
// slot j of thread t at slots[j * stride + t].
struct SlotSink {
    static constexpr bool kRecord = true;
    uint16_t* slots;
    uint32_t stride;
    uint32_t cap;
    uint32_t n;
    bool over;
    __device__ __forceinline__ void put(uint32_t off)
    {
        if (n < cap)
            slots[n * stride] = (uint16_t)off;
        else
            over = true;
        n++;
    }
};

// Writes positions straight to global memory (overflow re-walk).
struct GlobalSink {
    static constexpr bool kRecord = true;
    int64_t* pos;
    int64_t cap;
    int64_t idx;
    int64_t start0;       // start position of end offset 0
    __device__ __forceinline__ void put(uint32_t off)
    {
        if (idx < cap) pos[idx] = start0 + (int64_t)off;
        idx++;
    }
};

// ---------------------------------------------------------------- walk

template <int LAYOUT, bool LIM, class Sink>
struct Walker {
    const SmemTab& T;
    Sink& sink;
    uint32_t e;      // K4: entry (state in byte 0); STT: state
    uint32_t cnt;

    __device__ __forceinline__ void accept_mask(uint32_t acc, uint32_t r)
    {
        if (Sink::kRecord) {
            while (acc) {
                uint32_t i = __ffs(acc) - 1;
                sink.put(r + i);
                acc &= acc - 1;
            }
        }
    }

    __device__ __forceinline__ void word_k4(uint32_t x, uint32_t r, uint32_t lim)
    {
        e = k4_next<LAYOUT>(T.k4, e, x);
        if (LIM) {
            uint32_t acc = ((e >> K4_ACC_SHIFT) & 0xFu) & lim_mask(r, lim);
            cnt += __popc(acc);
            accept_mask(acc, r);
        } else {
            cnt += e >> K4_CNT_SHIFT;
            if (Sink::kRecord) {
                uint32_t acc = (e >> K4_ACC_SHIFT) & 0xFu;
                if (acc) accept_mask(acc, r);
            }
        }
    }

    __device__ __forceinline__ void byte_d1(uint32_t c, uint32_t r, uint32_t lim)
    {
        e = byte_next(T.d1, e, c);
        if (e == T.m && (!LIM || r < lim)) {
            cnt++;
            if (Sink::kRecord) sink.put(r);
        }
    }

    // Four exact single steps on a word of four bases (no base test).
    __device__ __forceinline__ void word_exact(uint32_t x, uint32_t r, uint32_t lim)
    {
#pragma unroll
        for (uint32_t i = 0; i < 4; i++) {
            e = lds_u8(T.d1 + e * 4u + ((x >> (8 * i + 1)) & 3u));
            if (e == T.m && (!LIM || r + i < lim)) {
                cnt++;
                if (Sink::kRecord) sink.put(r + i);
            }
        }
    }

    // k4s fast path over n words of bases: one lookup per word, the states
    // at the start of every group OR-ed; only a group starting at a state
    // >= m - 4 can accept (the state grows by at most one per byte), so if
    // the OR shows no such state nothing was accepted, else the words are
    // walked again exactly from the saved state.
    template <int N>
    __device__ __forceinline__ void words_s(const uint32_t (&x)[N], uint32_t r, uint32_t lim)
    {
        const uint32_t e_in = e;
        uint32_t orq = e | T.force;
#pragma unroll
        for (int k = 0; k < N; k++) {
            const uint32_t code = (x[k] & 0x06060606u) * 0x00820820u;
            e = tab8(__byte_perm(code, e, 0x7743u));
            if (k + 1 < N) orq |= e;
        }
        if ((orq >> T.sh) != 0u) {
            e = e_in;
#pragma unroll
            for (int k = 0; k < N; k++) word_exact(x[k], r + 4 * k, lim);
        }
    }

    __device__ __forceinline__ void word_stt(uint32_t x, uint32_t r, uint32_t lim)
    {
#pragma unroll
        for (uint32_t i = 0; i < 4; i++) {
            e = tab8(__byte_perm(x, e, 0x7740u | i));
            if (e == T.m && (!LIM || r + i < lim)) {
                cnt++;
                if (Sink::kRecord) sink.put(r + i);
            }
        }
    }

    // Slow path for a 16-byte vector holding at least one non-base byte:
    // word by word, a word of four bases takes the four-step table, a word of
    // four non-bases resets the walk, anything else goes byte by byte.
    __device__ __forceinline__ void slow_vec(uint4 v, uint32_t r, uint32_t lim)
    {
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const uint32_t b = word_bad(w[k]);
            if (b == 0u) {
                if (LAYOUT == kLayoutK4S) {
                    const uint32_t one[1] = {w[k]};
                    words_s<1>(one, r + 4 * k, lim);
                } else {
                    word_k4(w[k], r + 4 * k, lim);
                }
            } else if (((((b & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | b) & 0x80808080u) == 0x80808080u) {
                e = 0u;                       // four non-bases: back to q0, nothing accepted
            } else {
                e &= 0xFFu;
#pragma unroll
                for (int i = 0; i < 4; i++) byte_d1((w[k] >> (8 * i)) & 0xFFu, r + 4 * k + i, lim);
            }
        }
    }

    // 64 contiguous bytes (four vectors) starting at offset r, one test for
    // the common case of 64 bases.
    __device__ __forceinline__ void vec4(uint4 v0, uint4 v1, uint4 v2, uint4 v3, uint32_t r)
    {
        if (LAYOUT == kLayoutK4S) {
            const uint32_t bad = word_bad(v0.x) | word_bad(v0.y) | word_bad(v0.z) | word_bad(v0.w) |
                                 word_bad(v1.x) | word_bad(v1.y) | word_bad(v1.z) | word_bad(v1.w) |
                                 word_bad(v2.x) | word_bad(v2.y) | word_bad(v2.z) | word_bad(v2.w) |
                                 word_bad(v3.x) | word_bad(v3.y) | word_bad(v3.z) | word_bad(v3.w);
            if (bad == 0u) {
                const uint32_t x[16] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w,
                                        v2.x, v2.y, v2.z, v2.w, v3.x, v3.y, v3.z, v3.w};
                words_s<16>(x, r, 0);
            } else {
                slow_vec(v0, r, 0);
                slow_vec(v1, r + 16, 0);
                slow_vec(v2, r + 32, 0);
                slow_vec(v3, r + 48, 0);
            }
        } else if (LAYOUT == kLayoutK4 || LAYOUT == kLayoutK4F) {
            const uint32_t bad = word_bad(v0.x) | word_bad(v0.y) | word_bad(v0.z) | word_bad(v0.w) |
                                 word_bad(v1.x) | word_bad(v1.y) | word_bad(v1.z) | word_bad(v1.w) |
                                 word_bad(v2.x) | word_bad(v2.y) | word_bad(v2.z) | word_bad(v2.w) |
                                 word_bad(v3.x) | word_bad(v3.y) | word_bad(v3.z) | word_bad(v3.w);
            if (bad == 0u) {
                word_k4(v0.x, r, 0); word_k4(v0.y, r + 4, 0); word_k4(v0.z, r + 8, 0); word_k4(v0.w, r + 12, 0);
                word_k4(v1.x, r + 16, 0); word_k4(v1.y, r + 20, 0); word_k4(v1.z, r + 24, 0); word_k4(v1.w, r + 28, 0);
                word_k4(v2.x, r + 32, 0); word_k4(v2.y, r + 36, 0); word_k4(v2.z, r + 40, 0); word_k4(v2.w, r + 44, 0);
                word_k4(v3.x, r + 48, 0); word_k4(v3.y, r + 52, 0); word_k4(v3.z, r + 56, 0); word_k4(v3.w, r + 60, 0);
            } else {
                slow_vec(v0, r, 0);
                slow_vec(v1, r + 16, 0);
                slow_vec(v2, r + 32, 0);
                slow_vec(v3, r + 48, 0);
            }
        } else {
            vec(v0, r, 0);
            vec(v1, r + 16, 0);
            vec(v2, r + 32, 0);
            vec(v3, r + 48, 0);
        }
    }

    // vec4 for a recording K4 walk of a dense pattern: the accept masks of the
    // 16 words are gathered into a 64-bit map of end offsets (bit j = end
    // r + j) without branches, then counted and handed to the sink once.
    __device__ __forceinline__ void vec4_map(uint4 v0, uint4 v1, uint4 v2, uint4 v3, uint32_t r)
    {
        const uint32_t x[16] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w,
                                v2.x, v2.y, v2.z, v2.w, v3.x, v3.y, v3.z, v3.w};
        uint32_t bad = 0u;
#pragma unroll
        for (int k = 0; k < 16; k++) bad |= word_bad(x[k]);
        if (bad != 0u) {
            slow_vec(v0, r, 0);
            slow_vec(v1, r + 16, 0);
            slow_vec(v2, r + 32, 0);
            slow_vec(v3, r + 48, 0);
            return;
        }
        uint32_t lo = 0u, hi = 0u;
#pragma unroll
        for (int k = 0; k < 16; k++) {
            e = k4_next<LAYOUT>(T.k4, e, x[k]);
            const uint32_t acc = e & (0xFu << K4_ACC_SHIFT);      // bits 8..11
            const int sh = 4 * (k & 7) - (int)K4_ACC_SHIFT;       // to bits 4k..4k+3 of its half
            const uint32_t a = sh >= 0 ? acc << (sh & 31) : acc >> ((-sh) & 31);
            if (k < 8) lo |= a; else hi |= a;
        }
        cnt += __popc(lo) + __popc(hi);
        if (Sink::kRecord) {
            while (lo) {
                sink.put(r + (uint32_t)(__ffs(lo) - 1));
                lo &= lo - 1u;
            }
            while (hi) {
                sink.put(r + 32u + (uint32_t)(__ffs(hi) - 1));
                hi &= hi - 1u;
            }
        }
    }

    // vec4_map of a dense pattern (m <= 8) without the up-front base test:
    // the words are walked through their 2-bit codes alone (a relaxed walk:
    // a non-base is read as the base with its code), which never misses an
    // exact accept (see relaxed_words).  The relaxed state equals the exact
    // one whenever the last 8 >= m bytes are bases: both are then the longest
    // suffix within those bytes that is a prefix of P.  So a stage whose
    // relaxed walk accepts nothing has no accept, and each relaxed accept is
    // exact iff its m-byte window holds only bases (window_exact, which the
    // caller applies).  Returns the 64-bit map of relaxed accept ends (bit j:
    // end r + j).
    __device__ __forceinline__ uint2 vec4_relaxed_map(uint4 v0, uint4 v1, uint4 v2, uint4 v3)
    {
        const uint32_t x[16] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w,
                                v2.x, v2.y, v2.z, v2.w, v3.x, v3.y, v3.z, v3.w};
        uint32_t lo = 0u, hi = 0u;
#pragma unroll
        for (int k = 0; k < 16; k++) {
            e = k4_next<LAYOUT>(T.k4, e, x[k]);
            const uint32_t acc = e & (0xFu << K4_ACC_SHIFT);
            const int sh = 4 * (k & 7) - (int)K4_ACC_SHIFT;
            const uint32_t a = sh >= 0 ? acc << (sh & 31) : acc >> ((-sh) & 31);
            if (k < 8) lo |= a; else hi |= a;
        }
        return make_uint2(lo, hi);
    }

    // Count and record a map of accept ends (bit j: end r + j).
    __device__ __forceinline__ void put_map(uint2 map, uint32_t r)
    {
        uint32_t lo = map.x, hi = map.y;
        cnt += __popc(lo) + __popc(hi);
        if (Sink::kRecord) {
            while (lo) {
                sink.put(r + (uint32_t)(__ffs(lo) - 1));
                lo &= lo - 1u;
            }
            while (hi) {
                sink.put(r + 32u + (uint32_t)(__ffs(hi) - 1));
                hi &= hi - 1u;
            }
        }
    }

    __device__ __forceinline__ void vec(uint4 v, uint32_t r, uint32_t lim)
    {
        if (LAYOUT == kLayoutK4S) {
            if ((word_bad(v.x) | word_bad(v.y) | word_bad(v.z) | word_bad(v.w)) == 0u) {
                const uint32_t x[4] = {v.x, v.y, v.z, v.w};
                words_s<4>(x, r, lim);
            } else {
                slow_vec(v, r, lim);
            }
        } else if (LAYOUT == kLayoutK4 || LAYOUT == kLayoutK4F) {
            uint32_t bad = word_bad(v.x) | word_bad(v.y) | word_bad(v.z) | word_bad(v.w);
            if (bad == 0u) {
                word_k4(v.x, r, lim);
                word_k4(v.y, r + 4, lim);
                word_k4(v.z, r + 8, lim);
                word_k4(v.w, r + 12, lim);
            } else {
                slow_vec(v, r, lim);
            }
        } else {
            word_stt(v.x, r, lim);
            word_stt(v.y, r + 4, lim);
            word_stt(v.z, r + 8, lim);
            word_stt(v.w, r + 12, lim);
        }
    }
};

// Walk the chunk [s, e) of the text: from q0 at s through min(e + m - 1, n),
// counting (and handing to the sink) the occurrences that start in [s, e),
// i.e. whose last byte lies below e + m - 1.  Returns the count.
template <int LAYOUT, class Sink>
__device__ uint32_t walk_chunk(const ScanArgs& a, const SmemTab& T, int64_t s, int64_t e, Sink& sink)
{
    const uint32_t m = T.m;
    const int64_t len = e - s;
    const uint32_t lim = (uint32_t)len + m - 1;               // end offsets must be < lim
    const uint32_t h16 = (m - 1 + 15) & ~15u;                 // halo rounded to vectors
    if (a.aligned && len > 0 && ((s | len) & 15) == 0 && s + len + h16 <= a.n) {
        const uint4* p = reinterpret_cast<const uint4*>(a.text + s);
        const int nv = (int)(len >> 4);
        Walker<LAYOUT, false, Sink> w{T, sink, 0u, 0u};
        uint4 cur = ldg16(p);
#pragma unroll 1
        for (int i = 0; i < nv - 1; i++) {
            uint4 nxt = ldg16(p + i + 1);
            w.vec(cur, (uint32_t)i << 4, 0);
            cur = nxt;
        }
        w.vec(cur, (uint32_t)(nv - 1) << 4, 0);
        Walker<LAYOUT, true, Sink> h{T, sink, w.e, w.cnt};
        for (uint32_t r = (uint32_t)len; r < (uint32_t)len + h16; r += 16)
            h.vec(ldg16(reinterpret_cast<const uint4*>(a.text + s + r)), r, lim);
        return h.cnt;
    }
    // boundary chunk: byte loads, exact bounds
    const int64_t hi = min(e + (int64_t)m - 1, a.n);
    uint32_t q = 0, cnt = 0;
    for (int64_t j = s; j < hi; j++) {
        uint32_t c = a.text[j];
        if (LAYOUT != kLayoutStt)
            q = byte_next(T.d1, q, c);
        else
            q = tab8((q << 8) | c);
        if (q == m) {
            cnt++;
            if (Sink::kRecord) sink.put((uint32_t)(j - s));
        }
    }
    return cnt;
}

// Where load_tables puts each table of a layout (shared addresses), from
// the launch arguments alone.
template <int LAYOUT>
__device__ __forceinline__ SmemTab tab_view(const ScanArgs& a)
{
    SmemTab T;
    const uint32_t base = (uint32_t)__cvta_generic_to_shared(g_smem);
    T.m = (uint32_t)a.m;
    // a group of four steps accepts only from a state q >= m - 4; every such q
    // has a bit at position >= floor(log2(m - 4)), so the OR of the groups'
    // start states shifted right by that much is non-zero whenever a group
    // may accept (for m <= 4 every group may)
    T.sh = a.m > 4 ? 31u - (uint32_t)__clz(a.m - 4) : 0u;
    T.force = a.m <= 4 ? 1u : 0u;
    T.fl = (uint32_t)(a.k4f_bytes >> 8) - (uint32_t)a.m - 1u;
    T.k4 = 0;
    T.d1 = 0;
    T.stt = 0;
    T.k4s = 0;
    if (LAYOUT == kLayoutK4S) {            // [k4s][d1]
        T.k4s = base;
        T.d1 = base + (uint32_t)a.k4s_bytes;
    } else if (LAYOUT == kLayoutK4F) {     // [k4f][k4][d1]
        T.k4 = base + (uint32_t)a.k4f_bytes;
        T.d1 = T.k4 + (uint32_t)a.k4_bytes;
    } else if (LAYOUT == kLayoutK4) {      // [k4][d1]
        T.k4 = base;
        T.d1 = base + (uint32_t)a.k4_bytes;
    } else {                               // [stt]
        T.stt = base;
    }
    return T;
}

// Copy the layout's tables from global memory to shared offset 0 (every
// thread of the CTA takes part; the caller synchronises).
template <int LAYOUT>
__device__ __forceinline__ void load_tables(const ScanArgs& a, uint8_t* smem)
{
    // (destination offset, source offset, bytes) of up to two ranges
    int d0 = 0, s0, n0, d1 = 0, s1 = 0, n1 = 0;
    if (LAYOUT == kLayoutK4S) {
        s0 = a.k4_bytes + a.d1_bytes + a.stt_bytes;
        n0 = a.k4s_bytes;
        d1 = a.k4s_bytes;
        s1 = a.k4_bytes;
        n1 = a.d1_bytes;
    } else if (LAYOUT == kLayoutK4F) {
        s0 = a.k4_bytes + a.d1_bytes + a.stt_bytes + a.k4s_bytes;
        n0 = a.k4f_bytes;
        d1 = a.k4f_bytes;
        s1 = 0;
        n1 = a.k4_bytes + a.d1_bytes;
    } else if (LAYOUT == kLayoutK4) {
        s0 = 0;
        n0 = a.k4_bytes + a.d1_bytes;
    } else {
        s0 = a.k4_bytes + a.d1_bytes;
        n0 = a.stt_bytes;
    }
    const uint4* src0 = reinterpret_cast<const uint4*>(a.tab + s0);
    uint4* dst0 = reinterpret_cast<uint4*>(smem + d0);
    for (int i = threadIdx.x; i < (n0 >> 4); i += blockDim.x) dst0[i] = src0[i];
    const uint4* src1 = reinterpret_cast<const uint4*>(a.tab + s1);
    uint4* dst1 = reinterpret_cast<uint4*>(smem + d1);
    for (int i = threadIdx.x; i < (n1 >> 4); i += blockDim.x) dst1[i] = src1[i];
}

__device__ __forceinline__ int table_smem_bytes_dev(const ScanArgs& a, int layout)
{
    return layout == kLayoutK4    ? a.k4_bytes + a.d1_bytes
           : layout == kLayoutK4S ? a.k4s_bytes + a.d1_bytes
           : layout == kLayoutK4F ? a.k4f_bytes + a.k4_bytes + a.d1_bytes
                                  : a.stt_bytes;
}

// ---------------------------------------------------------------- kernels

template <int LAYOUT, int THREADS>
__global__ void __launch_bounds__(THREADS) k_count(const ScanArgs a)
{
    uint8_t* smem = g_smem;
    __shared__ unsigned long long s_warp[THREADS / 32];
    load_tables<LAYOUT>(a, smem);
    const SmemTab T = tab_view<LAYOUT>(a);
    __syncthreads();
    const int64_t tb = (int64_t)THREADS * a.chunk;
    unsigned long long total = 0;
    CountSink sink;
    for (int64_t tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
        const int64_t s = tile * tb + (int64_t)threadIdx.x * a.chunk;
        if (s < a.n_own) total += walk_chunk<LAYOUT>(a, T, s, min(s + a.chunk, a.n_own), sink);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) total += __shfl_xor_sync(0xffffffffu, total, o);
    if ((threadIdx.x & 31) == 0) s_warp[threadIdx.x >> 5] = total;
    __syncthreads();
    if (threadIdx.x < 32) {
        unsigned long long v = threadIdx.x < THREADS / 32 ? s_warp[threadIdx.x] : 0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0 && v) atomicAdd(a.count, v);
    }
}

// Decoupled look-back: publish this tile's sum, add up predecessors' sums
// until one with an inclusive prefix is found, publish the inclusive prefix.
// Returns the tile's exclusive offset.  Every wait is bounded; on give-up
// bit 0 of the status word is set and the walk back stops.
__device__ unsigned long long lookback(unsigned long long* work, int64_t tile, unsigned long long total)
{
    unsigned long long* desc = work + kWorkHeader;
    if (tile == 0) {
        st_release(desc, kFlagPre | total);
        return 0ull;
    }
    st_release(desc + tile, kFlagAgg | total);
    unsigned long long excl = 0;
    for (int64_t j = tile - 1; j >= 0; j--) {
        unsigned long long d;
        unsigned spins = 0, ns = 32;
        while (((d = ld_acquire(desc + j)) >> 62) == 0ull) {
            if (++spins > kSpinLimit) {
                atomicOr(reinterpret_cast<unsigned long long*>(work + 1), 1ull);
                d = kFlagPre;
                break;
            }
            __nanosleep(ns);
            if (ns < 1024) ns <<= 1;
        }
        excl += d & kValMask;
        if ((d >> 62) == 2ull) break;
    }
    st_release(desc + tile, kFlagPre | (excl + total));
    return excl;
}

template <int LAYOUT, int THREADS>
__global__ void __launch_bounds__(THREADS) k_find(const ScanArgs a)
{
    uint8_t* smem = g_smem;
    __shared__ uint32_t s_warp[THREADS / 32];
    __shared__ int64_t s_tile;
    __shared__ unsigned long long s_off;
    load_tables<LAYOUT>(a, smem);
    const SmemTab T = tab_view<LAYOUT>(a);
    uint16_t* slots = reinterpret_cast<uint16_t*>(smem + ((table_smem_bytes_dev(a, LAYOUT) + 15) & ~15));
    const unsigned long long base = a.base_in ? *a.base_in : 0ull;
    const int64_t tb = (int64_t)THREADS * a.chunk;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (;;) {
        if (threadIdx.x == 0) s_tile = (int64_t)atomicAdd(a.work, 1ull);
        __syncthreads();
        const int64_t tile = s_tile;
        if (tile >= a.ntiles) break;
        const int64_t s = tile * tb + (int64_t)threadIdx.x * a.chunk;
        const int64_t e = min(s + a.chunk, a.n_own);
        SlotSink sink{slots + threadIdx.x, THREADS, (uint32_t)kSlots, 0u, false};
        uint32_t cnt = 0;
        if (s < a.n_own) cnt = walk_chunk<LAYOUT>(a, T, s, e, sink);

        // block-wide exclusive scan of the per-thread counts
        uint32_t v = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += y;
        }
        if (lane == 31) s_warp[warp] = v;
        __syncthreads();
        if (warp == 0) {
            uint32_t w = lane < THREADS / 32 ? s_warp[lane] : 0u;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            if (lane < THREADS / 32) s_warp[lane] = w;
        }
        __syncthreads();
        const uint32_t excl = v - cnt + (warp ? s_warp[warp - 1] : 0u);
        const uint32_t total = s_warp[THREADS / 32 - 1];
        if (threadIdx.x == 0) s_off = lookback(a.work, tile, total);
        __syncthreads();
        const unsigned long long off = s_off;
        const int64_t g0 = (int64_t)(base + off + excl);
        const int64_t start0 = a.pos_base + s - (a.m - 1);
        if (cnt) {
            if (!sink.over) {
                for (uint32_t j = 0; j < cnt; j++) {
                    int64_t g = g0 + j;
                    if (g < a.cap) a.pos[g] = start0 + slots[j * THREADS + threadIdx.x];
                }
            } else if (g0 < a.cap) {
                GlobalSink gs{a.pos, a.cap, g0, start0};
                walk_chunk<LAYOUT>(a, T, s, e, gs);
            }
        }
        if (tile == a.ntiles - 1 && threadIdx.x == 0) *a.count = base + off + total;
        __syncthreads();
    }
}

// ---------------------------------------------------------------- TMA-staged kernel
//
// Persistent, warp-specialised form of the same walk, one CTA per SM.  A
// tile is 512 rows of C bytes (row r of tile k = text[(512k + r)C, ...+C)),
// walked by 8 warps; each lane walks two rows (32 apart) with their two
// automaton chains interleaved, which hides the latency of the table lookups.
// The text is viewed as a 2-D tensor of C-byte rows.  Each walker warp
// streams its own 64 rows through a private ring of shared-memory stages
// (64 bytes x 64 rows, one TMA box with 64-byte swizzle,
// cp.async.bulk.tensor.2d); its lane 0 reloads a slot as soon as the warp has
// read it, so warps never wait for one another inside a tile.  After the C
// bytes of its rows a warp receives one more "halo" box, the first 64 bytes
// of rows r+1: the m-1 bytes of overlap each row needs (Algorithm 1).
//   warp 8 (tickets): hands out tile ids through a small ring (in text order
//           for find, by a static schedule for count);
//   warp 9 (scheduler, find only): sums the walker warps' counts of a tile,
//           publishes them and resolves the tile's global offset by a
//           warp-parallel decoupled look-back while the walkers go on; a
//           tile's positions are written kDefer - 1 tiles later, which hides
//           the look-back's latency.
// In find mode a sparse pattern (few occurrences expected) is walked without
// looking at accept bits; a stage whose count moved is walked again from its
// saved start state to record the positions.  Dense patterns record inline.
// Rows whose chunk or overlap runs past the full rows of the tensor (the end
// of the text) are walked from global memory by their thread instead.

constexpr int kWalkWarps = 16;
constexpr int kRPL = 1;                          // rows walked by each lane (16 warps x 1 row measured best)
constexpr int kWarpRows = 32 * kRPL;             // rows of one warp's box
constexpr int kRows = kWalkWarps * kWarpRows;    // rows of a tile
constexpr int kWalkThreads = kWalkWarps * 32;
constexpr int kStageW = 64;
constexpr int kWarpStage = kWarpRows * kStageW;  // one TMA box
constexpr int kTmaThreads = kWalkThreads + 64;
constexpr int kProducerWarp = kWalkWarps;
constexpr int kSchedulerWarp = kWalkWarps + 1;
constexpr int kTSlots = 8;                       // staged positions per row (sparse patterns)
constexpr int kTSlotsDense = 16;                 // staged positions per row (dense patterns)
// Stages in flight per warp ring.  With rings of 64-byte rows a depth of 3-4
// streams at the HBM rate on GB300; deeper rings were measured to lose up to
// half the throughput, so the depth is capped here.
constexpr int kMaxStages = 4;
constexpr int kRelaxedCountStages = 2;           // ring depth of the relaxed count pass
// Default row length (stages of 64 bytes) of a long text: relaxed layouts 12
// stages, layout 1 finds (the staged dense pass) 16, other exact scans 15.
// Measured on 3.2e9 bytes (device time of one call): finds of m = 8 and 16
// 0.614/0.550 ms at 12 stages, 0.615/0.562 at 14, 0.623/0.574 at 16, 0.633/0.560
// at 10, m = 16 and 64 0.62 at 20; the dense find of m = 4 (m = 5) 0.650
// (0.583) at 16, 0.662 (0.658) at 15, 0.682 (0.639) at 14, 0.696 (0.625) at
// 12: rows of a multiple of 128 bytes stream better (at 15 stages the dense
// pass read 1.12x its text from DRAM); counts of m = 4 0.684 at 15, 0.696
// at 16.
constexpr int kDefaultStagesRelaxed = 12;
constexpr int kDefaultStagesExact = 15;
constexpr int kDefaultStagesDenseFind = 16;
constexpr int kDefer = 4;                        // tiles whose positions wait for their offset
constexpr int kTicketRing = 8;
// How many tiles ahead of the slowest walker warp the ticket warp may claim
// in find mode.  Tickets fix the text order that the look-back follows, so a
// CTA must not hold tiles it will only start much later (its successors'
// offsets would wait for them).  A warp still walking tile k prefetches the
// stages of tiles up to k + 1 + (nst - 1) / (stages per tile), which needs
// ahead >= 2 + (nst - 1) / (stages per tile); the host adds one tile of slack
// so that one slow warp does not hold back the others' prefetch
// (TmaArgs::ahead).  Counting uses a static schedule and runs a full ring
// ahead.
constexpr int kDenseMaxM = 6;                     // patterns this short record inline
static_assert(kDenseMaxM <= 8, "the relaxed dense walk settles the exact state from the last 8 bytes");
constexpr long long kWaitCycles = 4000000000ll;   // ~2 s at 2 GHz

struct TmaArgs {
    ScanArgs a;
    int64_t nrows_full;   // rows of C bytes fully inside [0, n): the tensor's rows
    int32_t nst;          // stages in each warp's ring
    int32_t sps;          // body stages per tile (C / 64)
    int32_t table_bytes;  // shared bytes of the table, 128-aligned
    int32_t ahead;        // find: tiles the ticket warp may claim ahead (see above)
    int32_t rings_off;    // byte offset of the TMA rings in dynamic shared memory
    // where a wait that gave up is reported: the find workspace's status
    // word (bit 1), or bit 63 of the count for a count without workspace
    unsigned long long* fail_word;
    unsigned long long fail_bit;
    // count mode, first pass of a two-pass find: every row's count (u16) and
    // every tile's total (added up) go here; null otherwise
    uint16_t* rows;
    unsigned long long* tile_sum;
    // and either (layout 1) the rows' exact accept end offsets (u16, relative
    // to the row start): each walker warp of tile t writes those of its 32
    // rows, at most KS a row, packed in row order into its own region of
    // 32 * KS entries at stage + (t * kWalkWarps + warp) * 32 * KS; or
    // (relaxed layouts) for every row with a count the mask of the 64-byte
    // stages holding its exact accepts at masks[row] (bit s: body stage s; bit
    // sps: the overlap; all ones: the whole row)
    uint16_t* stage;
    unsigned long long* masks;
    // layout 1: each walker warp's total count of the tile, at
    // warp_sum[t * kWalkWarps + warp]
    uint32_t* warp_sum;
    // first pass of a two-pass find on a relaxed layout: the last CTA to
    // finish turns tile_sum into each tile's first index (scan_base added)
    // and writes the total to scan_count; a.count then counts the finished
    // CTAs. Null otherwise (layout 1 scans in k_tile_offsets).
    unsigned long long* scan_count;
    const unsigned long long* scan_base;
};

// Exclusive scan of ntiles tile totals by one CTA (blockDim.x a multiple of
// 32): tile_sum[t] becomes base + the totals of the tiles before t, *count
// base + all of them. Each thread scans its own contiguous run of tiles,
// then one block scan of the runs. The totals were added by other CTAs'
// atomics: read at L2.
__device__ __forceinline__ void scan_tile_totals(unsigned long long* tile_sum, int64_t ntiles,
                                                 unsigned long long base, unsigned long long* count)
{
    __shared__ unsigned long long s_warp[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (int)(blockDim.x >> 5);
    const int64_t per = (ntiles + blockDim.x - 1) / blockDim.x;
    const int64_t t0 = min((int64_t)threadIdx.x * per, ntiles), t1 = min(t0 + per, ntiles);
    unsigned long long sum = 0;
#pragma unroll 4
    for (int64_t t = t0; t < t1; t++) sum += __ldcg(tile_sum + t);
    unsigned long long x = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        unsigned long long w = lane < nw ? s_warp[lane] : 0ull;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        s_warp[lane] = w;                      // inclusive over warps
    }
    __syncthreads();
    unsigned long long run = base + (warp ? s_warp[warp - 1] : 0ull) + x - sum;
    for (int64_t t = t0; t < t1; t++) {
        const unsigned long long v = __ldcg(tile_sum + t);
        tile_sum[t] = run;
        run += v;
    }
    if (threadIdx.x == 0) *count = base + s_warp[nw - 1];
}

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar)
{
    asm volatile(
        "{\n\t.reg .b64 st;\n\t"
        "mbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile(
        "{\n\t.reg .b64 st;\n\t"
        "mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(smem_u32(bar)),
        "r"(bytes)
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int32_t x, int32_t y,
                                            uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// 16-byte shared-memory load that is always issued (never merged with an
// earlier load of the same address), so a value need not stay in registers.
__device__ __forceinline__ uint4 lds128_fresh(const void* p)
{
    uint4 v;
    asm volatile("ld.shared.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "r"(smem_u32(p)));
    return v;
}

__device__ __forceinline__ void named_sync_walkers()
{
    asm volatile("bar.sync 1, %0;" ::"n"(kWalkThreads) : "memory");
}

// Bounded wait on an mbarrier phase.  Gives up after ~2 s (reported through
// p.fail_word, and the CTA's abort flag set) or when another role aborted.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                          const TmaArgs& p)
{
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    for (;;) {
        if (mbar_try_wait(bar, parity)) return true;
        if (*abort_flag) return false;
        if (clock64() - t0 > kWaitCycles) {
            *abort_flag = 1;
            atomicOr(p.fail_word, p.fail_bit);
            return false;
        }
    }
}

// mbar_wait for a whole warp: every lane gets the same outcome, so that an
// abort racing with a completing phase cannot split the warp.
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                          const TmaArgs& p)
{
    const bool ok = mbar_wait(bar, parity, abort_flag, p);
    return __all_sync(0xffffffffu, ok);
}

// Warp-parallel decoupled look-back: lane l inspects the descriptor of tile
// (end - l); the window slides back 32 tiles at a time until it holds an
// inclusive prefix.  Returns the tile's exclusive offset (all lanes).
__device__ unsigned long long lookback_warp(unsigned long long* work, int64_t tile,
                                            unsigned long long total, int lane)
{
    unsigned long long* desc = work + kWorkHeader;
    if (tile == 0) {
        if (lane == 0) st_release(desc, kFlagPre | total);
        return 0ull;
    }
    if (lane == 0) st_release(desc + tile, kFlagAgg | total);
    unsigned long long excl = 0;
    for (int64_t end = tile - 1;; end -= 32) {
        const int64_t j = end - lane;
        unsigned long long d = kFlagPre;           // before tile 0: an empty inclusive prefix
        if (j >= 0) {
            d = ld_acquire(desc + j);
            if ((d >> 62) == 0ull) {
                const long long t0 = clock64();
                unsigned ns = 32;
                while (((d = ld_acquire(desc + j)) >> 62) == 0ull) {
                    if (clock64() - t0 > kWaitCycles) {
                        atomicOr(work + 1, 1ull);
                        d = kFlagPre;
                        break;
                    }
                    __nanosleep(ns);
                    if (ns < 512) ns <<= 1;
                }
            }
        }
        const unsigned pre = __ballot_sync(0xffffffffu, (d >> 62) == 2ull);
        const int first = pre ? __ffs(pre) - 1 : 32;
        unsigned long long v = lane <= first ? (d & kValMask) : 0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        excl += v;
        if (pre) break;
    }
    if (lane == 0) st_release(desc + tile, kFlagPre | (excl + total));
    return excl;
}

// A TMA walker row's staged end offsets: entry j at shared byte address
// base + j * kRows * 2 (the tile's rows interleaved, so a warp's stores fall
// in distinct banks).  n counts every accept put; n > CAP means the row
// overflowed its slots and is walked again from global memory at flush.
template <uint32_t CAP>
struct RowSlots {
    static constexpr bool kRecord = true;
    uint32_t base;
    uint32_t n;
    __device__ __forceinline__ void put(uint32_t off)
    {
        if (n < CAP) asm volatile("st.shared.u16 [%0], %1;" ::"r"(base + n * (uint32_t)(kRows * 2)), "h"((uint16_t)off));
        n++;
    }
};

// The exact accepts among a dense stage's relaxed accepts (m <= 8).  The
// relaxed walk is the automaton run on the text with every byte replaced by
// the base of its 2-bit code, so it accepts at end j exactly when the codes
// of the m bytes ending at j are those of P; the exact automaton accepts
// there exactly when, in addition, those m bytes are bases (each base is the
// one byte, in either case, with its code).  So an accept is exact iff its
// window holds no non-base, whatever came before it.  map: bit j = a relaxed
// accept ending at stage offset j; the stage is the lane's 64 bytes in its
// ring slot (16-byte piece k at q + (ob ^ (k << 4))), preceded by the 8
// bytes p0, p1.  Each exact accept goes to the sink at end offset r + j;
// returns their number.
template <class Sink>
__device__ __forceinline__ uint32_t window_exact(uint2 map, uint32_t r, uint32_t m, uint32_t p0, uint32_t p1,
                                                 const uint8_t* q, uint32_t ob, Sink& sink)
{
    uint32_t c = 0u, lo = map.x, hi = map.y;
    while ((lo | hi) != 0u) {
        const bool low = lo != 0u;
        const uint32_t j = (uint32_t)(__ffs(low ? lo : hi) - 1) + (low ? 0u : 32u);
        if (low)
            lo &= lo - 1u;
        else
            hi &= hi - 1u;
        // the window ends in byte jl of stage word j >> 2 (wh); with the word
        // before it (wl) and, for m > 5, the one before that (w0)
        const uint32_t jl = j & 3u;
        const uint32_t wh = *reinterpret_cast<const uint32_t*>(q + (ob ^ (j & 0x30u)) + (j & 0xCu));
        uint32_t wl = p1;
        if (j >= 4u) {
            const uint32_t jp = j - 4u;
            wl = *reinterpret_cast<const uint32_t*>(q + (ob ^ (jp & 0x30u)) + (jp & 0xCu));
        }
        if (m <= 4u) {
            // the window in one word: bytes jl + 1 .. jl + 4 of wl:wh, its
            // first 4 - m bytes outside the window
            const uint32_t w = __funnelshift_rc(wl, wh, 8u * (jl + 1u));
            if ((word_bad(w) & (0xFFFFFFFFu << (8u * (4u - m)))) == 0u) {
                sink.put(r + j);
                c++;
            }
            continue;
        }
        // bytes of wl inside the window: from 5 + jl - m on (all of them
        // when that is below 0, none when it is past 3: shl by >= 32 is 0)
        uint32_t keep_l;
        asm("shl.b32 %0, %1, %2;" : "=r"(keep_l) : "r"(0xFFFFFFFFu), "r"(5u + jl > m ? 8u * (5u + jl - m) : 0u));
        // bytes of wh inside the window: from jl + 1 - m (when above 0) to jl
        const uint32_t keep_h = (0xFFFFFFFFu >> (24u - 8u * jl)) & (0xFFFFFFFFu << (jl + 1u > m ? 8u * (jl + 1u - m) : 0u));
        uint32_t bad = (word_bad(wh) & keep_h) | (word_bad(wl) & keep_l);
        if (m > 5u && 5u + jl < m) {
            uint32_t w0 = p0;
            if (j >= 8u) {
                const uint32_t jq = j - 8u;
                w0 = *reinterpret_cast<const uint32_t*>(q + (ob ^ (jq & 0x30u)) + (jq & 0xCu));
            } else if (j >= 4u) {
                w0 = p1;
            }
            bad |= word_bad(w0) & (0xFFFFFFFFu << (8u * (9u + jl - m)));
        }
        if (bad == 0u) {
            sink.put(r + j);
            c++;
        }
    }
    return c;
}

// Cold paths of the TMA walkers, kept out of line so that the hot loop's
// register allocation does not pay for them.
//   replay_stage: walk a 64-byte stage again from its start entry and record
//                 the accepts (a sparse pattern's stage whose count moved);
//   replay_halo:  the same for the overlap stage, ends limited to lim;
//   walk_cold:    a row walked from global memory (edge rows, overflow).
template <int LAYOUT>
__device__ __noinline__ uint32_t replay_stage(SmemTab T, uint32_t slots, uint32_t n, uint32_t e_in,
                                              const uint8_t* rp, uint32_t ob, uint32_t r)
{
    RowSlots<kTSlots> ss{slots, n};
    Walker<LAYOUT, false, RowSlots<kTSlots>> rw{T, ss, e_in, 0u};
    rw.vec4(lds128_fresh(rp + ob), lds128_fresh(rp + (ob ^ 16u)), lds128_fresh(rp + (ob ^ 32u)),
            lds128_fresh(rp + (ob ^ 48u)), r);
    return ss.n;
}

template <int LAYOUT>
__device__ __noinline__ uint32_t replay_halo(SmemTab T, uint32_t slots, uint32_t n, uint32_t e_in,
                                             const uint8_t* rp, uint32_t ob, uint32_t C, uint32_t lim)
{
    RowSlots<kTSlots> ss{slots, n};
    Walker<LAYOUT, true, RowSlots<kTSlots>> hr{T, ss, e_in, 0u};
    const uint32_t m = T.m;
    hr.vec(lds128_fresh(rp + ob), C, lim);
    if (m > 17) hr.vec(lds128_fresh(rp + (ob ^ 16u)), C + 16, lim);
    if (m > 33) hr.vec(lds128_fresh(rp + (ob ^ 32u)), C + 32, lim);
    if (m > 49) hr.vec(lds128_fresh(rp + (ob ^ 48u)), C + 48, lim);
    return ss.n;
}

// The exact state after the 8 bytes of (p0, p1), walked from q0; for a
// pattern of m <= 8 it is the exact state after any text ending in them.
__device__ __forceinline__ uint32_t exact_state8(const SmemTab& T, uint32_t p0, uint32_t p1)
{
    uint32_t q = 0u;
#pragma unroll
    for (int i = 0; i < 4; i++) q = byte_next(T.d1, q, (p0 >> (8 * i)) & 0xFFu);
#pragma unroll
    for (int i = 0; i < 4; i++) q = byte_next(T.d1, q, (p1 >> (8 * i)) & 0xFFu);
    return q;
}

template <int LAYOUT, class Sink>
__device__ __noinline__ uint32_t walk_cold(const ScanArgs* a, int64_t s, int64_t e, Sink* sink)
{
    const SmemTab T = tab_view<LAYOUT>(*a);
    return walk_chunk<LAYOUT>(*a, T, s, e, *sink);
}

// walk_cold recording into a row's slots, which go in and out by value (no
// address of the caller's row state is taken, so it stays in registers).
// Returns (count, slots used).
template <int LAYOUT, uint32_t CAP>
__device__ __noinline__ uint2 walk_cold_rec(const ScanArgs* a, int64_t s, int64_t e, uint32_t base, uint32_t n)
{
    RowSlots<CAP> ss{base, n};
    const SmemTab T = tab_view<LAYOUT>(*a);
    const uint32_t c = walk_chunk<LAYOUT>(*a, T, s, e, ss);
    return make_uint2(c, ss.n);
}

// Relaxed walk of layouts 3 and 4 (patterns of kOptMinM and more).  The
// text is read through the 2-bit codes alone, i.e. every byte that is not a
// base is taken as the base with the same code, and no byte is tested.
// Against the exact walk (a non-base resets to q0) this relaxed walk is
// never behind: its state is the longest suffix of the relaxed text that is
// a prefix of P, the exact state the longest such suffix holding no
// non-base, which is also a suffix of the relaxed text.  So every exact
// accept is a relaxed accept, and a stage whose relaxed walk shows none has
// none.  A stage that may hold one is walked again exactly (replay_exact).
//   layout 4: entries carry a flag for "one of the four steps accepted";
//   layout 3: states only; a group of four steps can accept only from a
//             state q >= m - 4, i.e. with (q >> T.sh) != 0 (force for m <= 4).
// Returns non-zero when the words may hold an accept.
// tmask: layout 4: the flag; layout 3: the bits of the states >= 2^sh (all
// bits, with orq forced non-zero, when m <= 4).
template <int LAYOUT, int N>
__device__ __forceinline__ uint32_t relaxed_words(uint32_t tmask, uint32_t& e, const uint32_t (&x)[N])
{
    uint32_t orq = LAYOUT == kLayoutK4S ? (e | (tmask == ~0u ? 1u : 0u)) : 0u;
#pragma unroll
    for (int k = 0; k < N; k++) {
        const uint32_t code = (x[k] & 0x06060606u) * 0x00820820u;
        e = tab8(__byte_perm(code, e, 0x7743u));
        if (LAYOUT == kLayoutK4F || k + 1 < N) orq |= e;
    }
    return orq & tmask;
}

template <int LAYOUT>
__device__ __forceinline__ uint32_t relaxed_mask(uint32_t m)
{
    if (LAYOUT == kLayoutK4F) return 1u << (32 - __clz(m));
    if (m <= 4) return ~0u;
    return ~((1u << (31u - (uint32_t)__clz(m - 4))) - 1u);
}

// Exact walk, at the end of a tile, of the stages of one row (starting at
// text offset rs) that its relaxed walk flagged: bit s of mask for body
// stage s (64 bytes at rs + 64 s), bit sps for the overlap stage (ends
// limited to C + m - 1).  The exact state at a stage start depends on at
// most the m <= 64 bytes before it (Algorithm 1's overlap argument), so each
// stage is walked from q0 at the previous 64 bytes of the row (from the row
// start for stage 0).  Every byte is read again from global memory, where
// the tile was just streamed from.  With REC the accepts go to the row's
// slots (base, n), in ascending order.  Returns (count, n, and the mask of
// the stages that hold exact accepts in .z (bits 0..31) and .w (32..63)).
// MODE 0: count only; 1: accepts to the row's shared-memory slots (base, n).
template <int LAYOUT, int MODE>
__device__ __noinline__ uint4 replay_row(const ScanArgs* a, int64_t rs, uint32_t sps, uint64_t mask,
                                         uint32_t slot_base, uint32_t slot_n)
{
    constexpr bool REC = MODE == 1;
    uint64_t hit = 0ull;
    const SmemTab T = tab_view<LAYOUT>(*a);
    const uint32_t m = (uint32_t)a->m;
    const uint32_t C = sps * kStageW;
    using Sink = typename std::conditional<REC, RowSlots<kTSlots>, CountSink>::type;
    Sink sink{};
    if (REC) {
        reinterpret_cast<RowSlots<kTSlots>*>(&sink)->base = slot_base;
        reinterpret_cast<RowSlots<kTSlots>*>(&sink)->n = slot_n;
    }
    uint32_t cnt = 0;
    while (mask) {
        const uint32_t s = (uint32_t)__ffsll((long long)mask) - 1u;
        mask &= mask - 1ull;
        const uint4* g = reinterpret_cast<const uint4*>(a->text + rs + (int64_t)s * kStageW);
        uint32_t e0 = 0u;
        if (s) {
            CountSink cs;
            Walker<LAYOUT, false, CountSink> w{T, cs, 0u, 0u};
            w.vec4(ldg16(g - 4), ldg16(g - 3), ldg16(g - 2), ldg16(g - 1), 0u);
            e0 = w.e;
        }
        if (s < sps) {
            Walker<LAYOUT, false, Sink> w{T, sink, e0, 0u};
            w.vec4(ldg16(g), ldg16(g + 1), ldg16(g + 2), ldg16(g + 3), s * kStageW);
            cnt += w.cnt;
            if (w.cnt) hit |= 1ull << s;
        } else {
            const uint32_t lim = C + m - 1;
            Walker<LAYOUT, true, Sink> h{T, sink, e0, 0u};
            h.vec(ldg16(g), C, lim);
            if (m > 17) h.vec(ldg16(g + 1), C + 16, lim);
            if (m > 33) h.vec(ldg16(g + 2), C + 32, lim);
            if (m > 49) h.vec(ldg16(g + 3), C + 48, lim);
            cnt += h.cnt;
            if (h.cnt) hit |= 1ull << s;
        }
    }
    return make_uint4(cnt, REC ? reinterpret_cast<RowSlots<kTSlots>*>(&sink)->n : 0u, (uint32_t)hit,
                      (uint32_t)(hit >> 32));
}

// The common case of a stage: kRPL rows of 64 bytes each, counted only.
// The rows' automaton chains are advanced word by word in turn so that their
// table lookups overlap; a stage holding any non-base byte takes the
// per-row slow path.  Rows with ok[i] false are walked on whatever bytes the
// stage holds (every table index stays in range) and their result discarded.
template <int LAYOUT>
__device__ __forceinline__ void count_stage(const SmemTab& T, uint32_t (&e)[kRPL], uint32_t (&cnt)[kRPL],
                                            const uint4 (&v)[kRPL][4], const bool (&ok)[kRPL], uint32_t r)
{
    if (LAYOUT == kLayoutK4) {
        uint32_t bad = 0;
#pragma unroll
        for (int i = 0; i < kRPL; i++) {
            const uint32_t b = word_bad(v[i][0].x) | word_bad(v[i][0].y) | word_bad(v[i][0].z) |
                               word_bad(v[i][0].w) | word_bad(v[i][1].x) | word_bad(v[i][1].y) |
                               word_bad(v[i][1].z) | word_bad(v[i][1].w) | word_bad(v[i][2].x) |
                               word_bad(v[i][2].y) | word_bad(v[i][2].z) | word_bad(v[i][2].w) |
                               word_bad(v[i][3].x) | word_bad(v[i][3].y) | word_bad(v[i][3].z) |
                               word_bad(v[i][3].w);
            bad |= ok[i] ? b : 0u;
        }
        if (bad == 0u) {
#pragma unroll
            for (int q = 0; q < 4; q++) {
#pragma unroll
                for (int c = 0; c < 4; c++) {
#pragma unroll
                    for (int i = 0; i < kRPL; i++) {
                        const uint32_t x = c == 0 ? v[i][q].x : c == 1 ? v[i][q].y : c == 2 ? v[i][q].z : v[i][q].w;
                        e[i] = k4_next(T.k4, e[i], x);
                        cnt[i] += e[i] >> K4_CNT_SHIFT;
                    }
                }
            }
            return;
        }
    }
#pragma unroll
    for (int i = 0; i < kRPL; i++) {
        CountSink cs;
        Walker<LAYOUT, false, CountSink> w{T, cs, e[i], cnt[i]};
        w.vec4(v[i][0], v[i][1], v[i][2], v[i][3], r);
        e[i] = w.e;
        cnt[i] = w.cnt;
    }
}


// One tile's worth of a walker row's state, kept in one register until its
// positions are written: the row's count (bits 0..12; at most a chunk of
// 4096 bytes), its exclusive offset among the warp's rows (bits 13..29; at
// most 31 x 4096) and the slot-overflow flag (bit 31).  The tile id comes
// from the scheduler with the tile's offset.
constexpr uint32_t kPendCntBits = 13;
constexpr uint32_t kPendExclBits = 17;
__device__ __forceinline__ uint32_t pend_pack(uint32_t cnt, uint32_t excl, bool over)
{
    return cnt | (excl << kPendCntBits) | (over ? 0x80000000u : 0u);
}
__device__ __forceinline__ uint32_t pend_cnt(uint32_t pr) { return pr & ((1u << kPendCntBits) - 1u); }
__device__ __forceinline__ uint32_t pend_excl(uint32_t pr)
{
    return (pr >> kPendCntBits) & ((1u << kPendExclBits) - 1u);
}
__device__ __forceinline__ bool pend_over(uint32_t pr) { return (pr >> 31) != 0u; }

template <int LAYOUT, bool FIND, bool DENSE>
// A count has static tiles and no offsets to resolve: its CTA is the 16
// walker warps alone (128 registers a thread); a find adds the ticket and
// scheduler warps (96 registers a thread).  The staged pass of layout 1 runs
// two CTAs per SM (64 registers a thread, 32 walker warps to hide its table
// lookups behind: 3.2e9 bytes, m = 4, find 0.934 -> 0.852 ms).
__global__ void __launch_bounds__(FIND ? kTmaThreads : kWalkThreads, (!FIND && DENSE && LAYOUT == kLayoutK4) ? 2 : 1)
    k_scan_tma(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ TmaArgs p)
{
    uint8_t* smem = g_smem;
    __shared__ __align__(8) uint64_t s_full[kWalkWarps][kMaxStages];
    __shared__ __align__(8) uint64_t s_tready[kTicketRing];
    __shared__ __align__(8) uint64_t s_tfree[kTicketRing];
    __shared__ __align__(8) uint64_t s_counted[kDefer];
    __shared__ __align__(8) uint64_t s_ready[kDefer];
    __shared__ int64_t s_tiles[kTicketRing];
    __shared__ int64_t s_tile_of[kDefer];
    __shared__ uint32_t s_wtot[kDefer][kWalkWarps];
    __shared__ uint32_t s_woff[kDefer][kWalkWarps];
    __shared__ unsigned long long s_tile_off[kDefer];
    __shared__ int64_t s_tile_done[kDefer];       // the tile s_tile_off[b] belongs to
    __shared__ unsigned long long s_sum[kWalkWarps];
    __shared__ int s_abort;

    // layouts 3 and 4: relaxed walk, exact replay of the rare flagged stages;
    // dense patterns: every accept recorded inline during the walk.
    // STAGED (count mode with DENSE, layout 1): pass 1 of the two-pass find
    // of a dense pattern, every exact accept recorded to the row's slots and,
    // at the end of the tile, written out (TmaArgs::stage).  The relaxed
    // layouts' pass 1 is their count kernel with TmaArgs::rows set.
    constexpr bool STAGED = !FIND && DENSE;
    constexpr bool OPT = LAYOUT == kLayoutK4S || LAYOUT == kLayoutK4F;
    constexpr bool INLINE_REC = DENSE && !OPT;
    constexpr int KS = INLINE_REC ? kTSlotsDense : kTSlots;
    static_assert(!STAGED || kRPL == 1, "the staged pass writes one row per lane");
    static_assert(!STAGED || LAYOUT == kLayoutK4, "the staged pass records on the four-step table");
    const ScanArgs& a = p.a;
    const int nst = p.nst;
    // [tables][position slots][rings], rings 1024-byte aligned for the TMA swizzle
    load_tables<LAYOUT>(a, smem);
    const SmemTab T = tab_view<LAYOUT>(a);
    uint16_t* slots = reinterpret_cast<uint16_t*>(smem + p.table_bytes);
    const uint32_t slots_sa = (uint32_t)__cvta_generic_to_shared(slots);
    uint8_t* rings = smem + p.rings_off;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int w = 0; w < kWalkWarps; w++)
            for (int i = 0; i < nst; i++) mbar_init(&s_full[w][i], 1);
        for (int i = 0; i < kTicketRing; i++) {
            mbar_init(&s_tready[i], 1);
            mbar_init(&s_tfree[i], kWalkWarps);
        }
        for (int i = 0; i < kDefer; i++) {
            mbar_init(&s_counted[i], kWalkWarps);
            mbar_init(&s_ready[i], 1);
        }
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    volatile int* abort_flag = &s_abort;
    const uint32_t sps = (uint32_t)p.sps;
    // stages per tile, the halo (the next row's first 64 bytes) included;
    // the staged dense pass (m <= 8) takes its halo from the next lane's
    // first stage instead
    const uint32_t spt = sps + (STAGED ? 0u : 1u);
    const int64_t C = a.chunk;

    if (FIND && warp == kProducerWarp) {
        // ------------------------------------------------------ tickets
        if (lane != 0) return;
        const int64_t ahead = FIND ? (int64_t)p.ahead : (int64_t)kTicketRing;
        for (int64_t kk = 0;; kk++) {
            const int slot = (int)((uint64_t)kk % kTicketRing);
            // wait until every walker warp is done with tile kk - ahead
            // (which also frees this slot, since kk - kTicketRing <= kk - ahead)
            if (kk >= ahead) {
                const uint64_t kf = (uint64_t)(kk - ahead);
                if (!mbar_wait(&s_tfree[kf % kTicketRing], (uint32_t)(kf / kTicketRing) & 1u, abort_flag, p))
                    return;
            }
            int64_t tile = FIND ? (int64_t)atomicAdd(a.work, 1ull)
                                : (int64_t)blockIdx.x + kk * (int64_t)gridDim.x;
            if (tile >= a.ntiles) tile = -1;
            s_tiles[slot] = tile;
            mbar_arrive(&s_tready[slot]);
            if (tile < 0) return;
        }
    }

    if (FIND && warp == kSchedulerWarp) {
        // ------------------------------------------------------ scheduler
        if (!FIND) return;
        const unsigned long long base = a.base_in ? *a.base_in : 0ull;
        for (int64_t k = 0;; k++) {
            const int b = (int)((uint64_t)k % kDefer);
            if (!warp_wait(&s_counted[b], (uint32_t)((uint64_t)k / kDefer) & 1u, abort_flag, p)) return;
            const int64_t tile = s_tile_of[b];
            if (tile < 0) return;
            const uint32_t wt = lane < kWalkWarps ? s_wtot[b][lane] : 0u;
            uint32_t inc = wt;
#pragma unroll
            for (int o = 1; o < kWalkWarps; o <<= 1) {
                uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += y;
            }
            const uint32_t total = __shfl_sync(0xffffffffu, inc, kWalkWarps - 1);
            if (lane < kWalkWarps) s_woff[b][lane] = inc - wt;
            const unsigned long long off = lookback_warp(a.work, tile, total, lane);
            if (lane == 0) {
                s_tile_off[b] = base + off;
                s_tile_done[b] = tile;
                if (tile == a.ntiles - 1) *a.count = base + off + total;
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&s_ready[b]);
        }
    }

    // ---------------------------------------------------------- walkers
    const uint32_t m = (uint32_t)a.m;
    uint8_t* ring = rings + (size_t)warp * nst * kWarpStage;
    uint64_t* full = s_full[warp];
    // row i of this lane is box row 32i + lane; its 16-byte piece j sits at
    // ob + i*32*64 ^ (j << 4) (64-byte swizzle of the box)
    const uint32_t ob = lane * kStageW + ((((uint32_t)lane >> 1) & 3u) << 4);
    const uint32_t wrow0 = (uint32_t)warp * kWarpRows + lane;    // row 0 of this lane in the tile
    bool aborted = false;

    // tile ids and per-CTA tile counts fit 32 bits (a tile is at least 64 KiB)
    auto tile_id = [&](uint32_t kk, int32_t* out) -> bool {
        if (!FIND) {                              // count: static tiles
            const int64_t t = (int64_t)blockIdx.x + (int64_t)kk * gridDim.x;
            *out = t < a.ntiles ? (int32_t)t : -1;
            return true;
        }
        const uint32_t slot = kk % kTicketRing;
        if (!warp_wait(&s_tready[slot], (kk / kTicketRing) & 1u, abort_flag, p)) return false;
        *out = (int32_t)s_tiles[slot];
        return true;
    };
    // refill cursor: the next stage of this warp's rows to load, kept as
    // (tile index, stage within the tile, ring slot) without divisions; the
    // warp's lane 0 loads a slot again as soon as the warp has read it
    uint32_t i_k = 0;
    int32_t i_tile = 0;
    uint32_t i_s = 0, i_slot = 0, n_issued = 0, n_consumed = 0;
    bool i_done = false;
    auto issue_next = [&]() -> bool {
        if (i_done) return true;
        if (i_s == 0) {
            if (!tile_id(i_k, &i_tile)) return false;
            if (i_tile < 0) {
                i_done = true;
                return true;
            }
        }
        if (lane == 0) {
            mbar_arrive_expect_tx(&full[i_slot], kWarpStage);
            const int32_t x = i_s < sps ? (int32_t)(i_s * kStageW) : 0;
            const int32_t y = i_tile * kRows + warp * kWarpRows + (i_s < sps ? 0 : 1);
            tma_load_2d(ring + (size_t)i_slot * kWarpStage, &tmap, x, y, &full[i_slot]);
        }
        n_issued++;
        if (++i_slot == (uint32_t)nst) i_slot = 0;
        if (++i_s == spt) {
            i_s = 0;
            i_k++;
        }
        return true;
    };
    for (int i = 0; i < nst && !aborted; i++) aborted = !issue_next();

    unsigned long long total = 0;
    // pend[d] holds tile k-1-d, for d = 0 .. kDefer-2
    uint32_t pend[kDefer - 1][kRPL];
#pragma unroll
    for (int d = 0; d < kDefer - 1; d++)
#pragma unroll
        for (int i = 0; i < kRPL; i++) pend[d][i] = 0u;
    auto flush = [&](const uint32_t (&pr)[kRPL], int64_t kp) -> bool {
        const int b = (int)((uint64_t)kp % kDefer);
        if (!warp_wait(&s_ready[b], (uint32_t)((uint64_t)kp / kDefer) & 1u, abort_flag, p)) return false;
#pragma unroll
        for (int i = 0; i < kRPL; i++) {
            const uint32_t pc = pend_cnt(pr[i]);
            if (pc == 0) continue;
            const int64_t g0 = (int64_t)(s_tile_off[b] + s_woff[b][warp] + pend_excl(pr[i]));
            const int64_t ps = (s_tile_done[b] * kRows + wrow0 + 32 * i) * C;
            const int64_t pe = min(ps + C, a.n_own);
            const int64_t start0 = a.pos_base + ps - (int64_t)(m - 1);
            if (!pend_over(pr[i])) {
                // a row that did not overflow recorded exactly pc <= KS ends;
                // the bound keeps every read inside the slot array regardless
                const uint16_t* sl = slots + (size_t)b * KS * kRows + wrow0 + 32 * i;
                const uint32_t nrec = min(pc, (uint32_t)KS);
                for (uint32_t j = 0; j < nrec; j++) {
                    const int64_t gi = g0 + j;
                    if (gi < a.cap) a.pos[gi] = start0 + sl[j * kRows];
                }
            } else if (g0 < a.cap) {
                GlobalSink gs{a.pos, a.cap, g0, start0};
                walk_cold<LAYOUT>(&a, ps, pe, &gs);
            }
        }
        return true;
    };

    uint32_t c_slot = 0, c_par = 0;               // consume cursor
    uint32_t k = 0;
    while (!aborted) {
        const int tslot = (int)(k % kTicketRing);
        int32_t tile;
        if (!tile_id(k, &tile)) {
            aborted = true;
            break;
        }
        if (tile < 0) break;
        const int kb = (int)(k % kDefer);
        bool ok[kRPL];
        uint32_t e[kRPL], cnt[kRPL];
        uint64_t fmask[kRPL];                     // relaxed walks: stages to replay exactly
        uint32_t tl0[kRPL], tl1[kRPL];            // dense finds: the row's last 8 bytes walked
        uint32_t hf0 = 0u, hf1 = 0u;              // staged: the row's first 8 bytes
        uint2 hn = make_uint2(0u, 0u);            // staged, lane 31: the next warp's row's first 8
        RowSlots<KS> ss[kRPL];
#pragma unroll
        for (int i = 0; i < kRPL; i++) {
            // a full row whose successor row is complete too (its halo is the
            // next row's first bytes); every other row is walked cold below
            const int64_t row = (int64_t)tile * kRows + wrow0 + 32 * i;
            ok[i] = (row + 1) * C <= a.n_own && row + 1 < p.nrows_full;
            if (STAGED && lane == 31 && ok[i]) {
                // the row after the warp's last: another warp's (or tile's)
                asm volatile("ld.global.nc.v2.u32 {%0,%1}, [%2];"
                             : "=r"(hn.x), "=r"(hn.y)
                             : "l"(a.text + (row + 1) * C));
            }
            e[i] = 0;
            cnt[i] = 0;
            fmask[i] = 0;
            tl0[i] = 0x41414141u;                 // no byte before the row start: bases
            tl1[i] = 0x41414141u;
            ss[i] = RowSlots<KS>{slots_sa + (uint32_t)(((uint32_t)(FIND ? kb : 0) * KS * kRows + wrow0 + 32 * i) * 2), 0u};
        }
        for (uint32_t s = 0; s < spt; s++) {
            if (!warp_wait(&full[c_slot], c_par, abort_flag, p)) {
                aborted = true;
                break;
            }
            const uint8_t* rp = ring + (size_t)c_slot * kWarpStage;
            if (s < sps) {
                const uint32_t r = s * kStageW;
                uint4 v[kRPL][4];
#pragma unroll
                for (int i = 0; i < kRPL; i++) {
                    const uint8_t* q = rp + ob + i * 32 * kStageW;
                    v[i][0] = *reinterpret_cast<const uint4*>(q);
                    v[i][1] = *reinterpret_cast<const uint4*>(rp + ((ob + i * 32 * kStageW) ^ 16u));
                    v[i][2] = *reinterpret_cast<const uint4*>(rp + ((ob + i * 32 * kStageW) ^ 32u));
                    v[i][3] = *reinterpret_cast<const uint4*>(rp + ((ob + i * 32 * kStageW) ^ 48u));
                }
                if (OPT) {
#pragma unroll
                    for (int i = 0; i < kRPL; i++) {
                        const uint32_t x[16] = {v[i][0].x, v[i][0].y, v[i][0].z, v[i][0].w,
                                                v[i][1].x, v[i][1].y, v[i][1].z, v[i][1].w,
                                                v[i][2].x, v[i][2].y, v[i][2].z, v[i][2].w,
                                                v[i][3].x, v[i][3].y, v[i][3].z, v[i][3].w};
                        const uint32_t flag = relaxed_words<LAYOUT, 16>(relaxed_mask<LAYOUT>(m), e[i], x);
                        fmask[i] |= (uint64_t)(flag != 0u) << s;
                    }
                } else if (INLINE_REC) {
                    if (STAGED && s == 0u) {              // the previous lane's halo
                        hf0 = v[0][0].x;
                        hf1 = v[0][0].y;
                    }
#pragma unroll
                    for (int i = 0; i < kRPL; i++) {
                        if (!ok[i]) continue;
                        Walker<LAYOUT, false, RowSlots<KS>> wd{T, ss[i], e[i], cnt[i]};
                        if (LAYOUT == kLayoutK4) {
                            const uint32_t p0 = tl0[i], p1 = tl1[i];
                            tl0[i] = v[i][3].z;
                            tl1[i] = v[i][3].w;
                            const uint2 map = wd.vec4_relaxed_map(v[i][0], v[i][1], v[i][2], v[i][3]);
                            if ((map.x | map.y) != 0u)        // accepts: each window tested for bases
                                wd.cnt += window_exact(map, r, m, p0, p1, rp + i * 32 * kStageW, ob, ss[i]);
                        } else {
                            wd.vec4(v[i][0], v[i][1], v[i][2], v[i][3], r);
                        }
                        e[i] = wd.e;
                        cnt[i] = wd.cnt;
                    }
                } else {
                    uint32_t e_in[kRPL], c_in[kRPL];
#pragma unroll
                    for (int i = 0; i < kRPL; i++) {
                        e_in[i] = e[i];
                        c_in[i] = cnt[i];
                    }
                    if (!FIND && LAYOUT == kLayoutK4 && m <= 8u) {
                        // count of a short pattern: the relaxed walk of the
                        // dense find, each relaxed accept's window tested
#pragma unroll
                        for (int i = 0; i < kRPL; i++) {
                            if (!ok[i]) continue;
                            const uint32_t p0 = tl0[i], p1 = tl1[i];
                            tl0[i] = v[i][3].z;
                            tl1[i] = v[i][3].w;
                            CountSink cs;
                            Walker<LAYOUT, false, CountSink> wc{T, cs, e[i], 0u};
                            const uint2 map = wc.vec4_relaxed_map(v[i][0], v[i][1], v[i][2], v[i][3]);
                            if ((map.x | map.y) != 0u)        // accepts: each window tested for bases
                                cnt[i] += window_exact(map, r, m, p0, p1, rp + i * 32 * kStageW, ob, cs);
                            e[i] = wc.e;
                        }
                    } else {
                        count_stage<LAYOUT>(T, e, cnt, v, ok, r);
                    }
                    if (FIND) {
#pragma unroll
                        for (int i = 0; i < kRPL; i++) {
                            if (ok[i] && cnt[i] != c_in[i]) {
                                // a match in this stage: walk it again to record where
                                // (the stage is re-read from its slot, released below)
                                ss[i].n = replay_stage<LAYOUT>(T, ss[i].base, ss[i].n, e_in[i],
                                                               rp + i * 32 * kStageW, ob, r);
                            }
                        }
                    }
                }
            } else {
                // the overlap: ends below C + m - 1 belong to this row
                const uint32_t lim = (uint32_t)C + m - 1;
#pragma unroll
                for (int i = 0; i < kRPL; i++) {
                    if (!ok[i]) continue;
                    const uint8_t* q = rp + i * 32 * kStageW;
                    const uint4 h0 = *reinterpret_cast<const uint4*>(q + ob);
                    if (OPT) {
                        const uint32_t x0[4] = {h0.x, h0.y, h0.z, h0.w};
                        uint32_t flag = relaxed_words<LAYOUT, 4>(relaxed_mask<LAYOUT>(m), e[i], x0);
#pragma unroll
                        for (uint32_t j = 1; j < 4; j++) {
                            if (m > 16 * j + 1) {
                                const uint4 hj = *reinterpret_cast<const uint4*>(q + (ob ^ (j << 4)));
                                const uint32_t xj[4] = {hj.x, hj.y, hj.z, hj.w};
                                flag |= relaxed_words<LAYOUT, 4>(relaxed_mask<LAYOUT>(m), e[i], xj);
                            }
                        }
                        fmask[i] |= (uint64_t)(flag != 0u) << s;
                    } else if (INLINE_REC) {
                        // the relaxed walk's state is exact unless the last 8
                        // bytes hold a non-base (vec4_map_relaxed)
                        if (LAYOUT == kLayoutK4 && (word_bad(tl0[i]) | word_bad(tl1[i])) != 0u)
                            e[i] = exact_state8(T, tl0[i], tl1[i]);
                        Walker<LAYOUT, true, RowSlots<KS>> h{T, ss[i], e[i], cnt[i]};
                        h.vec(h0, (uint32_t)C, lim);
                        if (m > 17) h.vec(*reinterpret_cast<const uint4*>(q + (ob ^ 16u)), (uint32_t)C + 16, lim);
                        if (m > 33) h.vec(*reinterpret_cast<const uint4*>(q + (ob ^ 32u)), (uint32_t)C + 32, lim);
                        if (m > 49) h.vec(*reinterpret_cast<const uint4*>(q + (ob ^ 48u)), (uint32_t)C + 48, lim);
                        cnt[i] = h.cnt;
                    } else {
                        // a short pattern's relaxed count: the exact state
                        // from the last 8 bytes when they hold a non-base
                        if (!FIND && LAYOUT == kLayoutK4 && m <= 8u && (word_bad(tl0[i]) | word_bad(tl1[i])) != 0u)
                            e[i] = exact_state8(T, tl0[i], tl1[i]);
                        CountSink cs;
                        Walker<LAYOUT, true, CountSink> h{T, cs, e[i], cnt[i]};
                        h.vec(h0, (uint32_t)C, lim);
                        if (m > 17) h.vec(*reinterpret_cast<const uint4*>(q + (ob ^ 16u)), (uint32_t)C + 16, lim);
                        if (m > 33) h.vec(*reinterpret_cast<const uint4*>(q + (ob ^ 32u)), (uint32_t)C + 32, lim);
                        if (m > 49) h.vec(*reinterpret_cast<const uint4*>(q + (ob ^ 48u)), (uint32_t)C + 48, lim);
                        if (FIND && h.cnt != cnt[i]) {
                            ss[i].n = replay_halo<LAYOUT>(T, ss[i].base, ss[i].n, e[i], q, ob, (uint32_t)C, lim);
                        }
                        cnt[i] = h.cnt;
                    }
                }
            }
            // The slot is reloaded only after the walk: every lane's walk has
            // consumed each word it read from the slot, so its shared loads
            // are complete before the warp syncs and lane 0 starts the TMA
            // that overwrites them.  (Reloading right after the loads, before
            // the walk, raced with them in the dense find.)
            __syncwarp();
            n_consumed++;
            if (++c_slot == (uint32_t)nst) {
                c_slot = 0;
                c_par ^= 1u;
            }
            if (!issue_next()) {                  // reload the slot just read
                aborted = true;
                break;
            }
        }
        if (aborted) break;
        if (STAGED) {
            // the overlap (m - 1 <= 7 bytes) of a dense pattern: the next
            // row's first 8 bytes, which the next lane read in its first
            // stage (lane 31: the next warp's row, loaded at the tile start);
            // the relaxed state is exact unless the last 8 bytes hold a
            // non-base (the relaxed dense walk)
            const uint32_t n0 = __shfl_down_sync(0xffffffffu, hf0, 1);
            const uint32_t n1 = __shfl_down_sync(0xffffffffu, hf1, 1);
            const uint32_t lim = (uint32_t)C + m - 1;
            if (ok[0]) {
                if ((word_bad(tl0[0]) | word_bad(tl1[0])) != 0u) e[0] = exact_state8(T, tl0[0], tl1[0]);
                Walker<LAYOUT, true, RowSlots<KS>> h{T, ss[0], e[0], cnt[0]};
                h.vec(make_uint4(lane == 31 ? hn.x : n0, lane == 31 ? hn.y : n1, 0u, 0u), (uint32_t)C, lim);
                cnt[0] = h.cnt;
            }
        }
#pragma unroll
        for (int i = 0; i < kRPL; i++) {
            const int64_t s0 = ((int64_t)tile * kRows + wrow0 + 32 * i) * C;
            const int64_t e0 = min(s0 + C, a.n_own);
            if (s0 >= a.n_own) {
                cnt[i] = 0;
            } else if (!ok[i]) {
                ss[i].n = 0;
                fmask[i] = ~0ull;                 // a row walked cold: the third pass takes it whole
                if (STAGED) {
                    const uint2 w2 = walk_cold_rec<LAYOUT, KS>(&a, s0, e0, ss[i].base, 0u);
                    cnt[i] = w2.x;
                    ss[i].n = w2.y;
                } else if (FIND)
                    cnt[i] = walk_cold<LAYOUT>(&a, s0, e0, &ss[i]);
                else {
                    CountSink cs;
                    cnt[i] = walk_cold<LAYOUT>(&a, s0, e0, &cs);
                }
            } else if (OPT && fmask[i] != 0ull) {
                const uint4 rc = replay_row<LAYOUT, FIND ? 1 : 0>(&a, s0, sps, fmask[i], ss[i].base, ss[i].n);
                cnt[i] += rc.x;
                if (FIND) ss[i].n = rc.y;
                fmask[i] = (uint64_t)rc.z | ((uint64_t)rc.w << 32);
            }
        }
        __syncwarp();
        if (FIND && lane == 0) mbar_arrive(&s_tfree[tslot]);

        if (!FIND) {
#pragma unroll
            for (int i = 0; i < kRPL; i++) total += cnt[i];
            if (STAGED || p.rows) {
                uint32_t ws = 0;
#pragma unroll
                for (int i = 0; i < kRPL; i++) {
                    const int64_t row = (int64_t)tile * kRows + wrow0 + 32 * i;
                    p.rows[row] = (uint16_t)cnt[i];
                    // the stages holding the row's exact accepts (all ones:
                    // the whole row), for the third pass of a relaxed layout
                    if (OPT && p.masks && cnt[i]) p.masks[row] = fmask[i];
                    ws += cnt[i];
                }
                if (STAGED && INLINE_REC) {
                    // the row's recorded end offsets (at most KS; a row with
                    // more is walked again by the third pass), packed in row
                    // order into this warp's region of the tile
                    const uint32_t stw = min(cnt[0], (uint32_t)KS);
                    if (__any_sync(0xffffffffu, stw != 0u)) {
                        uint32_t x = stw;
#pragma unroll
                        for (int o = 1; o < 32; o <<= 1) {
                            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
                            if (lane >= o) x += y;
                        }
                        uint16_t* region = p.stage + ((size_t)tile * kWalkWarps + warp) * (32 * KS) + (x - stw);
                        for (uint32_t j = 0; j < stw; j++) {
                            uint32_t v;
                            asm volatile("ld.shared.u16 %0, [%1];" : "=r"(v) : "r"(ss[0].base + j * (uint32_t)(kRows * 2)));
                            region[j] = (uint16_t)v;
                        }
                    }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) ws += __shfl_xor_sync(0xffffffffu, ws, o);
                if (lane == 0 && ws) atomicAdd(p.tile_sum + tile, (unsigned long long)ws);
                if (STAGED && lane == 0) p.warp_sum[(size_t)tile * kWalkWarps + warp] = ws;
            }
        } else {
            // exclusive offsets of this lane's rows among the warp's rows
            // (row i of every lane, then row i+1 of every lane)
            uint32_t excl[kRPL], wsum = 0;
#pragma unroll
            for (int i = 0; i < kRPL; i++) {
                uint32_t v = cnt[i];
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
                    if (lane >= o) v += y;
                }
                excl[i] = wsum + v - cnt[i];
                wsum += __shfl_sync(0xffffffffu, v, 31);
            }
            if (lane == 0) {
                s_wtot[kb][warp] = wsum;
                if (warp == 0) s_tile_of[kb] = tile;
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&s_counted[kb]);
            if (k >= kDefer - 1 && !flush(pend[kDefer - 2], k - (kDefer - 1))) {
                aborted = true;
                break;
            }
#pragma unroll
            for (int d = kDefer - 2; d > 0; d--)
#pragma unroll
                for (int i = 0; i < kRPL; i++) pend[d][i] = pend[d - 1][i];
#pragma unroll
            for (int i = 0; i < kRPL; i++) pend[0][i] = pend_pack(cnt[i], excl[i], ss[i].n > (uint32_t)KS);
        }
        k++;
    }
    if (aborted) {
        // wait for this warp's loads still in flight before the CTA's memory goes away
        for (uint32_t i = n_consumed; i < n_issued; i++) {
            const long long t0 = clock64();
            while (!mbar_try_wait(&full[c_slot], c_par) && clock64() - t0 < kWaitCycles) {
            }
            if (++c_slot == (uint32_t)nst) {
                c_slot = 0;
                c_par ^= 1u;
            }
        }
    }
    if (!FIND) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) total += __shfl_xor_sync(0xffffffffu, total, o);
        if (lane == 0) s_sum[warp] = total;
        if (OPT && p.scan_count) {
            // pass 1 of a two-pass find (relaxed layouts): the CTAs count
            // themselves out; the last one scans the tile totals (every
            // warp's atomics on them are fenced before its CTA's ticket; no
            // CTA waits for another)
            __shared__ int s_last;
            if (lane == 0) __threadfence();
            named_sync_walkers();
            if (threadIdx.x == 0) {
                __threadfence();
                s_last = atomicAdd(a.count, 1ull) == (unsigned long long)gridDim.x - 1ull;
            }
            named_sync_walkers();
            if (!s_last) return;
            __threadfence();
            scan_tile_totals(p.tile_sum, a.ntiles, p.scan_base ? *p.scan_base : 0ull, p.scan_count);
            return;
        }
        named_sync_walkers();
        if (threadIdx.x == 0 && !*abort_flag) {
            unsigned long long v = 0;
            for (int i = 0; i < kWalkWarps; i++) v += s_sum[i];
            if (v) atomicAdd(a.count, v);
        }
        return;
    }
    if (aborted) return;
    // end of work: tell the scheduler, then write the last tiles' positions
    const int b = (int)((uint64_t)k % kDefer);
    if (lane == 0 && warp == 0) s_tile_of[b] = -1;
    __syncwarp();
    if (lane == 0) mbar_arrive(&s_counted[b]);
#pragma unroll
    for (int d = kDefer - 2; d >= 0; d--)
        if (k >= d + 1 && !flush(pend[d], k - 1 - d)) return;
}

// ------------------------------------------------ two-pass find, passes 2, 3
//
// For the relaxed-walk layouts a find is: the count kernel writing every
// row's count and every tile's total (pass 1), an exclusive scan of the tile
// totals (pass 2, done by pass 1's last CTA: scan_tile_totals), and an exact
// walk of just the rows that hold an accept, each writing its positions at
// its own offset (pass 3).  Sparse patterns have few such rows, so the find
// costs little more than the count.

// Pass 2 of layout 1's two-pass find (one CTA of 1024 threads): tile_sum[t]
// becomes the global index of tile t's first position (base included);
// *count becomes base + total.  (The relaxed layouts scan in pass 1's last
// CTA; on the dense pass that tail cost more than this launch.)
__global__ void __launch_bounds__(1024)
    k_tile_offsets(unsigned long long* tile_sum, int64_t ntiles, const unsigned long long* base_in,
                   unsigned long long* count)
{
    __shared__ unsigned long long s_base;     // read before anyone writes *count
    if (threadIdx.x == 0) s_base = base_in ? *base_in : 0ull;
    __syncthreads();
    scan_tile_totals(tile_sum, ntiles, s_base, count);
}

// Pass 3 of the staged two-pass find, one warp per (tile, walker warp)
// unit: a row's first index is its tile's offset (pass 2) + the totals of the
// tile's earlier walker warps + a scan of the row counts within the warp.
// Layout 1 staged each row's exact end offsets (up to ks, packed in row order
// in the warp's region): they are copied.  The relaxed layouts left, per row
// with accepts, the mask of the stages holding them: the warp walks those
// bytes again.  Rows past their slots are walked again too.

// Every occurrence starting in [s, e) (the starts of one row, or a part of
// them that holds all its occurrences), found by the whole warp and written
// in order from index g0: lane l takes the l-th slice of the starts and reads
// m - 1 bytes past it (Algorithm 1 within the range), walking exactly with
// the single-step table (shared memory) over 16-byte loads of the text (16-B
// aligned: the staged find runs on aligned texts only).  The first four
// occurrences of each slice are kept in registers, so one walk serves count
// and positions; a slice with more walks again after the warp's scan.
// An exact walk of the starts [ls, le) by one lane, reading bytes up to hi
// in 16-byte loads (16-B aligned: the two-pass find runs on aligned texts
// only; never past n) with the single-step table d1s in shared memory.
// WRITE: every position to pos[g ...]; else the count, the first four
// positions kept in keep.
template <bool WRITE>
__device__ __forceinline__ uint32_t place_slice(const ScanArgs& a, const uint8_t* d1s, int64_t ls, int64_t le,
                                                int64_t hi, int64_t g, int64_t (&keep)[4])
{
    const uint32_t m = (uint32_t)a.m;
    uint32_t c = 0, q = 0;
    if (ls >= le) return 0;
    for (int64_t base = ls & ~(int64_t)15; base < hi; base += 16) {
        uint4 v;
        if (base + 16 <= a.n) {
            v = ldg16(reinterpret_cast<const uint4*>(a.text + base));
        } else {                                  // the text's last bytes: no read past n
            uint32_t w[4] = {0u, 0u, 0u, 0u};
            for (int64_t j = base; j < a.n; j++) w[(j - base) >> 2] |= (uint32_t)__ldg(a.text + j) << (8 * ((j - base) & 3));
            v = make_uint4(w[0], w[1], w[2], w[3]);
        }
        const int64_t j0 = max(ls, base), j1 = min(hi, base + 16);
        for (int64_t j = j0; j < j1; j++) {
            const uint32_t off = (uint32_t)(j - base);
            const uint32_t wd = off < 8u ? (off < 4u ? v.x : v.y) : (off < 12u ? v.z : v.w);
            const uint32_t b = (wd >> (8u * (off & 3u))) & 0xFFu;
            const uint32_t t = (b >> 2) & ~(b >> 1) & 1u;
            q = ((b ^ (t * 0x11u)) & 0xD9u) == 0x41u ? (uint32_t)d1s[q * 4u + ((b >> 1) & 3u)] : 0u;
            if (q == m) {
                const int64_t st = a.pos_base + j - (int64_t)(m - 1);
                if (WRITE) {
                    if (g + c < a.cap) a.pos[g + c] = st;
                } else if (c < 4u) {
                    keep[c] = st;
                }
                c++;
            }
        }
    }
    return c;
}

// Every occurrence starting in [s, e) (a row, or the part of one that holds
// all its occurrences), found by the whole warp and written in order from
// index g0: lane l takes the l-th slice of the starts and reads m - 1 bytes
// past it (Algorithm 1 within the range); a count (the first four positions
// kept), a warp scan, and a second walk only in slices with more than four.
// For the long ranges (a row walked whole): one lane alone would keep its
// warp waiting for a thousand dependent steps.
__device__ __noinline__ void place_range(const ScanArgs& a, const uint8_t* d1s, int64_t s, int64_t e, int64_t g0,
                                         int lane)
{
    const int64_t span = (e - s + 31) / 32;
    const int64_t ls = min(s + lane * span, e), le = min(ls + span, e);
    const int64_t hi = min(le + (int64_t)a.m - 1, a.n);
    int64_t keep[4];
    const uint32_t c = place_slice<false>(a, d1s, ls, le, hi, 0, keep);
    uint32_t x = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    const int64_t g = g0 + (int64_t)(x - c);
    if (c <= 4u) {
        for (uint32_t k = 0; k < c; k++)
            if (g + k < a.cap) a.pos[g + k] = keep[k];
    } else {
        place_slice<true>(a, d1s, ls, le, hi, g, keep);
    }
}

// Ranges up to this many starts are walked by one lane; longer ones by the
// warp (place_range).
constexpr int64_t kLaneRange = 128;

// Every occurrence starting in [s, e), walked by one lane alone (through
// min(e + m - 1, n)) and written in order from index g: the walk of
// place_slice with the next 16-byte load in flight while a block is walked,
// and a block's words of four bases stepped without the per-byte base test
// (out of line, so the calling kernel's own registers do not pay for it).
__device__ __noinline__ void place_row_lane(const ScanArgs& a, const uint8_t* d1s, int64_t s, int64_t e, int64_t g)
{
    const int64_t hi = min(e + (int64_t)a.m - 1, a.n);
    const uint32_t m = (uint32_t)a.m;
    if (s >= e) return;
    uint32_t q = 0;
    auto load16 = [&](int64_t base) -> uint4 {
        if (base + 16 <= a.n) return ldg16(reinterpret_cast<const uint4*>(a.text + base));
        uint32_t w[4] = {0u, 0u, 0u, 0u};            // the text's last bytes: no read past n
        for (int64_t j = base; j < a.n; j++) w[(j - base) >> 2] |= (uint32_t)__ldg(a.text + j) << (8 * ((j - base) & 3));
        return make_uint4(w[0], w[1], w[2], w[3]);
    };
    auto hit = [&](int64_t j) {
        if (g < a.cap) a.pos[g] = a.pos_base + j - (int64_t)(m - 1);
        g++;
    };
    auto step = [&](uint32_t b) {                   // one byte, any value
        const uint32_t t = (b >> 2) & ~(b >> 1) & 1u;
        q = ((b ^ (t * 0x11u)) & 0xD9u) == 0x41u ? (uint32_t)d1s[q * 4u + ((b >> 1) & 3u)] : 0u;
    };
    int64_t base = s & ~(int64_t)15;
    uint4 v = load16(base);
    for (; base < hi; base += 16) {
        const uint4 vn = base + 16 < hi ? load16(base + 16) : make_uint4(0u, 0u, 0u, 0u);
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
        if (s <= base && base + 16 <= hi) {
#pragma unroll
            for (int k = 0; k < 4; k++) {
                if (word_bad(w[k]) == 0u) {
#pragma unroll
                    for (int i = 0; i < 4; i++) {
                        q = d1s[q * 4u + ((w[k] >> (8 * i + 1)) & 3u)];
                        if (q == m) hit(base + 4 * k + i);
                    }
                } else {
                    for (int i = 0; i < 4; i++) {
                        step((w[k] >> (8 * i)) & 0xFFu);
                        if (q == m) hit(base + 4 * k + i);
                    }
                }
            }
        } else {
            const int64_t j0 = max(s, base), j1 = min(hi, base + 16);
            for (int64_t j = j0; j < j1; j++) {
                const uint32_t off = (uint32_t)(j - base);
                step((w[off >> 2] >> (8u * (off & 3u))) & 0xFFu);
                if (q == m) hit(j);
            }
        }
        v = vn;
    }
}

// The single-step table of the pattern, (m+1) x 4 bytes, into shared memory.
__device__ __forceinline__ const uint8_t* place_table(const ScanArgs& a)
{
    __shared__ uint8_t d1s[(DFA_MAX_M + 1) * 4];
    for (int i = threadIdx.x; i < (a.m + 1) * 4; i += blockDim.x) d1s[i] = a.tab[a.k4_bytes + i];
    __syncthreads();
    return d1s;
}

// A tile's 512 row counts, 16 a lane (lane l: rows 16 l .. 16 l + 15, from
// two 16-byte loads), and the lane's first index within the tile (an
// exclusive warp scan of the lanes' sums).
__device__ __forceinline__ uint32_t tile_rows(const uint16_t* rows, int64_t tile, int lane, uint32_t (&c)[16])
{
    const uint4* src = reinterpret_cast<const uint4*>(rows + tile * kRows + lane * 16);
    const uint4 u = src[0], v = src[1];
    const uint32_t w[8] = {u.x, u.y, u.z, u.w, v.x, v.y, v.z, v.w};
    uint32_t tot = 0;
#pragma unroll
    for (int k = 0; k < 8; k++) {
        c[2 * k] = w[k] & 0xFFFFu;
        c[2 * k + 1] = w[k] >> 16;
        tot += c[2 * k] + c[2 * k + 1];
    }
    uint32_t x = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    return x - tot;
}

// Pass 3 of the two-pass find.  A row's first index is its tile's offset
// (pass 2) + a scan of the counts of the tile's earlier rows.

// Layout 1, one warp per (tile, walker warp) region of 32 rows: the count
// pass staged each row's exact end offsets (up to kTSlotsDense), packed in
// row order in the region, and each walker warp's total; the offsets are
// copied, each row by its lane, the region's first index adding the totals
// of the tile's earlier walker warps.  Rows past their slots are walked
// again by the warp.
__global__ void __launch_bounds__(256)
    k_place(const __grid_constant__ ScanArgs a, const uint16_t* rows, const unsigned long long* tile_off,
            const uint16_t* stage, const uint32_t* warp_sum)
{
    constexpr uint32_t KS = kTSlotsDense;
    const uint8_t* d1s = place_table(a);
    const int lane = threadIdx.x & 31;
    const unsigned long long end_all = *a.count;
    const int64_t C = a.chunk;
    const int64_t units = a.ntiles * kWalkWarps;
    const int64_t stride = ((int64_t)gridDim.x * blockDim.x) >> 5;
    // two regions a round, their loads issued together
    for (int64_t u0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u0 < units; u0 += 2 * stride) {
        int64_t uu[2] = {u0, u0 + stride};
        unsigned long long off[2], nxt[2];
        uint32_t pre[2], rc[2];
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int64_t u = uu[h] < units ? uu[h] : u0;
            const int64_t tile = u / kWalkWarps;
            const int w = (int)(u % kWalkWarps);
            off[h] = tile_off[tile];
            nxt[h] = tile + 1 < a.ntiles ? tile_off[tile + 1] : end_all;
            // the counts of the tile's rows before this region: the totals of
            // the walker warps before it
            pre[h] = lane < w ? warp_sum[tile * kWalkWarps + lane] : 0u;
            rc[h] = rows[tile * kRows + w * 32 + lane];
        }
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int64_t u = uu[h];
            if (u >= units || off[h] == nxt[h]) continue;       // no accepts in the tile
            const int64_t tile = u / kWalkWarps;
            const int w = (int)(u % kWalkWarps);
            uint32_t p = pre[h];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) p += __shfl_xor_sync(0xffffffffu, p, o);
            const uint32_t st = min(rc[h], KS);
            uint32_t x = rc[h], y = st;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t q = __shfl_up_sync(0xffffffffu, x, o);
                const uint32_t r = __shfl_up_sync(0xffffffffu, y, o);
                if (lane >= o) {
                    x += q;
                    y += r;
                }
            }
            const int64_t rs = (tile * kRows + w * 32 + lane) * C;
            const int64_t g0 = (int64_t)(off[h] + p + x - rc[h]);
            if (rc[h] <= KS) {
                const int64_t start0 = a.pos_base + rs - (int64_t)(a.m - 1);
                const uint16_t* src = stage + u * (32 * (int64_t)KS) + (y - st);
                for (uint32_t j = 0; j < rc[h]; j++)
                    if (g0 + j < a.cap) a.pos[g0 + j] = start0 + src[j];
            }
            // rows past their slots: each walked again by the whole warp
            uint32_t over = __ballot_sync(0xffffffffu, rc[h] > KS);
            while (over) {
                const int r = __ffs(over) - 1;
                over &= over - 1u;
                const int64_t rr = __shfl_sync(0xffffffffu, rs, r);
                place_range(a, d1s, rr, min(rr + C, a.n_own), __shfl_sync(0xffffffffu, g0, r), lane);
            }
        }
    }
}

// Relaxed layouts, one warp per tile: the tile's rows with accepts are listed
// (their index in the tile and first index) in shared memory, then walked
// side by side, one listed row per lane, over the bytes the row's stage mask
// names: the starts from m - 1 bytes before its first masked stage to the
// end of its last one (every accept of the row ends in a masked stage, and
// every occurrence starting there is one of them).
constexpr int kPlaceWarps = 8;
__global__ void __launch_bounds__(kPlaceWarps * 32)
    k_place_masked(const __grid_constant__ ScanArgs a, const uint16_t* rows, const unsigned long long* tile_off,
                   const unsigned long long* masks)
{
    __shared__ uint32_t s_row[kPlaceWarps][kRows];     // row in the tile
    __shared__ uint32_t s_first[kPlaceWarps][kRows];   // first index within the tile
    const uint8_t* d1s = place_table(a);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned long long end_all = *a.count;
    const int64_t C = a.chunk;
    for (int64_t tile = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; tile < a.ntiles;
         tile += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const unsigned long long off = tile_off[tile];
        if (off == (tile + 1 < a.ntiles ? tile_off[tile + 1] : end_all)) continue;
        uint32_t c[16];
        uint32_t first = tile_rows(rows, tile, lane, c);
        uint32_t nr = 0;
#pragma unroll
        for (int k = 0; k < 16; k++) nr += c[k] != 0u ? 1u : 0u;
        uint32_t slot = nr;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t v = __shfl_up_sync(0xffffffffu, slot, o);
            if (lane >= o) slot += v;
        }
        const uint32_t total = __shfl_sync(0xffffffffu, slot, 31);
        slot -= nr;
#pragma unroll
        for (int k = 0; k < 16; k++) {
            if (c[k]) {
                s_row[wid][slot] = (uint32_t)(lane * 16 + k);
                s_first[wid][slot] = first;
                slot++;
            }
            first += c[k];
        }
        __syncwarp();
        for (uint32_t i0 = 0; i0 < total; i0 += 32) {
            const uint32_t i = i0 + (uint32_t)lane;
            int64_t s = 0, e = 0, g = 0;
            if (i < total) {
                const int64_t row = tile * kRows + s_row[wid][i];
                const int64_t rs = row * C;
                s = rs;
                e = min(rs + C, a.n_own);
                g = (int64_t)(off + s_first[wid][i]);
                const unsigned long long mask = masks[row];
                if (mask != ~0ull) {
                    const int64_t lo_stage = __ffsll((long long)mask) - 1;
                    const int64_t hi_stage = 63 - __clzll((long long)mask);
                    s = max(rs, rs + lo_stage * kStageW - (int64_t)(a.m - 1));
                    e = min(e, rs + (hi_stage + 1) * kStageW);
                }
            }
            const bool lng = e - s > kLaneRange;
            if (i < total && !lng) place_row_lane(a, d1s, s, e, g);
            uint32_t big = __ballot_sync(0xffffffffu, lng);      // long ranges: the whole warp
            while (big) {
                const int r = __ffs(big) - 1;
                big &= big - 1u;
                place_range(a, d1s, __shfl_sync(0xffffffffu, s, r), __shfl_sync(0xffffffffu, e, r),
                            __shfl_sync(0xffffffffu, g, r), lane);
            }
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------- host side

// Text of the last CUDA failure seen by this thread (dfa_last_error).
thread_local char g_last_error[256] = "";

int cuda_fail(cudaError_t err, const char* what)
{
    snprintf(g_last_error, sizeof(g_last_error), "%s: %s", what, cudaGetErrorString(err));
    return DFA_ECUDA;
}

int fail(const char* what)
{
    snprintf(g_last_error, sizeof(g_last_error), "%s", what);
    return DFA_ECUDA;
}

#define CUDA_TRY(x)                                   \
    do {                                              \
        cudaError_t err_ = (x);                       \
        if (err_ != cudaSuccess) return cuda_fail(err_, #x); \
    } while (0)

struct DeviceInfo {
    int sms = 0;
    int smem_optin = 0;
    int smem_per_sm = 0;
    bool ok = false;
};

std::mutex g_mu;
DeviceInfo g_dev[64];

const DeviceInfo* device_info(int dev)
{
    if (dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(g_mu);
    DeviceInfo& d = g_dev[dev];
    if (!d.ok) {
        if (cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return nullptr;
        if (cudaDeviceGetAttribute(&d.smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
            cudaSuccess)
            return nullptr;
        if (cudaDeviceGetAttribute(&d.smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) !=
            cudaSuccess)
            return nullptr;
        d.ok = true;
    }
    return &d;
}

// Per (kernel, device): raise the dynamic shared memory limit once, and cache
// occupancy by shared memory size.
struct KernelCache {
    const void* fn;
    int dev;
    int smem;
    int occ;
};
std::vector<KernelCache> g_kc;

int occupancy(const void* fn, int threads, int smem, int dev, int smem_optin)
{
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto& k : g_kc)
        if (k.fn == fn && k.dev == dev && k.smem == smem) return k.occ;
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, fn) != cudaSuccess) return 0;
    const int dyn_max = smem_optin - (int)fa.sharedSizeBytes;
    if (smem > dyn_max) return 0;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_max) != cudaSuccess)
        return 0;
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, threads, (size_t)smem) != cudaSuccess)
        occ = 0;
    g_kc.push_back({fn, dev, smem, occ});
    return occ;
}

struct Resolved {
    int layout, threads, loader, ctas_per_sm;
    int64_t chunk;
};

constexpr int64_t kMinDefaultTile = 256 * 64;   // workspace sizing for cfg == NULL

// Launch configuration for a scan of n bytes (n_avail readable).  The TMA
// loader needs a 16-byte aligned text holding at least two full rows.
int resolve(const dfa_config* cfg, int64_t n, int64_t n_avail, bool aligned, int sms, int m, bool find,
            Resolved* r)
{
    // default layout (the TMA kernel's): short patterns walk the four-step
    // table exactly; from kOptMinM on the relaxed walk takes the flagged
    // four-step table
    const bool user_layout = cfg && cfg->layout;
    r->layout = user_layout ? cfg->layout
                            : (m >= kOptMinM ? kLayoutK4F : kLayoutK4);
    r->ctas_per_sm = cfg ? cfg->ctas_per_sm : 0;
    if (r->layout != kLayoutK4 && r->layout != kLayoutStt && r->layout != kLayoutK4S && r->layout != kLayoutK4F)
        return DFA_EINVAL;
    if (r->ctas_per_sm < 0 || r->ctas_per_sm > 32) return DFA_EINVAL;
    const int req_loader = cfg ? cfg->loader : 0;
    if (req_loader < 0 || req_loader > 2) return DFA_EINVAL;
    if (sms <= 0) sms = 152;
    const bool tma_chunk = !(cfg && cfg->chunk) ||
                           (cfg->chunk % kStageW == 0 && cfg->chunk >= 2 * kStageW && cfg->chunk <= kStageW * 63);
    if (req_loader == 2 && !tma_chunk) return DFA_EINVAL;
    if (req_loader == 2 || (req_loader == 0 && tma_chunk)) {
        // TMA-staged tiles of 256 rows x chunk bytes, chunk a multiple of 80
        int64_t chunk;
        if (cfg && cfg->chunk) {
            chunk = cfg->chunk;
        } else {
            // at least four tiles per SM, rows of at most the measured best
            const int64_t per = (int64_t)kRows * kStageW * 4 * sms;
            int64_t sps = (n + per - 1) / per;
            const bool relaxed = r->layout == kLayoutK4F || r->layout == kLayoutK4S;
            const int64_t cap = relaxed ? kDefaultStagesRelaxed
                                : (find && r->layout == kLayoutK4 && m <= 8) ? kDefaultStagesDenseFind
                                                                            : kDefaultStagesExact;
            sps = std::min<int64_t>(std::max<int64_t>(sps, 2), cap);
            chunk = sps * kStageW;
        }
        const bool ok = aligned && n_avail / chunk >= 2;
        if (ok || req_loader == 2) {
            if (!ok) return DFA_EINVAL;
            r->loader = 2;
            r->threads = kRows;
            r->chunk = chunk;
            return DFA_OK;
        }
    }
    // the direct-load kernels have no k4s or k4f variant
    if (r->layout == kLayoutK4S || r->layout == kLayoutK4F) {
        if (user_layout && req_loader == 1) return DFA_EINVAL;
        r->layout = kLayoutK4;
    }
    r->loader = 1;
    r->threads = cfg && cfg->threads ? cfg->threads : 256;
    if (cfg && cfg->chunk && !(req_loader == 0 && tma_chunk)) {
        r->chunk = cfg->chunk;
    } else {
        int64_t per = (int64_t)r->threads * sms * 8;
        int64_t c = (n + per - 1) / per;
        c = (c + 15) & ~(int64_t)15;
        r->chunk = std::min<int64_t>(std::max<int64_t>(c, kMinDefaultTile / r->threads), 1024);
    }
    if (r->threads != 128 && r->threads != 256 && r->threads != 512) return DFA_EINVAL;
    if (r->chunk < 16 || r->chunk > 32768 || (r->chunk & 15)) return DFA_EINVAL;
    return DFA_OK;
}

typedef void (*KernelFn)(const ScanArgs);

KernelFn pick_count(int layout, int threads)
{
    if (layout == kLayoutK4) {
        if (threads == 128) return k_count<kLayoutK4, 128>;
        if (threads == 256) return k_count<kLayoutK4, 256>;
        return k_count<kLayoutK4, 512>;
    }
    if (threads == 128) return k_count<kLayoutStt, 128>;
    if (threads == 256) return k_count<kLayoutStt, 256>;
    return k_count<kLayoutStt, 512>;
}

KernelFn pick_find(int layout, int threads)
{
    if (layout == kLayoutK4) {
        if (threads == 128) return k_find<kLayoutK4, 128>;
        if (threads == 256) return k_find<kLayoutK4, 256>;
        return k_find<kLayoutK4, 512>;
    }
    if (threads == 128) return k_find<kLayoutStt, 128>;
    if (threads == 256) return k_find<kLayoutStt, 256>;
    return k_find<kLayoutStt, 512>;
}

int table_smem(const dfa_table* t, int layout)
{
    return layout == kLayoutK4    ? t->view.k4_bytes + t->view.d1_bytes
           : layout == kLayoutK4S ? t->view.k4s_bytes + t->view.d1_bytes
           : layout == kLayoutK4F ? t->view.k4f_bytes + t->view.k4_bytes + t->view.d1_bytes
                                  : t->view.stt_bytes;
}

typedef void (*TmaKernelFn)(const CUtensorMap, const TmaArgs);

// Finds of patterns this short record every accept inline (layouts 1, 2).
bool tma_dense(int layout, int m)
{
    return m <= kDenseMaxM && (layout == kLayoutK4 || layout == kLayoutStt);
}

// staged: pass 1 of the two-pass find of a dense pattern on layout 1 (count
// mode recording every exact accept); the relaxed layouts' pass 1 is their
// count kernel.
TmaKernelFn pick_tma(int layout, bool find, int m, bool staged)
{
    const bool dense = tma_dense(layout, m);
    if (layout == kLayoutK4S) return find ? k_scan_tma<kLayoutK4S, true, false> : k_scan_tma<kLayoutK4S, false, false>;
    if (layout == kLayoutK4F) return find ? k_scan_tma<kLayoutK4F, true, false> : k_scan_tma<kLayoutK4F, false, false>;
    if (layout == kLayoutK4) {
        if (staged) return k_scan_tma<kLayoutK4, false, true>;
        if (!find) return k_scan_tma<kLayoutK4, false, false>;
        return dense ? k_scan_tma<kLayoutK4, true, true> : k_scan_tma<kLayoutK4, true, false>;
    }
    if (!find) return k_scan_tma<kLayoutStt, false, false>;
    return dense ? k_scan_tma<kLayoutStt, true, true> : k_scan_tma<kLayoutStt, true, false>;
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

int tensor_map_encoder(PFN_cuTensorMapEncodeTiled_v12000* fn)
{
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_encode) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !p)
            return fail("cuTensorMapEncodeTiled entry point not found");
        g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    *fn = g_encode;
    return DFA_OK;
}

// Launch the TMA-staged kernel for the filled-in arguments `a`.
int launch_tma(const Resolved& r, const ScanArgs& a, const dfa_table* t, bool find, int dev,
               const DeviceInfo* di, cudaStream_t st, uint16_t* rows = nullptr, uint16_t* stage = nullptr,
               unsigned long long* masks = nullptr, uint32_t* warp_sum = nullptr,
               unsigned long long* scan_count = nullptr, const unsigned long long* scan_base = nullptr)
{
    PFN_cuTensorMapEncodeTiled_v12000 encode;
    int rc = tensor_map_encoder(&encode);
    if (rc) return rc;
    const int64_t C = r.chunk;
    TmaArgs p;
    p.a = a;
    p.nrows_full = a.n / C;
    p.sps = (int32_t)(C / kStageW);
    p.table_bytes = (table_smem(t, r.layout) + 127) & ~127;
    // a wait that gave up: the find workspace's status word (also for the
    // count pass of a two-pass find), else bit 63 of the count
    p.fail_word = find || rows ? a.work + 1 : a.count;
    p.fail_bit = find || rows ? 2ull : (1ull << 63);
    p.rows = rows;
    p.tile_sum = rows ? a.work + kWorkHeader : nullptr;
    p.stage = stage;
    p.masks = masks;
    p.warp_sum = warp_sum;
    p.scan_count = scan_count;
    p.scan_base = scan_base;
    CUtensorMap map;
    cuuint64_t dims[2] = {(cuuint64_t)C, (cuuint64_t)p.nrows_full};
    cuuint64_t strides[1] = {(cuuint64_t)C};
    cuuint32_t box[2] = {(cuuint32_t)kStageW, (cuuint32_t)kWarpRows};
    cuuint32_t estr[2] = {1, 1};
    if (encode(&map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<uint8_t*>(a.text), dims, strides, box,
               estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return fail("cuTensorMapEncodeTiled failed");
    const bool staged = !find && stage != nullptr;
    TmaKernelFn fn = pick_tma(r.layout, find, t->m, staged);
    cudaFuncAttributes fa;
    CUDA_TRY(cudaFuncGetAttributes(&fa, (const void*)fn));
    const int slot_bytes = find     ? kDefer * (tma_dense(r.layout, t->m) ? kTSlotsDense : kTSlots) * kRows * 2
                           : staged ? kTSlotsDense * kRows * 2
                                    : 0;
    p.rings_off = (p.table_bytes + slot_bytes + 1023) & ~1023;
    const int budget = di->smem_optin - (int)fa.sharedSizeBytes - p.rings_off;
    int nst = std::min(budget / (kWalkWarps * kWarpStage), kMaxStages);
    if (nst < 2) return DFA_EINVAL;
    // the relaxed count pass streams faster with two stages per warp ring
    // than with four (3.2e9 bytes, m = 16: 0.572 against 0.603 ms; the exact
    // count is the same with 2, 3 or 4)
    if (!find && (r.layout == kLayoutK4F || r.layout == kLayoutK4S)) nst = std::min(nst, kRelaxedCountStages);
    // the staged pass of layout 1: two CTAs per SM, each with two-stage rings
    const int ctas = staged ? 2 : 1;
    if (ctas == 2) nst = std::min(nst, 2);
    p.nst = nst;
    p.ahead = std::min(3 + (nst - 1) / (p.sps + 1), kTicketRing);
    const int smem = p.rings_off + kWalkWarps * nst * kWarpStage;
    const int threads = find ? kTmaThreads : kWalkThreads;
    int occ = occupancy((const void*)fn, threads, smem, dev, di->smem_optin);
    if (occ <= 0) return fail("TMA scan kernel does not fit on an SM (occupancy 0)");
    if (occ < ctas) return fail("TMA scan kernel: two CTAs do not fit on an SM");
    const int64_t grid = std::min<int64_t>(a.ntiles, (int64_t)di->sms * ctas);
    fn<<<(unsigned)grid, threads, smem, st>>>(map, p);
    CUDA_TRY(cudaGetLastError());
    return DFA_OK;
}

void fill_args(ScanArgs* a, const uint8_t* text, int64_t n, int64_t n_own, const dfa_table* t,
               const Resolved& r)
{
    memset(a, 0, sizeof(*a));
    a->text = text;
    a->n = n;
    a->n_own = n_own;
    a->chunk = r.chunk;
    const int64_t tb = (int64_t)r.threads * r.chunk;
    a->ntiles = (n_own + tb - 1) / tb;
    a->tab = static_cast<const uint8_t*>(t->d_mem);
    a->m = t->m;
    a->k4_bytes = t->view.k4_bytes;
    a->d1_bytes = t->view.d1_bytes;
    a->stt_bytes = t->view.stt_bytes;
    a->k4s_bytes = t->view.k4s_bytes;
    a->k4f_bytes = t->view.k4f_bytes;
    a->aligned = ((uintptr_t)text & 15u) == 0;
}

int current_device_info(const DeviceInfo** di, int* dev)
{
    if (cudaGetDevice(dev) != cudaSuccess) return DFA_ECUDA;
    *di = device_info(*dev);
    return *di ? DFA_OK : DFA_ECUDA;
}

int launch_count(const uint8_t* d_text, int64_t n, const dfa_table* t, uint64_t* d_count,
                 const dfa_config* cfg, cudaStream_t st)
{
    const DeviceInfo* di;
    int dev;
    int rc = current_device_info(&di, &dev);
    if (rc) return rc;
    if (dev != t->device) return DFA_EINVAL;
    Resolved r;
    rc = resolve(cfg, n, n, ((uintptr_t)d_text & 15u) == 0, di->sms, t->m, false, &r);
    if (rc) return rc;
    CUDA_TRY(cudaMemsetAsync(d_count, 0, sizeof(uint64_t), st));
    if (n < t->m) return DFA_OK;
    ScanArgs a;
    fill_args(&a, d_text, n, n, t, r);
    a.count = reinterpret_cast<unsigned long long*>(d_count);
    if (r.loader == 2) return launch_tma(r, a, t, false, dev, di, st);
    KernelFn fn = pick_count(r.layout, r.threads);
    const int smem = table_smem(t, r.layout);
    int occ = occupancy((const void*)fn, r.threads, smem, dev, di->smem_optin);
    if (occ <= 0) return fail("scan kernel does not fit on an SM (occupancy 0)");
    if (r.ctas_per_sm) occ = std::min(occ, r.ctas_per_sm);
    int64_t grid = std::min<int64_t>(a.ntiles, (int64_t)occ * di->sms);
    fn<<<(unsigned)grid, r.threads, smem, st>>>(a);
    CUDA_TRY(cudaGetLastError());
    return DFA_OK;
}

int64_t work_bytes_for(int64_t ntiles) { return 8 * (kWorkHeader + ntiles); }

// Two-pass find: [header][one word per tile][one u16 count per row of every
// tile, 16-byte aligned][16-byte aligned: layout 1, kTSlotsDense u16 end
// offsets per row, then one u32 total per walker warp of every tile;
// relaxed layouts, one u64 stage mask per row].
int64_t staged_rows_off(int64_t ntiles) { return (work_bytes_for(ntiles) + 15) & ~(int64_t)15; }
int64_t staged_tail_off(int64_t ntiles) { return (staged_rows_off(ntiles) + ntiles * kRows * 2 + 15) & ~(int64_t)15; }
int64_t staged_row_bytes(int layout) { return layout == kLayoutK4 ? 2 * kTSlotsDense : 8; }
int64_t staged_wsum_off(int64_t ntiles) { return staged_tail_off(ntiles) + ntiles * kRows * 2 * kTSlotsDense; }
int64_t work_bytes_two_pass(int64_t ntiles, int layout)
{
    const int64_t b = staged_tail_off(ntiles) + ntiles * kRows * staged_row_bytes(layout);
    return layout == kLayoutK4 ? b + ntiles * kWalkWarps * 4 : b;
}

// The staged two-pass find serves the TMA kernel's four-step layouts: the
// relaxed ones (3, 4) at any m, layout 1 for m <= 8 (its accepts are tested
// against their m-byte windows, which the 8 bytes kept before each stage
// cover).
bool two_pass_layout(const Resolved& r, int m)
{
    return r.loader == 2 && (r.layout == kLayoutK4F || r.layout == kLayoutK4S || (r.layout == kLayoutK4 && m <= 8));
}

// Passes 1-3 of the staged two-pass find (see scan_tile_totals, k_tile_offsets, k_place); the
// header and tile words of the workspace are already zero.
int launch_two_pass(const Resolved& r, const ScanArgs& a, const dfa_table* t, int dev, const DeviceInfo* di,
                    cudaStream_t st)
{
    unsigned long long* tile_sum = a.work + kWorkHeader;
    uint8_t* wb = reinterpret_cast<uint8_t*>(a.work);
    uint16_t* rows = reinterpret_cast<uint16_t*>(wb + staged_rows_off(a.ntiles));
    const bool dense = r.layout == kLayoutK4;
    uint16_t* stage = dense ? reinterpret_cast<uint16_t*>(wb + staged_tail_off(a.ntiles)) : nullptr;
    unsigned long long* masks = dense ? nullptr : reinterpret_cast<unsigned long long*>(wb + staged_tail_off(a.ntiles));
    ScanArgs a1 = a;
    // the unused ticket word: pass 1's total (layout 1), else its count of
    // finished CTAs (pass 2, the tile scan, runs in its last CTA)
    a1.count = a.work;
    uint32_t* wsum = dense ? reinterpret_cast<uint32_t*>(wb + staged_wsum_off(a.ntiles)) : nullptr;
    int rc = launch_tma(r, a1, t, false, dev, di, st, rows, stage, masks, wsum, dense ? nullptr : a.count,
                        a.base_in);
    if (rc) return rc;
    if (dense) {
        k_tile_offsets<<<1, 1024, 0, st>>>(tile_sum, a.ntiles, a.base_in, a.count);
        CUDA_TRY(cudaGetLastError());
    }
    const void* fn = dense ? (const void*)k_place : (const void*)k_place_masked;
    int occ = occupancy(fn, 256, 0, dev, di->smem_optin);
    if (occ <= 0) return fail("placement kernel does not fit on an SM (occupancy 0)");
    // warps: one per 32-row region (layout 1) or one per tile
    const int64_t warps = dense ? a.ntiles * kWalkWarps : a.ntiles;
    const int64_t grid = std::min<int64_t>((warps + 7) / 8, (int64_t)occ * di->sms);
    if (dense)
        k_place<<<(unsigned)grid, 256, 0, st>>>(a, rows, tile_sum, stage, wsum);
    else
        k_place_masked<<<(unsigned)grid, 256, 0, st>>>(a, rows, tile_sum, masks);
    CUDA_TRY(cudaGetLastError());
    return DFA_OK;
}

// Shared by dfa_find and the segmented host path.
int launch_find(const uint8_t* d_text, int64_t n, int64_t n_own, const dfa_table* t, int64_t* d_pos,
                int64_t cap, uint64_t* d_count, const uint64_t* d_base, int64_t pos_base, void* d_work,
                int64_t work_bytes, const dfa_config* cfg, cudaStream_t st)
{
    const DeviceInfo* di;
    int dev;
    int rc = current_device_info(&di, &dev);
    if (rc) return rc;
    if (dev != t->device) return DFA_EINVAL;
    Resolved r;
    rc = resolve(cfg, n_own, n, ((uintptr_t)d_text & 15u) == 0, di->sms, t->m, true, &r);
    if (rc) return rc;
    ScanArgs a;
    fill_args(&a, d_text, n, n_own, t, r);
    const int64_t need = work_bytes_for(a.ntiles);
    if (work_bytes < need) return DFA_EWORKSPACE;
    if ((reinterpret_cast<uintptr_t>(d_work) & 15u) != 0) return DFA_EINVAL;   // u64 words, 16-byte parts
    CUDA_TRY(cudaMemsetAsync(d_work, 0, (size_t)need, st));
    if (a.ntiles == 0) {
        if (d_base)
            CUDA_TRY(cudaMemcpyAsync(d_count, d_base, 8, cudaMemcpyDeviceToDevice, st));
        else
            CUDA_TRY(cudaMemsetAsync(d_count, 0, 8, st));
        return DFA_OK;
    }
    a.count = reinterpret_cast<unsigned long long*>(d_count);
    a.pos = d_pos;
    a.cap = d_pos ? cap : 0;
    a.pos_base = pos_base;
    a.base_in = reinterpret_cast<const unsigned long long*>(d_base);
    a.work = static_cast<unsigned long long*>(d_work);
    if (two_pass_layout(r, t->m) && work_bytes >= work_bytes_two_pass(a.ntiles, r.layout))
        return launch_two_pass(r, a, t, dev, di, st);
    if (r.loader == 2) return launch_tma(r, a, t, true, dev, di, st);
    KernelFn fn = pick_find(r.layout, r.threads);
    const int smem = ((table_smem(t, r.layout) + 15) & ~15) + kSlots * r.threads * 2;
    int occ = occupancy((const void*)fn, r.threads, smem, dev, di->smem_optin);
    if (occ <= 0) return fail("scan kernel does not fit on an SM (occupancy 0)");
    if (r.ctas_per_sm) occ = std::min(occ, r.ctas_per_sm);
    int64_t grid = std::min<int64_t>(a.ntiles, (int64_t)occ * di->sms);
    fn<<<(unsigned)grid, r.threads, smem, st>>>(a);
    CUDA_TRY(cudaGetLastError());
    return DFA_OK;
}

}  // namespace

namespace dnadfa {
int set_last_error(int code, const char* msg)
{
    snprintf(g_last_error, sizeof(g_last_error), "%s", msg);
    return code;
}
}  // namespace dnadfa

namespace {
// acc |= the status word of a find's workspace (its bounded waits).
__global__ void k_or_status(const unsigned long long* work, unsigned long long* acc)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) *acc |= work[1];
}

// A wait of the find that just ran gave up: mark its count (bit 63).
__global__ void k_status_to_count(const unsigned long long* work, unsigned long long* count)
{
    if (threadIdx.x == 0 && blockIdx.x == 0 && work[1]) *count |= 1ull << 63;
}

// One warp runs the ordered compaction's look-back for `tile` on a
// workspace (dfa_debug_wait_timeout).
__global__ void k_debug_lookback(unsigned long long* work, int64_t tile)
{
    lookback_warp(work, tile, 1ull, (int)(threadIdx.x & 31));
}
}  // namespace

// ==================================================================== C ABI

namespace {

// Host part of dfa_build / dfa_build_into: validated pattern, host tables,
// sizes of the device image and the image itself in t->img.
int make_table(const char* pattern, int32_t m, dfa_table** out)
{
    if (!pattern || !out || m < 1 || m > DFA_MAX_M) return DFA_EINVAL;
    *out = nullptr;
    dfa_table* t = new (std::nothrow) dfa_table();
    if (!t) return DFA_ENOMEM;
    t->m = m;
    for (int j = 0; j < m; j++) {
        uint32_t c = (uint8_t)pattern[j];
        if (!code_valid(c)) {
            delete t;
            return DFA_EINVAL;
        }
        t->pattern[j] = (uint8_t)(c & 0xDFu);
    }
    int rc = build_host_tables(t);
    if (rc) {
        delete t;
        return rc;
    }
    t->view.m = m;
    t->view.k4_bytes = (m + 1) * 512;
    t->view.d1_bytes = ((m + 1) * 4 + 15) & ~15;
    t->view.stt_bytes = (m + 1) * 256;
    t->view.k4s_bytes = (m + 1) * 256;
    t->view.k4f_bytes = (int32_t)t->k4f.size();
    t->d_bytes = (size_t)t->view.k4_bytes + t->view.d1_bytes + t->view.stt_bytes + t->view.k4s_bytes +
                 t->view.k4f_bytes;
    std::vector<uint8_t>& img = t->img;
    img.assign(t->d_bytes, 0);
    memcpy(img.data(), t->k4.data(), (size_t)t->view.k4_bytes);
    memcpy(img.data() + t->view.k4_bytes, t->d1.data(), t->d1.size());
    memcpy(img.data() + t->view.k4_bytes + t->view.d1_bytes, t->stt.data(), t->stt.size());
    memcpy(img.data() + t->view.k4_bytes + t->view.d1_bytes + t->view.stt_bytes, t->k4s.data(), t->k4s.size());
    if (!t->k4f.empty())
        memcpy(img.data() + t->view.k4_bytes + t->view.d1_bytes + t->view.stt_bytes + t->view.k4s_bytes,
               t->k4f.data(), t->k4f.size());
    *out = t;
    return DFA_OK;
}

}  // namespace

extern "C" {

int dfa_build(const char* pattern, int32_t m, dfa_table** out)
{
    dfa_table* t = nullptr;
    int rc = make_table(pattern, m, &t);
    if (rc) return rc;
    if (cudaGetDevice(&t->device) != cudaSuccess || cudaMalloc(&t->d_mem, t->d_bytes) != cudaSuccess) {
        cudaGetLastError();
        delete t;
        return DFA_ECUDA;
    }
    if (cudaMemcpy(t->d_mem, t->img.data(), t->d_bytes, cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(t->d_mem);
        delete t;
        return DFA_ECUDA;
    }
    std::vector<uint8_t>().swap(t->img);
    t->view.base = static_cast<const uint8_t*>(t->d_mem);
    *out = t;
    return DFA_OK;
}

int64_t dfa_table_bytes(int32_t m)
{
    if (m < 1 || m > DFA_MAX_M) return -1;
    return (int64_t)(m + 1) * 512 + (((m + 1) * 4 + 15) & ~15) + (int64_t)(m + 1) * 256 * 2 +
           (int64_t)(k4f_flag(m) + m + 1) * 256;
}

int dfa_build_into(const char* pattern, int32_t m, void* d_mem, int64_t bytes, void* stream, dfa_table** out)
{
    if (!out) return DFA_EINVAL;
    *out = nullptr;
    if (!d_mem || (reinterpret_cast<uintptr_t>(d_mem) & 15u) || bytes < dfa_table_bytes(m))
        return DFA_EINVAL;
    dfa_table* t = nullptr;
    int rc = make_table(pattern, m, &t);
    if (rc) return rc;
    cudaError_t err;
    if ((err = cudaGetDevice(&t->device)) != cudaSuccess ||
        (err = cudaMemcpyAsync(d_mem, t->img.data(), t->d_bytes, cudaMemcpyHostToDevice,
                               static_cast<cudaStream_t>(stream))) != cudaSuccess) {
        delete t;
        return cuda_fail(err, "dfa_build_into");
    }
    t->d_mem = d_mem;
    t->owns_mem = false;
    t->view.base = static_cast<const uint8_t*>(d_mem);
    *out = t;
    return DFA_OK;
}

void dfa_free(dfa_table* table)
{
    if (!table) return;
    if (table->d_mem && table->owns_mem) {
        int cur = -1;
        cudaGetDevice(&cur);
        if (cur != table->device) cudaSetDevice(table->device);
        cudaFree(table->d_mem);
        if (cur >= 0 && cur != table->device) cudaSetDevice(cur);
    }
    delete table;
}

int32_t dfa_pattern_length(const dfa_table* table) { return table ? table->m : -1; }

int dfa_export_stt(const dfa_table* table, uint8_t* h_stt, int64_t bytes)
{
    if (!table || !h_stt || bytes < (int64_t)table->stt.size()) return DFA_EINVAL;
    memcpy(h_stt, table->stt.data(), table->stt.size());
    return DFA_OK;
}

int dfa_count(const uint8_t* d_text, int64_t n, const dfa_table* table, uint64_t* d_count,
              const dfa_config* cfg, void* stream)
{
    if (!table || !d_count || n < 0 || (n > 0 && !d_text)) return DFA_EINVAL;
    return launch_count(d_text, n, table, d_count, cfg, static_cast<cudaStream_t>(stream));
}

int64_t dfa_find_workspace_bytes(int64_t n, const dfa_config* cfg)
{
    if (n < 0) return -1;
    int64_t tb;
    if (cfg && cfg->threads && cfg->chunk) {
        tb = (int64_t)cfg->threads * cfg->chunk;
        if (tb <= 0) return -1;
    } else {
        tb = kMinDefaultTile;
    }
    const int64_t single = work_bytes_for((n + tb - 1) / tb);
    // room for the two-pass find of the TMA kernel as well: its tiles are
    // kRows rows of the chunk resolve picks on the current device
    int sms = 0, dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) {
        const DeviceInfo* di = device_info(dev);
        if (di) sms = di->sms;
    }
    if (sms <= 0) {
        (void)cudaGetLastError();
        sms = 152;
    }
    // the default layout and rows depend on m (layout 1 below kOptMinM,
    // a relaxed layout from there on): size for both
    int64_t need = single;
    for (int m : {1, kOptMinM}) {
        Resolved r;
        if (resolve(cfg, n, n, true, sms, m, true, &r) == DFA_OK && two_pass_layout(r, m)) {
            const int64_t tile_bytes = (int64_t)kRows * r.chunk;
            need = std::max(need, work_bytes_two_pass((n + tile_bytes - 1) / tile_bytes, r.layout));
        }
    }
    return need;
}

int dfa_find(const uint8_t* d_text, int64_t n, const dfa_table* table, int64_t* d_pos, int64_t cap,
             uint64_t* d_count, void* d_work, int64_t work_bytes, const dfa_config* cfg, void* stream)
{
    if (!table || !d_count || !d_work || n < 0 || (n > 0 && !d_text) || cap < 0 ||
        (cap > 0 && !d_pos))
        return DFA_EINVAL;
    return launch_find(d_text, n, n, table, d_pos, cap, d_count, nullptr, 0, d_work, work_bytes, cfg,
                       static_cast<cudaStream_t>(stream));
}

int dfa_find_status(const void* d_work, const uint64_t* d_count, int64_t cap, uint64_t* h_count,
                    void* stream)
{
    if (!d_work || !d_count) return DFA_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned long long hdr[2] = {0, 0};
    uint64_t cnt = 0;
    if (cudaStreamSynchronize(st) != cudaSuccess) return DFA_ECUDA;
    if (cudaMemcpy(hdr, d_work, sizeof(hdr), cudaMemcpyDeviceToHost) != cudaSuccess) return DFA_ECUDA;
    if (cudaMemcpy(&cnt, d_count, 8, cudaMemcpyDeviceToHost) != cudaSuccess) return DFA_ECUDA;
    if (h_count) *h_count = cnt;
    if (hdr[1]) return DFA_ETIMEOUT;
    if ((int64_t)cnt > cap) return DFA_ETRUNC;
    return DFA_OK;
}

// Segmented host path: staging = [2 segment buffers][positions][2 counters][workspace]
static int64_t stage_layout(int64_t seg, int64_t cap, int64_t* seg_stride, int64_t* pos_off,
                            int64_t* cnt_off, int64_t* work_off)
{
    *seg_stride = (seg + DFA_MAX_M + 255) & ~(int64_t)255;
    *pos_off = 2 * *seg_stride;
    *cnt_off = *pos_off + ((cap * 8 + 255) & ~(int64_t)255);
    *work_off = *cnt_off + 256;
    int64_t wb = dfa_find_workspace_bytes(seg, nullptr);
    return *work_off + wb;
}

int64_t dfa_host_stage_bytes(int64_t seg, int64_t cap)
{
    if (seg < (1 << 20) || cap < 0) return -1;
    int64_t a, b, c, d;
    return stage_layout(seg, cap, &a, &b, &c, &d);
}

int dfa_find_host(const uint8_t* h_text, int64_t n, const dfa_table* table, int64_t* h_pos, int64_t cap,
                  uint64_t* h_count, void* d_stage, int64_t stage_bytes, int64_t seg, void* stream)
{
    if (!table || !h_count || !d_stage || n < 0 || (n > 0 && !h_text) || cap < 0 ||
        (cap > 0 && !h_pos) || seg < (1 << 20))
        return DFA_EINVAL;
    int64_t seg_stride, pos_off, cnt_off, work_off;
    int64_t need = stage_layout(seg, cap, &seg_stride, &pos_off, &cnt_off, &work_off);
    if (stage_bytes < need) return DFA_EWORKSPACE;
    uint8_t* stage = static_cast<uint8_t*>(d_stage);
    int64_t* d_pos = cap > 0 ? reinterpret_cast<int64_t*>(stage + pos_off) : nullptr;
    uint64_t* d_cnt = reinterpret_cast<uint64_t*>(stage + cnt_off);   // two ping-pong counters
    void* d_work = stage + work_off;
    const int64_t work_bytes = stage_bytes - work_off;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int m = table->m;

    cudaStream_t cp;
    cudaEvent_t copied[2], scanned[2];
    if (cudaStreamCreateWithFlags(&cp, cudaStreamNonBlocking) != cudaSuccess) return DFA_ECUDA;
    int rc = DFA_OK;
    for (int i = 0; i < 2; i++) {
        cudaEventCreateWithFlags(&copied[i], cudaEventDisableTiming);
        cudaEventCreateWithFlags(&scanned[i], cudaEventDisableTiming);
    }
    if (cudaMemsetAsync(d_cnt, 0, 16, st) != cudaSuccess) rc = DFA_ECUDA;
    // the copy stream starts after the counters are cleared
    cudaEventRecord(scanned[1], st);
    cudaEventRecord(scanned[0], st);
    const int64_t nseg = n > 0 ? (n + seg - 1) / seg : 0;
    for (int64_t k = 0; k < nseg && rc == DFA_OK; k++) {
        const int b = (int)(k & 1);
        const int64_t lo = k * seg;
        const int64_t own = std::min(seg, n - lo);
        const int64_t avail = std::min(own + m - 1, n - lo);
        uint8_t* buf = stage + b * seg_stride;
        // buffer b was last read by scan k-2
        if (cudaStreamWaitEvent(cp, scanned[b], 0) != cudaSuccess ||
            cudaMemcpyAsync(buf, h_text + lo, (size_t)avail, cudaMemcpyHostToDevice, cp) != cudaSuccess ||
            cudaEventRecord(copied[b], cp) != cudaSuccess || cudaStreamWaitEvent(st, copied[b], 0) != cudaSuccess) {
            rc = DFA_ECUDA;
            break;
        }
        const uint64_t* base = d_cnt + ((k + 1) & 1);     // previous segment's running total
        uint64_t* outc = d_cnt + (k & 1);
        rc = launch_find(buf, avail, own, table, d_pos, cap, outc, k ? base : nullptr, lo, d_work,
                         work_bytes, nullptr, st);
        if (rc == DFA_OK && cudaEventRecord(scanned[b], st) != cudaSuccess) rc = DFA_ECUDA;
    }
    uint64_t cnt = 0;
    unsigned long long hdr[2] = {0, 0};
    if (rc == DFA_OK) {
        const uint64_t* last = nseg ? d_cnt + ((nseg - 1) & 1) : d_cnt;
        if (cudaMemcpyAsync(&cnt, last, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaMemcpyAsync(hdr, d_work, 16, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            rc = DFA_ECUDA;
    }
    if (rc == DFA_OK && cap > 0 && cnt > 0) {
        int64_t k = std::min<int64_t>((int64_t)cnt, cap);
        if (cudaMemcpyAsync(h_pos, d_pos, (size_t)k * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            rc = DFA_ECUDA;
    }
    cudaStreamSynchronize(cp);
    for (int i = 0; i < 2; i++) {
        cudaEventDestroy(copied[i]);
        cudaEventDestroy(scanned[i]);
    }
    cudaStreamDestroy(cp);
    if (rc != DFA_OK) return rc;
    *h_count = cnt;
    if (hdr[1]) return DFA_ETIMEOUT;
    if ((int64_t)cnt > cap) return DFA_ETRUNC;
    return DFA_OK;
}

// Segmented host path for several patterns: [2 segment buffers][positions
// of each pattern][2 counters per pattern][status accumulator][workspace]
static int64_t stage_layout_multi(int64_t seg, const int64_t* caps, int32_t npat, int64_t* seg_stride,
                                  int64_t* pos_off, int64_t* cnt_off, int64_t* work_off)
{
    *seg_stride = (seg + DFA_MAX_M + 255) & ~(int64_t)255;
    int64_t o = 2 * *seg_stride;
    for (int32_t i = 0; i < npat; i++) {
        if (pos_off) pos_off[i] = o;
        o += (caps[i] * 8 + 255) & ~(int64_t)255;
    }
    *cnt_off = o;
    o += ((int64_t)npat * 16 + 8 + 255) & ~(int64_t)255;
    *work_off = o;
    return o + dfa_find_workspace_bytes(seg, nullptr);
}

constexpr int32_t kHostMaxPat = 1024;

int64_t dfa_host_stage_bytes_multi(int64_t seg, const int64_t* caps, int32_t npat)
{
    if (seg < (1 << 20) || !caps || npat < 1 || npat > kHostMaxPat) return -1;
    for (int32_t i = 0; i < npat; i++)
        if (caps[i] < 0) return -1;
    int64_t a, c, d;
    return stage_layout_multi(seg, caps, npat, &a, nullptr, &c, &d);
}

int dfa_find_host_multi(const uint8_t* h_text, int64_t n, const dfa_table* const* tables, int32_t npat,
                        int64_t* const* h_pos, const int64_t* caps, uint64_t* h_counts, void* d_stage,
                        int64_t stage_bytes, int64_t seg, void* stream)
{
    if (!tables || !caps || !h_counts || !d_stage || npat < 1 || npat > kHostMaxPat || n < 0 ||
        (n > 0 && !h_text) || seg < (1 << 20))
        return DFA_EINVAL;
    int mmax = 1;
    for (int32_t i = 0; i < npat; i++) {
        if (!tables[i] || caps[i] < 0 || (caps[i] > 0 && (!h_pos || !h_pos[i]))) return DFA_EINVAL;
        mmax = std::max(mmax, (int)tables[i]->m);
    }
    std::vector<int64_t> pos_off(npat);
    int64_t seg_stride, cnt_off, work_off;
    const int64_t need = stage_layout_multi(seg, caps, npat, &seg_stride, pos_off.data(), &cnt_off, &work_off);
    if (stage_bytes < need) return DFA_EWORKSPACE;
    uint8_t* stage = static_cast<uint8_t*>(d_stage);
    uint64_t* d_cnt = reinterpret_cast<uint64_t*>(stage + cnt_off);   // 2 per pattern, then the status
    unsigned long long* d_status = reinterpret_cast<unsigned long long*>(d_cnt + 2 * npat);
    void* d_work = stage + work_off;
    const int64_t work_bytes = stage_bytes - work_off;
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    cudaStream_t cp;
    cudaEvent_t copied[2], scanned[2];
    if (cudaStreamCreateWithFlags(&cp, cudaStreamNonBlocking) != cudaSuccess) return DFA_ECUDA;
    int rc = DFA_OK;
    for (int i = 0; i < 2; i++) {
        cudaEventCreateWithFlags(&copied[i], cudaEventDisableTiming);
        cudaEventCreateWithFlags(&scanned[i], cudaEventDisableTiming);
    }
    if (cudaMemsetAsync(d_cnt, 0, (size_t)npat * 16 + 8, st) != cudaSuccess) rc = DFA_ECUDA;
    cudaEventRecord(scanned[1], st);
    cudaEventRecord(scanned[0], st);
    const int64_t nseg = n > 0 ? (n + seg - 1) / seg : 0;
    for (int64_t k = 0; k < nseg && rc == DFA_OK; k++) {
        const int b = (int)(k & 1);
        const int64_t lo = k * seg;
        const int64_t own = std::min(seg, n - lo);
        const int64_t avail = std::min(own + mmax - 1, n - lo);
        uint8_t* buf = stage + b * seg_stride;
        // one copy of the segment (with the longest pattern's overlap) for
        // every pattern; buffer b was last read by the scans of segment k-2
        if (cudaStreamWaitEvent(cp, scanned[b], 0) != cudaSuccess ||
            cudaMemcpyAsync(buf, h_text + lo, (size_t)avail, cudaMemcpyHostToDevice, cp) != cudaSuccess ||
            cudaEventRecord(copied[b], cp) != cudaSuccess || cudaStreamWaitEvent(st, copied[b], 0) != cudaSuccess) {
            rc = DFA_ECUDA;
            break;
        }
        for (int32_t i = 0; i < npat && rc == DFA_OK; i++) {
            uint64_t* ci = d_cnt + 2 * i;
            const uint64_t* base = ci + ((k + 1) & 1);       // this pattern's running total
            int64_t* d_pos = caps[i] > 0 ? reinterpret_cast<int64_t*>(stage + pos_off[i]) : nullptr;
            rc = launch_find(buf, avail, own, tables[i], d_pos, caps[i], ci + (k & 1), k ? base : nullptr, lo,
                             d_work, work_bytes, nullptr, st);
            if (rc == DFA_OK) {
                k_or_status<<<1, 32, 0, st>>>(static_cast<const unsigned long long*>(d_work), d_status);
                if (cudaGetLastError() != cudaSuccess) rc = DFA_ECUDA;
            }
        }
        if (rc == DFA_OK && cudaEventRecord(scanned[b], st) != cudaSuccess) rc = DFA_ECUDA;
    }
    std::vector<unsigned long long> hc((size_t)npat * 2 + 1, 0);
    if (rc == DFA_OK) {
        if (cudaMemcpyAsync(hc.data(), d_cnt, hc.size() * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            rc = DFA_ECUDA;
    }
    bool trunc = false;
    for (int32_t i = 0; rc == DFA_OK && i < npat; i++) {
        const uint64_t c = nseg ? hc[2 * i + ((nseg - 1) & 1)] : 0;
        h_counts[i] = c;
        trunc |= (int64_t)c > caps[i];
        const int64_t kk = std::min<int64_t>((int64_t)c, caps[i]);
        if (kk > 0 && cudaMemcpyAsync(h_pos[i], stage + pos_off[i], (size_t)kk * 8, cudaMemcpyDeviceToHost, st) !=
                          cudaSuccess)
            rc = DFA_ECUDA;
    }
    if (rc == DFA_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = DFA_ECUDA;
    cudaStreamSynchronize(cp);
    for (int i = 0; i < 2; i++) {
        cudaEventDestroy(copied[i]);
        cudaEventDestroy(scanned[i]);
    }
    cudaStreamDestroy(cp);
    if (rc != DFA_OK) return rc;
    if (hc[(size_t)npat * 2]) return DFA_ETIMEOUT;
    return trunc ? DFA_ETRUNC : DFA_OK;
}

int dfa_find_batched(const uint8_t* d_text, int64_t n, const dfa_table* const* tables, int32_t npat,
                     int64_t* const* d_pos, const int64_t* caps, uint64_t* d_counts, void* d_work,
                     int64_t work_bytes, const dfa_config* cfg, void* stream)
{
    if (!tables || !caps || !d_counts || !d_work || npat < 1 || npat > kHostMaxPat || n < 0 ||
        (n > 0 && !d_text))
        return DFA_EINVAL;
    for (int32_t i = 0; i < npat; i++)
        if (!tables[i] || caps[i] < 0 || (caps[i] > 0 && (!d_pos || !d_pos[i]))) return DFA_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    for (int32_t i = 0; i < npat; i++) {
        const int rc = launch_find(d_text, n, n, tables[i], caps[i] > 0 ? d_pos[i] : nullptr, caps[i],
                                   d_counts + i, nullptr, 0, d_work, work_bytes, cfg, st);
        if (rc) return rc;
        if (n > 0) {
            k_status_to_count<<<1, 32, 0, st>>>(static_cast<const unsigned long long*>(d_work),
                                                reinterpret_cast<unsigned long long*>(d_counts + i));
            CUDA_TRY(cudaGetLastError());
        }
    }
    return DFA_OK;
}

int dfa_debug_wait_timeout(void* d_work, int64_t work_bytes, int64_t tile, void* stream)
{
    if (!d_work || tile < 1 || work_bytes < work_bytes_for(tile + 1)) return DFA_EINVAL;
    k_debug_lookback<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(
        static_cast<unsigned long long*>(d_work), tile);
    CUDA_TRY(cudaGetLastError());
    return DFA_OK;
}

const char* dfa_strerror(int code)
{
    switch (code) {
    case DFA_OK: return "ok";
    case DFA_EINVAL: return "invalid argument";
    case DFA_ETRUNC: return "more occurrences than the position buffer holds";
    case DFA_ETIMEOUT: return "a bounded device-side wait gave up";
    case DFA_ECUDA: return "CUDA runtime error";
    case DFA_EWORKSPACE: return "workspace too small";
    case DFA_ENOMEM: return "out of memory";
    default: return "unknown error";
    }
}

const char* dfa_version(void) { return "dnadfa 0.1 (sm_103a)"; }

const char* dfa_last_error(void) { return g_last_error; }

}  // extern "C"

// ================================================= find without an allocation
//
// dfa_find_noalloc runs dfa_find with its workspace (the ticket, the status
// word and one look-back descriptor per tile) in a fixed array of this
// library's device memory instead of memory the caller provides.  The paper
// has no counterpart: it exists for callers that may not allocate device
// memory at all (see include/dnadfa.h).

namespace {

// Tiles the static workspace can describe.  A tile is the text one CTA
// takes per ticket (threads x chunk bytes of the resolved launch; by default
// for multi-GB texts 384 KiB for patterns of 8 and more and 480 KiB below,
// so the default limit is about 24 GiB).
constexpr int64_t kNoAllocTiles = 65536;
constexpr int kNoAllocMaxDevices = 64;

}  // namespace

// The shared workspace: [0] ticket, [1] status, then one word per tile
// (512 KiB + 16 bytes, held on every device that loads the library until the
// process exits).  In host code this name is only a handle for
// cudaGetSymbolAddress, never a device address.
static __device__ __align__(256) unsigned long long g_noalloc_work[kWorkHeader + kNoAllocTiles];

namespace {

std::mutex g_noalloc_mu;
void* g_noalloc_addr[kNoAllocMaxDevices];      // device address of g_noalloc_work, per device
CUcontext g_noalloc_ctx[kNoAllocMaxDevices];   // the context that address belongs to

typedef CUresult (*CtxGetCurrentFn)(CUcontext*);

// cuCtxGetCurrent from the driver (the library links the runtime only).
CtxGetCurrentFn ctx_get_current()
{
    static CtxGetCurrentFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<CtxGetCurrentFn>(p);
    }
    return fn;
}

// Set-up, once per device, with that device current: resolve the address of
// g_noalloc_work on it.  The address belongs to the device's current context;
// when a call finds another context current (a different handle after a
// device reset, or a context the caller made current), set-up runs again.
int noalloc_workspace(int dev, void** out)
{
    if (dev < 0 || dev >= kNoAllocMaxDevices) {
        snprintf(g_last_error, sizeof(g_last_error),
                 "dfa_find_noalloc: device %d is beyond the %d devices it serves", dev,
                 kNoAllocMaxDevices);
        return DFA_EINVAL;
    }
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    CUcontext ctx = nullptr;
    if (CtxGetCurrentFn get = ctx_get_current()) get(&ctx);
    if (!g_noalloc_addr[dev] || g_noalloc_ctx[dev] != ctx) {
        void* p = nullptr;
        cudaError_t err = cudaGetSymbolAddress(&p, g_noalloc_work);
        if (err != cudaSuccess) return cuda_fail(err, "cudaGetSymbolAddress(g_noalloc_work)");
        g_noalloc_addr[dev] = p;
        if (ctx == nullptr && ctx_get_current()) ctx_get_current()(&ctx);   // made by the call above
        g_noalloc_ctx[dev] = ctx;
    }
    *out = g_noalloc_addr[dev];
    return DFA_OK;
}

// Runs after the scan on the same stream: the status word is the caller's
// only view of a bounded wait that gave up, so it is folded into bit 63 of
// the count.
__global__ void k_noalloc_status(const unsigned long long* work, unsigned long long* count)
{
    if (work[1]) atomicOr(count, 1ull << 63);
}

}  // namespace

extern "C" int dfa_find_noalloc(const uint8_t* d_text, int64_t n, const dfa_table* table,
                                int64_t* d_pos, int64_t cap, uint64_t* d_count,
                                const dfa_config* cfg, void* stream)
{
    if (!table || !d_count || n < 0 || (n > 0 && !d_text) || cap < 0 || (cap > 0 && !d_pos))
        return DFA_EINVAL;
    int dev;
    if (cudaGetDevice(&dev) != cudaSuccess) return fail("dfa_find_noalloc: no current device");
    void* work = nullptr;
    int rc = noalloc_workspace(dev, &work);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // launch_find checks the tile count against the array before any GPU
    // work and clears the header and descriptors this call uses.
    rc = launch_find(d_text, n, n, table, d_pos, cap, d_count, nullptr, 0, work,
                     (int64_t)sizeof(g_noalloc_work), cfg, st);
    if (rc == DFA_EWORKSPACE) {
        snprintf(g_last_error, sizeof(g_last_error),
                 "dfa_find_noalloc: a text of %lld bytes needs more than the %lld tiles its "
                 "static workspace holds; use dfa_find with a caller workspace or a larger chunk",
                 (long long)n, (long long)kNoAllocTiles);
        return rc;
    }
    if (rc) return rc;
    k_noalloc_status<<<1, 1, 0, st>>>(static_cast<const unsigned long long*>(work),
                                      reinterpret_cast<unsigned long long*>(d_count));
    CUDA_TRY(cudaGetLastError());
    return DFA_OK;
}
