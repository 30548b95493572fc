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
// the walk back to q0 (Sec. III-B).  Counts go to per-CTA shared-memory
// counters per pattern and are added to the global per-(sequence, pattern)
// counts when the CTA moves to another sequence and at its end.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cstdio>
#include <cstring>
#include <new>
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
    int32_t delta_bytes = 0, out1_bytes = 0, off_bytes = 0, ids_bytes = 0, mlen_bytes = 0;
    bool owns_mem = true;               // false: d_mem is the caller's (dfa_multi_attach)
    std::vector<uint8_t> img;           // device image, kept until the table is freed
};

namespace {

constexpr int kMultiMaxSeq = 64;
constexpr int kMultiMaxStates = 16383;   // 4 * state fits the u16 entry
constexpr int kMultiMaxPat = 8192;       // per-CTA counters: 32 KiB

int round16(int64_t b) { return (int)((b + 15) & ~(int64_t)15); }

constexpr uint32_t kMany = 0xFFFFu;      // out1 entry of a state with 0 or >= 2 outputs

struct MultiArgs {
    const uint8_t* text[kMultiMaxSeq];
    int64_t n[kMultiMaxSeq];
    int64_t tile0[kMultiMaxSeq + 1];     // first tile of each sequence; tile0[nseq] = all tiles
    int32_t nseq, npat, mmax, chunk;
    int32_t delta_bytes, out1_bytes;     // the parts copied to shared memory
    const uint8_t* tab;                  // device image: [delta][out1][off][ids][mlen]
    const uint32_t* off;
    const uint16_t* ids;
    const uint8_t* mlen;
    unsigned long long* counts;         // [nseq][npat]
};

__device__ __forceinline__ uint4 ldg16m(const uint4* p)
{
    uint4 v;
    asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
}

// Per byte of x: zero iff the byte is a base (A C G T a c g t).
__device__ __forceinline__ uint32_t word_bad_m(uint32_t x)
{
    uint32_t t = (x >> 2) & ~(x >> 1) & 0x01010101u;
    return ((x ^ (t * 0x11u)) & 0xD9D9D9D9u) ^ 0x41414141u;
}

struct MultiTab {
    const uint16_t* delta;   // shared: 4 * state + code -> 4 * next | (out(next) not empty)
    const uint16_t* out1;    // shared: the one pattern a state outputs, or kMany
    uint32_t* hist;          // shared: per-pattern counts of this CTA
    const MultiArgs* args;   // the launch's arguments (output lists in global memory)
};

// Outputs of state st at end offset j, one by one from the list
// (ids[off[st] .. off[st+1])), each kept iff its start j - m_p + 1 lies
// below own (the chunk's owned starts).
__device__ __noinline__ void emit_list(const MultiArgs* a, uint32_t* hist, uint32_t st, uint32_t j, uint32_t own)
{
    const uint32_t* off = a->off;
    const uint32_t k1 = __ldg(off + st + 1);
    for (uint32_t k = __ldg(off + st); k < k1; k++) {
        const uint32_t p = __ldg(a->ids + k);
        if (j + 1u < own + __ldg(a->mlen + p)) atomicAdd(hist + p, 1u);
    }
}

// Entry e has its output flag set: count the patterns ending at j.  A state
// with one output inside the owned part (every start there is owned) takes
// the shared-memory fast path.
__device__ __forceinline__ void emit(const MultiTab& M, uint32_t e, uint32_t j, uint32_t own)
{
    const uint32_t st = e >> 2;
    const uint32_t p = M.out1[st];
    if (p != kMany && j < own)
        atomicAdd(M.hist + p, 1u);
    else
        emit_list(M.args, M.hist, st, j, own);
}

// Four bases of a word w, byte k ending at offset j + k: four dependent
// lookups, one test of the output flags.
__device__ __forceinline__ void word_bases(const MultiTab& M, uint32_t& ent, uint32_t w, uint32_t j, uint32_t own)
{
    const uint32_t c = (w >> 1) & 0x03030303u;
    const uint32_t e0 = M.delta[(ent & ~3u) | (c & 3u)];
    const uint32_t e1 = M.delta[(e0 & ~3u) | ((c >> 8) & 3u)];
    const uint32_t e2 = M.delta[(e1 & ~3u) | ((c >> 16) & 3u)];
    const uint32_t e3 = M.delta[(e2 & ~3u) | (c >> 24)];
    ent = e3;
    if ((e0 | e1 | e2 | e3) & 1u) {
        if (e0 & 1u) emit(M, e0, j, own);
        if (e1 & 1u) emit(M, e1, j + 1, own);
        if (e2 & 1u) emit(M, e2, j + 2, own);
        if (e3 & 1u) emit(M, e3, j + 3, own);
    }
}

// A word holding bases and non-bases: byte by byte, every non-base resets
// the walk to q0 (Sec. III-B: columns outside the alphabet lead to q0).
__device__ __noinline__ uint32_t word_mixed(const MultiTab M, uint32_t ent, uint32_t w, uint32_t j, uint32_t own)
{
    for (int k = 0; k < 4; k++) {
        const uint32_t b = (w >> (8 * k)) & 0xFFu;
        const uint32_t t = (b >> 2) & ~(b >> 1) & 1u;
        if (((b ^ (t * 0x11u)) & 0xD9u) == 0x41u) {
            ent = M.delta[(ent & ~3u) | ((b >> 1) & 3u)];
            if (ent & 1u) emit(M, ent, j + k, own);
        } else {
            ent = 0u;
        }
    }
    return ent;
}

__device__ __forceinline__ void word_any(const MultiTab& M, uint32_t& ent, uint32_t w, uint32_t j, uint32_t own)
{
    const uint32_t bad = word_bad_m(w);
    if (bad == 0u) {
        word_bases(M, ent, w, j, own);
    } else if (((bad - 0x01010101u) & ~bad & 0x80808080u) == 0u) {
        ent = 0u;                                   // four non-bases (an N block)
    } else {
        ent = word_mixed(M, ent, w, j, own);
    }
}

template <int THREADS>
__global__ void __launch_bounds__(THREADS, 1024 / THREADS) k_multi_count(const __grid_constant__ MultiArgs a)
{
    extern __shared__ __align__(16) uint8_t msm[];
    {
        const int bytes = a.delta_bytes + a.out1_bytes;
        const uint4* src = reinterpret_cast<const uint4*>(a.tab);
        uint4* dst = reinterpret_cast<uint4*>(msm);
        for (int i = threadIdx.x; i < (bytes >> 4); i += THREADS) dst[i] = src[i];
    }
    MultiTab M;
    M.delta = reinterpret_cast<const uint16_t*>(msm);
    M.out1 = reinterpret_cast<const uint16_t*>(msm + a.delta_bytes);
    M.hist = reinterpret_cast<uint32_t*>(msm + a.delta_bytes + a.out1_bytes);
    M.args = &a;
    for (int p = threadIdx.x; p < a.npat; p += THREADS) M.hist[p] = 0u;
    __syncthreads();

    auto flush = [&](int sq) {
        __syncthreads();
        for (int p = threadIdx.x; p < a.npat; p += THREADS) {
            const uint32_t v = M.hist[p];
            if (v) {
                atomicAdd(a.counts + (int64_t)sq * a.npat + p, (unsigned long long)v);
                M.hist[p] = 0u;
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
        }
        const int64_t n = a.n[sq];
        const uint8_t* text = a.text[sq];
        const int64_t s = (t - a.tile0[sq]) * tb + (int64_t)threadIdx.x * C;
        if (s >= n) continue;
        const int64_t e = min(s + C, n);
        const int64_t hi = min(e + (int64_t)a.mmax - 1, n);
        const uint32_t own = (uint32_t)(e - s);
        const uint32_t len = (uint32_t)(hi - s);
        uint32_t ent = 0u;
        uint32_t done = 0;
        if ((((uintptr_t)text) & 15u) == 0 && len >= 16) {
            // 16-byte vectors, two in flight ahead of the one walked
            const uint4* p = reinterpret_cast<const uint4*>(text + s);
            const uint32_t nv = len >> 4;
            uint4 b0 = ldg16m(p);
            uint4 b1 = nv > 1 ? ldg16m(p + 1) : b0;
            uint4 b2 = nv > 2 ? ldg16m(p + 2) : b0;
#pragma unroll 1
            for (uint32_t g = 0; g < nv; g++) {
                const uint4 v = b0;
                b0 = b1;
                b1 = b2;
                if (g + 3 < nv) b2 = ldg16m(p + g + 3);
                const uint32_t j = 16u * g;
                word_any(M, ent, v.x, j, own);
                word_any(M, ent, v.y, j + 4, own);
                word_any(M, ent, v.z, j + 8, own);
                word_any(M, ent, v.w, j + 12, own);
            }
            done = nv << 4;
        }
        for (uint32_t j = done; j < len; j++) {
            const uint32_t b = text[s + j];
            const uint32_t tt = (b >> 2) & ~(b >> 1) & 1u;
            if (((b ^ (tt * 0x11u)) & 0xD9u) == 0x41u) {
                ent = M.delta[(ent & ~3u) | ((b >> 1) & 3u)];
                if (ent & 1u) emit(M, ent, j, own);
            } else {
                ent = 0u;
            }
        }
    }
    if (cur >= 0) flush(cur);
}

typedef void (*MultiFn)(const MultiArgs);

MultiFn pick_multi(int threads)
{
    if (threads == 128) return k_multi_count<128>;
    if (threads == 512) return k_multi_count<512>;
    return k_multi_count<256>;
}

int multi_fail(const char* what, cudaError_t err)
{
    char buf[256];
    snprintf(buf, sizeof(buf), "%s: %s", what, cudaGetErrorString(err));
    return set_last_error(DFA_ECUDA, buf);
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
    int mmax = 0;
    for (int p = 0; p < npat; p++) {
        const int m = lengths[p];
        if (m < 1 || m > DFA_MAX_M || !patterns[p]) return DFA_EINVAL;
        mmax = std::max(mmax, m);
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
    dfa_multi* t = new (std::nothrow) dfa_multi();
    if (!t) return DFA_ENOMEM;
    t->npat = npat;
    t->nstates = S;
    t->mmax = mmax;
    t->mlen.resize(npat);
    for (int p = 0; p < npat; p++) t->mlen[p] = (uint8_t)lengths[p];
    t->delta.resize((size_t)S * 4);
    t->out_off.assign(S + 1, 0);
    for (int i = 0; i < S; i++) {
        const int u = order[i];
        for (int a = 0; a < 4; a++) {
            const int v = delta[u][a];
            t->delta[(size_t)i * 4 + a] = (uint16_t)(4 * num[v] + (outs[v].empty() ? 0 : 1));
        }
        t->out_off[i + 1] = t->out_off[i] + (uint32_t)outs[u].size();
        t->out_ids.insert(t->out_ids.end(), outs[u].begin(), outs[u].end());
    }
    // device image: [delta][out_off][out_ids][mlen], 16-byte aligned parts
    // out1[q]: the pattern of a state with exactly one output, else kMany
    std::vector<uint16_t> out1(S, (uint16_t)kMany);
    for (int i = 0; i < S; i++)
        if (t->out_off[i + 1] - t->out_off[i] == 1) out1[i] = t->out_ids[t->out_off[i]];
    t->delta_bytes = round16((int64_t)S * 4 * 2);
    t->out1_bytes = round16((int64_t)S * 2);
    t->off_bytes = round16((int64_t)(S + 1) * 4);
    t->ids_bytes = round16((int64_t)std::max<size_t>(t->out_ids.size(), 1) * 2);
    t->mlen_bytes = round16(npat);
    const size_t bytes = (size_t)t->delta_bytes + t->out1_bytes + t->off_bytes + t->ids_bytes + t->mlen_bytes;
    std::vector<uint8_t>& img = t->img;
    img.assign(bytes, 0);
    uint8_t* q = img.data();
    memcpy(q, t->delta.data(), t->delta.size() * 2);
    q += t->delta_bytes;
    memcpy(q, out1.data(), out1.size() * 2);
    q += t->out1_bytes;
    memcpy(q, t->out_off.data(), t->out_off.size() * 4);
    q += t->off_bytes;
    if (!t->out_ids.empty()) memcpy(q, t->out_ids.data(), t->out_ids.size() * 2);
    q += t->ids_bytes;
    memcpy(q, t->mlen.data(), npat);
    t->owns_mem = false;
    *out = t;
    return DFA_OK;
}

int dfa_multi_build(const char* const* patterns, const int32_t* lengths, int32_t npat, dfa_multi** out)
{
    if (!out) return DFA_EINVAL;
    dfa_multi* t = nullptr;
    int rc = dfa_multi_build_host(patterns, lengths, npat, &t);
    if (rc) return rc;
    const size_t bytes = t->img.size();
    cudaError_t err;
    if ((err = cudaGetDevice(&t->device)) != cudaSuccess || (err = cudaMalloc(&t->d_mem, bytes)) != cudaSuccess) {
        delete t;
        return multi_fail("dfa_multi_build", err);
    }
    t->owns_mem = true;
    if ((err = cudaMemcpy(t->d_mem, t->img.data(), bytes, cudaMemcpyHostToDevice)) != cudaSuccess) {
        cudaFree(t->d_mem);
        delete t;
        return multi_fail("dfa_multi_build", err);
    }
    *out = t;
    return DFA_OK;
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
    return (int64_t)t->delta_bytes + t->out1_bytes + (int64_t)t->npat * 4;
}

int dfa_multi_count(const uint8_t* const* d_texts, const int64_t* lengths, int32_t nseq, const dfa_multi* t,
                    uint64_t* d_counts, const dfa_config* cfg, void* stream)
{
    if (!t || !d_counts || !d_texts || !lengths || nseq < 1 || nseq > kMultiMaxSeq) return DFA_EINVAL;
    if (!t->d_mem) return set_last_error(DFA_EINVAL, "dfa_multi_count: the automaton has no device copy (dfa_multi_attach)");
    const int threads = cfg && cfg->threads ? cfg->threads : 256;
    const int chunk = cfg && cfg->chunk ? cfg->chunk : 1024;
    if (threads != 128 && threads != 256 && threads != 512) return DFA_EINVAL;
    if (chunk < 16 || chunk > 32768 || (chunk & 15)) return DFA_EINVAL;
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
    a.out1_bytes = t->out1_bytes;
    a.tab = static_cast<const uint8_t*>(t->d_mem);
    a.off = reinterpret_cast<const uint32_t*>(a.tab + t->delta_bytes + t->out1_bytes);
    a.ids = reinterpret_cast<const uint16_t*>(a.tab + t->delta_bytes + t->out1_bytes + t->off_bytes);
    a.mlen = a.tab + t->delta_bytes + t->out1_bytes + t->off_bytes + t->ids_bytes;
    a.counts = reinterpret_cast<unsigned long long*>(d_counts);
    if ((err = cudaMemsetAsync(d_counts, 0, (size_t)nseq * t->npat * 8, st)) != cudaSuccess)
        return multi_fail("dfa_multi_count", err);
    if (a.tile0[nseq] == 0) return DFA_OK;
    MultiFn fn = pick_multi(threads);
    const int smem = (int)dfa_multi_smem_bytes(t);
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

}  // extern "C"
