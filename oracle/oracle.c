/*
 * CPU ORACLE for the finite-automaton DNA pattern scan — TEST INFRASTRUCTURE.
 *
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg use
 * this file.  The product path (the CUDA library) never links, loads or calls
 * it, and it shares no code with that path: everything here is written
 * plainly from the paper (Memeti & Pllana, "Accelerating DNA Sequence
 * Analysis using Intel Xeon Phi", 2015) and from the mathematics of string
 * matching, in the most direct form, for a reader to check by eye.
 *
 * Contents
 *   oracle_find_brute   the result by definition (Sec. II-A problem
 *                       statement): every i with T[i..i+m) = P, overlaps
 *                       included, by comparing each window.
 *   oracle_dfa_delta    transition function of the string-matching automaton
 *                       (Sec. II-A quintuple (Q, Sigma, delta, q0, F)), built
 *                       from its definition: delta(q, a) = length of the
 *                       longest prefix of P that is a suffix of P[0..q)a.
 *   oracle_dfa_scan     the sequential automaton walk (the paper's sequential
 *                       version, p = v = 1 in Algorithm 1).
 *   oracle_alg1_scan    Algorithm 1 (Parallel DNA Analysis) with p chunks of
 *                       m-1 overlap (Sec. III-A, Fig. 2a) each split into v
 *                       lanes (Fig. 2b), emulated lane by lane, optionally
 *                       with one OpenMP thread per chunk.
 *   oracle_stt_ascii    the sparse 256-column state transition table of
 *                       Sec. III-B (Table I layout) of the failure-less
 *                       automaton (Fig. 4) of a set of strings, finals
 *                       numbered last.
 *   oracle_find_set     the definition for a set of patterns: every window
 *                       start compared with all patterns at once, patterns
 *                       that share a prefix sharing those comparisons (a
 *                       trie descent from each start, no failure links).
 *   oracle_kmer_census  count of every k-mer by definition.
 *   oracle_valid_windows number of windows of k bytes all in ACGTacgt,
 *                       computed from the lengths of the valid runs.
 *
 * Readings of the paper taken here (each one is listed in the design notes):
 *   - Matching is case-insensitive: text bytes a/c/g/t match A/C/G/T.  Any
 *     other byte (N, IUPAC codes, newline, >= 128) matches nothing and, in
 *     the automaton, sends the walk back to q0 (Sec. III-B: every cell outside
 *     the alphabet's columns holds q0).
 *   - Output positions are 0-based START indices (Algorithm 1 reports the
 *     index c of the last matched character; start = c - m + 1), ascending.
 *   - Algorithm 1 is read as: chunk i covers [i*L, (i+1)*L) with L = n/p and
 *     the last chunk taking the remainder; the scan of a chunk runs from q0 at
 *     its first byte through min(end + m - 1, n); lane k of a chunk walks a
 *     contiguous sub-range (Fig. 2b: lanes start at 0, 4, 8, 12 for v = 4 on a
 *     16-byte input), again with m-1 bytes of overlap.  A match is reported
 *     by the one piece that owns its start.
 *
 * Return convention: counts are >= 0; -1 means invalid arguments.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ASCII upper-casing of letters; other bytes are returned unchanged. */
static int fold(int c)
{
    if (c >= 'a' && c <= 'z') return c - 32;
    return c;
}

/* Index of a base in the automaton alphabet order A, C, G, T, or -1. */
static int base_index(int c)
{
    switch (fold(c)) {
    case 'A': return 0;
    case 'C': return 1;
    case 'G': return 2;
    case 'T': return 3;
    default: return -1;
    }
}

static const char BASES[4] = {'A', 'C', 'G', 'T'};

/* Normalise a pattern to upper case; 0 on success, -1 if any byte is not a
 * base or m < 1. */
static int normalise_pattern(const uint8_t* pattern, int32_t m, uint8_t* out)
{
    if (!pattern || m < 1) return -1;
    for (int32_t j = 0; j < m; j++) {
        int b = base_index(pattern[j]);
        if (b < 0) return -1;
        out[j] = (uint8_t)BASES[b];
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* The definition: compare every window.                               */
/* ------------------------------------------------------------------ */

int64_t oracle_find_brute(const uint8_t* text, int64_t n, const uint8_t* pattern, int32_t m,
                          int64_t* positions, int64_t cap)
{
    if (n < 0 || (n > 0 && !text)) return -1;
    uint8_t* P = (uint8_t*)malloc((size_t)(m > 0 ? m : 1));
    if (!P) return -1;
    if (normalise_pattern(pattern, m, P) != 0) {
        free(P);
        return -1;
    }
    int64_t count = 0;
    for (int64_t i = 0; i + m <= n; i++) {
        int32_t j = 0;
        while (j < m && fold(text[i + j]) == P[j]) j++;
        if (j == m) {
            if (positions && count < cap) positions[count] = i;
            count++;
        }
    }
    free(P);
    return count;
}

/* ------------------------------------------------------------------ */
/* The definition for a set of patterns.                               */
/* ------------------------------------------------------------------ */

/*
 * Every occurrence of every pattern of a set (Sec. II-A problem statement,
 * applied to each pattern; overlaps included): pattern p occurs at i iff
 * T[i..i+m_p) = P_p.  For each window start i the patterns are compared
 * together, character by character, by descending a trie of the patterns
 * (node = a distinct prefix, child[node][base]): the descent stops at the
 * first byte that is not a base or that no pattern continues with, and every
 * pattern that ends on a node passed counts one occurrence at i.  This is
 * the window compare of oracle_find_brute with the comparisons of patterns
 * that share a prefix done once; it is not the Aho-Corasick automaton (no
 * failure links: each window is compared from its first byte).
 *
 * Inputs: npat patterns concatenated in pats, lengths in lens (1..255 bytes
 * of ACGTacgt each; duplicates allowed and counted separately).
 * Outputs: counts[p] = occurrences of pattern p.  With pos non-NULL, pattern
 * p's start positions, ascending, go to pos[pos_off[p] ...] (the caller
 * sizes pos and pos_off from the counts of an earlier call).  nthreads > 1
 * splits the window starts into contiguous ranges over OpenMP threads.
 * Returns 0, or -1 for invalid arguments.
 */
typedef struct {
    int32_t child[4];
    int32_t first_end;      /* head of the list of patterns ending here, -1 */
} trie_node;

int oracle_find_set(const uint8_t* text, int64_t n, const uint8_t* pats, const int32_t* lens, int32_t npat,
                    uint64_t* counts, int64_t* pos, const int64_t* pos_off, int32_t nthreads)
{
    if (n < 0 || (n > 0 && !text) || !pats || !lens || npat < 1 || !counts) return -1;
    if (pos && !pos_off) return -1;
    int64_t total = 0;
    for (int32_t p = 0; p < npat; p++) {
        if (lens[p] < 1 || lens[p] > 255) return -1;
        total += lens[p];
    }
    trie_node* node = (trie_node*)malloc(sizeof(trie_node) * (size_t)(total + 1));
    int32_t* next_end = (int32_t*)malloc(sizeof(int32_t) * (size_t)npat);   /* list links */
    if (!node || !next_end) {
        free(node);
        free(next_end);
        return -1;
    }
    int32_t nodes = 1;
    for (int b = 0; b < 4; b++) node[0].child[b] = -1;
    node[0].first_end = -1;
    const uint8_t* q = pats;
    for (int32_t p = 0; p < npat; p++) {
        int32_t v = 0;
        for (int32_t j = 0; j < lens[p]; j++) {
            const int b = base_index(q[j]);
            if (b < 0) {
                free(node);
                free(next_end);
                return -1;
            }
            if (node[v].child[b] < 0) {
                for (int c = 0; c < 4; c++) node[nodes].child[c] = -1;
                node[nodes].first_end = -1;
                node[v].child[b] = nodes++;
            }
            v = node[v].child[b];
        }
        next_end[p] = node[v].first_end;
        node[v].first_end = p;
        q += lens[p];
    }
    const int T = nthreads > 0 ? nthreads : 1;
    /* per range r of window starts: its occurrence count of each pattern */
    uint64_t* part = (uint64_t*)calloc((size_t)T * (size_t)npat, sizeof(uint64_t));
    if (!part) {
        free(node);
        free(next_end);
        return -1;
    }
    for (int pass = 0; pass < (pos ? 2 : 1); pass++) {
        if (pass == 1) {
            /* exclusive offsets: pattern p's positions from range r start at
             * pos_off[p] + (occurrences of p in ranges before r) */
            for (int32_t p = 0; p < npat; p++) {
                uint64_t run = 0;
                for (int r = 0; r < T; r++) {
                    const uint64_t c = part[(size_t)r * npat + p];
                    part[(size_t)r * npat + p] = run;
                    run += c;
                }
            }
        }
#ifdef _OPENMP
#pragma omp parallel for schedule(static, 1) num_threads(T)
#endif
        for (int r = 0; r < T; r++) {
            const int64_t lo = n * r / T, hi = n * (r + 1) / T;
            uint64_t* mine = part + (size_t)r * npat;
            for (int64_t i = lo; i < hi; i++) {
                int32_t v = 0;
                for (int64_t j = i; j < n; j++) {
                    const int b = base_index(text[j]);
                    if (b < 0) break;
                    v = node[v].child[b];
                    if (v < 0) break;
                    for (int32_t p = node[v].first_end; p >= 0; p = next_end[p]) {
                        if (pass == 1) pos[pos_off[p] + (int64_t)mine[p]] = i;
                        mine[p]++;
                    }
                }
            }
        }
        if (pass == 0) {
            for (int32_t p = 0; p < npat; p++) {
                uint64_t c = 0;
                for (int r = 0; r < T; r++) c += part[(size_t)r * npat + p];
                counts[p] = c;
            }
        }
    }
    free(part);
    free(node);
    free(next_end);
    return 0;
}

/* ------------------------------------------------------------------ */
/* The automaton, from its definition.                                 */
/* ------------------------------------------------------------------ */

/* 1 if P[0..k) is a suffix of the string P[0..q) followed by the byte a. */
static int prefix_is_suffix(const uint8_t* P, int32_t k, int32_t q, uint8_t a)
{
    if (k == 0) return 1;
    if (P[k - 1] != a) return 0;
    /* P[0..k-1) must equal the last k-1 bytes of P[0..q) */
    for (int32_t i = 0; i < k - 1; i++)
        if (P[i] != P[q - (k - 1) + i]) return 0;
    return 1;
}

/*
 * delta[q*4 + b] for q = 0..m and b over A, C, G, T: the length of the
 * longest prefix of P that is a suffix of P[0..q)·BASES[b].  State m is the
 * one accepting state.  O(m^3) per column; plainly the definition.
 */
int oracle_dfa_delta(const uint8_t* pattern, int32_t m, int32_t* delta)
{
    uint8_t* P = (uint8_t*)malloc((size_t)(m > 0 ? m : 1));
    if (!P || !delta) {
        free(P);
        return -1;
    }
    if (normalise_pattern(pattern, m, P) != 0) {
        free(P);
        return -1;
    }
    for (int32_t q = 0; q <= m; q++) {
        for (int b = 0; b < 4; b++) {
            int32_t k = q + 1 < m ? q + 1 : m;
            while (k > 0 && !(k <= q + 1 && prefix_is_suffix(P, k, q, (uint8_t)BASES[b]))) k--;
            delta[q * 4 + b] = k;
        }
    }
    free(P);
    return 0;
}

/* One automaton step on a raw text byte: non-bases go to q0. */
static inline int32_t step(const int32_t* delta, int32_t q, uint8_t c)
{
    int b = base_index(c);
    return b < 0 ? 0 : delta[q * 4 + b];
}

/*
 * Walk the automaton over text[lo, hi) from q0 and record every match whose
 * start lies in [lo, own_end).  Used by the sequential and Algorithm 1 scans.
 */
static int64_t walk(const uint8_t* text, int64_t lo, int64_t hi, int64_t own_end,
                    const int32_t* delta, int32_t m, int64_t* positions, int64_t cap,
                    int64_t count)
{
    int32_t q = 0;
    for (int64_t c = lo; c < hi; c++) {
        q = step(delta, q, text[c]);
        if (q >= m) {                       /* accept test "q >= f" (Sec. III-B) */
            int64_t start = c - m + 1;
            if (start < own_end) {
                if (positions && count < cap) positions[count] = start;
                count++;
            }
        }
    }
    return count;
}

int64_t oracle_dfa_scan(const uint8_t* text, int64_t n, const int32_t* delta, int32_t m,
                        int64_t* positions, int64_t cap)
{
    if (n < 0 || (n > 0 && !text) || !delta || m < 1) return -1;
    return walk(text, 0, n, n, delta, m, positions, cap, 0);
}

/*
 * Algorithm 1 lane starts (for the Fig. 2b check): for chunk `i` of p chunks,
 * write the v lane start offsets into starts[0..v).  Returns the lane length.
 */
static void chunk_bounds(int64_t n, int64_t p, int64_t i, int64_t* s, int64_t* e)
{
    int64_t L = n / p;
    *s = i * L;
    *e = (i == p - 1) ? n : (i + 1) * L;
}

static void lane_bounds(int64_t cs, int64_t ce, int64_t v, int64_t k, int64_t* s, int64_t* e)
{
    int64_t len = ce - cs;
    int64_t L = (len + v - 1) / v;          /* lanes of equal length, last one short */
    int64_t a = cs + k * L;
    int64_t b = a + L;
    if (a > ce) a = ce;
    if (b > ce) b = ce;
    *s = a;
    *e = b;
}

int oracle_alg1_lane_starts(int64_t n, int64_t p, int64_t v, int64_t chunk, int64_t* starts)
{
    if (n < 0 || p < 1 || v < 1 || chunk < 0 || chunk >= p || !starts) return -1;
    int64_t cs, ce;
    chunk_bounds(n, p, chunk, &cs, &ce);
    for (int64_t k = 0; k < v; k++) {
        int64_t s, e;
        lane_bounds(cs, ce, v, k, &s, &e);
        starts[k] = s;
    }
    return 0;
}

/*
 * Algorithm 1: p chunks (thread level), v lanes per chunk (SIMD level).  Each
 * lane walks its contiguous sub-range plus m-1 bytes of overlap, from q0.
 * Matches are stored chunk by chunk and lane by lane, which is ascending
 * order.  `scanned` (optional) receives the number of automaton steps, so
 * that the overlap cost can be checked.  nthreads > 1 runs chunks in
 * parallel with OpenMP (one thread per chunk at a time), positions then
 * being gathered in chunk order.
 */
int64_t oracle_alg1_scan(const uint8_t* text, int64_t n, const int32_t* delta, int32_t m,
                         int64_t p, int64_t v, int32_t nthreads,
                         int64_t* positions, int64_t cap, int64_t* scanned)
{
    if (n < 0 || (n > 0 && !text) || !delta || m < 1 || p < 1 || v < 1) return -1;
    int64_t* cnt = (int64_t*)calloc((size_t)p, sizeof(int64_t));
    int64_t* steps = (int64_t*)calloc((size_t)p, sizeof(int64_t));
    if (!cnt || !steps) {
        free(cnt);
        free(steps);
        return -1;
    }
    /* pass 1: count per chunk */
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1)
#endif
    for (int64_t i = 0; i < p; i++) {
        int64_t cs, ce;
        chunk_bounds(n, p, i, &cs, &ce);
        int64_t c = 0, st = 0;
        for (int64_t k = 0; k < v; k++) {
            int64_t s, e;
            lane_bounds(cs, ce, v, k, &s, &e);
            if (s >= e) continue;
            int64_t hi = e + m - 1 < n ? e + m - 1 : n;
            c = walk(text, s, hi, e, delta, m, NULL, 0, c);
            st += hi - s;
        }
        cnt[i] = c;
        steps[i] = st;
    }
    int64_t total = 0, total_steps = 0;
    for (int64_t i = 0; i < p; i++) {
        int64_t c = cnt[i];
        cnt[i] = total;                      /* exclusive offset */
        total += c;
        total_steps += steps[i];
    }
    /* pass 2: write positions at each chunk's offset */
    if (positions && cap > 0) {
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1)
#endif
        for (int64_t i = 0; i < p; i++) {
            int64_t off = cnt[i];
            if (off >= cap) continue;
            int64_t cs, ce;
            chunk_bounds(n, p, i, &cs, &ce);
            int64_t c = 0;
            for (int64_t k = 0; k < v; k++) {
                int64_t s, e;
                lane_bounds(cs, ce, v, k, &s, &e);
                if (s >= e) continue;
                int64_t hi = e + m - 1 < n ? e + m - 1 : n;
                c = walk(text, s, hi, e, delta, m, positions + off, cap - off, c);
            }
        }
    }
    if (scanned) *scanned = total_steps;
    free(cnt);
    free(steps);
    return total;
}

/* ------------------------------------------------------------------ */
/* Sparse ASCII STT (Sec. III-B, Table I).                             */
/* ------------------------------------------------------------------ */

/*
 * The failure-less automaton of Fig. 4 as a sparse 256-column table.
 *
 * Input: k strings over A/C/G/T (concatenated, lengths in lens[]), each
 * flagged final or not.  The states are the distinct prefixes of the strings
 * (the Aho-Corasick trie, Sec. II-A), numbered in order of first appearance
 * as the strings are inserted one after the other, except that the final
 * states (prefixes equal to a flagged string) are renumbered last, keeping
 * their order (Sec. III-B).  The transition from state s on base a goes to
 * the state whose string is the longest suffix of s·a (no failure links:
 * Fig. 4).  Columns are raw byte values: only 'A','C','G','T' and their
 * lower-case forms hold transitions, every other column holds q0.
 *
 * Outputs: stt[row*256 + byte]; *first_final = f (the accept test is
 * q >= f); state_src[row] / state_len[row] name the state's string as a
 * prefix of length state_len of input string state_src.  Returns the number
 * of states, or -1.
 */
int32_t oracle_stt_ascii(const uint8_t* strings, const int32_t* lens, const int32_t* is_final,
                         int32_t k, int32_t* stt, int32_t max_states, int32_t* first_final,
                         int32_t* state_src, int32_t* state_len)
{
    if (!strings || !lens || !is_final || k < 1 || !stt) return -1;
    int64_t total = 0;
    for (int32_t i = 0; i < k; i++) {
        if (lens[i] < 1) return -1;
        total += lens[i];
    }
    int32_t cap = (int32_t)total + 1;
    uint8_t* s = (uint8_t*)malloc((size_t)total);
    int64_t* off = (int64_t*)malloc(sizeof(int64_t) * (size_t)k);
    int32_t* plen = (int32_t*)malloc(sizeof(int32_t) * (size_t)cap);
    int32_t* psrc = (int32_t*)malloc(sizeof(int32_t) * (size_t)cap);
    int32_t* fin = (int32_t*)malloc(sizeof(int32_t) * (size_t)cap);
    int32_t* num = (int32_t*)malloc(sizeof(int32_t) * (size_t)cap);
    uint8_t* cand = (uint8_t*)malloc((size_t)total + 1);
    int32_t ns = 0, f = 0;
    if (!s || !off || !plen || !psrc || !fin || !num || !cand) goto done;
    for (int32_t i = 0, o = 0; i < k; i++) {
        off[i] = o;
        if (normalise_pattern(strings + o, lens[i], s + o) != 0) goto done;
        o += lens[i];
    }
#define STR(st) (s + off[psrc[st]])
    /* distinct prefixes in insertion order; state 0 is the empty string */
    ns = 1;
    plen[0] = 0;
    psrc[0] = 0;
    for (int32_t i = 0; i < k; i++) {
        for (int32_t L = 1; L <= lens[i]; L++) {
            int32_t found = 0;
            for (int32_t t = 1; t < ns && !found; t++)
                if (plen[t] == L && memcmp(STR(t), s + off[i], (size_t)L) == 0) found = 1;
            if (!found) {
                plen[ns] = L;
                psrc[ns] = i;
                ns++;
            }
        }
    }
    if (ns > max_states) {
        ns = -1;
        goto done;
    }
    /* a state is final when its string equals a flagged string */
    for (int32_t t = 0; t < ns; t++) {
        fin[t] = 0;
        for (int32_t i = 0; i < k && t > 0; i++)
            if (is_final[i] && lens[i] == plen[t] && memcmp(s + off[i], STR(t), (size_t)plen[t]) == 0)
                fin[t] = 1;
    }
    int32_t next = 0;
    for (int32_t t = 0; t < ns; t++)
        if (!fin[t]) num[t] = next++;
    f = next;
    for (int32_t t = 0; t < ns; t++)
        if (fin[t]) num[t] = next++;

    for (int32_t t = 0; t < ns; t++) {
        int32_t row = num[t];
        for (int c = 0; c < 256; c++) stt[row * 256 + c] = 0;
        if (state_src) state_src[row] = psrc[t];
        if (state_len) state_len[row] = plen[t];
        int32_t L = plen[t] + 1;
        memcpy(cand, STR(t), (size_t)plen[t]);
        for (int b = 0; b < 4; b++) {
            cand[L - 1] = (uint8_t)BASES[b];
            int32_t best = 0, bestlen = 0;
            for (int32_t u = 1; u < ns; u++) {
                int32_t ul = plen[u];
                if (ul > L || ul <= bestlen) continue;
                if (memcmp(STR(u), cand + (L - ul), (size_t)ul) == 0) {
                    best = u;
                    bestlen = ul;
                }
            }
            stt[row * 256 + BASES[b]] = num[best];
            stt[row * 256 + (BASES[b] | 0x20)] = num[best];
        }
    }
#undef STR
    if (first_final) *first_final = f;
done:
    free(s);
    free(off);
    free(plen);
    free(psrc);
    free(fin);
    free(num);
    free(cand);
    return ns > 0 ? ns : -1;
}

/* ------------------------------------------------------------------ */
/* k-mer census and the window invariant.                              */
/* ------------------------------------------------------------------ */

/*
 * hist[code] for every window of k bytes that are all bases; code is base 4
 * with A=0, C=1, G=2, T=3 and the first byte most significant.
 */
int oracle_kmer_census(const uint8_t* text, int64_t n, int32_t k, uint64_t* hist)
{
    if (k < 1 || k > 15 || !hist || n < 0) return -1;
    memset(hist, 0, sizeof(uint64_t) * ((size_t)1 << (2 * k)));
    for (int64_t i = 0; i + k <= n; i++) {
        uint64_t code = 0;
        int ok = 1;
        for (int32_t j = 0; j < k; j++) {
            int b = base_index(text[i + j]);
            if (b < 0) {
                ok = 0;
                break;
            }
            code = code * 4 + (uint64_t)b;
        }
        if (ok) hist[code]++;
    }
    return 0;
}

/* Number of windows of k consecutive base bytes: the sum over maximal runs of
 * bases of max(0, run - k + 1). */
int64_t oracle_valid_windows(const uint8_t* text, int64_t n, int32_t k)
{
    if (k < 1 || n < 0) return -1;
    int64_t total = 0, run = 0;
    for (int64_t i = 0; i <= n; i++) {
        if (i < n && base_index(text[i]) >= 0) {
            run++;
        } else {
            if (run >= k) total += run - k + 1;
            run = 0;
        }
    }
    return total;
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
