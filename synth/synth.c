/*
 * Seeded synthetic DNA inputs for the finite-automaton scan.
 *
 * This module draws random numbers only: it holds none of the scan's
 * arithmetic (no automaton, no matching) and is the one piece of code that
 * both the CPU oracle and the CUDA path are fed from.  Every generator is a
 * pure function of its seed and arguments, computed with integer arithmetic
 * only, so that an x86-64 host and an aarch64 host produce the same bytes.
 *
 * Random source: SplitMix64 (Steele, Lea and Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014), used in counter mode: the
 * k-th draw of stream s under seed x is mix(key(x, s) + (k + 1) * gamma),
 * where mix is the SplitMix64 finaliser.  Counter mode lets the byte fill run
 * in parallel and still give the same text for any thread count.
 *
 * Workload shapes (they stand in for the paper's GenBank genomes, Table II,
 * and its 8-mer patterns, Table III, neither of which is available here):
 *   - uniform text: i.i.d. uniform A/C/G/T, 2 bits of a draw per base;
 *   - genome text: base composition with GC = 0.41 (A .295, C .205, G .205,
 *     T .295), soft-masked lower-case runs (alternating renewal process of
 *     unmasked and masked runs, both geometric with mean 300, starting
 *     unmasked) and 'N' blocks (alternating renewal process of non-N gaps,
 *     geometric mean 950000, and N runs, geometric mean 50000, i.e. 5% N);
 *   - patterns: i.i.d. uniform upper-case A/C/G/T.
 */
#include <stdint.h>
#include <stddef.h>
#include <string.h>

#define SM64_GAMMA 0x9E3779B97F4A7C15ULL

static inline uint64_t sm64_mix(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Key of stream `stream` under seed `seed`. */
static inline uint64_t sm64_key(uint64_t seed, uint64_t stream)
{
    return sm64_mix(seed * SM64_GAMMA + stream * 0x632BE59BD9B4E019ULL + 0x2545F4914F6CDD1DULL);
}

/* k-th draw of a keyed stream. */
static inline uint64_t sm64_at(uint64_t key, uint64_t k)
{
    return sm64_mix(key + (k + 1) * SM64_GAMMA);
}

uint64_t synth_draw(uint64_t seed, uint64_t stream, uint64_t k)
{
    return sm64_at(sm64_key(seed, stream), k);
}

/* ---- integer-only geometric sampling -------------------------------- */

/* log2(x) for x >= 1 in Q32 fixed point, by normalisation and repeated
 * squaring of the mantissa (one fractional bit per squaring).  Integer
 * arithmetic only, so it is bit-identical on every host. */
static int64_t ilog2_q32(uint64_t x)
{
    int e = 63 - __builtin_clzll(x);
    uint64_t y = (e >= 62) ? (x >> (e - 62)) : (x << (62 - e)); /* [2^62, 2^63) = [1,2) in Q62 */
    int64_t r = (int64_t)e << 32;
    for (int i = 1; i <= 32; i++) {
        unsigned __int128 sq = (unsigned __int128)y * y;
        y = (uint64_t)(sq >> 62);                  /* [1,4) in Q62 */
        if (y >= (1ULL << 63)) {
            y >>= 1;
            r += (int64_t)1 << (32 - i);
        }
    }
    return r;
}

/* Geometric run length on {1, 2, ...} with the given mean (>= 2), by
 * inversion: L = 1 + floor(log(U) / log(1 - 1/mean)), U uniform on (0,1]. */
static int64_t geo_scale(uint64_t mean)
{
    int64_t b = ilog2_q32(mean) - ilog2_q32(mean - 1);     /* -log2(1-1/mean) in Q32, > 0 */
    return b > 0 ? b : 1;
}

static int64_t geometric_b(uint64_t draw, int64_t b)
{
    uint64_t u = (draw >> 11) + 1;                         /* [1, 2^53] */
    int64_t a = ((int64_t)53 << 32) - ilog2_q32(u);        /* -log2(U) in Q32, >= 0 */
    return 1 + a / b;
}

static int64_t geometric(uint64_t draw, uint64_t mean)
{
    return geometric_b(draw, geo_scale(mean));
}

int64_t synth_geometric(uint64_t seed, uint64_t stream, uint64_t k, uint64_t mean)
{
    return geometric(synth_draw(seed, stream, k), mean);
}

/* ---- texts ----------------------------------------------------------- */

static const char ACGT[4] = {'A', 'C', 'G', 'T'};

/* Uniform i.i.d. A/C/G/T: base i takes bits 2*(i%32).. of draw i/32. */
void synth_uniform(uint8_t* out, int64_t n, uint64_t seed)
{
    const uint64_t key = sm64_key(seed, 0);
    int64_t nblk = (n + 31) / 32;
#pragma omp parallel for schedule(static)
    for (int64_t b = 0; b < nblk; b++) {
        uint64_t z = sm64_at(key, (uint64_t)b);
        int64_t i0 = b * 32;
        int64_t i1 = i0 + 32 < n ? i0 + 32 : n;
        for (int64_t i = i0; i < i1; i++) {
            out[i] = (uint8_t)ACGT[z & 3];
            z >>= 2;
        }
    }
}

/* Pattern of length m: uniform upper-case A/C/G/T (same recipe as the
 * uniform text, under the pattern's own seed). */
void synth_pattern(uint8_t* out, int32_t m, uint64_t seed)
{
    synth_uniform(out, m, seed);
}

/* Composition thresholds on a 32-bit uniform: A < .295, C < .500, G < .705. */
#define THR_A 1267015745ULL   /* 0.295 * 2^32 */
#define THR_C 2147483648ULL   /* 0.500 * 2^32 */
#define THR_G 3027951551ULL   /* 0.705 * 2^32 */

static inline uint8_t comp_base(uint32_t u)
{
    return (uint8_t)(u < THR_A ? 'A' : u < THR_C ? 'C' : u < THR_G ? 'G' : 'T');
}

/*
 * Genome-like text.  mask_mean == 0 disables soft-masking; n_gap_mean == 0
 * disables N blocks.  gc selects the composition recipe: 0 = uniform
 * (2 bits per base), 1 = GC 0.41 thresholds.
 */
void synth_genome(uint8_t* out, int64_t n, uint64_t seed, int32_t gc,
                  uint64_t mask_mean, uint64_t n_gap_mean, uint64_t n_run_mean)
{
    if (n <= 0) return;
    if (!gc) {
        synth_uniform(out, n, seed);
    } else {
        const uint64_t key = sm64_key(seed, 0);
        int64_t nblk = (n + 1) / 2;
#pragma omp parallel for schedule(static)
        for (int64_t b = 0; b < nblk; b++) {
            uint64_t z = sm64_at(key, (uint64_t)b);
            int64_t i = 2 * b;
            out[i] = comp_base((uint32_t)z);
            if (i + 1 < n) out[i + 1] = comp_base((uint32_t)(z >> 32));
        }
    }
    /* soft-mask: alternating unmasked / masked runs, first run unmasked */
    if (mask_mean >= 2) {
        const uint64_t key = sm64_key(seed, 1);
        const int64_t b = geo_scale(mask_mean);
        uint64_t k = 0;
        int64_t pos = 0;
        int masked = 0;
        while (pos < n) {
            int64_t len = geometric_b(sm64_at(key, k++), b);
            int64_t end = pos + len < n ? pos + len : n;
            if (masked)
                for (int64_t i = pos; i < end; i++) out[i] |= 0x20;
            pos = end;
            masked ^= 1;
        }
    }
    /* N blocks: alternating non-N gaps / N runs, first run a gap */
    if (n_gap_mean >= 2 && n_run_mean >= 2) {
        const uint64_t key = sm64_key(seed, 2);
        const int64_t b_run = geo_scale(n_run_mean), b_gap = geo_scale(n_gap_mean);
        uint64_t k = 0;
        int64_t pos = 0;
        int isn = 0;
        while (pos < n) {
            int64_t len = geometric_b(sm64_at(key, k++), isn ? b_run : b_gap);
            int64_t end = pos + len < n ? pos + len : n;
            if (isn) memset(out + pos, 'N', (size_t)(end - pos));
            pos = end;
            isn ^= 1;
        }
    }
}

/*
 * Copy `pattern` (length m) into `text` at each of the k positions (used to
 * plant occurrences for long patterns, whose random occurrences are ~0).
 * Positions that would run past the end are skipped.  When `lower` is set
 * the copy keeps the case of the bytes it overwrites.
 */
void synth_plant(uint8_t* text, int64_t n, const uint8_t* pattern, int32_t m,
                 const int64_t* positions, int64_t k, int32_t keep_case)
{
    for (int64_t j = 0; j < k; j++) {
        int64_t p = positions[j];
        if (p < 0 || p + m > n) continue;
        for (int32_t i = 0; i < m; i++) {
            uint8_t c = pattern[i];
            if (keep_case && (text[p + i] & 0x20) && text[p + i] != 'N') c |= 0x20;
            text[p + i] = c;
        }
    }
}

/* Uniform integers in [0, bound) (bound >= 1), k-th of a keyed stream. */
void synth_uniform_ints(int64_t* out, int64_t k, int64_t bound, uint64_t seed, uint64_t stream)
{
    const uint64_t key = sm64_key(seed, stream);
    for (int64_t j = 0; j < k; j++) {
        unsigned __int128 prod = (unsigned __int128)sm64_at(key, (uint64_t)j) * (uint64_t)bound;
        out[j] = (int64_t)(prod >> 64);
    }
}
