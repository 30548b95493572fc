/*
 * dnadfa — finite-automaton DNA pattern scan on GB300 (sm_103a): C ABI.
 *
 * The method is the automaton scan of Memeti & Pllana, "Accelerating DNA
 * Sequence Analysis using Intel Xeon Phi" (2015): a failure-less automaton
 * (Sec. III-B, Fig. 4) walks the text once, the text being split into chunks
 * that carry m-1 bytes of overlap so that occurrences across chunk borders
 * are found exactly once (Algorithm 1, Sec. III-A, Fig. 2a).  This library
 * runs that walk in hand-written CUDA kernels; every call below is a plain C
 * function on plain pointers and sizes.
 *
 * Conventions shared by every entry point
 *   - Text: raw bytes.  A, C, G, T match in either case; every other byte
 *     (N, IUPAC codes, newline, >= 128) matches nothing and resets the
 *     automaton to q0, as the sparse table of Sec. III-B does for every
 *     column outside the alphabet.
 *   - Results: the number of occurrences of the pattern, overlaps included
 *     (Sec. II-A problem statement), and their 0-based START positions in
 *     ascending order (Algorithm 1 reports the index of the last matched
 *     character; start = that index - m + 1).
 *   - Memory: "d_" arguments are device pointers owned by the caller, on the
 *     device that is current when the call is made; "h_" arguments are host
 *     pointers.  Tables (dfa_table) are owned by the library.
 *   - Streams: `stream` is a cudaStream_t passed as void* (NULL = the legacy
 *     default stream).  Device entry points only enqueue work: they return
 *     before it runs, do not synchronise, and allocate no memory.
 *   - Errors: every int-returning function returns a DFA_* code and never
 *     aborts the process.  Argument errors are detected before anything is
 *     enqueued.
 *   - Alignment: a text pointer that is 16-byte aligned gets the vectorised
 *     path; any other pointer is accepted and scanned with byte loads.
 *   - Device reset: tables and the per-device settings the library caches
 *     (kernel attributes, workspace addresses) belong to the CUDA context in
 *     which they were made.  cudaDeviceReset destroys them; build tables
 *     again afterwards, and expect the first launches to redo their set-up
 *     only where the library can see the change of context.
 */
#ifndef DNADFA_H
#define DNADFA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Return codes. */
#define DFA_OK 0          /* success */
#define DFA_EINVAL 1      /* bad argument: NULL pointer, n < 0, m out of range, bad pattern byte */
#define DFA_ETRUNC 2      /* more occurrences than the position buffer holds (count is still exact) */
#define DFA_ETIMEOUT 3    /* a bounded device-side wait gave up; results of that call are invalid */
#define DFA_ECUDA 4       /* a CUDA runtime call failed */
#define DFA_EWORKSPACE 5  /* workspace smaller than dfa_find_workspace_bytes() asks for */
#define DFA_ENOMEM 6      /* host or device allocation failed (dfa_build only) */

/* Bit of a count written by dfa_count that marks a device-side failure. */
#define DFA_COUNT_FAILED (1ull << 63)

/* Longest pattern accepted.  States 0..m must fit a byte and the tables of
 * the fast layouts must fit in one SM's shared memory beside the TMA rings:
 * the four-step tables hold (m+1)*256 entries each (layout 4: about
 * 2*(m+1)*256 bytes), so 64 rather than the 255 a byte of state would
 * allow (255 would need 190 KiB of tables). */
#define DFA_MAX_M 64

/* Opaque automaton for one pattern: host tables plus a device copy on the
 * device that was current at dfa_build.  Library-owned; free with dfa_free. */
typedef struct dfa_table dfa_table;

/*
 * Build the automaton of one pattern (Sec. III-B, Fig. 4; single pattern).
 *   pattern: m bytes from {A,C,G,T,a,c,g,t} (case is folded); need not be
 *            NUL-terminated.
 *   m:       1 <= m <= DFA_MAX_M.
 *   out:     receives the new table.
 * The transition function is delta(q, a) = the length of the longest prefix
 * of the pattern that is a suffix of (its first q bytes)·a, for q = 0..m; the
 * one final state is m, numbered last (Sec. III-B).  The device copy is
 * allocated and uploaded synchronously on the current device.
 * Errors: DFA_EINVAL (NULL, m out of range, non-base byte), DFA_ENOMEM,
 * DFA_ECUDA.
 */
int dfa_build(const char* pattern, int32_t m, dfa_table** out);

/* Bytes of device memory the tables of one pattern of length m occupy (every
 * layout of the automaton of Sec. III-B), for dfa_build_into; -1 if m is out
 * of range. */
int64_t dfa_table_bytes(int32_t m);

/*
 * dfa_build without a device allocation, for callers that manage device
 * memory themselves (a serving loop with its own arena; cudaMalloc and
 * cudaFree may synchronise the device and stall work in flight).
 *   d_mem / bytes: caller-owned device memory on the current device, 16-byte
 *            aligned, at least dfa_table_bytes(m) bytes; it must stay valid
 *            until the last call that uses the table has completed.
 *   stream:  the copy of the tables into d_mem is enqueued on this stream;
 *            calls that use the table must be ordered after it (the same
 *            stream, or an event).
 * The table behaves like one from dfa_build; dfa_free releases its host
 * memory only.  Errors: DFA_EINVAL (as dfa_build, or d_mem NULL, unaligned
 * or too small), DFA_ENOMEM, DFA_ECUDA.
 */
int dfa_build_into(const char* pattern, int32_t m, void* d_mem, int64_t bytes, void* stream,
                   dfa_table** out);

/* Release a table (host and device memory; for a table from dfa_build_into,
 * host memory only).  NULL is ignored.  The caller must make sure no enqueued
 * call still uses it. */
void dfa_free(dfa_table* table);

/* Pattern length m of a table, or -1 for NULL. */
int32_t dfa_pattern_length(const dfa_table* table);

/*
 * Copy the table's sparse ASCII state transition table (Sec. III-B, Table I
 * layout) to host memory: (m+1) rows of 256 bytes, row q column c holding
 * delta(q, c); only the columns of A, C, G, T and a, c, g, t are non-zero.
 *   h_stt: host buffer of at least (m+1)*256 bytes; bytes: its size.
 * Errors: DFA_EINVAL.
 */
int dfa_export_stt(const dfa_table* table, uint8_t* h_stt, int64_t bytes);

/*
 * Launch configuration (the knobs the autotuner sets).  Zero fields take the
 * library's defaults.
 *   layout:  0 = default (4 for m >= 8, else 1); 1 = four-step composite
 *            table over 2-bit codes (u16 entries, (m+1)*256), exact walk;
 *            2 = the paper's sparse ASCII STT (u8 entries, (m+1)*256, one
 *            lookup per byte: Sec. III-B); 3 = four-step table of states
 *            only and 4 = four-step states with an accept flag, both walked
 *            through the codes alone with exact replays of the stages that
 *            may hold an accept (loader 2 only).
 *   threads: threads per CTA for loader 1 (128, 256 or 512); loader 2 and
 *            dfa_multi_count fix their own.
 *   chunk:   bytes walked per thread (one row) per tile, each carrying m-1
 *            bytes of overlap (Algorithm 1): loader 1 a multiple of 16 in
 *            16..32768; loader 2 a multiple of 64 in 128..4032.
 *   loader:  0 = default (2 when the text is 16-byte aligned and holds two
 *            full rows, else 1); 1 = direct 16-byte global loads; 2 =
 *            TMA-staged tiles (cp.async.bulk.tensor into shared memory).
 *   ctas_per_sm: persistent CTAs per SM for loader 1 (0 = as many as fit).
 */
typedef struct dfa_config {
    int32_t layout;
    int32_t threads;
    int32_t chunk;
    int32_t loader;
    int32_t ctas_per_sm;
} dfa_config;

/*
 * Count every occurrence (overlaps included) of the table's pattern in
 * d_text[0..n) and store the count in *d_count (device, uint64), overwriting
 * it.  n < m gives 0.  Asynchronous on `stream`; allocates nothing.
 * Matches the paper's "count" output of Algorithm 1.
 *   cfg: launch configuration or NULL for the defaults.
 * Errors: DFA_EINVAL (NULL pointers with n > 0, n < 0, bad cfg), DFA_ECUDA.
 * Device-side failure: a bounded wait inside the kernel that gave up sets
 * bit 63 of *d_count (DFA_COUNT_FAILED); the count is then invalid.
 */
int dfa_count(const uint8_t* d_text, int64_t n, const dfa_table* table, uint64_t* d_count,
              const dfa_config* cfg, void* stream);

/* Bytes of device workspace that dfa_find needs for a text of n bytes under
 * `cfg` (NULL = defaults).  Returns -1 for bad arguments. */
int64_t dfa_find_workspace_bytes(int64_t n, const dfa_config* cfg);

/*
 * Count and locate every occurrence (overlaps included) of the table's
 * pattern in d_text[0..n) (Algorithm 1's two outputs: the number of matches
 * and where they are).  Writes the exact count to *d_count (device, uint64) and the
 * first min(count, cap) start positions, ascending, to d_pos[0..cap) (device,
 * int64).  When count > cap the extra positions are dropped and
 * dfa_find_status reports DFA_ETRUNC.
 *   d_work / work_bytes: caller-owned device workspace, 16-byte aligned, of
 *            at least dfa_find_workspace_bytes(n, cfg) bytes (a status word,
 *            per-tile totals and offsets, and per-row counts and recorded
 *            end offsets or stage masks for the two-pass find; with room for
 *            the tile words only, the ordered single-pass find).  Its
 *            contents need no initialisation; one workspace must not be
 *            shared by two calls that may overlap on the device.
 * Asynchronous on `stream`; allocates nothing.
 * Errors: DFA_EINVAL (also an unaligned d_work), DFA_EWORKSPACE, DFA_ECUDA.
 * Device-side outcomes (truncation, a wait that gave up) are read with
 * dfa_find_status.
 */
int dfa_find(const uint8_t* d_text, int64_t n, const dfa_table* table, int64_t* d_pos,
             int64_t cap, uint64_t* d_count, void* d_work, int64_t work_bytes,
             const dfa_config* cfg, void* stream);

/*
 * Synchronise `stream` and report the device-side outcome of the last
 * dfa_find that used d_work: DFA_ETIMEOUT if a bounded wait gave up,
 * DFA_ETRUNC if *d_count > cap, else DFA_OK (DFA_ECUDA on a CUDA error).
 * If h_count is not NULL it receives *d_count.
 */
int dfa_find_status(const void* d_work, const uint64_t* d_count, int64_t cap,
                    uint64_t* h_count, void* stream);

/*
 * End-to-end form with HOST buffers: the text is copied to the device in
 * segments (each carrying the m-1 byte overlap of Algorithm 1 from its
 * predecessor), scanned while the next segment is in flight, and the
 * positions copied back.  Blocking: returns when *h_count and h_pos are
 * final.
 *   h_text: host text (pinned memory gives full copy bandwidth).
 *   h_pos / cap: host buffer for up to cap start positions (NULL, 0 = count
 *            only).
 *   d_stage / stage_bytes: caller-owned device staging memory; at least
 *            dfa_host_stage_bytes(seg, cap) bytes, where seg is the segment
 *            size in bytes (>= 1 MiB).
 * Returns DFA_ETRUNC when count > cap, else as dfa_find.
 */
int64_t dfa_host_stage_bytes(int64_t seg, int64_t cap);
int dfa_find_host(const uint8_t* h_text, int64_t n, const dfa_table* table, int64_t* h_pos,
                  int64_t cap, uint64_t* h_count, void* d_stage, int64_t stage_bytes,
                  int64_t seg, void* stream);

/*
 * dfa_find of several patterns over one device text (Algorithm 1's output
 * for each): the finds run one after another on `stream`, sharing the one
 * workspace d_work (at least dfa_find_workspace_bytes(n, cfg) bytes).
 * Several texts are several calls (each pattern's positions need their own
 * capacity per text); counting many patterns over many texts in one launch
 * is dfa_multi_count, below.
 *   tables / npat: 1 <= npat <= 1024 automata.
 *   d_pos[i] / caps[i]: device buffer for up to caps[i] start positions of
 *            pattern i (d_pos may be NULL when every cap is 0).
 *   d_counts: device uint64[npat], overwritten with the exact counts;
 *            pattern i is truncated when d_counts[i] > caps[i].
 * A bounded wait that gave up sets bit 63 of that pattern's count
 * (DFA_COUNT_FAILED).  Asynchronous; allocates nothing.
 * Errors: DFA_EINVAL, DFA_EWORKSPACE, DFA_ECUDA.
 */
int dfa_find_batched(const uint8_t* d_text, int64_t n, const dfa_table* const* tables, int32_t npat,
                     int64_t* const* d_pos, const int64_t* caps, uint64_t* d_counts, void* d_work,
                     int64_t work_bytes, const dfa_config* cfg, void* stream);

/*
 * dfa_find_host for several patterns over one host text: each segment is
 * copied to the device once (with the m_max - 1 byte overlap of the longest
 * pattern, Algorithm 1) and every pattern's find runs on it, so the text
 * crosses the host link once for all patterns.  Blocking.
 *   tables / npat: 1 <= npat <= 1024 automata (dfa_build).
 *   h_pos[i] / caps[i]: host buffer for up to caps[i] start positions of
 *            pattern i (h_pos may be NULL when every cap is 0).
 *   h_counts: host uint64[npat], the exact counts.
 *   d_stage / stage_bytes: caller-owned device staging memory of at least
 *            dfa_host_stage_bytes_multi(seg, caps, npat) bytes; seg >= 1 MiB.
 * Returns DFA_ETRUNC when some count exceeds its cap (the counts are exact,
 * the first caps[i] positions valid), DFA_ETIMEOUT if a bounded device wait
 * gave up, else as dfa_find.
 */
int64_t dfa_host_stage_bytes_multi(int64_t seg, const int64_t* caps, int32_t npat);
int dfa_find_host_multi(const uint8_t* h_text, int64_t n, const dfa_table* const* tables, int32_t npat,
                        int64_t* const* h_pos, const int64_t* caps, uint64_t* h_counts, void* d_stage,
                        int64_t stage_bytes, int64_t seg, void* stream);

/*
 * dfa_find for callers that must not allocate device memory.  The paper has
 * no counterpart; this is a library service.  Some callers cannot allocate:
 * code running in a process where another allocator already holds the
 * device's memory (a framework's caching pool that reserved most of HBM, so
 * a fresh cudaMalloc fails although the pool has room), code on a
 * latency-bound stream (cudaMalloc and cudaFree can synchronise the whole
 * device), or a plug-in that is handed only its input and output buffers.
 * Such callers pass the text, positions and count buffers exactly as for
 * dfa_find; the workspace is a fixed array inside the library's device
 * image instead.
 *
 * Arguments, outputs and errors are those of dfa_find without d_work and
 * work_bytes.  The array holds 65536 tile descriptors (512 KiB on every
 * device that loads the library, until the process exits); a text that needs
 * more tiles under `cfg` is rejected with DFA_EWORKSPACE before any GPU work,
 * and dfa_last_error says so.
 *
 * Device-side outcome: there is no workspace to hand to dfa_find_status, so
 * a bounded wait that gave up sets bit 63 of *d_count (DFA_COUNT_FAILED) and
 * the count and positions are then invalid.  Truncation is count > cap, as
 * for dfa_find.
 *
 * First call on each device: it resolves the array's address on the current
 * device (cudaGetSymbolAddress), which may load the library's device code.
 * Make that first call before any stream capture begins.  The address belongs
 * to the context that was current then; a later call that finds a different
 * context current resolves it again.  After cudaDeviceReset the library's
 * tables and per-device state are invalid (see the conventions above).
 *
 * Every call on a device shares the one array, which keeps the previous
 * call's contents; each call clears the part it uses at its start, on
 * `stream`.  Two calls that may overlap on the GPU (different streams with no
 * ordering between them, or different host threads) race on the array and
 * give wrong results: order them.  Asynchronous on `stream`; calls no
 * cudaMalloc, cudaFree or other allocating routine.
 */
int dfa_find_noalloc(const uint8_t* d_text, int64_t n, const dfa_table* table, int64_t* d_pos,
                     int64_t cap, uint64_t* d_count, const dfa_config* cfg, void* stream);

/* ------------------------------------------------------------------
 * Many patterns at once: the multi-pattern failure-less automaton of
 * Sec. III-B (one automaton for a set of patterns, failure transitions
 * folded into the table, one lookup per character) and a batched count
 * over many sequences in one launch.  A batch of patterns is one automaton
 * rather than an array of single-pattern tables: each byte of each text is
 * then walked once for all the patterns, not once per pattern.
 * ------------------------------------------------------------------ */
typedef struct dfa_multi dfa_multi;

/*
 * Build the automaton of npat patterns (patterns[i]: lengths[i] bytes of
 * ACGTacgt, 1..DFA_MAX_M; case-insensitive; duplicates allowed and counted
 * separately).  At most 8192 patterns and 16384 automaton states (the trie
 * of the patterns).  Copies the tables to the current device.
 * Errors: DFA_EINVAL (bad pattern, too many states: see dfa_last_error),
 * DFA_ENOMEM, DFA_ECUDA.
 */
int dfa_multi_build(const char* const* patterns, const int32_t* lengths, int32_t npat,
                    dfa_multi** out);

/*
 * The same automaton built on the host only, with no device copy yet (for
 * callers that manage device memory themselves, as for dfa_build_into).
 * dfa_multi_image_bytes gives the size of its device image (-1 for NULL);
 * dfa_multi_attach enqueues, on `stream`, the copy of the image into
 * caller-owned device memory d_mem (current device, 16-byte aligned, at least
 * that many bytes, valid until the last use of the table) and makes the
 * table usable by dfa_multi_count on calls ordered after the copy.  A table
 * can be attached once.  Errors: as dfa_multi_build; DFA_EINVAL for an
 * attached table, a NULL, unaligned or too small d_mem.
 */
int dfa_multi_build_host(const char* const* patterns, const int32_t* lengths, int32_t npat,
                         dfa_multi** out);
int64_t dfa_multi_image_bytes(const dfa_multi* table);
int dfa_multi_attach(dfa_multi* table, void* d_mem, int64_t bytes, void* stream);

/*
 * Character-class patterns (the class cells of the paper's Table III,
 * Sec. IV): each position allows a set of bases.  patterns[i] holds
 * lengths[i] bytes of symbols, one position each: a base; an IUPAC
 * nucleotide code, R (A/G), Y (C/T), S (C/G), W (A/T), K (G/T), M (A/C),
 * B (not A), D (not C), H (not G), V (not T), N (any base); a bracket set
 * of those, e.g. "[CGT]"; or an alternation of single symbols as the paper
 * writes them, e.g. "(a|g)"; either case.  1..DFA_MAX_M positions a pattern.
 * An occurrence at i is a window T[i..i+m) whose every byte is a base (either
 * case) in its position's set: text bytes outside ACGTacgt still match
 * nothing.  The automaton (subset construction over the patterns'
 * positions: a state is the set of (pattern, matched length) pairs; for
 * patterns of single bases it is the trie automaton of dfa_multi_build)
 * is used like dfa_multi_build's by dfa_multi_count, dfa_multi_locate,
 * dfa_multi_attach and dfa_multi_export.  At most 8192 patterns and 16384
 * states; a pattern with many wide positions can need more.
 * Errors: DFA_EINVAL (bad syntax, too many states: see dfa_last_error),
 * DFA_ENOMEM, DFA_ECUDA (device copy).
 */
int dfa_multi_build_class(const char* const* patterns, const int32_t* lengths, int32_t npat,
                          dfa_multi** out);
int dfa_multi_build_class_host(const char* const* patterns, const int32_t* lengths, int32_t npat,
                               dfa_multi** out);

/* Positions (length m) of pattern p of the automaton; -1 for a bad table or p. */
int32_t dfa_multi_pattern_length(const dfa_multi* table, int32_t p);

/* Release an automaton (its device copy too, unless the caller attached it
 * to its own memory).  NULL is ignored. */
void dfa_multi_free(dfa_multi* table);

/* Number of automaton states (root 0, breadth-first order). */
int32_t dfa_multi_states(const dfa_multi* table);

/*
 * Host copy of the automaton for checking: h_next[q*4 + a] = delta(q, a)
 * with a the 2-bit code ((c >> 1) & 3: A 0, C 1, T 2, G 3), h_nout[q] = the
 * number of patterns that end in state q (own and via failure links).
 * Either pointer may be NULL.  cap_states >= dfa_multi_states.
 */
int dfa_multi_export(const dfa_multi* table, int32_t* h_next, int32_t* h_nout, int64_t cap_states);

/* Shared memory one CTA of dfa_multi_count needs for this automaton. */
int64_t dfa_multi_smem_bytes(const dfa_multi* table);

/*
 * Count every occurrence (overlaps included) of every pattern in every
 * sequence, in one launch.  d_texts: HOST array of nseq (1..64) DEVICE
 * pointers, lengths: HOST array of their byte counts.  d_counts: device
 * uint64[nseq * npat], row-major by sequence, overwritten.  Occurrences are
 * owned by the chunk holding their start (Algorithm 1 with patterns of
 * several lengths: each chunk reads m_max - 1 bytes past its end).
 *   cfg: threads (128, 256, 512 or 1024 per CTA) and chunk (bytes per
 *        thread per tile, multiple of 16); layout: the table in shared
 *        memory, 1 = one copy (2 bytes an entry), 2 = 32 per-lane copies
 *        (4 bytes an entry each, every warp's lookups conflict-free;
 *        DFA_EINVAL when they do not fit), 3, 4, 5 = one table copy and 2,
 *        4 or 8 copies of every state's output counter, lane l adding to
 *        copy l % copies so that the atomics of an output-dense automaton
 *        (a k-mer census) spread over more banks (512 or 1024 threads only;
 *        shared memory: the table + copies x 4 bytes a state; DFA_EINVAL
 *        when it does not fit), 0 = the per-lane table copies when CTAs of
 *        1024 threads a SM still fit in 200 KiB (about 198 states at 512
 *        threads), else layout 1; other fields ignored; NULL = 256 x 1024,
 *        layout 0.
 * Asynchronous on `stream`; allocates nothing (capturable in a CUDA graph).
 * Errors: DFA_EINVAL, DFA_ECUDA.
 */
int dfa_multi_count(const uint8_t* const* d_texts, const int64_t* lengths, int32_t nseq,
                    const dfa_multi* table, uint64_t* d_counts, const dfa_config* cfg,
                    void* stream);

/*
 * Diagnostics for failure detection (no counterpart in the paper): enqueue
 * one warp that runs dfa_find's ordered-compaction look-back for tile
 * `tile` (>= 1) on the workspace d_work (at least 8 * (2 + tile + 1)
 * bytes).  It waits for tiles tile-1, tile-2, ... to publish their
 * descriptors; on a zeroed workspace nothing ever publishes them, so every
 * wait gives up after its bound (about two seconds), records the failure in
 * the workspace's status word and returns.  dfa_find_status(d_work, ...)
 * then reports DFA_ETIMEOUT, and the device stays usable.
 * Errors: DFA_EINVAL, DFA_ECUDA.
 */
int dfa_debug_wait_timeout(void* d_work, int64_t work_bytes, int64_t tile, void* stream);

/*
 * Sorted start positions of every pattern of a multi-pattern automaton in one
 * text, in one walk (the multi-pattern automaton of Sec. III-B; Algorithm 1's
 * "location" output for each pattern).  For patterns with few occurrences:
 * each occurrence is written into its pattern's segment of d_pos during the
 * walk, then each segment is sorted on the device.
 *   d_text / n: the text (device).
 *   table:    the automaton (built with a device copy, or attached).
 *   h_counts: HOST uint64[npat], the exact counts of the patterns in this
 *             text (e.g. from dfa_multi_count); each at most DFA_LOCATE_MAX.
 *   d_pos / cap: device int64 buffer of at least the sum of the counts;
 *             pattern p's positions, ascending, start at index
 *             h_counts[0] + ... + h_counts[p-1].
 *   d_work / work_bytes: caller-owned device scratch of at least
 *             dfa_multi_locate_work_bytes(npat) bytes (bases, counts,
 *             cursors, a status word); not shared by calls that may overlap.
 * Asynchronous on `stream`; allocates nothing.  dfa_multi_locate_status
 * (synchronising) returns DFA_EINVAL when the counts did not match the text
 * (a segment over- or under-filled), else DFA_OK.
 * Errors: DFA_EINVAL (a count above DFA_LOCATE_MAX, cap too small, no device
 * copy), DFA_EWORKSPACE, DFA_ECUDA.
 */
#define DFA_LOCATE_MAX 4096
int64_t dfa_multi_locate_work_bytes(int32_t npat);
int dfa_multi_locate(const uint8_t* d_text, int64_t n, const dfa_multi* table, const uint64_t* h_counts,
                     int64_t* d_pos, int64_t cap, void* d_work, int64_t work_bytes, void* stream);
int dfa_multi_locate_status(const void* d_work, int32_t npat, void* stream);

/* Static text for a return code. */
const char* dfa_strerror(int code);

/* Library version string. */
const char* dfa_version(void);

/* Text of the last CUDA failure (DFA_ECUDA) seen by the calling thread: the
 * failing call and CUDA's message.  Empty if none.  Thread-local, static
 * storage owned by the library. */
const char* dfa_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* DNADFA_H */
