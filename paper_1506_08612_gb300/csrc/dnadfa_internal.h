// Internal declarations shared by the host automaton builder and the CUDA
// scan.  Not part of the public ABI (include/dnadfa.h).
#pragma once

#include <cstddef>
#include <cstdint>
#include <vector>

#include "../../include/dnadfa.h"

namespace dnadfa {

// 2-bit base code used by every device layout: code(c) = (c >> 1) & 3, which
// maps A/a -> 0, C/c -> 1, T/t -> 2, G/g -> 3 (the case bit 0x20 and the low
// bit drop out).  A byte is a base iff code_valid(c).
inline uint32_t base_code(uint32_t c) { return (c >> 1) & 3u; }

// Exact base test on one byte: with t = bit2 & ~bit1 (set only for T/t),
// a byte is one of A C G T a c g t iff ((c ^ t*0x11) & 0xD9) == 0x41.
inline bool code_valid(uint32_t c)
{
    uint32_t t = (c >> 2) & ~(c >> 1) & 1u;
    return ((c ^ (t * 0x11u)) & 0xD9u) == 0x41u;
}

// Entry of the four-step composite table (u16):
//   bits 0..7   state after the four steps
//   bits 8..11  accept mask: bit 8+i set iff the state after step i+1 is m
//   bits 12..14 popcount of the accept mask
constexpr uint32_t K4_ACC_SHIFT = 8;
constexpr uint32_t K4_CNT_SHIFT = 12;

// Four-step table with accept flags (u8): with F the smallest power of two
// above m, row q (and its copy, row q | F) holds, per code4, the state after
// the four steps with F added if one of the four steps reached state m.
// Rows are indexed by the previous entry as is, flag included, so the walk
// needs no masking; rows 0..m and F..F+m are used, F+m+1 rows in all.
inline int k4f_flag(int m)
{
    int f = 1;
    while (f <= m) f <<= 1;
    return f;
}

// Device copy layout, one allocation, every part 16-byte aligned:
//   [k4: (m+1)*256 u16][d1: (m+1)*4 u8, padded to 16][stt: (m+1)*256 u8]
//   [k4s: (m+1)*256 u8][k4f: (k4f_flag(m)+m+1)*256 u8]
// k4s is the four-step table holding only the state after the four steps.
struct DeviceTableView {
    const uint8_t* base;   // start of the allocation
    int32_t m;
    int32_t k4_bytes;      // (m+1)*512
    int32_t d1_bytes;      // (m+1)*4 rounded up to 16
    int32_t stt_bytes;     // (m+1)*256
    int32_t k4s_bytes;     // (m+1)*256
    int32_t k4f_bytes;     // (k4f_flag(m)+m+1)*256
};

}  // namespace dnadfa

struct dfa_table {
    int32_t m;
    uint8_t pattern[DFA_MAX_M];          // upper case
    std::vector<uint8_t> d1;             // (m+1)*4, column = base_code
    std::vector<uint16_t> k4;            // (m+1)*256
    std::vector<uint8_t> stt;            // (m+1)*256, the paper's sparse ASCII STT
    std::vector<uint8_t> k4s;            // (m+1)*256, state after four steps only
    std::vector<uint8_t> k4f;            // (k4f_flag(m)+m+1)*256, states + accept flag
    int device;
    void* d_mem;
    size_t d_bytes;
    dnadfa::DeviceTableView view;
    bool owns_mem = true;                // false: d_mem is the caller's (dfa_build_into)
    std::vector<uint8_t> img;            // device image kept for dfa_build_into's async copy
};

namespace dnadfa {
// Fill d1, k4, stt, k4s and k4f of t from t->pattern / t->m.  Returns DFA_OK or DFA_EINVAL.
int build_host_tables(dfa_table* t);

// Record the text of a failure for dfa_last_error (thread-local); returns code.
int set_last_error(int code, const char* msg);
}  // namespace dnadfa
