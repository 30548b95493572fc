// Host construction of the failure-less single-pattern automaton and of the
// table layouts the scan kernels read (Sec. III-B, Fig. 4 and Table I).
//
// delta(q, a), for q = 0..m and a in {A, C, G, T}, is the length of the
// longest prefix of P that is a suffix of P[0..q)·a; the final state is m,
// which is already the last state number, so the accept test of Sec. III-B
// ("next state >= a - b") reads "next state == m".  The construction here is
// the linear one that runs a second copy of the automaton one byte behind:
// a mismatch from state q behaves like the state X reached by reading
// P[1..q), so row q copies row X and overrides the column of P[q].
#include <cstring>

#include "dnadfa_internal.h"

namespace dnadfa {

int build_host_tables(dfa_table* t)
{
    const int m = t->m;
    if (m < 1 || m > DFA_MAX_M) return DFA_EINVAL;
    const int S = m + 1;
    int pc[DFA_MAX_M];
    for (int j = 0; j < m; j++) {
        uint32_t c = t->pattern[j];
        if (!code_valid(c)) return DFA_EINVAL;
        pc[j] = (int)base_code(c);
    }

    // single-step table in base_code column order
    std::vector<uint8_t>& d1 = t->d1;
    d1.assign((size_t)S * 4, 0);
    d1[0 * 4 + pc[0]] = 1;
    int X = 0;
    for (int q = 1; q <= m; q++) {
        for (int a = 0; a < 4; a++) d1[q * 4 + a] = d1[X * 4 + a];
        if (q < m) {
            d1[q * 4 + pc[q]] = (uint8_t)(q + 1);
            X = d1[X * 4 + pc[q]];
        }
    }

    // four-step composite table: index q*256 + code4 with
    // code4 = d0 | d1<<2 | d2<<4 | d3<<6, d0 the code of the first byte
    std::vector<uint16_t>& k4 = t->k4;
    k4.assign((size_t)S * 256, 0);
    std::vector<uint8_t>& k4s = t->k4s;
    k4s.assign((size_t)S * 256, 0);
    for (int q = 0; q < S; q++) {
        for (int code4 = 0; code4 < 256; code4++) {
            int s = q;
            uint32_t acc = 0;
            for (int i = 0; i < 4; i++) {
                s = d1[s * 4 + ((code4 >> (2 * i)) & 3)];
                if (s == m) acc |= 1u << i;
            }
            uint32_t pop = (uint32_t)__builtin_popcount(acc);
            k4[(size_t)q * 256 + code4] =
                (uint16_t)(s | (acc << K4_ACC_SHIFT) | (pop << K4_CNT_SHIFT));
            k4s[(size_t)q * 256 + code4] = (uint8_t)s;
        }
    }

    // four-step states with an accept flag, for the relaxed walk: the row of
    // an entry is the entry itself, so flagged rows repeat the plain ones
    const int F = k4f_flag(m);
    std::vector<uint8_t>& k4f = t->k4f;
    k4f.assign((size_t)(F + S) * 256, 0);
    for (int q = 0; q < S; q++)
        for (int code4 = 0; code4 < 256; code4++) {
            uint16_t v = k4[(size_t)q * 256 + code4];
            uint8_t f = (uint8_t)((v & 0xFFu) + (((v >> K4_ACC_SHIFT) & 0xFu) ? F : 0));
            k4f[(size_t)q * 256 + code4] = f;
            k4f[(size_t)(q | F) * 256 + code4] = f;
        }

    // the paper's sparse ASCII STT: columns are raw byte values; only the
    // eight base columns hold transitions, every other column holds q0
    std::vector<uint8_t>& stt = t->stt;
    stt.assign((size_t)S * 256, 0);
    static const char kBases[8] = {'A', 'C', 'G', 'T', 'a', 'c', 'g', 't'};
    for (int q = 0; q < S; q++)
        for (char ch : kBases) {
            uint32_t c = (uint8_t)ch;
            stt[(size_t)q * 256 + c] = d1[q * 4 + base_code(c)];
        }
    return DFA_OK;
}

}  // namespace dnadfa
