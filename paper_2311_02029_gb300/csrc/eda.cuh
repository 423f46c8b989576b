// SneakySnake edit-distance approximation on the GPU (Table 1, ref. [48]; pairs at
// approximate distance <= E pass, read-mapping "Evaluation Methodology").
//
// The neighbourhood map has one row per diagonal d in [-E, E]; M[d][j] = 0 iff read base j
// equals window base E + j + d. From column c the walk follows the longest zero run of any
// row, counts the obstacle that ends it and steps over it; more than E obstacles rejects.
//
// Bit-parallel form: a group of G lanes works on one pair. Each lane owns a contiguous range
// of ceil((2E+1)/G) diagonals (di = E + d is the window offset of the row). The run of a row
// from column c ends at its next mismatch, found 32 columns at a time by XOR-ing 64-bit
// slices of the 2-bit packed read and window, folding each 2-bit group to one bit and
// taking the lowest set bit. The group then takes the furthest run end with one
// redux.sync max. Window bases outside the genome (classification windows that overhang a
// genome end) are forced to mismatch with an edge mask.
#pragma once

#include "common.cuh"

// Mismatch flags (bit 2t) for window columns q0 .. q0+31 that lie outside [lo, hi).
MT_DEV uint64_t edge_mask(int32_t q0, int32_t lo, int32_t hi) {
    uint64_t m = 0;
    int32_t a = lo - q0;
    if (a > 0) m |= (a >= 32) ? EVEN_BITS : (((1ull << (2 * a)) - 1) & EVEN_BITS);
    int32_t b = hi - q0;
    if (b < 32) m |= (b <= 0) ? EVEN_BITS : (~((1ull << (2 * b)) - 1) & EVEN_BITS);
    return m;
}

// First column >= c at which the read and window offset `woff` differ, or n.
template <bool EDGES>
MT_DEV uint32_t next_mismatch(const uint64_t *rd, const uint64_t *wn, uint32_t n, uint32_t c,
                              uint32_t woff, int32_t lo, int32_t hi) {
    for (uint32_t p = c; p < n; p += 32) {
        uint64_t x = get32(rd, p) ^ get32(wn, p + woff);
        uint64_t m = (x | (x >> 1)) & EVEN_BITS;
        if (EDGES) m |= edge_mask((int32_t)(p + woff), lo, hi);
        if (m) return min(p + ((uint32_t)(__ffsll((long long)m) - 1) >> 1), n);
    }
    return n;
}

// The walk for one pair, executed by the G lanes of `gmask` (glane = lane within group).
// Lane glane owns the contiguous diagonal range [glane*T, glane*T + T), T = ceil((2E+1)/G).
// Per step it loads the read's 32 columns from c once and the window's bases from c + its
// first diagonal (up to 32 + T bases) once; each diagonal's 32 columns then come from a
// register funnel shift. Only a diagonal whose first 32 columns all match walks on further.
template <int G, bool EDGES>
MT_DEV uint32_t sneaky_walk(const uint64_t *rd, const uint64_t *wn, uint32_t n, uint32_t E,
                            int32_t lo, int32_t hi, unsigned gmask, uint32_t glane) {
    const uint32_t ndiag = 2 * E + 1;
    const uint32_t T = (ndiag + G - 1) / G;
    const uint32_t d0 = glane * T;
    const uint32_t d1 = min(d0 + T, ndiag);
    uint32_t c = 0, cnt = 0;
    while (c < n) {
        uint32_t best = c;
        if (d0 < d1) {
            const uint64_t r0 = get32(rd, c);
            for (uint32_t tb = d0; tb < d1; tb += 32) {   // blocks of 32 diagonals
                const uint32_t q = c + tb;
                const uint64_t w0 = get32(wn, q);
                const uint64_t w1 = get32(wn, q + 32);
                const uint32_t tn = min(32u, d1 - tb);
                for (uint32_t t = 0; t < tn; t++) {
                    const uint32_t sh = 2 * t;
                    const uint64_t x = t ? ((w0 >> sh) | (w1 << (64 - sh))) : w0;
                    const uint64_t y = r0 ^ x;
                    uint64_t m = (y | (y >> 1)) & EVEN_BITS;
                    if (EDGES) m |= edge_mask((int32_t)(q + t), lo, hi);
                    uint32_t e;
                    if (m) e = c + ((uint32_t)(__ffsll((long long)m) - 1) >> 1);
                    else e = next_mismatch<EDGES>(rd, wn, n, c + 32, tb + t, lo, hi);
                    e = e < n ? e : n;
                    best = e > best ? e : best;
                }
            }
        }
        if (G > 1) best = __reduce_max_sync(gmask, best);
        c = best;
        if (c >= n) break;
        cnt++;
        if (cnt > E) break;
        c++;
    }
    return cnt < E + 1 ? cnt : E + 1;
}

// Shared-memory words one pair needs: read ceil(n/32)+2, window ceil((n+2E)/32)+3.
__host__ __device__ __forceinline__ uint32_t eda_read_words(uint32_t maxn) {
    return (maxn + 31) / 32 + 2;
}
__host__ __device__ __forceinline__ uint32_t eda_win_words(uint32_t maxn, uint32_t maxE) {
    return (maxn + 2 * maxE + 31) / 32 + 3;
}
