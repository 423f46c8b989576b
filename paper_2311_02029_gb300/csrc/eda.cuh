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

// The walk when each lane has at most SNAKE_TMAX diagonals: the lanes keep 32-bit mismatch
// masks of their diagonals over one 16-column block [B, B + 16) in registers, refilled when
// the walk leaves the block, so a step inside the block costs a shift and a find-first-set a
// diagonal. A run that reaches the block end continues with next_mismatch from B + 16. Same
// result as the walk below.
static constexpr uint32_t SNAKE_TMAX = 4;

template <int G, bool EDGES>
MT_DEV uint32_t sneaky_walk_cached(const uint64_t *rd, const uint64_t *wn, uint32_t n, uint32_t E,
                                   int32_t lo, int32_t hi, unsigned gmask, uint32_t glane) {
    const uint32_t ndiag = 2 * E + 1;
    const uint32_t T = (ndiag + G - 1) / G;
    const uint32_t d0 = glane * T;
    const uint32_t nt = d0 < ndiag ? min(T, ndiag - d0) : 0u;
    uint32_t M[SNAKE_TMAX];
    uint32_t c = 0, cnt = 0, B = 0;
    bool fresh = false;
    while (c < n) {
        if (!fresh || c - B >= 16) {   // refill the masks at the current column
            B = c;
            fresh = true;
            const uint32_t r0 = (uint32_t)get32(rd, B);
            const uint64_t w0 = get32(wn, B + d0);
            const uint64_t em = EDGES ? edge_mask((int32_t)(B + d0), lo, hi) : 0ull;
#pragma unroll
            for (uint32_t t = 0; t < SNAKE_TMAX; t++) {
                if (t < nt) {
                    const uint32_t y = r0 ^ (uint32_t)(w0 >> (2 * t));
                    uint32_t m = (y | (y >> 1)) & 0x55555555u;
                    if (EDGES) m |= (uint32_t)(em >> (2 * t)) & 0x55555555u;
                    M[t] = m;
                }
            }
        }
        const uint32_t sh = 2 * (c - B);
        uint32_t best = c;
#pragma unroll
        for (uint32_t t = 0; t < SNAKE_TMAX; t++) {
            if (t < nt) {
                const uint32_t r = M[t] >> sh;
                uint32_t e = r ? c + ((uint32_t)(__ffs((int)r) - 1) >> 1)
                               : next_mismatch<EDGES>(rd, wn, n, B + 16, d0 + t, lo, hi);
                e = e < n ? e : n;
                best = e > best ? e : best;
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

// First mismatch at or after column c of the diagonals tb .. tb + tn - 1 (tn <= 17), the
// furthest of them and `best`. The read's columns c .. c + 15 are r16 (2 bits a base); one
// 64-bit window word (bases c + tb ..) holds columns c .. c + 15 of all tn diagonals, so each
// diagonal costs a shift, an XOR, a fold and a find-first-set on 32 bits. A diagonal whose 16
// columns all match (nearly only the location's own) walks on with next_mismatch. FULL: tn is
// 17, and the pass is unrolled (constant shifts; the walks-on come after it).
template <bool EDGES, bool FULL>
MT_DEV uint32_t snake_block16(const uint64_t *rd, const uint64_t *wn, uint32_t n, uint32_t c, uint32_t r16,
                              uint32_t tb, uint32_t tn, int32_t lo, int32_t hi, uint32_t best) {
    const uint32_t q = c + tb;
    const uint64_t w = get32(wn, q);
    const uint64_t em = EDGES ? edge_mask((int32_t)q, lo, hi) : 0ull;
    if (FULL) {
        uint32_t open = 0;
#pragma unroll
        for (uint32_t t = 0; t < 17; t++) {
            const uint32_t y = r16 ^ (uint32_t)(w >> (2 * t));
            uint32_t m = (y | (y >> 1)) & 0x55555555u;
            if (EDGES) m |= (uint32_t)(em >> (2 * t)) & 0x55555555u;
            const uint32_t e = m ? min(c + ((uint32_t)(__ffs((int)m) - 1) >> 1), n) : c;
            open |= (uint32_t)(m == 0) << t;
            best = e > best ? e : best;
        }
        while (open) {
            const uint32_t t = __ffs((int)open) - 1;
            open &= open - 1;
            const uint32_t e = min(next_mismatch<EDGES>(rd, wn, n, c + 16, tb + t, lo, hi), n);
            best = e > best ? e : best;
        }
    } else {
        for (uint32_t t = 0; t < tn; t++) {
            const uint32_t y = r16 ^ (uint32_t)(w >> (2 * t));
            uint32_t m = (y | (y >> 1)) & 0x55555555u;
            if (EDGES) m |= (uint32_t)(em >> (2 * t)) & 0x55555555u;
            uint32_t e;
            if (m) e = c + ((uint32_t)(__ffs((int)m) - 1) >> 1);
            else e = next_mismatch<EDGES>(rd, wn, n, c + 16, tb + t, lo, hi);
            e = e < n ? e : n;
            best = e > best ? e : best;
        }
    }
    return best;
}

// Furthest first mismatch at or after column c over the diagonals [d0, d1) and `best`.
template <bool EDGES>
MT_DEV uint32_t snake_diagonals(const uint64_t *rd, const uint64_t *wn, uint32_t n, uint32_t c, uint32_t d0,
                                uint32_t d1, int32_t lo, int32_t hi, uint32_t best) {
    const uint32_t r16 = (uint32_t)get32(rd, c);
    uint32_t tb = d0;
    for (; tb + 17 <= d1; tb += 17) best = snake_block16<EDGES, true>(rd, wn, n, c, r16, tb, 17, lo, hi, best);
    if (tb < d1) best = snake_block16<EDGES, false>(rd, wn, n, c, r16, tb, d1 - tb, lo, hi, best);
    return best;
}

// The walk for one pair, executed by the G lanes of `gmask` (glane = lane within group).
// Lane glane owns the contiguous diagonal range [glane*T, glane*T + T), T = ceil((2E+1)/G).
// Per step it loads the read's 16 columns from c once and, per block of 17 diagonals, one
// window word (snake_diagonals).
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
        if (d0 < d1) best = snake_diagonals<EDGES>(rd, wn, n, c, d0, d1, lo, hi, best);
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

// ---- the pipeline's other approximations (Table 1: HD [49], SHD [50]; Base Counting [46]
// and q-gram [52], the O(n) count comparisons of the Discussion) ----------------------------
// Readings: HD, Base Counting and q-gram compare the read with the window's central segment
// S = window[E, E + n) (the location's first diagonal); SHD uses all 2E+1 diagonals. A window
// base outside the genome equals no read base. Each result is min(estimate, E + 1).
enum EdaAlgo : int { ALGO_SNAKE = 0, ALGO_HD = 1, ALGO_BC = 2, ALGO_QGRAM = 3, ALGO_SHD = 4 };
static constexpr uint32_t QGRAM_Q = 5;
static constexpr uint32_t QGRAM_BINS = 1u << (2 * QGRAM_Q);

// Mismatch flags (bit 2t) of read columns p .. p+31 against window columns p+off .. (p < n);
// flags of columns >= n are cleared.
template <bool EDGES>
MT_DEV uint64_t mism32(const uint64_t *rd, const uint64_t *wn, uint32_t p, uint32_t off, uint32_t n,
                       int32_t lo, int32_t hi) {
    const uint64_t x = get32(rd, p) ^ get32(wn, p + off);
    uint64_t m = (x | (x >> 1)) & EVEN_BITS;
    if (EDGES) m |= edge_mask((int32_t)(p + off), lo, hi);
    if (n - p < 32) m &= (1ull << (2 * (n - p))) - 1;
    return m;
}

// Hamming distance on the central segment; each lane of the group takes 32-column blocks.
template <int G, bool EDGES>
MT_DEV uint32_t hamming_est(const uint64_t *rd, const uint64_t *wn, uint32_t n, uint32_t E, int32_t lo,
                            int32_t hi, unsigned gmask, uint32_t glane) {
    uint32_t cnt = 0;
    for (uint32_t p = 32 * glane; p < n; p += 32 * G) cnt += (uint32_t)__popcll(mism32<EDGES>(rd, wn, p, E, n, lo, hi));
    if (G > 1) cnt = __reduce_add_sync(gmask, cnt);
    return min(cnt, E + 1);
}

// Base Counting: ceil(sum over A, C, G, T and "outside" of |count in read - count in S| / 2).
template <int G, bool EDGES>
MT_DEV uint32_t basecount_est(const uint64_t *rd, const uint64_t *wn, uint32_t n, uint32_t E, int32_t lo,
                              int32_t hi, unsigned gmask, uint32_t glane) {
    int d0 = 0, d1 = 0, d2 = 0, d3 = 0, d4 = 0;   // read minus segment, per base (4: outside)
    for (uint32_t p = 32 * glane; p < n; p += 32 * G) {
        const uint32_t v = min(32u, n - p);
        const uint64_t V = v == 32 ? EVEN_BITS : (((1ull << (2 * v)) - 1) & EVEN_BITS);
        const uint64_t O = EDGES ? (edge_mask((int32_t)(p + E), lo, hi) & V) : 0ull;
        const uint64_t W = V & ~O;
        const uint64_t xr = get32(rd, p), xw = get32(wn, p + E);
        const uint64_t rl = xr & EVEN_BITS, rh = (xr >> 1) & EVEN_BITS;
        const uint64_t wl = xw & EVEN_BITS, wh = (xw >> 1) & EVEN_BITS;
        d0 += __popcll(~rl & ~rh & V) - __popcll(~wl & ~wh & W);
        d1 += __popcll(rl & ~rh & V) - __popcll(wl & ~wh & W);
        d2 += __popcll(~rl & rh & V) - __popcll(~wl & wh & W);
        d3 += __popcll(rl & rh & V) - __popcll(wl & wh & W);
        d4 -= __popcll(O);
    }
    if (G > 1) {
        d0 = __reduce_add_sync(gmask, d0); d1 = __reduce_add_sync(gmask, d1);
        d2 = __reduce_add_sync(gmask, d2); d3 = __reduce_add_sync(gmask, d3);
        d4 = __reduce_add_sync(gmask, d4);
    }
    const uint32_t sum = (uint32_t)(abs(d0) + abs(d1) + abs(d2) + abs(d3) + abs(d4));
    return min((sum + 1) / 2, E + 1);
}

// q-gram distance (q = 5), a whole warp per pair: the read's q-grams add 1 and the segment's
// subtract 1 in a shared-memory histogram `hist` (QGRAM_BINS counters, 16-byte aligned, zero
// on entry and on return); a segment q-gram holding an outside base adds 1 directly. The
// warp then sums |counter| over all bins (16-byte loads) and clears them. ceil(sum / 2q).
template <bool EDGES>
MT_DEV uint32_t qgram_est(const uint64_t *rd, const uint64_t *wn, uint32_t n, uint32_t E, int32_t lo,
                          int32_t hi, int *hist) {
    const uint32_t lane = lane_id();
    uint32_t s = 0;
    for (uint32_t j = lane; j + QGRAM_Q <= n; j += 32) {
        atomicAdd(&hist[(uint32_t)get32(rd, j) & (QGRAM_BINS - 1)], 1);
        const int32_t q0 = (int32_t)(E + j);
        if (EDGES && (q0 < lo || q0 + (int32_t)QGRAM_Q > hi)) s++;
        else atomicAdd(&hist[(uint32_t)get32(wn, E + j) & (QGRAM_BINS - 1)], -1);
    }
    __syncwarp();
    int4 *h4 = reinterpret_cast<int4 *>(hist);
#pragma unroll
    for (uint32_t b = lane; b < QGRAM_BINS / 4; b += 32) {
        const int4 v = h4[b];
        s += (uint32_t)(abs(v.x) + abs(v.y) + abs(v.z) + abs(v.w));
        h4[b] = make_int4(0, 0, 0, 0);
    }
    s = __reduce_add_sync(0xffffffffu, s);
    __syncwarp();
    return min((s + 2 * QGRAM_Q - 1) / (2 * QGRAM_Q), E + 1);
}

// SHD: each lane takes a contiguous range of the 2E+1 diagonals and walks its masks block by
// block, keeping the neighbouring blocks for two columns of context on each side (columns
// outside [0, n) count as matches, so runs touching an end are never filled). A match at
// column i is filled when it is a run of one (mismatch at i-1 and i+1) or one of a run of two
// (mismatches at i-1 and i+2, or at i-2 and i+1). Each amended mask is AND-ed into F
// (ceil(n/32) words of shared memory); the set flags left are counted.
template <int G, bool EDGES>
MT_DEV uint32_t shd_est(const uint64_t *rd, const uint64_t *wn, uint32_t n, uint32_t E, int32_t lo,
                        int32_t hi, unsigned gmask, uint32_t glane, unsigned long long *F) {
    const uint32_t nb = (n + 31) / 32;
    for (uint32_t b = glane; b < nb; b += G) F[b] = EVEN_BITS;
    __syncwarp(gmask);
    const uint32_t ndiag = 2 * E + 1, T = (ndiag + G - 1) / G;
    const uint32_t dlo = glane * T, dhi = min(dlo + T, ndiag);
    for (uint32_t di = dlo; di < dhi; di++) {
        uint64_t P = 0, C = nb ? mism32<EDGES>(rd, wn, 0, di, n, lo, hi) : 0ull;
        for (uint32_t b = 0; b < nb; b++) {
            const uint64_t N = b + 1 < nb ? mism32<EDGES>(rd, wn, 32 * (b + 1), di, n, lo, hi) : 0ull;
            const uint64_t L1 = ((C << 2) | (P >> 62)) & EVEN_BITS, L2 = ((C << 4) | (P >> 60)) & EVEN_BITS;
            const uint64_t R1 = ((C >> 2) | (N << 62)) & EVEN_BITS, R2 = ((C >> 4) | (N << 60)) & EVEN_BITS;
            const uint64_t fill = ~C & EVEN_BITS & ((L1 & R1) | (L1 & ~R1 & R2) | (L2 & ~L1 & R1));
            atomicAnd(&F[b], (unsigned long long)(C | fill));
            P = C;
            C = N;
        }
    }
    __syncwarp(gmask);
    uint32_t cnt = 0;
    for (uint32_t b = glane; b < nb; b += G) cnt += (uint32_t)__popcll(F[b]);
    if (G > 1) cnt = __reduce_add_sync(gmask, cnt);
    __syncwarp(gmask);
    return min(cnt, E + 1);
}
