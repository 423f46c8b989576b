// Read classification on the device: the paper's three stages ("The MetaTrinity Pipeline",
// Fig. 1) over one batch of reads.
//
//   k_seed     (stage 1 + 2a-c)  one warp per read: bytes -> 2-bit words in shared memory,
//              k-mer codes and keys, (w,k)-minimizers by warp-parallel window minima, one
//              open-addressing probe per minimizer (a 32-byte slot, occurrences inline),
//              seed matches into shared memory, per-genome containment counts (shared-memory
//              histogram), warp bitonic sort of the matches by (genome, strand, diagonal),
//              greedy locations via "next start" pointers, the qualifying locations ranked
//              and the first C stored. Locations are formed per (genome, strand), so masking
//              genomes later only removes whole locations: no second seeding pass.
//   k_mask     (stage 1d)  genome g kept iff hits[g] * den > max(hits) * num.
//   k_select   (stage 2c)  first top_n stored locations in kept genomes -> candidates.
//   k_fallback exact slow path, one CTA per read, for reads whose matches overflow shared
//              memory or whose stored locations run out after masking.
//   EDA        (stage 2d)  SneakySnake on every candidate (eda.cu).
//   k_decide   (stage 3a)  per-read decision, unique counts, multi-mapped reads.
//   k_multi / k_abund (stage 3a-b) multi-read split, relative abundances, 0.01% cutoff.
#include <algorithm>
#include <type_traits>
#include <cstdio>
#include <cstring>
#include <vector>

#include "eda.cuh"
#include "internal.h"

namespace mt {
bool eda_mode_ok(uint32_t mode);
int launch_classify_eda(const IndexView &ix, const uint64_t *rw, const IoBlock *io,
                        const uint32_t *cl, const uint64_t *cl_count, uint64_t max_items,
                        const Cluster *cand, uint32_t top_n, uint32_t e_abs, uint32_t e_permille,
                        uint32_t maxn, uint32_t maxE, uint32_t mode, uint8_t *dist,
                        unsigned long long *counter, cudaStream_t s, bool tune, mt_eda_shape *used);

static constexpr unsigned FULL = 0xffffffffu;
static constexpr int SEED_WARPS = 8;
static constexpr int SEED_THREADS = SEED_WARPS * 32;
static constexpr uint32_t TILE = 128;                     // windows per tile
static constexpr uint32_t KEYS = TILE + MT_MAX_W + 4;     // k-mers a tile may read (<= TILE+w+2)
static constexpr uint32_t HCAP = 256;                     // seed matches held per read
static constexpr uint32_t W11_TILE = 150;                 // windows per pass of the w = 11 path
static constexpr uint32_t MPOS = W11_TILE > TILE ? W11_TILE : TILE;   // minimizers a pass may select
static constexpr uint32_t RDW = MT_MAX_READ_LEN / 32 + 2;
static constexpr uint32_t CSTORE = 8;                     // locations stored per read
static constexpr uint32_t QOVF = 0xFFFFFFFFu;
static constexpr uint32_t SMEM_HIST_MAX = 4096;           // genomes counted in shared memory
static constexpr uint32_t MULTI_UNROLL = 2;     // key-filter loads in flight per lane (several indexes)
static constexpr int FB_CTAS = 16;
static constexpr int FB_THREADS = 256;

// Per-warp shared memory of the seeding kernel. HitT is the seed-match key: 32 bits when the
// index's genome count and lengths allow (see HitKey), else 64. The w = 11 block path keeps no
// per-position keys (W11: key[] shrinks to one word).
template <typename HitT, bool W11 = false>
struct WarpSmem {
    unsigned long long stat[4];     // the warp's minimizers, matches, list occurrences, stored locations
    uint32_t nmr;                   // minimizers of the current read
    uint32_t pad_;
    uint64_t rd[RDW];               // packed read
    HitT hits[HCAP];                // seed-match keys of the read
    union {                         // the tiles of a read, then its location walk
        struct {
            uint64_t key[W11 ? 1 : KEYS];   // k-mer keys of the tile (general path)
            uint64_t code[KEYS];    // canonical code | strand << 63
            uint16_t mpos[MPOS];    // minimizer positions of the tile
            // lookups of one round, by rank among those with matches
            uint64_t e_w[32 * 3];   // inline occurrences, or the occurrence-list offset
            uint32_t e_pre[32];     // first match of the lookup within the round
            uint32_t e_meta[32];    // rpos | strand << 16 | inline << 17
        } t;
        struct {
            uint16_t gs[HCAP + 1];  // starts of (genome, strand) groups in the sorted matches
            // qualifying locations: 32-bit match keys as one rank word each,
            // (0xFFFF - seed count) << 32 | key of the first match; 64-bit keys as key and count
            uint64_t qr[sizeof(HitT) == 4 ? HCAP : 1];
            HitT qk[sizeof(HitT) == 4 ? 1 : HCAP];
            uint16_t qn[sizeof(HitT) == 4 ? 1 : HCAP];
            uint32_t qcount;
        } wk;
    } u;
};

enum StatIdx { ST_MINS = 0, ST_HITS, ST_CAND, ST_ACC, ST_MULTI, ST_FB, ST_EXT, ST_STORED, ST_N };

struct Counters {
    uint32_t err;
    uint32_t pad;
    unsigned long long stat[ST_N];
    uint64_t cl_count;
    uint64_t fb_count;
    uint64_t multi_count;
    unsigned long long eda_counter;
    uint32_t maxn;
    uint32_t pad2;
};

// one index among several counted in one pass
struct BatchView {
    const ulonglong2 *table;
    uint64_t slot_mask;
    const uint64_t *occ;
    const uint64_t *filter;   // the index's key filter: a key it rejects is not in the table
    uint32_t slot_shift;
    uint32_t filter_shift;
    uint32_t base;            // first counter of the batch's genomes
    uint32_t pad;
};

struct SeedArgs {
    IndexView ix;
    const IoBlock *io;
    uint32_t e_abs, e_permille, min_seeds, max_occ;
    uint64_t *rw;
    uint32_t *qcnt;
    Cluster *clus;
    unsigned long long *ghits;
    uint32_t *fb_list;
    Counters *ctr;
    uint64_t r_begin, r_end;   // the reads this launch takes: [r_begin, min(r_end, n_reads))
    // counting over several indexes of one (k, w, canonical, compression) at once: every
    // minimizer is looked up in each batch's table and counted at base + genome
    const BatchView *bv = nullptr;
    uint32_t n_bv = 0, n_hist = 0;
    uint32_t div_magic = 0;    // ceil(2^32 / n_bv): pair / n_bv = umulhi(pair, div_magic) (n_bv > 1)
};

// ---- read packing (one warp) ------------------------------------------------------------
// Four bytes at a time: code = ((b >> 1) & 3) with G/T swapped; a byte is valid iff the
// ASCII letter of its code (picked with a byte permute from "ACGT") equals the byte. Bytes
// outside `m` give code 0 and are not checked. Returns the four codes as 8 bits, first byte
// lowest (one multiply gathers the 2-bit fields: the partial products never overlap).
MT_DEV uint32_t swar_pack4(uint32_t u, uint32_t m, bool &bad) {
    uint32_t c = (u >> 1) & 0x03030303u;
    c ^= (c >> 1) & 0x01010101u;
    c &= m;
    const uint32_t t = c | (c >> 4);
    const uint32_t sel = (t & 0xFFu) | ((t >> 8) & 0xFF00u);     // code of byte i in nibble i
    bad |= ((__byte_perm(0x54474341u, 0u, sel) ^ u) & m) != 0u;
    return (c * 0x01041040u) >> 24;
}

// Bytes [0, nb) of a 4-byte word, nb clamped to [0, 4].
MT_DEV uint32_t low_bytes(int32_t nb) {
    return nb >= 4 ? 0xFFFFFFFFu : nb <= 0 ? 0u : ((1u << (8 * nb)) - 1u);
}

// Packs bases [start, start + n) of `reads` into rd[0, nw) (2 bits a base, base i at bits
// 2(i%32) of word i/32, the tail of the last word zero) and into `dst`, and zeroes rd[nw],
// rd[nw + 1]. Each lane converts 8 bases a pass from two aligned 8-byte loads; four lanes
// assemble one word with two shuffles. Returns true (on every lane) if a byte is not ACGT.
MT_DEV bool warp_pack(const uint8_t *reads, uint64_t n_bases, int vec_ok, uint64_t start, uint32_t n,
                      uint64_t *rd, uint64_t *dst) {
    const uint32_t lane = lane_id();
    const uint32_t nw = (n + 31) / 32;
    const uint32_t sh = (uint32_t)(start & 7u) * 8u;
    const uint64_t a0 = start & ~7ull;
    bool bad = false;
    __syncwarp();                                 // rd of the previous read is no longer read
    for (uint32_t b0 = 0; b0 < n; b0 += 256) {
        const uint32_t j = b0 + 8 * lane;         // first base of this lane
        uint32_t c16 = 0;
        if (j < n) {
            uint32_t x0, x1;
            const uint64_t a = a0 + j;            // aligned: bases start + j .. + 7 lie in [a, a + 16)
            if (vec_ok && a + 16 <= n_bases) {
                const uint2 lo = __ldg(reinterpret_cast<const uint2 *>(reads + a));
                const uint2 hi = __ldg(reinterpret_cast<const uint2 *>(reads + a + 8));
                if (sh < 32) {
                    x0 = __funnelshift_r(lo.x, lo.y, sh);
                    x1 = __funnelshift_r(lo.y, hi.x, sh);
                } else {
                    x0 = __funnelshift_r(lo.y, hi.x, sh - 32);
                    x1 = __funnelshift_r(hi.x, hi.y, sh - 32);
                }
            } else {
                x0 = x1 = 0;
                const uint64_t p0 = start + j, end = start + n;
#pragma unroll 1
                for (int q = 0; q < 8; q++) {
                    const uint32_t by = (p0 + q < end) ? reads[p0 + q] : 'A';
                    if (q < 4) x0 |= by << (8 * q); else x1 |= by << (8 * (q - 4));
                }
            }
            const int32_t nb = (int32_t)(n - j);
            c16 = swar_pack4(x0, low_bytes(nb), bad) | (swar_pack4(x1, low_bytes(nb - 4), bad) << 8);
        }
        uint32_t v = c16 << (16 * (lane & 1u));
        v |= __shfl_xor_sync(FULL, v, 1);
        const uint32_t hi = __shfl_xor_sync(FULL, v, 2);
        const uint32_t t = (b0 >> 5) + (lane >> 2);
        if ((lane & 3u) == 0 && t < nw) {
            const uint64_t word = (uint64_t)v | ((uint64_t)hi << 32);
            rd[t] = word;
            if (dst) dst[t] = word;
        }
    }
    if (lane < 2) rd[nw + lane] = 0;
    __syncwarp();
    return __any_sync(FULL, bad);
}

// Homopolymer compression of a packed read in place (the containment seeds of an index built
// with MT_INDEX_HPC): each run of one base becomes a single base. Pass t reads word t: a lane
// keeps base 32t+lane when it differs from the base before it, a ballot gives the kept
// bases' output positions, and each output word is assembled with redux OR; an output word is
// stored once complete, at an index <= t, so no word is written before it has been read.
// Zeroes the words after the result (up to the old end + 2). Returns the new length.
MT_DEV uint32_t warp_hpc(uint64_t *rd, uint32_t n) {
    const uint32_t lane = lane_id();
    const uint32_t nw = (n + 31) / 32;
    uint32_t out = 0, prev = 4;   // bases kept so far; last base of the previous word (4: none)
    uint64_t acc = 0;              // the output word being filled
    for (uint32_t t = 0; t < nw; t++) {
        const uint64_t word = rd[t];
        __syncwarp();
        const uint32_t b = (uint32_t)(word >> (2 * lane)) & 3u;
        uint32_t pb = __shfl_up_sync(FULL, b, 1);
        if (lane == 0) pb = prev;
        const bool keep = 32 * t + lane < n && b != pb;
        const unsigned bal = __ballot_sync(FULL, keep);
        const uint32_t o = out + __popc(bal & ((1u << lane) - 1u));
        const uint32_t cur = out >> 5;
        uint64_t lo = 0, hi = 0;
        if (keep) {
            if ((o >> 5) == cur) lo = (uint64_t)b << (2 * (o & 31));
            else hi = (uint64_t)b << (2 * (o & 31));
        }
        acc |= ((uint64_t)__reduce_or_sync(FULL, (uint32_t)(lo >> 32)) << 32) | __reduce_or_sync(FULL, (uint32_t)lo);
        const uint64_t nxt = ((uint64_t)__reduce_or_sync(FULL, (uint32_t)(hi >> 32)) << 32) |
                             __reduce_or_sync(FULL, (uint32_t)hi);
        const uint32_t cnt = __popc(bal);
        if (((out + cnt) >> 5) != cur) {   // word cur is complete
            if (lane == 0) rd[cur] = acc;
            acc = nxt;
        }
        out += cnt;
        prev = __shfl_sync(FULL, b, 31);
    }
    if (lane == 0) rd[out >> 5] = acc;
    __syncwarp();
    for (uint32_t t = (out >> 5) + 1 + lane; t < nw + 2; t += 32) rd[t] = 0;
    __syncwarp();
    return out;
}

template <typename T>
MT_DEV uint32_t lower_bound_t(const T *a, uint32_t lo, uint32_t hi, T key) {
    while (lo < hi) {
        uint32_t mid = (lo + hi) >> 1;
        if (a[mid] < key) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Seed-match keys in the seeding kernel. Both forms order matches by (genome, relative
// strand, diagonal); the 32-bit form packs genome << (db + 1) | rel << db | diag + bias and
// is used when the index guarantees those fields fit (bias + diagonal + E + 1 < 2^db too,
// so a band bound key + E + 1 never leaves its (genome, strand) group).
template <bool HK32> struct HitKey;
template <> struct HitKey<true> {
    using T = uint32_t;
    uint32_t db;
    MT_DEV T make(uint64_t occ, uint32_t rpos, uint32_t rst, uint32_t nk) const {
        const uint32_t rel = ((uint32_t)occ & 1u) ^ rst;
        const uint32_t rp = rel ? nk - rpos : rpos;
        return ((uint32_t)(occ >> 33) << (db + 1)) | (rel << db) | ((uint32_t)(occ >> 1) + DIAG_BIAS - rp);
    }
    MT_DEV uint32_t grel(T h) const { return h >> db; }
    MT_DEV uint32_t genome(T h) const { return h >> (db + 1); }
    MT_DEV uint64_t wide(T h) const {
        return ((uint64_t)(h >> (db + 1)) << 34) | ((uint64_t)((h >> db) & 1u) << 33) | (h & ((1u << db) - 1u));
    }
};
template <> struct HitKey<false> {
    using T = uint64_t;
    uint32_t db;
    MT_DEV T make(uint64_t occ, uint32_t rpos, uint32_t rst, uint32_t nk) const {
        const uint32_t rel = ((uint32_t)occ & 1u) ^ rst;
        const int64_t rp = rel ? (int64_t)(nk - rpos) : (int64_t)rpos;
        const int64_t diag = (int64_t)((occ >> 1) & 0xFFFFFFFFull) - rp;
        return ((occ >> 33) << 34) | ((uint64_t)rel << 33) | (uint64_t)(diag + DIAG_BIAS);
    }
    MT_DEV uint64_t grel(T h) const { return h >> 33; }
    MT_DEV uint32_t genome(T h) const { return (uint32_t)(h >> 34); }
    MT_DEV uint64_t wide(T h) const { return h; }
};

// One merge stage of a bitonic sort in registers (element r*32 + lane in v[r]), in its
// mirrored form: blocks of k keys whose halves are each ascending become ascending. Key i is
// first compared with its mirror i ^ (k - 1) in the block, then with i ^ j for j = k/4 .. 1;
// every compare keeps the smaller key at the lower index, so its direction depends only on the
// lane bit (or register slot) it exchanges across. Exchanges across lanes are shuffles.
template <int R, typename T>
MT_DEV void bitonic_stage(T (&v)[R], uint32_t k) {
    const uint32_t lane = lane_id();
    if (k <= 32) {
#pragma unroll
        for (int r = 0; r < R; r++) {
            const T o = __shfl_xor_sync(FULL, v[r], k - 1);
            v[r] = (lane & (k >> 1)) == 0 ? min(v[r], o) : max(v[r], o);
        }
    } else {
        const int rm = (int)(k >> 5) - 1;          // mirrored register slots: r ^ rm, lane ^ 31
#pragma unroll
        for (int r = 0; r < R; r++) {
            const int pr = r ^ rm;
            if (pr > r) {
                const T a = v[r], b = v[pr];
                const T ob = __shfl_xor_sync(FULL, b, 31), oa = __shfl_xor_sync(FULL, a, 31);
                v[r] = min(a, ob);
                v[pr] = max(b, oa);
            }
        }
    }
#pragma unroll
    for (uint32_t j = k >> 2; j > 0; j >>= 1) {
        if (j >= 32) {
#pragma unroll
            for (int r = 0; r < R; r++) {
                const int pr = r ^ (int)(j >> 5);
                if (pr > r) { const T a = v[r], b = v[pr]; v[r] = min(a, b); v[pr] = max(a, b); }
            }
        } else {
#pragma unroll
            for (int r = 0; r < R; r++) {
                const T o = __shfl_xor_sync(FULL, v[r], j);
                v[r] = (lane & j) == 0 ? min(v[r], o) : max(v[r], o);
            }
        }
    }
}

// Bitonic sort of 32*R keys held in registers, ascending: element r*32 + lane in v[r].
template <int R, typename T>
MT_DEV void bitonic_regs(T (&v)[R]) {
#pragma unroll
    for (uint32_t k = 2; k <= 32u * R; k <<= 1) bitonic_stage<R, T>(v, k);
}

template <int R, typename T>
MT_DEV void sort_regs(T *h, uint32_t H) {
    const uint32_t lane = lane_id();
    T v[R];
#pragma unroll
    for (int r = 0; r < R; r++) {
        const uint32_t i = (uint32_t)r * 32u + lane;
        v[r] = i < H ? h[i] : (T)~(T)0;
    }
    bitonic_regs<R, T>(v);
#pragma unroll
    for (int r = 0; r < R; r++) {
        const uint32_t i = (uint32_t)r * 32u + lane;
        if (i < H) h[i] = v[r];
    }
    __syncwarp();
}

// Mirrored bitonic sort of 64 keys in registers with key 2*lane + r in v[r], so that the
// compares at distance 1 stay in the lane and the others exchange with lane ^ (distance / 2).
template <typename T>
MT_DEV void bitonic_pairs64(T (&v)[2]) {
    const uint32_t lane = lane_id();
#pragma unroll
    for (uint32_t k = 2; k <= 64; k <<= 1) {
        if (k > 2) {   // mirror: key i with i ^ (k - 1), i.e. slot r ^ 1 of lane ^ ((k - 1) / 2)
            const uint32_t m = (k - 1) >> 1;
            const bool lo = (lane & (k >> 2)) == 0;
            const T o0 = __shfl_xor_sync(FULL, v[1], m), o1 = __shfl_xor_sync(FULL, v[0], m);
            v[0] = lo ? min(v[0], o0) : max(v[0], o0);
            v[1] = lo ? min(v[1], o1) : max(v[1], o1);
        }
#pragma unroll
        for (uint32_t j = (k == 2 ? 1u : k >> 2); j > 1; j >>= 1) {
            const bool lo = (lane & (j >> 1)) == 0;
#pragma unroll
            for (int r = 0; r < 2; r++) {
                const T o = __shfl_xor_sync(FULL, v[r], j >> 1);
                v[r] = lo ? min(v[r], o) : max(v[r], o);
            }
        }
        const T a = v[0], b = v[1];   // distance 1 (and the mirror of k = 2)
        v[0] = min(a, b);
        v[1] = max(a, b);
    }
}

// 33..128 keys: each 64-key half sorted in registers by one copy of the 64-key network, then
// one mirrored merge stage over all 128 (key 64q + 2*lane + r in v[2q + r]).
template <typename T>
MT_DEV void sort_regs128(T *h, uint32_t H) {
    const uint32_t lane = lane_id();
    const uint32_t halves = H > 64 ? 2u : 1u;
#pragma unroll 1
    for (uint32_t q = 0; q < halves; q++) {
        T v[2];
#pragma unroll
        for (int r = 0; r < 2; r++) {
            const uint32_t i = 64u * q + 2u * lane + (uint32_t)r;
            v[r] = i < H ? h[i] : (T)~(T)0;
        }
        bitonic_pairs64<T>(v);
#pragma unroll
        for (int r = 0; r < 2; r++) {
            const uint32_t i = 64u * q + 2u * lane + (uint32_t)r;
            if (i < H || halves == 2) h[i] = v[r];
        }
    }
    if (halves == 2) {
        __syncwarp();
        T v[4];
#pragma unroll
        for (int r = 0; r < 4; r++) v[r] = h[64u * (r >> 1) + 2u * lane + (uint32_t)(r & 1)];
        {   // mirror: key i of the first half with 127 - i (slot 3 - r of lane ^ 31)
            const T o3 = __shfl_xor_sync(FULL, v[3], 31), o2 = __shfl_xor_sync(FULL, v[2], 31);
            const T o1 = __shfl_xor_sync(FULL, v[1], 31), o0 = __shfl_xor_sync(FULL, v[0], 31);
            v[0] = min(v[0], o3);
            v[1] = min(v[1], o2);
            v[2] = max(v[2], o1);
            v[3] = max(v[3], o0);
        }
#pragma unroll
        for (uint32_t j = 32; j > 1; j >>= 1) {
            const bool lo = (lane & (j >> 1)) == 0;
#pragma unroll
            for (int r = 0; r < 4; r++) {
                const T o = __shfl_xor_sync(FULL, v[r], j >> 1);
                v[r] = lo ? min(v[r], o) : max(v[r], o);
            }
        }
#pragma unroll
        for (int r = 0; r < 4; r += 2) { const T a = v[r], b = v[r + 1]; v[r] = min(a, b); v[r + 1] = max(a, b); }
#pragma unroll
        for (int r = 0; r < 4; r++) {
            const uint32_t i = 64u * (r >> 1) + 2u * lane + (uint32_t)(r & 1);
            if (i < H) h[i] = v[r];
        }
    }
    __syncwarp();
}

// warp bitonic sort of a[0, P) in shared memory, P a power of two >= 2
template <typename T>
MT_DEV void warp_bitonic(T *a, uint32_t P) {
    const uint32_t lane = lane_id();
    for (uint32_t k = 2; k <= P; k <<= 1) {
        for (uint32_t j = k >> 1; j > 0; j >>= 1) {
            for (uint32_t i = lane; i < P / 2; i += 32) {
                uint32_t lo = ((i & ~(j - 1)) << 1) | (i & (j - 1));
                uint32_t hi = lo + j;
                bool up = (lo & k) == 0;
                T x = a[lo], y = a[hi];
                if ((x > y) == up) { a[lo] = y; a[hi] = x; }
            }
            __syncwarp();
        }
    }
}

// Up to 128 matches are sorted in registers; the rare larger sets (<= HCAP) in shared memory.
template <typename T>
MT_DEV void sort_hits(T *h, uint32_t H) {
    if (H <= 32) sort_regs<1, T>(h, H);
    else if (H <= 128) sort_regs128<T>(h, H);
    else {
        uint32_t P = 128;
        while (P < H) P <<= 1;
        for (uint32_t i = H + lane_id(); i < P; i += 32) h[i] = (T)~(T)0;
        __syncwarp();
        warp_bitonic<T>(h, P);
    }
}

// Top 32 bits of the k-mer key mix64(code) of a code below 2^56 (k <= 28), from the first
// multiply, the middle xor-shift and the high word of the second multiply (the last xor-shift
// changes only bit 0 of them). z >> 30 then fits in 32 bits, so the first xor-shift touches
// the low word only.
MT_DEV uint32_t mix64_hi(uint64_t z) {
    z = (z ^ (uint64_t)(uint32_t)(z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z ^= z >> 27;
    const uint32_t lo = (uint32_t)z, hi = (uint32_t)(z >> 32);
    return __umulhi(lo, 0x133111ebu) + lo * 0x94d049bbu + hi * 0x133111ebu;
}

// (w,k)-minimizers of one pass over the windows [t0, t0 + tw) of a read for w = 11, k <= 28
// (tw <= W11_TILE). Lane l computes the k-mers at local positions 5l .. 5l + 4 from one 32-base
// slice of the packed read (forward codes from the slice's 2-bit reversal, reverse-complement
// codes from its complement) and stores code | strand << 63 at code[local position]. A window
// of 11 k-mers starting at local 5l + a (a < 5) is the last 5 - a k-mers of lane l, all five
// of lane l + 1 and the first a + 1 of lane l + 2, so its minimum is min(suffix_l[a],
// block_{l+1}, prefix_{l+2}[a]) (van Herk / Gil-Werman with blocks of five). Minima are taken
// on 32-bit words (key bits 40..63) << 8 | local position, so one unsigned min orders by key
// and keeps the leftmost of equal words. The same minima with the position bits reversed find
// the rightmost k-mer of the smallest top bits; when the two differ, two k-mers of the window
// share them and the window is redone on full 64-bit keys. Appends the selected positions
// (absolute, each once) to mpos and returns their number; carry is the selection of the
// previous pass's last window (-1 before the first pass).
template <typename WS>
MT_DEV uint32_t minimizers_w11(WS &ws, uint32_t t0, uint32_t tw, uint32_t k, uint32_t canonical,
                               int32_t &carry) {
    const uint32_t lane = lane_id();
    const uint32_t b = 5u * lane;                 // first local position of this lane
    uint32_t v[5], u[5];                          // leftmost / rightmost words
    {
        // every lane computes its five k-mers without branching; positions at or past tw + 10
        // (past the pass's last k-mer) read zero or stale words (the slice's word index is
        // clamped to the read buffer), but no window of the pass reaches them: window
        // 5l + a < tw ends at 5l + a + 10 < tw + 10, and
        // its three parts (suffix of lane l, lane l + 1, prefix of lane l + 2) hold only its
        // own positions
        const uint64_t mask = (1ull << (2 * k)) - 1;
        const uint32_t p = min(t0 + b, 32u * (RDW - 2));
        const uint64_t x = get32(ws.rd, p);                       // bases t0+b.., first lowest
        const uint64_t nx = ~x;
        const uint64_t rv = rev2(x) >> (56 - 2 * k);              // forward code of k-mer 4 in bits 0..2k-1
#pragma unroll
        for (int i = 0; i < 5; i++) {
            const uint64_t rc = (nx >> (2 * i)) & mask;
            const uint64_t fwd = (rv >> (8 - 2 * i)) & mask;
            const bool r = canonical && rc < fwd;
            const uint64_t code = r ? rc : fwd;
            ws.u.t.code[b + i] = code | ((uint64_t)r << 63);
            v[i] = (mix64_hi(code) & 0xFFFFFF00u) | (b + i);
            u[i] = v[i] ^ 0xFFu;                                  // position bits reversed: 255 - (b + i)
        }
    }
    uint32_t sel[5];
    bool tie[5];
    {
        uint32_t pre[5], suf[5], qre[5], quf[5];
        pre[0] = v[0]; qre[0] = u[0];
#pragma unroll
        for (int i = 1; i < 5; i++) { pre[i] = min(pre[i - 1], v[i]); qre[i] = min(qre[i - 1], u[i]); }
        suf[4] = v[4]; quf[4] = u[4];
#pragma unroll
        for (int i = 3; i >= 0; i--) { suf[i] = min(v[i], suf[i + 1]); quf[i] = min(u[i], quf[i + 1]); }
        const uint32_t f1 = __shfl_down_sync(FULL, pre[4], 1), g1 = __shfl_down_sync(FULL, qre[4], 1);
#pragma unroll
        for (int a = 0; a < 5; a++) {
            const uint32_t p2 = __shfl_down_sync(FULL, pre[a], 2), q2 = __shfl_down_sync(FULL, qre[a], 2);
            const uint32_t m = min(min(suf[a], f1), p2), q = min(min(quf[a], g1), q2);
            sel[a] = t0 + (m & 0xFFu);
            tie[a] = b + a < tw && ((m ^ q) & 0xFFu) != 0xFFu;
        }
    }
    __syncwarp();                                 // codes of the pass are in shared memory
    uint32_t tied = 0;
#pragma unroll
    for (int a = 0; a < 5; a++) tied |= (uint32_t)tie[a] << a;
    if (__any_sync(FULL, tied != 0)) {
        while (tied) {                            // leftmost smallest full key of the window
            const uint32_t a = __ffs(tied) - 1;
            tied &= tied - 1;
            const uint32_t j = b + a;
            uint32_t best = j;
            uint64_t bk = mix64(ws.u.t.code[j] & CODE_MASK62);
#pragma unroll 1
            for (uint32_t t = j + 1; t < j + 11; t++) {
                const uint64_t kk = mix64(ws.u.t.code[t] & CODE_MASK62);
                if (kk < bk) { bk = kk; best = t; }
            }
#pragma unroll
            for (int q = 0; q < 5; q++) if ((uint32_t)q == a) sel[q] = t0 + best;
        }
    }
    // each selected position once: a window's selection is new when it differs from the
    // previous window's (selections never decrease along the read)
    int32_t prv = __shfl_up_sync(FULL, (int32_t)sel[4], 1);
    if (lane == 0) prv = carry;
    bool em[5];
    uint32_t ne = 0;
#pragma unroll
    for (int a = 0; a < 5; a++) {
        const bool ok = b + a < tw;
        em[a] = ok && (int32_t)sel[a] != prv;
        ne += em[a];
        if (ok) prv = (int32_t)sel[a];
    }
    const uint32_t incl = warp_incl_scan(ne);
    uint32_t o = incl - ne;
#pragma unroll
    for (int a = 0; a < 5; a++)
        if (em[a]) ws.u.t.mpos[o++] = (uint16_t)sel[a];
    // prv is now the selection of the lane's last window: the pass's last window's, for the next
    carry = __shfl_sync(FULL, prv, (tw - 1) / 5u);
    return __shfl_sync(FULL, incl, 31);
}

// COUNT: containment only (every occurrence of every minimizer counted per genome, no
// locations, no outputs per read); HPC: the reads' seeds are taken after homopolymer
// compression (an index built with MT_INDEX_HPC).
// Adds c seed hits of genome g into the CTA's 32-bit shared counter (or straight to the 64-bit
// global counter). CHECKED adds (the per-occurrence counting of containment and of overflowing
// reads, which max_occ alone does not bound) move the counter to the global one once it reaches
// 2^31; unchecked adds come from the location walk, at most HCAP a read, so a CTA's share of a
// launch (fewer than 2^32 / MT_MAX_TOPN reads over at least min(reads / 8, SMs) CTAs) adds under
// 2^28 a genome: the counter never wraps.
template <bool SMEM_HIST, bool CHECKED>
MT_DEV void add_hits(uint32_t *hist, unsigned long long *ghits, uint32_t g, uint32_t c) {
    if (SMEM_HIST) {
        if (CHECKED) {
            const uint32_t old = atomicAdd(&hist[g], c);
            if (old + c >= 0x80000000u) {
                const uint32_t v = atomicExch(&hist[g], 0u);
                if (v) atomicAdd(&ghits[g], (unsigned long long)v);
            }
        } else {
            atomicAdd(&hist[g], c);
        }
    } else {
        atomicAdd(&ghits[g], (unsigned long long)c);
    }
}

// Shared memory of one seeding CTA: 32-bit genome counters, then the warps' areas.
template <bool HK32, bool W11>
static size_t seed_smem_bytes(uint32_t hist_n) {
    using HitT = typename std::conditional<HK32, uint32_t, uint64_t>::type;
    return (((size_t)hist_n * 4 + 15) & ~(size_t)15) + SEED_WARPS * sizeof(WarpSmem<HitT, W11>);
}

// Resident CTAs per SM of a seeding kernel. The mapping kernel of the w = 11 path with 32-bit
// match keys fits five in shared memory, and 48 registers a thread; it then keeps its
// statistics and the batch description in shared memory, not in registers.
template <bool HK32, bool COUNT, bool W11>
struct SeedLean {
    static constexpr bool value = HK32 && W11 && !COUNT;
    static constexpr int ctas = value ? 5 : 4;
};

// W11: the index has w = 11 and k <= 28, and the minimizers come from the block path
// (minimizers_w11); otherwise the general window-minimum path runs.
template <bool SMEM_HIST, bool HK32, bool COUNT = false, bool HPC = false, bool MULTI = false, bool W11 = false>
__global__ void __launch_bounds__(SEED_THREADS, (SeedLean<HK32, COUNT, W11>::ctas)) k_seed(SeedArgs A) {
    static_assert(!MULTI || (COUNT && !HK32), "several indexes are only counted");
    static_assert(!(MULTI && W11), "the block path keeps no keys for several tables");
    using HitT = typename HitKey<HK32>::T;
    extern __shared__ __align__(16) unsigned char smraw[];
    using WS = WarpSmem<HitT, W11>;
    uint32_t *hist = reinterpret_cast<uint32_t *>(smraw);
    const uint32_t hist_n = SMEM_HIST ? (MULTI ? A.n_hist : A.ix.G) : 0;
    WS *wsall = reinterpret_cast<WS *>(smraw + ((hist_n * 4 + 15) & ~15u));
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
    WS &ws = wsall[warp];
    if (SMEM_HIST) {
        for (uint32_t g = threadIdx.x; g < hist_n; g += blockDim.x) hist[g] = 0;
        __syncthreads();
    }
    const uint32_t k = A.ix.k, w = A.ix.w, canonical = A.ix.canonical;
    HitKey<HK32> hf;
    hf.db = A.ix.hk_db;
    // statistics: minimizers, matches, list occurrences, stored locations (warp-uniform)
    constexpr bool LEAN = SeedLean<HK32, COUNT, W11>::value;
    unsigned long long st_mins = 0, st_hits = 0, st_ext = 0, st_stored = 0;
    if (LEAN && lane < 4) ws.stat[lane] = 0;
    __shared__ IoBlock s_io;
    IoBlock io_r;
    if (LEAN) {
        if (threadIdx.x == 0) s_io = *A.io;
        __syncthreads();
    } else {
        io_r = *A.io;
    }
    const IoBlock &io = LEAN ? s_io : io_r;
    const uint64_t total_warps = (uint64_t)gridDim.x * SEED_WARPS;
    const uint64_t r_end = umin64(A.r_end, io.n_reads);
    for (uint64_t r = A.r_begin + (uint64_t)blockIdx.x * SEED_WARPS + warp; r < r_end; r += total_warps) {
        const uint64_t start = io.roff[r], end = io.roff[r + 1];
        if (end < start || end > io.n_bases) {
            if (lane == 0) { atomicOr(&A.ctr->err, ERR_BAD_OFFSETS); if (!COUNT) A.qcnt[r] = 0; }
            continue;
        }
        const uint64_t n64 = end - start;
        if (n64 > io.max_len) {
            if (lane == 0) { atomicOr(&A.ctr->err, ERR_READ_TOO_LONG); if (!COUNT) A.qcnt[r] = 0; }
            continue;
        }
        uint32_t n = (uint32_t)n64;
        // packed read, also kept in rw for the approximation stage
        if (warp_pack(io.reads, io.n_bases, io.vec_ok, start, n, ws.rd,
                      COUNT ? nullptr : A.rw + seq_word(start, io.off0, r))) {
            if (lane == 0) { atomicOr(&A.ctr->err, ERR_BAD_BASE); if (!COUNT) A.qcnt[r] = 0; }
            continue;
        }
        if (HPC) n = warp_hpc(ws.rd, n);
        const uint32_t E = edit_threshold(n, A.e_abs, A.e_permille);
        if (n < k || n - k + 1 < w) {
            if (lane == 0 && !COUNT) A.qcnt[r] = 0;
            continue;
        }
        const uint32_t nwin = n - k - w + 2, nk = n - k;
        uint32_t H = 0;
        bool ovf = COUNT;   // counting only from the start
        if (lane == 0) ws.nmr = 0;
        int32_t carry = -1;
        constexpr bool w11 = W11;
        const uint32_t tile = w11 ? W11_TILE : TILE;
        for (uint32_t t0 = 0; t0 < nwin; t0 += tile) {
            const uint32_t tw = min(tile, nwin - t0);
            const uint32_t npos = tw + w - 1;
            uint32_t nm = 0;
            if constexpr (W11) {
                nm = minimizers_w11(ws, t0, tw, k, canonical, carry);
            } else {
            // codes and keys of the tile's k-mers
            for (uint32_t i = lane; i < npos; i += 32) {
                uint64_t fwd, rc, code;
                uint32_t st;
                kmer_codes(get32(ws.rd, t0 + i), k, fwd, rc);
                canon(fwd, rc, canonical, code, st);
                ws.u.t.key[i] = mix64(code);
                ws.u.t.code[i] = code | ((uint64_t)st << 63);
            }
            __syncwarp();
            // (w,k)-minimizers: leftmost smallest key of each window, each position once.
            // Lane l takes windows 4l..4l+3 of the tile; for w >= 4 the four windows share
            // the k-mers [4l+3, 4l+w-1], so that minimum is found once.
            {
                const uint64_t *key = ws.u.t.key;
                const uint32_t j0 = 4 * lane;
                int32_t sel[4] = {-1, -1, -1, -1};
                if (j0 < tw) {
                    if (w >= 4) {
                        uint32_t cp = j0 + 3;   // argmin of the shared part
                        uint64_t ck = key[cp];
                        for (uint32_t t = j0 + 4; t < j0 + w; t++) {
                            uint64_t kk = key[t];
                            if (kk < ck) { ck = kk; cp = t; }
                        }
                        // left parts [j0+a, j0+2] (a = 0..2), right parts [j0+w, j0+a+w-1] (a = 1..3)
                        uint64_t k0 = key[j0], k1 = key[j0 + 1], k2 = key[j0 + 2];
                        uint64_t r0 = key[j0 + w], r1 = key[j0 + w + 1], r2 = key[j0 + w + 2];
                        uint32_t lp2 = j0 + 2; uint64_t lk2 = k2;
                        uint32_t lp1 = (k1 <= lk2) ? j0 + 1 : lp2; uint64_t lk1 = (k1 <= lk2) ? k1 : lk2;
                        uint32_t lp0 = (k0 <= lk1) ? j0 : lp1; uint64_t lk0 = (k0 <= lk1) ? k0 : lk1;
                        uint32_t rp1 = j0 + w; uint64_t rk1 = r0;
                        uint32_t rp2 = (r1 < rk1) ? j0 + w + 1 : rp1; uint64_t rk2 = (r1 < rk1) ? r1 : rk1;
                        uint32_t rp3 = (r2 < rk2) ? j0 + w + 2 : rp2; uint64_t rk3 = (r2 < rk2) ? r2 : rk2;
                        // window a = left part, shared part, right part, in position order
                        const uint32_t b0 = (lk0 <= ck) ? lp0 : cp;
                        uint32_t b1 = (lk1 <= ck) ? lp1 : cp; const uint64_t bk1 = (lk1 <= ck) ? lk1 : ck;
                        b1 = (rk1 < bk1) ? rp1 : b1;
                        uint32_t b2 = (lk2 <= ck) ? lp2 : cp; const uint64_t bk2 = (lk2 <= ck) ? lk2 : ck;
                        b2 = (rk2 < bk2) ? rp2 : b2;
                        const uint32_t b3 = (rk3 < ck) ? rp3 : cp;
                        sel[0] = (int32_t)(t0 + b0);
                        if (j0 + 1 < tw) sel[1] = (int32_t)(t0 + b1);
                        if (j0 + 2 < tw) sel[2] = (int32_t)(t0 + b2);
                        if (j0 + 3 < tw) sel[3] = (int32_t)(t0 + b3);
                    } else {
#pragma unroll
                        for (int a = 0; a < 4; a++) {
                            const uint32_t j = j0 + a;
                            if (j < tw) {
                                uint32_t b = j;
                                uint64_t bk = key[j];
                                for (uint32_t t = 1; t < w; t++) {
                                    uint64_t kk = key[j + t];
                                    if (kk < bk) { bk = kk; b = j + t; }
                                }
                                sel[a] = (int32_t)(t0 + b);
                            }
                        }
                    }
                }
                int32_t prv = __shfl_up_sync(FULL, sel[3], 1);
                if (lane == 0) prv = carry;
                bool em[4];
                uint32_t ne = 0;
#pragma unroll
                for (int a = 0; a < 4; a++) {
                    em[a] = sel[a] >= 0 && sel[a] != prv;
                    ne += em[a];
                    if (sel[a] >= 0) prv = sel[a];
                }
                const uint32_t incl = warp_incl_scan(ne);
                uint32_t o = nm + incl - ne;
#pragma unroll
                for (int a = 0; a < 4; a++)
                    if (em[a]) ws.u.t.mpos[o++] = (uint16_t)sel[a];
                nm += __shfl_sync(FULL, incl, 31);
                // selection of the tile's last window, for the next tile
                const uint32_t last_lane = (tw - 1) / 4;
                int32_t lastsel = sel[0];
#pragma unroll
                for (int a = 1; a < 4; a++) if (((tw - 1) & 3) == (uint32_t)a) lastsel = sel[a];
                carry = __shfl_sync(FULL, lastsel, last_lane);
            }
            }
            __syncwarp();
            if (lane == 0) ws.nmr += nm;
            if (!LEAN) st_mins += nm;
            else if (lane == 0) ws.stat[0] += nm;
            if (MULTI) {
                // (minimizer, batch) pairs: the batches' key filters (small, in L2) are tested
                // MULTI_UNROLL pairs a lane at a time (their loads in flight together); the pairs that pass
                // (about one batch per minimizer) are queued in the idle match buffer and
                // probed one a lane, matches counted into the batch's genome counters.
                const uint32_t B = A.n_bv, np = nm * B;
                // the match buffer is idle when counting: the queue in its first 1 KB, the
                // tile's minimizer keys in minimizer order in its second
                uint32_t *queue = reinterpret_cast<uint32_t *>(ws.hits);
                uint64_t *mkey = reinterpret_cast<uint64_t *>(ws.hits) + HCAP / 2;
                static_assert(HCAP / 2 >= TILE && HCAP >= 32 * (MULTI_UNROLL + 1), "queue and keys fit");
                for (uint32_t m = lane; m < nm; m += 32) mkey[m] = ws.u.t.key[ws.u.t.mpos[m] - t0];
                __syncwarp();
                uint32_t nq = 0;
                for (uint32_t p0 = 0; p0 < np; p0 += 32 * MULTI_UNROLL) {
                    uint32_t pass = 0;
                    // branch-free, so the four filter loads can be in flight together
#pragma unroll
                    for (uint32_t u = 0; u < MULTI_UNROLL; u++) {
                        const uint32_t pq = min(p0 + u * 32 + lane, np - 1);
                        const uint32_t m = B == 1 ? pq : __umulhi(pq, A.div_magic), b = pq - m * B;
                        const uint64_t key = mkey[m];
                        const uint64_t fb = filter_bits(key);
                        const uint64_t v = __ldg(&A.bv[b].filter[filter_block(key, A.bv[b].filter_shift)]);
                        pass |= (uint32_t)((v & fb) == fb && p0 + u * 32 + lane < np) << u;
                    }
#pragma unroll
                    for (uint32_t u = 0; u < MULTI_UNROLL; u++) {
                        const unsigned bal = __ballot_sync(FULL, (pass >> u) & 1u);
                        if ((pass >> u) & 1u) queue[nq + __popc(bal & ((1u << lane) - 1u))] = p0 + u * 32 + lane;
                        nq += __popc(bal);
                    }
                    __syncwarp();
                    const bool last = p0 + 32 * MULTI_UNROLL >= np;
                    uint32_t done = 0;
                    for (; done < nq && (last || nq - done >= 32); done += 32) {
                        const uint32_t qi = done + lane;
                        uint32_t cnt = 0, ni = 0, base = 0;
                        uint64_t w1 = 0, w2 = 0, w3 = 0;
                        const uint64_t *occ = nullptr;
                        if (qi < nq) {
                            const uint32_t pq = queue[qi];
                            const uint32_t m = B == 1 ? pq : __umulhi(pq, A.div_magic), b = pq - m * B;
                            const BatchView bv = A.bv[b];
                            const uint32_t xi = ws.u.t.mpos[m] - t0;
                            const uint64_t want = (ws.u.t.code[xi] & CODE_MASK62) + 1;
                            uint64_t s = slot_of(ws.u.t.key[xi], bv.slot_shift);
                            for (uint64_t it = 0; it <= bv.slot_mask; it++) {
                                const ulonglong2 a = __ldg(&bv.table[2 * s]);
                                const ulonglong2 c2 = __ldg(&bv.table[2 * s + 1]);
                                if (a.x == 0) break;
                                if ((a.x & CODE_MASK62) == want) {
                                    ni = (uint32_t)(a.x >> 62);
                                    w1 = a.y; w2 = c2.x; w3 = c2.y;
                                    cnt = ni ? ni : (uint32_t)(a.y >> 40);
                                    break;
                                }
                                s = (s + 1) & bv.slot_mask;
                            }
                            if (cnt > A.max_occ) cnt = 0;
                            base = bv.base;
                            occ = bv.occ;
                        }
                        H += __shfl_sync(FULL, warp_incl_scan(cnt), 31);
                        {
                            const uint32_t ext = __reduce_add_sync(FULL, ni ? 0u : cnt);
                            if (!LEAN) st_ext += ext;
                            else if (lane == 0) ws.stat[2] += ext;
                        }
                        if (ni && cnt) {
#pragma unroll
                            for (uint32_t t = 0; t < 3; t++)
                                if (t < cnt) add_hits<SMEM_HIST, true>(hist, A.ghits, base + (uint32_t)((t == 0 ? w1 : (t == 1 ? w2 : w3)) >> 33), 1u);
                        }
                        unsigned ext = __ballot_sync(FULL, ni == 0 && cnt != 0);
                        while (ext) {
                            const int src = __ffs(ext) - 1;
                            ext &= ext - 1;
                            const uint32_t c = __shfl_sync(FULL, cnt, src);
                            const uint32_t bb = __shfl_sync(FULL, base, src);
                            const uint64_t off = __shfl_sync(FULL, w1 & OFF_MASK40, src);
                            const uint64_t *oc = (const uint64_t *)__shfl_sync(FULL, (unsigned long long)occ, src);
                            for (uint32_t q = lane; q < c; q += 32) add_hits<SMEM_HIST, true>(hist, A.ghits, bb + (uint32_t)(__ldg(&oc[off + q]) >> 33), 1u);
                        }
                    }
                    // keep the unprobed tail (fewer than 32) at the front of the queue
                    const uint32_t left = nq > done ? nq - done : 0;
                    const uint32_t keep_v = lane < left ? queue[done + lane] : 0u;
                    __syncwarp();
                    if (lane < left) queue[lane] = keep_v;
                    nq = left;
                    __syncwarp();
                }
                continue;
            }
            // Index lookups, one minimizer a lane, both halves of a slot loaded together; then
            // the round's matches are expanded across the warp.
            for (uint32_t m0 = 0; m0 < nm; m0 += 32) {
                const uint32_t m = m0 + lane;
                uint32_t cnt = 0, ni = 0, rpos = 0, rst = 0;
                uint64_t w1 = 0, w2 = 0, w3 = 0;
                if (m < nm) {
                    rpos = ws.u.t.mpos[m];
                    const uint32_t xi = rpos - t0;
                    const uint64_t cs = ws.u.t.code[xi];
                    uint64_t key;
                    if constexpr (W11) key = mix64(cs & CODE_MASK62);
                    else key = ws.u.t.key[xi];
                    rst = (uint32_t)(cs >> 63);
                    const uint64_t want = (cs & CODE_MASK62) + 1;
                    uint64_t s = slot_of(key, A.ix.slot_shift);
                    for (uint64_t it = 0; it <= A.ix.slot_mask; it++) {
                        const ulonglong2 a = __ldg(&A.ix.table[2 * s]);
                        const ulonglong2 b = __ldg(&A.ix.table[2 * s + 1]);
                        if (a.x == 0) break;
                        if ((a.x & CODE_MASK62) == want) {
                            ni = (uint32_t)(a.x >> 62);
                            w1 = a.y; w2 = b.x; w3 = b.y;
                            cnt = ni ? ni : (uint32_t)(a.y >> 40);
                            break;
                        }
                        s = (s + 1) & A.ix.slot_mask;
                    }
                    if (cnt > A.max_occ) cnt = 0;
                }
                {
                    const uint32_t ext = __reduce_add_sync(FULL, ni ? 0u : cnt);
                    if (!LEAN) st_ext += ext;
                    else if (lane == 0) ws.stat[2] += ext;
                }
                const uint32_t incl = warp_incl_scan(cnt);
                const uint32_t total = __shfl_sync(FULL, incl, 31);
                const uint32_t pre = incl - cnt;
                if (!ovf && H + total > HCAP) {
                    // switch to counting only: count what is buffered so far
                    for (uint32_t i = lane; i < H; i += 32) add_hits<SMEM_HIST, true>(hist, A.ghits, hf.genome(ws.hits[i]), 1u);
                    ovf = true;
                }
                if (!ovf) {
                    // stage the lookups with matches by rank, then expand: one match a lane a
                    // pass; a match's lookup is the last one starting at or before it
                    const unsigned nz = __ballot_sync(FULL, cnt != 0);
                    if (cnt) {
                        const uint32_t c = __popc(nz & ((1u << lane) - 1u));
                        ws.u.t.e_pre[c] = pre;
                        ws.u.t.e_meta[c] = rpos | (rst << 16) | ((ni ? 1u : 0u) << 17);
                        ws.u.t.e_w[3 * c] = ni ? w1 : (w1 & OFF_MASK40);
                        if (ni) { ws.u.t.e_w[3 * c + 1] = w2; ws.u.t.e_w[3 * c + 2] = w3; }
                    }
                    __syncwarp();
                    uint32_t before = 0;    // lookups starting before this pass
#pragma unroll 1
                    for (uint32_t q0 = 0; q0 < total; q0 += 32) {
                        const uint32_t bit = (cnt && pre >= q0 && pre < q0 + 32) ? (1u << (pre - q0)) : 0u;
                        const uint32_t M = __reduce_or_sync(FULL, bit);
                        const uint32_t q = q0 + lane;
                        if (q < total) {
                            const uint32_t c = before + __popc(M & (0xFFFFFFFFu >> (31 - lane))) - 1;
                            const uint32_t t = q - ws.u.t.e_pre[c];
                            const uint32_t meta = ws.u.t.e_meta[c];
                            const uint64_t occ = (meta >> 17) ? ws.u.t.e_w[3 * c + t] : __ldg(&A.ix.occ[ws.u.t.e_w[3 * c] + t]);
                            ws.hits[H + q] = hf.make(occ, meta & 0xFFFFu, (meta >> 16) & 1u, nk);
                        }
                        before += __popc(M);
                    }
                } else {
                    if (ni && cnt) {
#pragma unroll 1
                        for (uint32_t t = 0; t < 3; t++)
                            if (t < cnt) add_hits<SMEM_HIST, true>(hist, A.ghits, (uint32_t)((t == 0 ? w1 : (t == 1 ? w2 : w3)) >> 33), 1u);
                    }
                    unsigned ext = __ballot_sync(FULL, ni == 0 && cnt != 0);
                    while (ext) {
                        const int src = __ffs(ext) - 1;
                        ext &= ext - 1;
                        const uint32_t c = __shfl_sync(FULL, cnt, src);
                        const uint64_t off = __shfl_sync(FULL, w1 & OFF_MASK40, src);
                        for (uint32_t q = lane; q < c; q += 32) add_hits<SMEM_HIST, true>(hist, A.ghits, (uint32_t)(__ldg(&A.ix.occ[off + q]) >> 33), 1u);
                    }
                }
                __syncwarp();
                H += total;
            }
            __syncwarp();
        }
        if (!LEAN) st_hits += H;
        else if (lane == 0) ws.stat[1] += H;
        if (COUNT) continue;
        if (ovf) {
            if (lane == 0) {
                A.qcnt[r] = QOVF;
                unsigned long long slot = atomicAdd(reinterpret_cast<unsigned long long *>(&A.ctr->fb_count), 1ull);
                A.fb_list[slot] = (uint32_t)r;
            }
            continue;
        }
        if (H == 0) {
            if (lane == 0) A.qcnt[r] = 0;
            continue;
        }
        sort_hits<HitT>(ws.hits, H);
        // (genome, strand) groups of the sorted matches, in order
        uint32_t ng = 0;
        for (uint32_t i0 = 0; i0 < H; i0 += 32) {
            const uint32_t i = i0 + lane;
            const bool st = i < H && (i == 0 || hf.grel(ws.hits[i]) != hf.grel(ws.hits[i - 1]));
            const unsigned bal = __ballot_sync(FULL, st);
            if (st) ws.u.wk.gs[ng + __popc(bal & ((1u << lane) - 1u))] = (uint16_t)i;
            ng += __popc(bal);
        }
        if (lane == 0) { ws.u.wk.gs[ng] = (uint16_t)H; ws.u.wk.qcount = 0; }
        __syncwarp();
        // containment counts (one atomic per group) and greedy locations per group: a
        // location starting at match s ends before the first match with key >= key_s + E + 1
        for (uint32_t gi = lane; gi < ng; gi += 32) {
            uint32_t s = ws.u.wk.gs[gi];
            const uint32_t ge = ws.u.wk.gs[gi + 1];
            add_hits<SMEM_HIST, false>(hist, A.ghits, hf.genome(ws.hits[s]), ge - s);
            const HitT last = ws.hits[ge - 1];
            while (s < ge) {
                const HitT lim = (HitT)(ws.hits[s] + E + 1);
                // most groups hold one location: the group's last match is already below lim
                const uint32_t e = last < lim ? ge : lower_bound_t<HitT>(ws.hits, s + 1, ge, lim);
                if (e - s >= A.min_seeds) {
                    const uint32_t qi = atomicAdd(&ws.u.wk.qcount, 1u);
                    if constexpr (HK32) {
                        ws.u.wk.qr[qi] = ((uint64_t)(0xFFFFu - (e - s)) << 32) | ws.hits[s];
                    } else {
                        ws.u.wk.qk[qi] = ws.hits[s];
                        ws.u.wk.qn[qi] = (uint16_t)(e - s);
                    }
                }
                s = e;
            }
        }
        __syncwarp();
        const uint32_t Q = ws.u.wk.qcount;
        // rank the qualifying locations: seeds descending, then (genome, strand, diagonal)
        for (uint32_t qi = lane; qi < Q; qi += 32) {
            uint32_t seeds_i, rank = 0;
            HitT hk_i;
            if constexpr (HK32) {   // one compare of rank words (they are distinct)
                const uint64_t ri = ws.u.wk.qr[qi];
                for (uint32_t qj = 0; qj < Q; qj++) rank += ws.u.wk.qr[qj] < ri;
                seeds_i = 0xFFFFu - (uint32_t)(ri >> 32);
                hk_i = (HitT)ri;
            } else {
                seeds_i = ws.u.wk.qn[qi];
                hk_i = ws.u.wk.qk[qi];
                for (uint32_t qj = 0; qj < Q; qj++) {
                    const uint32_t seeds_j = ws.u.wk.qn[qj];
                    const HitT hk_j = ws.u.wk.qk[qj];
                    rank += (seeds_j > seeds_i) || (seeds_j == seeds_i && hk_j < hk_i);
                }
            }
            if (rank < CSTORE) {
                Cluster c;
                c.hkey = hf.wide(hk_i); c.seeds = seeds_i; c.pad = ws.nmr;
                A.clus[r * CSTORE + rank] = c;
            }
        }
        if (lane == 0) {
            A.qcnt[r] = Q;
            if (!LEAN) st_stored += min(Q, CSTORE);
            else ws.stat[3] += min(Q, CSTORE);
        }
        __syncwarp();
    }
    __syncwarp();
    if (lane == 0) {
        atomicAdd(&A.ctr->stat[ST_MINS], LEAN ? ws.stat[0] : st_mins);
        atomicAdd(&A.ctr->stat[ST_HITS], LEAN ? ws.stat[1] : st_hits);
        atomicAdd(&A.ctr->stat[ST_EXT], LEAN ? ws.stat[2] : st_ext);
        atomicAdd(&A.ctr->stat[ST_STORED], LEAN ? ws.stat[3] : st_stored);
    }
    if (SMEM_HIST) {
        __syncthreads();
        for (uint32_t g = threadIdx.x; g < hist_n; g += blockDim.x)
            if (hist[g]) atomicAdd(&A.ghits[g], (unsigned long long)hist[g]);
    }
}

// ---- containment mask ----------------------------------------------------------------------
__global__ void k_mask(const unsigned long long *hits, uint32_t G, uint32_t num, uint32_t den, uint8_t *keep) {
    __shared__ unsigned long long smax[32];
    unsigned long long m = 0;
    for (uint32_t g = threadIdx.x; g < G; g += blockDim.x) m = max(m, hits[g]);
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(FULL, m, o));
    if ((threadIdx.x & 31) == 0) smax[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        m = threadIdx.x < (blockDim.x + 31) / 32 ? smax[threadIdx.x] : 0;
        for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(FULL, m, o));
        if (threadIdx.x == 0) smax[0] = m;
    }
    __syncthreads();
    const unsigned long long mx = smax[0];
    for (uint32_t g = threadIdx.x; g < G; g += blockDim.x) {
        unsigned long long h = hits[g];
        // compare h * den > mx * num exactly in 128 bits
        unsigned long long lo1 = h * den, hi1 = __umul64hi(h, den);
        unsigned long long lo2 = mx * num, hi2 = __umul64hi(mx, num);
        bool gt = (hi1 > hi2) || (hi1 == hi2 && lo1 > lo2);
        keep[g] = (mx > 0 && gt) ? 1 : 0;
    }
}

// ---- candidate selection ----------------------------------------------------------------------
// A tile's candidates enter the compact list ordered by missing seeds: the read's minimizers
// (kept by the seeding kernel in the location record's spare word) minus the location's seeds,
// fewest first, a counting sort over 64 bins in shared memory. A location holding nearly all of
// its read's minimizers is usually a near-exact match whose approximation ends in a step or
// two, one missing many a divergent genome walked to E + 1 obstacles, so a warp of the
// approximation kernel that takes consecutive candidates walks them for similar numbers of
// steps, for reads of any length. The order of the list changes no result (each distance goes
// to its candidate's slot).
static constexpr int SELECT_CTAS = 6;   // resident k_select CTAs an SM (40 registers)

__global__ void __launch_bounds__(256, SELECT_CTAS)
k_select(const IoBlock *io, const uint32_t *qcnt, const Cluster *clus, const uint8_t *keep, uint32_t top_n,
         Cluster *cand, uint8_t *nloc_ws, uint32_t *cl, uint32_t *fb_list, Counters *ctr) {
    constexpr uint32_t BINS = 64;
    __shared__ uint32_t s_bin[BINS];
    __shared__ unsigned long long s_base;
    const uint64_t n_reads = io->n_reads;
    for (uint64_t r0 = (uint64_t)blockIdx.x * blockDim.x; r0 < n_reads; r0 += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t r = r0 + threadIdx.x;
        uint32_t taken = 0;
        uint64_t bins = 0;       // bin of candidate t in bits 6t .. 6t+5
        bool fb = false;
        if (threadIdx.x < BINS) s_bin[threadIdx.x] = 0;
        __syncthreads();
        if (r < n_reads) {
            uint32_t q = qcnt[r];
            if (q == QOVF) {
                fb = false;   // queued by the seeding pass
                nloc_ws[r] = 0;
            } else {
                const uint32_t lim = min(q, CSTORE);
                // the first four locations and their genomes' verdicts are loaded together
                Cluster c4[4];
                bool k4[4];
#pragma unroll
                for (uint32_t i = 0; i < 4; i++) {
                    c4[i].hkey = 0; c4[i].seeds = 0; c4[i].pad = 0;
                    if (i < lim) c4[i] = clus[r * CSTORE + i];
                }
#pragma unroll
                for (uint32_t i = 0; i < 4; i++) k4[i] = i < lim && keep[hk_genome(c4[i].hkey)];
#pragma unroll
                for (uint32_t i = 0; i < 4; i++) {
                    if (k4[i] && taken < top_n) {
                        const uint32_t bin = min(c4[i].pad > c4[i].seeds ? c4[i].pad - c4[i].seeds : 0u, BINS - 1);
                        bins |= (uint64_t)bin << (6 * taken);
                        cand[r * top_n + taken++] = c4[i];
                    }
                }
                for (uint32_t i = 4; i < lim && taken < top_n; i++) {
                    Cluster c = clus[r * CSTORE + i];
                    if (keep[hk_genome(c.hkey)]) {
                        const uint32_t bin = min(c.pad > c.seeds ? c.pad - c.seeds : 0u, BINS - 1);
                        bins |= (uint64_t)bin << (6 * taken);
                        cand[r * top_n + taken++] = c;
                    }
                }
                if (taken < top_n && q > CSTORE) { fb = true; taken = 0; }
                nloc_ws[r] = (uint8_t)taken;
            }
        }
        if (fb) {
            unsigned long long slot = atomicAdd(reinterpret_cast<unsigned long long *>(&ctr->fb_count), 1ull);
            fb_list[slot] = (uint32_t)r;
        }
        for (uint32_t t = 0; t < taken; t++) atomicAdd(&s_bin[(bins >> (6 * t)) & (BINS - 1)], 1u);
        __syncthreads();
        if (threadIdx.x < 32) {   // bin starts within the tile, and the tile's place in the list
            const uint32_t lane = threadIdx.x;
            const uint32_t c0 = s_bin[2 * lane], c1 = s_bin[2 * lane + 1];
            const uint32_t incl = warp_incl_scan(c0 + c1);
            const uint32_t run = __shfl_sync(FULL, incl, 31);
            s_bin[2 * lane] = incl - c0 - c1;
            s_bin[2 * lane + 1] = incl - c1;
            if (lane == 0)
                s_base = run ? atomicAdd(reinterpret_cast<unsigned long long *>(&ctr->cl_count), (unsigned long long)run) : 0;
        }
        __syncthreads();
        const unsigned long long base = s_base;
        for (uint32_t t = 0; t < taken; t++) {
            const uint32_t pos = atomicAdd(&s_bin[(bins >> (6 * t)) & (BINS - 1)], 1u);
            cl[base + pos] = (uint32_t)(r * top_n + t);
        }
        __syncthreads();   // s_bin and s_base are reused by the next tile
    }
}

// ---- exact slow path -------------------------------------------------------------------------------
struct FbArgs {
    IndexView ix;
    const uint64_t *rw;
    const IoBlock *io;
    uint32_t e_abs, e_permille, min_seeds, max_occ, top_n;
    const uint8_t *keep;
    const uint32_t *fb_list;
    Cluster *cand;
    uint8_t *nloc_ws;
    uint32_t *cl;
    Counters *ctr;
    uint64_t *scratch;     // FB_CTAS * cap hit keys, then FB_CTAS * cap u32 next pointers
    uint64_t cap;          // power of two
};

MT_DEV void read_kmer(const uint64_t *rd, uint32_t p, uint32_t k, uint32_t canonical, uint64_t &code,
                      uint32_t &st, uint64_t &key) {
    uint64_t fwd, rc;
    kmer_codes(get32(rd, p), k, fwd, rc);
    canon(fwd, rc, canonical, code, st);
    key = mix64(code);
}

MT_DEV uint32_t window_sel(const uint64_t *rd, uint32_t j, uint32_t k, uint32_t w, uint32_t canonical) {
    uint64_t c, kk, bk;
    uint32_t st, b = j;
    read_kmer(rd, j, k, canonical, c, st, bk);
    for (uint32_t t = j + 1; t < j + w; t++) {
        read_kmer(rd, t, k, canonical, c, st, kk);
        if (kk < bk) { bk = kk; b = t; }
    }
    return b;
}

__global__ void __launch_bounds__(FB_THREADS) k_fallback(FbArgs A) {
    __shared__ unsigned long long s_H;
    __shared__ uint32_t s_best_start[MT_MAX_TOPN], s_best_seeds[MT_MAX_TOPN];
    __shared__ uint32_t s_nbest;
    uint64_t *hits = A.scratch + (uint64_t)blockIdx.x * A.cap;
    uint32_t *nxt = reinterpret_cast<uint32_t *>(A.scratch + (uint64_t)FB_CTAS * A.cap) + (uint64_t)blockIdx.x * A.cap;
    const uint32_t k = A.ix.k, w = A.ix.w, canonical = A.ix.canonical;
    for (uint64_t fi = blockIdx.x; fi < A.ctr->fb_count; fi += gridDim.x) {
        const uint32_t r = A.fb_list[fi];
        const uint64_t start = A.io->roff[r];
        const uint32_t n = (uint32_t)(A.io->roff[r + 1] - start);
        const uint32_t E = edit_threshold(n, A.e_abs, A.e_permille);
        const uint64_t *rd = A.rw + seq_word(start, A.io->off0, r);
        if (threadIdx.x == 0) s_H = 0;
        __syncthreads();
        const uint32_t nwin = n - k - w + 2;   // the read reached here, so it has windows
        for (uint32_t j = threadIdx.x; j < nwin; j += blockDim.x) {
            uint32_t sel = window_sel(rd, j, k, w, canonical);
            if (j > 0 && window_sel(rd, j - 1, k, w, canonical) == sel) continue;
            uint64_t code, key;
            uint32_t st;
            read_kmer(rd, sel, k, canonical, code, st, key);
            Lookup L = probe(A.ix, code, key, &A.ctr->err);
            if (L.cnt > A.max_occ) continue;
            for (uint32_t t = 0; t < L.cnt; t++) {
                uint64_t o = occ_at(A.ix, L, t);
                if (!A.keep[o >> 33]) continue;
                unsigned long long pos = atomicAdd(&s_H, 1ull);
                if (pos < A.cap) hits[pos] = hit_key(o, sel, st, n, k);
                else atomicOr(&A.ctr->err, ERR_SCRATCH);
            }
        }
        __syncthreads();
        const uint32_t H = (uint32_t)umin64(s_H, A.cap);
        uint32_t P = 2;
        while (P < H) P <<= 1;
        for (uint32_t i = H + threadIdx.x; i < P; i += blockDim.x) hits[i] = ~0ull;
        __syncthreads();
        for (uint32_t kk = 2; kk <= P; kk <<= 1) {
            for (uint32_t j = kk >> 1; j > 0; j >>= 1) {
                for (uint32_t i = threadIdx.x; i < P / 2; i += blockDim.x) {
                    uint32_t lo = ((i & ~(j - 1)) << 1) | (i & (j - 1));
                    uint32_t hi = lo + j;
                    bool up = (lo & kk) == 0;
                    uint64_t x = hits[lo], y = hits[hi];
                    if ((x > y) == up) { hits[lo] = y; hits[hi] = x; }
                }
                __syncthreads();
            }
        }
        for (uint32_t i = threadIdx.x; i < H; i += blockDim.x) {
            uint64_t key = hits[i] + E + 1;
            uint32_t lo = i + 1, hi = H;
            while (lo < hi) {
                uint32_t mid = (lo + hi) >> 1;
                if (hits[mid] < key) lo = mid + 1; else hi = mid;
            }
            nxt[i] = lo;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            // walk the locations; keep the top_n by (seeds desc, key asc) in a small list
            uint32_t nb = 0;
            uint32_t s = 0;
            while (s < H) {
                uint32_t e = nxt[s];
                uint32_t seeds = e - s;
                if (seeds >= A.min_seeds) {
                    uint32_t pos = nb;
                    while (pos > 0) {
                        uint32_t ps = s_best_seeds[pos - 1];
                        bool before = ps > seeds || (ps == seeds && hits[s_best_start[pos - 1]] < hits[s]);
                        if (before) break;
                        pos--;
                    }
                    if (pos < A.top_n) {
                        uint32_t last = min(nb, A.top_n - 1);
                        for (uint32_t q = last; q > pos; q--) {
                            s_best_seeds[q] = s_best_seeds[q - 1];
                            s_best_start[q] = s_best_start[q - 1];
                        }
                        s_best_seeds[pos] = seeds;
                        s_best_start[pos] = s;
                        if (nb < A.top_n) nb++;
                    }
                }
                s = e;
            }
            s_nbest = nb;
            unsigned long long base = nb ? atomicAdd(reinterpret_cast<unsigned long long *>(&A.ctr->cl_count), (unsigned long long)nb) : 0;
            for (uint32_t q = 0; q < nb; q++) {
                Cluster c;
                c.hkey = hits[s_best_start[q]];
                c.seeds = s_best_seeds[q];
                c.pad = 0;
                A.cand[(uint64_t)r * A.top_n + q] = c;
                A.cl[base + q] = r * A.top_n + q;
            }
            A.nloc_ws[r] = (uint8_t)nb;
            atomicAdd(&A.ctr->stat[ST_FB], 1ull);
        }
        __syncthreads();
    }
}

// ---- per-read decision -------------------------------------------------------------------------------
struct DecideArgs {
    const IoBlock *io;
    uint32_t e_abs, e_permille, top_n;
    const uint8_t *nloc_ws;
    const Cluster *cand;
    const uint8_t *dist;
    unsigned long long *U;
    int32_t *multi_set;
    uint32_t *multi_list;
    Counters *ctr;
    uint32_t G;
    uint32_t hist;   // 1: unique counts are gathered per block in shared memory first
};

// A block takes tiles of DECIDE_THREADS consecutive reads: their candidate records, distances
// and location counts come into shared memory with contiguous loads, a thread decides its read
// from there, and the location records go out as contiguous 8-byte words.
static constexpr int DECIDE_THREADS = 256;

// TNMAX: the largest top_n of the launch (the per-read arrays below are sized by it).
template <uint32_t TNMAX>
__global__ void __launch_bounds__(DECIDE_THREADS, (TNMAX <= 3 ? 6 : 3)) k_decide(DecideArgs A) {
    extern __shared__ __align__(16) unsigned char dsm[];
    const uint32_t tn = A.top_n;
    // unique counts of the block (G counters), flushed once at the end
    unsigned long long *s_U = reinterpret_cast<unsigned long long *>(dsm);
    const uint32_t hist_n = A.hist ? A.G : 0;
    for (uint32_t g = threadIdx.x; g < hist_n; g += DECIDE_THREADS) s_U[g] = 0;
    unsigned long long *U = A.hist ? s_U : A.U;
    Cluster *s_cand = reinterpret_cast<Cluster *>(dsm + (((size_t)hist_n * 8 + 15) & ~(size_t)15));   // DECIDE_THREADS * tn
    uint64_t *s_locs = reinterpret_cast<uint64_t *>(s_cand + DECIDE_THREADS * tn);  // 3 words a location
    uint8_t *s_dist = reinterpret_cast<uint8_t *>(s_locs + 3 * DECIDE_THREADS * tn);
    uint8_t *s_nloc = s_dist + DECIDE_THREADS * tn;
    const uint32_t lane = threadIdx.x & 31u;
    unsigned long long acc = 0, mul = 0, cand = 0;
    const IoBlock io = *A.io;
    for (uint64_t r0 = (uint64_t)blockIdx.x * DECIDE_THREADS; r0 < io.n_reads; r0 += (uint64_t)gridDim.x * DECIDE_THREADS) {
        const uint32_t nr = (uint32_t)umin64(DECIDE_THREADS, io.n_reads - r0);
        __syncthreads();   // the previous tile's locations are out
        for (uint32_t i = threadIdx.x; i < nr * tn; i += DECIDE_THREADS) {
            s_cand[i] = A.cand[r0 * tn + i];
            s_dist[i] = A.dist[r0 * tn + i];
        }
        if (threadIdx.x < nr) s_nloc[threadIdx.x] = A.nloc_ws[r0 + threadIdx.x];
        __syncthreads();
        const uint64_t r = r0 + threadIdx.x;
        int32_t uniq = -1;
        bool is_multi = false;
        if (threadIdx.x < nr) {
            const uint32_t n = (uint32_t)(io.roff[r + 1] - io.roff[r]);
            const uint32_t E = edit_threshold(n, A.e_abs, A.e_permille);
            const uint32_t nl = s_nloc[threadIdx.x];
            cand += nl;
            // every loop below runs over the at most TNMAX slots with static indices
            uint32_t d[TNMAX];
            Cluster cl[TNMAX];
            uint32_t best = E + 1;
#pragma unroll
            for (uint32_t t = 0; t < TNMAX; t++) {
                d[t] = 0xFFu;
                cl[t].hkey = 0; cl[t].seeds = 0; cl[t].pad = 0;
                if (t < nl) {
                    d[t] = s_dist[threadIdx.x * tn + t];
                    cl[t] = s_cand[threadIdx.x * tn + t];
                    if (d[t] <= E && d[t] < best) best = d[t];
                }
            }
            int32_t tax = -1;
            int32_t S[TNMAX];
            uint32_t ns = 0;
#pragma unroll
            for (uint32_t t = 0; t < TNMAX; t++) {
                S[t] = -1;
                if (t < nl && best <= E && d[t] == best) {
                    const int32_t g = (int32_t)hk_genome(cl[t].hkey);
                    if (tax < 0) tax = g;
                    bool seen = false;
#pragma unroll
                    for (uint32_t q = 0; q < t; q++) seen |= (S[q] == g);
                    if (!seen) { S[t] = g; ns++; }
                }
            }
#pragma unroll
            for (uint32_t t = 0; t < TNMAX; t++) {
                if (t < tn && io.locs) {
                    mt_loc L;
                    memset(&L, 0, sizeof(L));
                    L.genome = -1;
                    if (t < nl) {
                        L.wstart = hk_diag(cl[t].hkey) - (int64_t)E;
                        L.genome = (int32_t)hk_genome(cl[t].hkey);
                        L.seeds = cl[t].seeds;
                        L.strand = (uint8_t)hk_rel(cl[t].hkey);
                        L.dist = (uint8_t)d[t];
                    }
                    memcpy(&s_locs[3 * (threadIdx.x * tn + t)], &L, sizeof(L));
                }
            }
            io.taxon[r] = tax;
            if (io.nloc) io.nloc[r] = (uint8_t)nl;
            if (ns == 1) uniq = tax;
            if (ns >= 2) {
                is_multi = true;
                // the distinct genomes at the best distance, in rank order, then -1
                uint32_t o = 0;
#pragma unroll
                for (uint32_t t = 0; t < TNMAX; t++)
                    if (S[t] >= 0) { A.multi_set[r * tn + o] = S[t]; o++; }
#pragma unroll
                for (uint32_t t = 0; t < TNMAX; t++)
                    if (t >= o && t < tn) A.multi_set[r * tn + t] = -1;
            }
            acc += (best <= E);
            mul += is_multi;
        }
        // unique counts, aggregated over lanes hitting the same genome
        unsigned act = __ballot_sync(FULL, uniq >= 0);
        if (uniq >= 0) {
            unsigned peers = __match_any_sync(act, uniq);
            if (lane == (uint32_t)(__ffs(peers) - 1)) atomicAdd(&U[uniq], (unsigned long long)__popc(peers));
        }
        unsigned mb = __ballot_sync(FULL, is_multi);
        unsigned long long base = 0;
        if (lane == 0 && mb) base = atomicAdd(reinterpret_cast<unsigned long long *>(&A.ctr->multi_count), (unsigned long long)__popc(mb));
        base = __shfl_sync(FULL, base, 0);
        if (is_multi) A.multi_list[base + __popc(mb & ((1u << lane) - 1u))] = (uint32_t)r;
        if (io.locs) {
            __syncthreads();
            uint64_t *dst = reinterpret_cast<uint64_t *>(io.locs + r0 * tn);
            for (uint32_t i = threadIdx.x; i < 3 * nr * tn; i += DECIDE_THREADS) dst[i] = s_locs[i];
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        acc += __shfl_xor_sync(FULL, acc, o);
        mul += __shfl_xor_sync(FULL, mul, o);
        cand += __shfl_xor_sync(FULL, cand, o);
    }
    if (lane == 0) {
        atomicAdd(&A.ctr->stat[ST_ACC], acc);
        atomicAdd(&A.ctr->stat[ST_MULTI], mul);
        atomicAdd(&A.ctr->stat[ST_CAND], cand);
    }
    if (A.hist) {
        __syncthreads();
        for (uint32_t g = threadIdx.x; g < hist_n; g += DECIDE_THREADS)
            if (s_U[g]) atomicAdd(&A.U[g], s_U[g]);
    }
}

// ---- location lists of several genome shards: merged by rank, then decided --------------------
struct MergeArgs {
    const mt_loc *lists;      // list q of read r: lists[(q * n_reads + r) * top_n ...], rank order, genome -1 ends it
    const uint64_t *roff;
    uint64_t n_reads;
    uint32_t R, top_n, e_abs, e_permille, G, hist;
    int32_t *taxon;
    uint8_t *nloc;
    mt_loc *locs;
    unsigned long long *U;
    int32_t *multi_set;
    uint32_t *multi_list;
    Counters *ctr;
};

// rank order of locations: seeds descending, then genome, strand, window start ascending
MT_DEV bool loc_before(const mt_loc &a, const mt_loc &b) {
    if (a.seeds != b.seeds) return a.seeds > b.seeds;
    if (a.genome != b.genome) return a.genome < b.genome;
    if (a.strand != b.strand) return a.strand < b.strand;
    return a.wstart < b.wstart;
}

// Thread per read: the t-th merged location is the first in rank order after the (t-1)-th
// among every shard's list (the shards' genomes are disjoint, so no two locations tie); the
// first top_n are decided like a single index's (k_decide).
__global__ void __launch_bounds__(256) k_merge_decide(MergeArgs A) {
    extern __shared__ unsigned long long s_mU[];
    const uint32_t hist_n = A.hist ? A.G : 0;
    for (uint32_t g = threadIdx.x; g < hist_n; g += blockDim.x) s_mU[g] = 0;
    __syncthreads();
    unsigned long long *U = A.hist ? s_mU : A.U;
    const uint32_t lane = threadIdx.x & 31u, tn = A.top_n;
    for (uint64_t r0 = (uint64_t)blockIdx.x * blockDim.x; r0 < A.n_reads; r0 += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t r = r0 + threadIdx.x;
        int32_t uniq = -1;
        bool is_multi = false;
        if (r < A.n_reads) {
            const uint32_t E = edit_threshold((uint32_t)(A.roff[r + 1] - A.roff[r]), A.e_abs, A.e_permille);
            uint32_t d[MT_MAX_TOPN];
            int32_t gg[MT_MAX_TOPN];
            uint32_t nl = 0;
            mt_loc prev;
            memset(&prev, 0, sizeof(prev));
            for (uint32_t t = 0; t < tn; t++) {
                bool found = false;
                mt_loc best;
                memset(&best, 0, sizeof(best));
                for (uint32_t q = 0; q < A.R; q++) {
                    const mt_loc *L = A.lists + (q * A.n_reads + r) * tn;
                    for (uint32_t u = 0; u < tn; u++) {
                        const mt_loc c = L[u];
                        if (c.genome < 0) break;
                        if (t > 0 && !loc_before(prev, c)) continue;
                        if (!found || loc_before(c, best)) { best = c; found = true; }
                    }
                }
                if (!found) break;
                A.locs[r * tn + t] = best;
                prev = best;
                nl++;
            }
#pragma unroll
            for (uint32_t t = 0; t < MT_MAX_TOPN; t++) {
                d[t] = 0xFFu; gg[t] = -1;
                if (t < nl) { d[t] = A.locs[r * tn + t].dist; gg[t] = A.locs[r * tn + t].genome; }
            }
            for (uint32_t t = nl; t < tn; t++) {
                mt_loc L;
                memset(&L, 0, sizeof(L));
                L.genome = -1;
                A.locs[r * tn + t] = L;
            }
            uint32_t best_d = E + 1;
#pragma unroll
            for (uint32_t t = 0; t < MT_MAX_TOPN; t++)
                if (t < nl && d[t] <= E && d[t] < best_d) best_d = d[t];
            int32_t tax = -1;
            int32_t S[MT_MAX_TOPN];
            uint32_t ns = 0;
#pragma unroll
            for (uint32_t t = 0; t < MT_MAX_TOPN; t++) {
                S[t] = -1;
                if (t < nl && best_d <= E && d[t] == best_d) {
                    if (tax < 0) tax = gg[t];
                    bool seen = false;
#pragma unroll
                    for (uint32_t q = 0; q < t; q++) seen |= (S[q] == gg[t]);
                    if (!seen) { S[t] = gg[t]; ns++; }
                }
            }
            A.taxon[r] = tax;
            A.nloc[r] = (uint8_t)nl;
            if (ns == 1) uniq = tax;
            if (ns >= 2) {
                is_multi = true;
                uint32_t o = 0;
#pragma unroll
                for (uint32_t t = 0; t < MT_MAX_TOPN; t++)
                    if (S[t] >= 0) { A.multi_set[r * tn + o] = S[t]; o++; }
                for (uint32_t t = o; t < tn; t++) A.multi_set[r * tn + t] = -1;
            }
        }
        const unsigned act = __ballot_sync(FULL, uniq >= 0);
        if (uniq >= 0) {
            const unsigned peers = __match_any_sync(act, uniq);
            if (lane == (uint32_t)(__ffs(peers) - 1)) atomicAdd(&U[uniq], (unsigned long long)__popc(peers));
        }
        const unsigned mb = __ballot_sync(FULL, is_multi);
        unsigned long long base = 0;
        if (lane == 0 && mb) base = atomicAdd(reinterpret_cast<unsigned long long *>(&A.ctr->multi_count), (unsigned long long)__popc(mb));
        base = __shfl_sync(FULL, base, 0);
        if (is_multi) A.multi_list[base + __popc(mb & ((1u << lane) - 1u))] = (uint32_t)r;
    }
    if (A.hist) {
        __syncthreads();
        for (uint32_t g = threadIdx.x; g < hist_n; g += blockDim.x)
            if (s_mU[g]) atomicAdd(&A.U[g], s_mU[g]);
    }
}

// multi-mapped reads: split by the genomes' unique counts (equally when they have none)
__global__ void k_multi(const uint32_t *multi_list, const Counters *ctr, const int32_t *multi_set, uint32_t top_n,
                        const unsigned long long *U, double *M) {
    const uint64_t cnt = ctr->multi_count;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t r = multi_list[i];
        const int32_t *S = multi_set + (uint64_t)r * top_n;
        uint32_t ns = 0;
        unsigned long long tot = 0;
        while (ns < top_n && S[ns] >= 0) { tot += U[S[ns]]; ns++; }
        for (uint32_t q = 0; q < ns; q++)
            atomicAdd(&M[S[q]], tot ? (double)U[S[q]] / (double)tot : 1.0 / (double)ns);
    }
}

MT_DEV double block_sum(double v, double *sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0;
    if (threadIdx.x == 0) {
        for (uint32_t i = 0; i < (blockDim.x + 31) / 32; i++) t += sh[i];
        sh[32] = t;
    }
    __syncthreads();
    return sh[32];
}

// relative abundances: a = (U + M) / sum; entries below the cutoff dropped; renormalised.
// One block; per-thread partial sums in a fixed order, so the result is deterministic for
// a given U and M.
__global__ void k_abund(uint32_t G, const unsigned long long *U, const double *M, double cutoff, double *out) {
    __shared__ double sh[33];
    double part = 0;
    for (uint32_t g = threadIdx.x; g < G; g += blockDim.x) part += (double)U[g] + M[g];
    double sum = block_sum(part, sh);
    double part2 = 0;
    for (uint32_t g = threadIdx.x; g < G; g += blockDim.x) {
        double a = sum > 0 ? ((double)U[g] + M[g]) / sum : 0.0;
        if (a < cutoff) a = 0.0;
        out[g] = a;
        part2 += a;
    }
    double kept = block_sum(part2, sh);
    if (kept > 0)
        for (uint32_t g = threadIdx.x; g < G; g += blockDim.x) out[g] /= kept;
}

// longest read and offset sanity for device-resident inputs
__global__ void k_maxlen(const uint64_t *roff, uint64_t n_reads, uint64_t n_bases, Counters *ctr) {
    unsigned int mx = 0;
    bool bad = false;
    for (uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n_reads; r += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t a = roff[r], b = roff[r + 1];
        if (b < a || b > n_bases) { bad = true; continue; }
        uint64_t n = b - a;
        mx = max(mx, (unsigned int)umin64(n, 0xFFFFFFFFull));
    }
    mx = __reduce_max_sync(FULL, mx);   // one atomic a warp
    bad = __any_sync(FULL, bad);
    if ((threadIdx.x & 31u) == 0) {
        atomicMax(&ctr->maxn, mx);
        if (bad) atomicOr(&ctr->err, ERR_BAD_OFFSETS);
    }
}

}  // namespace mt

using namespace mt;

// ---- host orchestration ---------------------------------------------------------------------------------
namespace {

struct Layout {
    size_t rw, qcnt, clus, keep, ghits, cand, nloc_ws, cl, dist, fb_list, multi_list, multi_set, U, M, abund,
        ctr, io, fb_scratch, taxon, nloc, locs, reads, roff, total;
    uint64_t rw_words, fb_cap;
};

uint64_t fb_cap_for(uint32_t maxn, uint32_t k, uint32_t w, uint32_t max_occ) {
    uint64_t nmin = (maxn >= k + w - 1) ? (uint64_t)(maxn - k - w + 2) : 1;
    uint64_t need = nmin * std::max<uint32_t>(max_occ, 1);
    uint64_t cap = 2;
    while (cap < need) cap <<= 1;
    return cap;
}

// host_io: the call's own copies of the host outputs and inputs are carved too (reads_in_ws:
// the reads' bytes as well; a call that uploads them before its layout is known keeps them in
// an allocation of their own).
Layout plan_layout(const mt_index *ix, uint64_t n_bases, uint64_t n_reads, uint32_t top_n, uint32_t maxn,
                   uint32_t max_occ, bool host_io, bool reads_in_ws = true) {
    Layout L{};
    Carver c;
    L.rw_words = (n_bases >> 5) + n_reads + 2;
    L.rw = c.take<uint64_t>(L.rw_words);
    L.qcnt = c.take<uint32_t>(n_reads);
    L.clus = c.take<Cluster>(n_reads * CSTORE);
    L.keep = c.take<uint8_t>(ix->G);
    L.ghits = c.take<uint64_t>(ix->G);
    L.cand = c.take<Cluster>(n_reads * top_n);
    L.nloc_ws = c.take<uint8_t>(n_reads);
    L.cl = c.take<uint32_t>(n_reads * top_n);
    L.dist = c.take<uint8_t>(n_reads * top_n);
    L.fb_list = c.take<uint32_t>(n_reads);
    L.multi_list = c.take<uint32_t>(n_reads);
    L.multi_set = c.take<int32_t>(n_reads * top_n);
    L.U = c.take<uint64_t>(ix->G);
    L.M = c.take<double>(ix->G);
    L.abund = c.take<double>(ix->G);
    L.ctr = c.take<Counters>(1);
    L.io = c.take<IoBlock>(1);
    L.fb_cap = fb_cap_for(maxn, ix->k, ix->w, max_occ);
    L.fb_scratch = c.take<uint8_t>((uint64_t)FB_CTAS * L.fb_cap * 12);
    if (host_io) {
        L.taxon = c.take<int32_t>(n_reads);
        L.nloc = c.take<uint8_t>(n_reads);
        L.locs = c.take<mt_loc>(n_reads * top_n);
        if (reads_in_ws) L.reads = c.take<uint8_t>(n_bases + 16);
        L.roff = c.take<uint64_t>(n_reads + 1);
    }
    L.total = c.off + 256;
    return L;
}

int check_params(const mt_classify_params *p) {
    if (!p) return MT_EINVAL;
    if (p->top_n < 1 || p->top_n > MT_MAX_TOPN) return MT_EINVAL;
    if (p->min_seeds < 1) return MT_EINVAL;
    if (p->max_occ > MT_MAX_OCC_LIMIT) return MT_EINVAL;
    if (p->cont_den == 0) return MT_EINVAL;
    if (!eda_mode_ok(p->eda_mode)) return MT_EINVAL;
    if (p->e_permille > 1000) return MT_EINVAL;
    if (p->e_permille == 0 && p->e_abs > MT_MAX_E) return MT_EINVAL;
    if (!(p->abund_cutoff >= 0.0)) return MT_EINVAL;
    return MT_OK;
}

}  // namespace

namespace mt {

// Everything one classification enqueues once its inputs are on the device and its IoBlock
// is written: no allocation, no synchronisation and no host read, so it can be captured into
// a CUDA graph. Grids are sized for the capacity `cap_reads`; the kernels take the actual
// batch size from the IoBlock and later counts from device counters.
struct EnqueueCtx {
    const mt_index *ix;
    const mt_classify_params *p;
    const Layout *L;
    unsigned char *ws;
    uint64_t cap_reads;
    uint32_t maxn, maxE;
    bool tune;             // time the approximation kernel's shapes on this batch (autotune calls)
    cudaEvent_t *ev;       // 5 events or null
    uint64_t launches;
    mt_allreduce_fn xfn;   // sum over the ranks of a sharded batch, or null
    void *xctx;
    const uint8_t *keep_in;   // a caller's genome mask replacing the containment mask, or null
    bool keep_dev;            // keep_in is a device pointer
    // reads arriving in chunks (host buffers): chunk i holds reads [chunk_r[i], chunk_r[i+1])
    // and is usable once chunk_ev[i] has fired; none: all reads are resident
    uint32_t n_chunks;
    const uint64_t *chunk_r;
    const cudaEvent_t *chunk_ev;
    bool capturing;           // the enqueue is being captured: chunk events are external waits
    mt_eda_shape *shape = nullptr;   // receives the approximation kernel's shape, or null
};

// Replaces the G-vector at `dev` with its sum over the ranks of a sharded batch (a no-op for an
// unsharded call): device -> host, the caller's allreduce, host -> device.
static int exchange(const EnqueueCtx &c, cudaStream_t s, void *dev, uint32_t G, int kind) {
    if (!c.xfn) return MT_OK;
    std::vector<uint64_t> h(std::max<uint32_t>(G, 1u), 0);
    if (G) MT_CK(cudaMemcpyAsync(h.data(), dev, G * 8ull, cudaMemcpyDeviceToHost, s));
    MT_CK(cudaStreamSynchronize(s));
    if (c.xfn(c.xctx, kind, h.data(), G) != 0) return MT_EXCHANGE;
    if (G) MT_CK(cudaMemcpyAsync(dev, h.data(), G * 8ull, cudaMemcpyHostToDevice, s));
    MT_CK(cudaStreamSynchronize(s));
    return MT_OK;
}

// The seeding kernel's block path serves indexes with w = 11 and k <= 28 (minimap2's short-read
// seeds, the mapping index of the paper's read mapper).
static bool seed_w11(const mt_index *ix) { return ix->w == 11 && ix->k <= 28; }

template <bool SH, bool HK32, bool COUNT = false, bool HPC = false, bool MULTI = false, bool W11 = false>
static int launch_seed(const SeedArgs &A, size_t smem, uint64_t need, cudaStream_t s) {
    auto kern = k_seed<SH, HK32, COUNT, HPC, MULTI, W11>;
    MT_CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    MT_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, SEED_THREADS, smem));
    per_sm = std::max(per_sm, 1);
    const unsigned grid = (unsigned)std::min<uint64_t>(need, (uint64_t)sm_count() * per_sm);
    kern<<<grid, SEED_THREADS, smem, s>>>(A);
    MT_CK(cudaGetLastError());
    return MT_OK;
}

static int enqueue_classify(EnqueueCtx &c, cudaStream_t s) {
    const Layout &L = *c.L;
    const mt_classify_params *p = c.p;
    const mt_index *ix = c.ix;
    const uint32_t G = ix->G, top_n = p->top_n;
    auto P = [&](size_t off) { return (void *)(c.ws + off); };
    static const char *const stage_name[5] = {
        "mt stage 1-2c: pack, minimizers, lookups, containment counts, locations",
        "mt stage 1d-2c: containment cutoff, candidate selection", "mt stage 2d: edit-distance approximation",
        "mt stage 3: decision, multi-mapped split, abundances", nullptr};
    StageTrace trace;
    auto mark = [&](int i) {
        if (c.ev) cudaEventRecord(c.ev[i], s);
        if (stage_name[i]) trace.next(stage_name[i]);
        else if (trace.open) { nvtxRangePop(); trace.open = false; }
    };
    Counters *ctr = (Counters *)P(L.ctr);
    unsigned long long *ghits = (unsigned long long *)P(L.ghits);
    unsigned long long *U = (unsigned long long *)P(L.U);
    double *M = (double *)P(L.M);
    const IoBlock *io = (const IoBlock *)P(L.io);
    MT_CK(cudaMemsetAsync(ctr, 0, sizeof(Counters), s));
    MT_CK(cudaMemsetAsync(ghits, 0, G * 8, s));
    MT_CK(cudaMemsetAsync(U, 0, G * 8, s));
    MT_CK(cudaMemsetAsync(M, 0, G * 8, s));
    const IndexView iv = ix->view();
    mark(0);
    if (c.cap_reads) {
        SeedArgs A;
        A.ix = iv;
        A.io = io;
        A.e_abs = p->e_abs; A.e_permille = p->e_permille; A.min_seeds = p->min_seeds; A.max_occ = p->max_occ;
        A.rw = (uint64_t *)P(L.rw);
        A.qcnt = (uint32_t *)P(L.qcnt);
        A.clus = (Cluster *)P(L.clus);
        A.ghits = ghits;
        A.fb_list = (uint32_t *)P(L.fb_list);
        A.ctr = ctr;
        const bool smem_hist = G <= SMEM_HIST_MAX;
        const bool hk32 = ix->hk_db != 0;
        const uint32_t hist_n = smem_hist ? G : 0;
        const bool w11 = seed_w11(ix);
        const size_t smem = hk32 ? (w11 ? seed_smem_bytes<true, true>(hist_n) : seed_smem_bytes<true, false>(hist_n))
                                 : (w11 ? seed_smem_bytes<false, true>(hist_n) : seed_smem_bytes<false, false>(hist_n));
        auto seed = [&](uint64_t rb, uint64_t re) {
            A.r_begin = rb;
            A.r_end = re;
            const uint64_t need = (std::min<uint64_t>(re, c.cap_reads) - rb + SEED_WARPS - 1) / SEED_WARPS;
            if (seed_w11(ix))
                return hk32 ? (smem_hist ? launch_seed<true, true, false, false, false, true>(A, smem, need, s)
                                         : launch_seed<false, true, false, false, false, true>(A, smem, need, s))
                            : (smem_hist ? launch_seed<true, false, false, false, false, true>(A, smem, need, s)
                                         : launch_seed<false, false, false, false, false, true>(A, smem, need, s));
            return hk32 ? (smem_hist ? launch_seed<true, true>(A, smem, need, s) : launch_seed<false, true>(A, smem, need, s))
                        : (smem_hist ? launch_seed<true, false>(A, smem, need, s) : launch_seed<false, false>(A, smem, need, s));
        };
        int rc = MT_OK;
        if (c.n_chunks) {   // seed each chunk of reads as soon as its bytes have arrived
            for (uint32_t i = 0; i < c.n_chunks && !rc; i++) {
                MT_CK(cudaStreamWaitEvent(s, c.chunk_ev[i], c.capturing ? cudaEventWaitExternal : 0));
                rc = seed(c.chunk_r[i], c.chunk_r[i + 1]);
            }
            c.launches += c.n_chunks - 1;
        } else {
            rc = seed(0, ~0ull);
        }
        if (rc) return rc;
        mark(1);
        if ((rc = exchange(c, s, ghits, G, MT_XCHG_GENOME_HITS))) return rc;

        if (c.keep_in) {
            MT_CK(cudaMemcpyAsync(P(L.keep), c.keep_in, G, c.keep_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
        } else {
            k_mask<<<1, 1024, 0, s>>>(ghits, G, p->cont_num, p->cont_den, (uint8_t *)P(L.keep));
            MT_CK(cudaGetLastError());
        }
        const unsigned rblocks = (unsigned)std::min<uint64_t>((c.cap_reads + 255) / 256, (uint64_t)sm_count() * SELECT_CTAS);
        k_select<<<rblocks, 256, 0, s>>>(io, A.qcnt, A.clus, (const uint8_t *)P(L.keep), top_n, (Cluster *)P(L.cand),
                                         (uint8_t *)P(L.nloc_ws), (uint32_t *)P(L.cl), A.fb_list, ctr);
        MT_CK(cudaGetLastError());
        FbArgs F;
        F.ix = iv;
        F.rw = A.rw;
        F.io = io;
        F.e_abs = p->e_abs; F.e_permille = p->e_permille; F.min_seeds = p->min_seeds; F.max_occ = p->max_occ;
        F.top_n = top_n;
        F.keep = (const uint8_t *)P(L.keep);
        F.fb_list = A.fb_list;
        F.cand = (Cluster *)P(L.cand);
        F.nloc_ws = (uint8_t *)P(L.nloc_ws);
        F.cl = (uint32_t *)P(L.cl);
        F.ctr = ctr;
        F.scratch = (uint64_t *)P(L.fb_scratch);
        F.cap = L.fb_cap;
        k_fallback<<<FB_CTAS, FB_THREADS, 0, s>>>(F);
        MT_CK(cudaGetLastError());
        mark(2);

        rc = launch_classify_eda(iv, A.rw, io, (const uint32_t *)P(L.cl), &ctr->cl_count, c.cap_reads * top_n,
                                     (const Cluster *)P(L.cand), top_n, p->e_abs, p->e_permille, c.maxn, c.maxE,
                                     p->eda_mode, (uint8_t *)P(L.dist), &ctr->eda_counter, s, c.tune, c.shape);
        if (rc) return rc;
        mark(3);

        DecideArgs D;
        D.io = io;
        D.e_abs = p->e_abs; D.e_permille = p->e_permille; D.top_n = top_n;
        D.nloc_ws = (const uint8_t *)P(L.nloc_ws);
        D.cand = (const Cluster *)P(L.cand);
        D.dist = (const uint8_t *)P(L.dist);
        D.U = U;
        D.multi_set = (int32_t *)P(L.multi_set);
        D.multi_list = (uint32_t *)P(L.multi_list);
        D.ctr = ctr;
        {
            static_assert(sizeof(mt_loc) == 24, "a location is three 8-byte words");
            D.G = G;
            D.hist = G <= SMEM_HIST_MAX;
            const size_t dsmem = (D.hist ? (((size_t)G * 8 + 15) & ~(size_t)15) : 0) +
                                 (size_t)DECIDE_THREADS * top_n * (sizeof(Cluster) + sizeof(mt_loc) + 1) + DECIDE_THREADS;
            // the paper's top 3 runs a variant with per-read arrays of 3 (fewer registers, more
            // resident CTAs); one wave of resident CTAs walks the reads
            auto kern = top_n <= 3 ? k_decide<3> : k_decide<MT_MAX_TOPN>;
            if (dsmem > 48 * 1024)
                MT_CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsmem));
            int per_sm = 0;
            MT_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, DECIDE_THREADS, dsmem));
            const unsigned dblocks = (unsigned)std::min<uint64_t>((c.cap_reads + DECIDE_THREADS - 1) / DECIDE_THREADS,
                                                                  (uint64_t)sm_count() * std::max(per_sm, 1));
            kern<<<dblocks, DECIDE_THREADS, dsmem, s>>>(D);
        }
        MT_CK(cudaGetLastError());
        if ((rc = exchange(c, s, U, G, MT_XCHG_UNIQUE))) return rc;
        k_multi<<<(unsigned)sm_count() * 4, 256, 0, s>>>(D.multi_list, ctr, D.multi_set, top_n, U, M);
        MT_CK(cudaGetLastError());
        if ((rc = exchange(c, s, M, G, MT_XCHG_MULTI))) return rc;
        c.launches += 7;   // seed, mask, select, fallback, approximation, decide, multi
    } else {
        mark(1); mark(2); mark(3);
        int rc;   // an empty shard still takes part in every exchange, with zeros
        if ((rc = exchange(c, s, ghits, G, MT_XCHG_GENOME_HITS))) return rc;
        if ((rc = exchange(c, s, U, G, MT_XCHG_UNIQUE))) return rc;
        if ((rc = exchange(c, s, M, G, MT_XCHG_MULTI))) return rc;
    }
    k_abund<<<1, 1024, 0, s>>>(G, U, M, p->abund_cutoff, (double *)P(L.abund));
    MT_CK(cudaGetLastError());
    c.launches += 1;
    mark(4);
    return MT_OK;
}

static void fill_stats(mt_stats *st, const Counters &h, uint64_t n_reads, uint64_t ws_bytes, uint64_t launches,
                       cudaEvent_t *ev) {
    if (!st) return;
    st->n_reads = n_reads;
    st->n_minimizers = h.stat[ST_MINS];
    st->n_hits = h.stat[ST_HITS];
    st->n_candidates = h.stat[ST_CAND];
    st->n_accepted = h.stat[ST_ACC];
    st->n_multi = h.stat[ST_MULTI];
    st->n_fallback = h.stat[ST_FB];
    st->workspace_bytes = ws_bytes;
    st->n_ext_occ = h.stat[ST_EXT];
    st->n_stored = h.stat[ST_STORED];
    st->n_launches = launches;
    st->err_bits = h.err;
    st->ms_seed = st->ms_select = st->ms_eda = st->ms_profile = st->ms_total = 0;
    if (ev) {
        float t[4] = {0, 0, 0, 0}, tot = 0;
        for (int i = 0; i < 4; i++) cudaEventElapsedTime(&t[i], ev[i], ev[i + 1]);
        cudaEventElapsedTime(&tot, ev[0], ev[4]);
        st->ms_seed = t[0]; st->ms_select = t[1]; st->ms_eda = t[2]; st->ms_profile = t[3]; st->ms_total = tot;
    }
}

static int status_of(uint32_t err) {
    if (err & (ERR_BAD_BASE | ERR_BAD_OFFSETS | ERR_READ_TOO_LONG)) return MT_EINVAL;
    if (err) return MT_ECUDA;
    return MT_OK;
}

}  // namespace mt

using namespace mt;

uint64_t mt::classify_ws_bytes(const mt_index *ix, uint64_t n_bases, uint64_t n_reads,
                               const mt_classify_params *p, uint32_t maxn, bool host_io) {
    if (!ix || !p || check_params(p)) return 0;
    return plan_layout(ix, n_bases, n_reads, p->top_n, std::max<uint32_t>(maxn, 1), p->max_occ, host_io).total;
}

extern "C" uint64_t mt_classify_workspace_bytes(const mt_index *ix, uint64_t n_bases, uint64_t n_reads,
                                                uint32_t max_read_len, const mt_classify_params *p) {
    if (!ix || !p || check_params(p)) return 0;
    uint32_t maxn = max_read_len ? std::min<uint32_t>(max_read_len, MT_MAX_READ_LEN)
                                 : (uint32_t)std::min<uint64_t>(n_bases, MT_MAX_READ_LEN);
    return plan_layout(ix, n_bases, n_reads, p->top_n, std::max<uint32_t>(maxn, 1), p->max_occ, true).total;
}

static int classify_impl(const mt_index *ix, const uint8_t *reads, uint64_t n_bases, const uint64_t *offsets,
                         uint64_t n_reads, const mt_classify_params *p, int device_ptrs, void *stream,
                         mt_allreduce_fn xfn, void *xctx, const uint8_t *keep_in, int32_t *taxon,
                         uint8_t *nloc, mt_loc *locs, uint64_t *genome_hits, double *abundance,
                         mt_stats *stats, bool tune = false, mt_eda_shape *shape = nullptr) {
    if (!ix || !offsets || (!taxon && n_reads) || (!reads && n_bases)) return MT_EINVAL;
    if (ix->hpc) return MT_EINVAL;   // a containment index: positions are in compressed coordinates
    Trace trace("mt_classify");
    int rc = check_params(p);
    if (rc) return rc;
    if (n_reads >= 0xFFFFFFFFull / MT_MAX_TOPN) return MT_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const uint32_t G = ix->G, top_n = p->top_n;
    const bool host_io = !device_ptrs;
    if (stats) memset(stats, 0, sizeof(*stats));

    // Host batches: the offsets and the reads' bytes go to allocations of their own, the bytes
    // in chunks on a second stream that start at once, so that they move while the offsets
    // are checked below; the seeding of a chunk waits only for its own bytes.
    uint64_t *d_roff = nullptr;
    uint8_t *d_reads = nullptr;
    cudaStream_t cs = nullptr;
    std::vector<cudaEvent_t> chunk_ev;
    std::vector<uint64_t> chunk_r;
    auto release = [&]() {
        if (cs) cudaStreamSynchronize(cs);
        for (auto e : chunk_ev) cudaEventDestroy(e);
        if (cs) cudaStreamDestroy(cs);
        if (d_roff) dfree(d_roff, s);
        if (d_reads) dfree(d_reads, s);
    };
    uint32_t maxn = 0;
    uint64_t off0 = 0, launches = 0;
    if (host_io && n_reads) {
        off0 = offsets[0];
        if ((rc = dalloc((void **)&d_roff, (n_reads + 1) * 8, s))) return rc;
        if ((rc = dalloc((void **)&d_reads, n_bases + 16, s))) { release(); return rc; }
        MT_CK(cudaMemcpyAsync(d_roff, offsets, (n_reads + 1) * 8, cudaMemcpyHostToDevice, s));
        // chunk i: reads [chunk_r[i], chunk_r[i+1]), its bytes copied on cs, then chunk_ev[i + 1].
        // The copies queue behind the offsets' copy (one copy engine takes a direction's copies
        // in issue order) and the first chunks are small (16 MB, doubling), so that seeding
        // starts soon after the offsets are checked. The offsets are not checked yet (k_maxlen
        // below does that, and a bad batch returns before any kernel reads the bytes), so every
        // copy is clamped to the n_bases buffer.
        const uint64_t span = offsets[n_reads] >= off0 ? offsets[n_reads] - off0 : 0;
        const uint64_t chunk = std::max<uint64_t>(32ull << 20, span / 16);
        if (span > chunk) {
            int e_ok = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) == cudaSuccess;
            cudaEvent_t ready = nullptr;
            e_ok = e_ok && cudaEventCreateWithFlags(&ready, cudaEventDisableTiming) == cudaSuccess;
            if (ready) chunk_ev.push_back(ready);
            // the copies follow the allocations, which are ordered on s
            e_ok = e_ok && cudaEventRecord(ready, s) == cudaSuccess && cudaStreamWaitEvent(cs, ready, 0) == cudaSuccess;
            chunk_r.push_back(0);
            uint64_t csz = std::min<uint64_t>(16ull << 20, chunk);
            for (uint64_t rb = 0; e_ok && rb < n_reads;) {
                const uint64_t limit = offsets[rb] + csz;
                csz = std::min<uint64_t>(csz * 2, chunk);
                uint64_t re = (uint64_t)(std::upper_bound(offsets + rb + 1, offsets + n_reads + 1, limit) - offsets) - 1;
                if (re <= rb) re = rb + 1;
                cudaEvent_t ev = nullptr;
                e_ok = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess;
                if (ev) chunk_ev.push_back(ev);
                const uint64_t b0 = std::min(offsets[rb], n_bases);
                const uint64_t b1 = std::min(std::max(offsets[re], b0), n_bases);
                if (e_ok && b1 > b0)
                    e_ok = cudaMemcpyAsync(d_reads + b0, reads + b0, b1 - b0, cudaMemcpyHostToDevice, cs) == cudaSuccess;
                e_ok = e_ok && cudaEventRecord(ev, cs) == cudaSuccess;
                chunk_r.push_back(re);
                rb = re;
            }
            if (!e_ok) {
                cuda_ok(cudaGetLastError(), "chunked read copies");
                release();
                return MT_ECUDA;
            }
        } else if (n_bases) {
            MT_CK(cudaMemcpyAsync(d_reads, reads, n_bases, cudaMemcpyHostToDevice, s));
        }
    }
    // longest read and offset checks, on the device
    if (n_reads) {
        Counters *pre = nullptr;
        if ((rc = dalloc((void **)&pre, sizeof(Counters), s))) { release(); return rc; }
        MT_CK(cudaMemsetAsync(pre, 0, sizeof(Counters), s));
        unsigned blocks = (unsigned)std::min<uint64_t>((n_reads + 255) / 256, (uint64_t)sm_count() * 4);
        k_maxlen<<<blocks, 256, 0, s>>>(host_io ? d_roff : offsets, n_reads, n_bases, pre);
        MT_CK(cudaGetLastError());
        launches++;
        Counters h{};
        MT_CK(cudaMemcpyAsync(&h, pre, sizeof(h), cudaMemcpyDeviceToHost, s));
        if (!host_io) MT_CK(cudaMemcpyAsync(&off0, offsets, 8, cudaMemcpyDeviceToHost, s));
        MT_CK(cudaStreamSynchronize(s));
        dfree(pre, s);
        if (h.err) { release(); return MT_EINVAL; }
        maxn = h.maxn;
    }
    const uint32_t maxE = edit_threshold(maxn, p->e_abs, p->e_permille);
    if (maxn > MT_MAX_READ_LEN || maxE > MT_MAX_E) {
        release();
        return MT_EINVAL;
    }

    Layout L = plan_layout(ix, n_bases, n_reads, top_n, std::max<uint32_t>(maxn, 1), p->max_occ, host_io, false);
    unsigned char *ws = nullptr;
    if ((rc = dalloc((void **)&ws, L.total, s))) { release(); return rc; }
    auto P = [&](size_t off) { return (void *)(ws + off); };
    IoBlock hio;
    hio.reads = reads;
    hio.roff = offsets;
    hio.n_reads = n_reads;
    hio.n_bases = n_bases;
    hio.off0 = off0;
    hio.max_len = MT_MAX_READ_LEN;
    hio.taxon = taxon;
    hio.nloc = nloc;
    hio.locs = locs;
    if (host_io) {
        hio.reads = d_reads;
        hio.roff = n_reads ? d_roff : (const uint64_t *)P(L.roff);
        hio.taxon = (int32_t *)P(L.taxon);
        hio.nloc = (uint8_t *)P(L.nloc);
        hio.locs = locs ? (mt_loc *)P(L.locs) : nullptr;
        if (!n_reads) MT_CK(cudaMemcpyAsync((void *)hio.roff, offsets, 8, cudaMemcpyHostToDevice, s));
    }
    hio.vec_ok = ((uintptr_t)hio.reads & 15u) == 0;
    MT_CK(cudaMemcpyAsync(P(L.io), &hio, sizeof(hio), cudaMemcpyHostToDevice, s));

    cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    if (stats)
        for (auto &e : ev) MT_CK(cudaEventCreate(&e));
    EnqueueCtx ctx{ix, p, &L, ws, n_reads, std::max<uint32_t>(maxn, 1), maxE, tune, stats ? ev : nullptr, launches,
                   xfn, xctx, keep_in, !host_io, 0, nullptr, nullptr};
    if (cs) {
        ctx.n_chunks = (uint32_t)(chunk_r.size() - 1);
        ctx.chunk_r = chunk_r.data();
        ctx.chunk_ev = chunk_ev.data() + 1;
    }
    ctx.shape = shape;
    rc = enqueue_classify(ctx, s);
    if (rc) {
        if (cs) cudaStreamSynchronize(cs);
        dfree(ws, s);
        cudaStreamSynchronize(s);
        release();
        return rc;
    }

    cudaMemcpyKind kind = host_io ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    if (genome_hits) MT_CK(cudaMemcpyAsync(genome_hits, P(L.ghits), G * 8, kind, s));
    if (abundance) MT_CK(cudaMemcpyAsync(abundance, P(L.abund), G * 8, kind, s));
    if (host_io && n_reads) {
        MT_CK(cudaMemcpyAsync(taxon, hio.taxon, n_reads * 4, cudaMemcpyDeviceToHost, s));
        if (nloc) MT_CK(cudaMemcpyAsync(nloc, hio.nloc, n_reads, cudaMemcpyDeviceToHost, s));
        if (locs) MT_CK(cudaMemcpyAsync(locs, hio.locs, n_reads * top_n * sizeof(mt_loc), cudaMemcpyDeviceToHost, s));
    }
    Counters h{};
    MT_CK(cudaMemcpyAsync(&h, P(L.ctr), sizeof(h), cudaMemcpyDeviceToHost, s));
    dfree(ws, s);
    MT_CK(cudaStreamSynchronize(s));
    release();
    fill_stats(stats, h, n_reads, L.total + (d_reads ? n_bases + 16 : 0), ctx.launches, stats ? ev : nullptr);
    if (stats)
        for (auto &e : ev) cudaEventDestroy(e);
    return status_of(h.err);
}

extern "C" int mt_classify(const mt_index *ix, const uint8_t *reads, uint64_t n_bases, const uint64_t *offsets,
                           uint64_t n_reads, const mt_classify_params *p, int device_ptrs, void *stream,
                           int32_t *taxon, uint8_t *nloc, mt_loc *locs, uint64_t *genome_hits, double *abundance,
                           mt_stats *stats) {
    return classify_impl(ix, reads, n_bases, offsets, n_reads, p, device_ptrs, stream, nullptr, nullptr, nullptr,
                         taxon, nloc, locs, genome_hits, abundance, stats);
}

extern "C" int mt_classify_autotune(const mt_index *ix, const uint8_t *reads, uint64_t n_bases,
                                    const uint64_t *offsets, uint64_t n_reads, const mt_classify_params *p,
                                    int device_ptrs, void *stream, int32_t *taxon, uint8_t *nloc, mt_loc *locs,
                                    uint64_t *genome_hits, double *abundance, mt_stats *stats,
                                    mt_eda_shape *shape) {
    if (shape) memset(shape, 0, sizeof(*shape));
    const bool tune = p && (p->eda_mode & 15u) == MT_EDA_BATCHED;
    int rc = classify_impl(ix, reads, n_bases, offsets, n_reads, p, device_ptrs, stream, nullptr, nullptr, nullptr,
                           taxon, nloc, locs, genome_hits, abundance, stats, tune, shape);
    if (shape && shape->lanes_per_pair) shape->tuned = tune ? 1u : 0u;
    return rc;
}

extern "C" int mt_classify_masked(const mt_index *ix, const uint8_t *reads, uint64_t n_bases, const uint64_t *offsets,
                                  uint64_t n_reads, const mt_classify_params *p, int device_ptrs, void *stream,
                                  const uint8_t *keep, int32_t *taxon, uint8_t *nloc, mt_loc *locs,
                                  uint64_t *genome_hits, double *abundance, mt_stats *stats) {
    if (!keep) return MT_EINVAL;
    return classify_impl(ix, reads, n_bases, offsets, n_reads, p, device_ptrs, stream, nullptr, nullptr, keep, taxon,
                         nloc, locs, genome_hits, abundance, stats);
}

extern "C" int mt_classify_sharded(const mt_index *ix, const uint8_t *reads, uint64_t n_bases,
                                   const uint64_t *offsets, uint64_t n_reads, const mt_classify_params *p,
                                   int device_ptrs, void *stream, mt_allreduce_fn allreduce, void *ctx,
                                   int32_t *taxon, uint8_t *nloc, mt_loc *locs, uint64_t *genome_hits,
                                   double *abundance, mt_stats *stats) {
    if (!allreduce) return MT_EINVAL;
    return classify_impl(ix, reads, n_bases, offsets, n_reads, p, device_ptrs, stream, allreduce, ctx, nullptr, taxon,
                         nloc, locs, genome_hits, abundance, stats);
}

// ---- containment alone (stage 1): seed hits per genome and the kept-genome mask ------------------
extern "C" int mt_containment(const mt_index *ix, const uint8_t *reads, uint64_t n_bases, const uint64_t *offsets,
                              uint64_t n_reads, uint32_t max_occ, uint32_t cont_num, uint32_t cont_den,
                              int device_ptrs, void *stream, uint64_t *genome_hits, uint8_t *keep) {
    if (!ix || !offsets || (!reads && n_bases) || !genome_hits) return MT_EINVAL;
    if (max_occ > MT_MAX_OCC_LIMIT || cont_den == 0) return MT_EINVAL;
    Trace trace("mt_containment");
    cudaStream_t s = (cudaStream_t)stream;
    const uint32_t G = ix->G;
    const bool host_io = !device_ptrs;
    uint64_t off0 = 0;
    if (host_io && n_reads) {
        off0 = offsets[0];
        for (uint64_t r = 0; r < n_reads; r++)
            if (offsets[r + 1] < offsets[r] || offsets[r + 1] > n_bases) return MT_EINVAL;
    } else if (n_reads) {
        MT_CK(cudaMemcpyAsync(&off0, offsets, 8, cudaMemcpyDeviceToHost, s));
        MT_CK(cudaStreamSynchronize(s));
    }
    // workspace: counters | hits | mask | I/O block | host-buffer staging (reads, offsets)
    auto up = [](size_t x) { return (x + 255) & ~size_t(255); };
    const size_t o_ctr = 0, o_hits = up(sizeof(Counters)), o_keep = o_hits + up(G * 8ull);
    const size_t o_io = o_keep + up(G), o_reads = o_io + up(sizeof(IoBlock));
    const size_t o_off = o_reads + (host_io ? up(std::max<uint64_t>(n_bases, 1)) : 0);
    const size_t total = o_off + (host_io ? up((n_reads + 1) * 8) : 0);
    unsigned char *ws = nullptr;
    int rc = dalloc((void **)&ws, total, s);
    if (rc) return rc;
    Counters *ctr = (Counters *)(ws + o_ctr);
    unsigned long long *ghits = (unsigned long long *)(ws + o_hits);
    uint8_t *dkeep = ws + o_keep;
    auto fail = [&](int code) { dfree(ws, s); return code; };
    if (cudaMemsetAsync(ws, 0, o_keep, s) != cudaSuccess) return fail(MT_ECUDA);
    IoBlock hio{};
    hio.reads = reads;
    hio.roff = offsets;
    hio.n_reads = n_reads;
    hio.n_bases = n_bases;
    hio.off0 = off0;
    hio.max_len = MT_MAX_READ_LEN;
    if (host_io) {
        hio.reads = ws + o_reads;
        hio.roff = (const uint64_t *)(ws + o_off);
        if (n_bases && cudaMemcpyAsync((void *)hio.reads, reads, n_bases, cudaMemcpyHostToDevice, s) != cudaSuccess)
            return fail(MT_ECUDA);
        if (cudaMemcpyAsync((void *)hio.roff, offsets, (n_reads + 1) * 8, cudaMemcpyHostToDevice, s) != cudaSuccess)
            return fail(MT_ECUDA);
    }
    hio.vec_ok = ((uintptr_t)hio.reads & 15u) == 0;
    if (cudaMemcpyAsync(ws + o_io, &hio, sizeof(hio), cudaMemcpyHostToDevice, s) != cudaSuccess) return fail(MT_ECUDA);
    if (n_reads) {
        SeedArgs A{};
        A.ix = ix->view();
        A.io = (const IoBlock *)(ws + o_io);
        A.min_seeds = 1;
        A.max_occ = max_occ;
        A.ghits = ghits;
        A.ctr = ctr;
        A.r_begin = 0;
        A.r_end = ~0ull;
        const bool smem_hist = G <= SMEM_HIST_MAX;
        const size_t smem = (!ix->hpc && seed_w11(ix)) ? seed_smem_bytes<false, true>(smem_hist ? G : 0)
                                                       : seed_smem_bytes<false, false>(smem_hist ? G : 0);
        const uint64_t need = (n_reads + SEED_WARPS - 1) / SEED_WARPS;
        if (ix->hpc) rc = smem_hist ? launch_seed<true, false, true, true>(A, smem, need, s)
                                    : launch_seed<false, false, true, true>(A, smem, need, s);
        else if (seed_w11(ix)) rc = smem_hist ? launch_seed<true, false, true, false, false, true>(A, smem, need, s)
                                              : launch_seed<false, false, true, false, false, true>(A, smem, need, s);
        else rc = smem_hist ? launch_seed<true, false, true, false>(A, smem, need, s)
                            : launch_seed<false, false, true, false>(A, smem, need, s);
        if (rc) return fail(rc);
    }
    k_mask<<<1, 1024, 0, s>>>(ghits, G, cont_num, cont_den, dkeep);
    if (!cuda_ok(cudaGetLastError(), "k_mask")) return fail(MT_ECUDA);
    const cudaMemcpyKind kind = host_io ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    if (cudaMemcpyAsync(genome_hits, ghits, G * 8ull, kind, s) != cudaSuccess) return fail(MT_ECUDA);
    if (keep && cudaMemcpyAsync(keep, dkeep, G, kind, s) != cudaSuccess) return fail(MT_ECUDA);
    Counters h{};
    if (cudaMemcpyAsync(&h, ctr, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess) return fail(MT_ECUDA);
    dfree(ws, s);
    MT_CK(cudaStreamSynchronize(s));
    return status_of(h.err);
}

// Seed hits of several indexes built with one (k, w, canonical, compression) in one pass over
// device-resident reads: each read's minimizers are found once and looked up in every
// index's table; hits[base_b + g] counts genome g of index b, base_b = the number of genomes
// of the indexes before b. Equal to one counting pass per index.
int mt::contain_multi(const mt_index *const *batches, uint32_t n_batches, const uint8_t *reads, uint64_t n_bases,
                      const uint64_t *offsets, uint64_t n_reads, uint32_t max_occ, uint64_t *hits, cudaStream_t s) {
    if (!n_batches) return MT_OK;
    if (!batches || !batches[0] || !hits || !offsets || (!reads && n_bases) || max_occ > MT_MAX_OCC_LIMIT ||
        n_batches > MULTI_MAX_INDEXES)
        return MT_EINVAL;
    const mt_index *b0 = batches[0];
    std::vector<BatchView> hv(n_batches);
    uint64_t T = 0;
    for (uint32_t b = 0; b < n_batches; b++) {
        const mt_index *ix = batches[b];
        if (!ix || ix->k != b0->k || ix->w != b0->w || ix->canonical != b0->canonical || ix->hpc != b0->hpc)
            return MT_EINVAL;
        hv[b].table = ix->d_table;
        hv[b].slot_mask = ix->slots - 1;
        hv[b].occ = ix->d_occ;
        hv[b].slot_shift = ix->slot_shift;
        hv[b].filter = ix->d_filter;
        hv[b].filter_shift = ix->filter_shift;
        hv[b].base = (uint32_t)T;
        hv[b].pad = 0;
        T += ix->G;
    }
    if (T >= (1ull << 31)) return MT_EINVAL;
    uint64_t off0 = 0;
    if (n_reads) {
        MT_CK(cudaMemcpyAsync(&off0, offsets, 8, cudaMemcpyDeviceToHost, s));
        MT_CK(cudaStreamSynchronize(s));
    }
    auto up = [](size_t x) { return (x + 255) & ~size_t(255); };
    const size_t o_io = up(sizeof(Counters)), o_bv = o_io + up(sizeof(IoBlock));
    const size_t total = o_bv + up(n_batches * sizeof(BatchView));
    unsigned char *ws = nullptr;
    int rc = dalloc((void **)&ws, total, s);
    if (rc) return rc;
    auto fail = [&](int code) { dfree(ws, s); cudaStreamSynchronize(s); return code; };
    Counters *ctr = (Counters *)ws;
    IoBlock hio{};
    hio.reads = reads;
    hio.roff = offsets;
    hio.n_reads = n_reads;
    hio.n_bases = n_bases;
    hio.off0 = off0;
    hio.max_len = MT_MAX_READ_LEN;
    hio.vec_ok = ((uintptr_t)reads & 15u) == 0;
    if (cudaMemsetAsync(ctr, 0, sizeof(Counters), s) != cudaSuccess ||
        cudaMemsetAsync(hits, 0, T * 8, s) != cudaSuccess ||
        cudaMemcpyAsync(ws + o_io, &hio, sizeof(hio), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(ws + o_bv, hv.data(), n_batches * sizeof(BatchView), cudaMemcpyHostToDevice, s) != cudaSuccess)
        return fail(MT_ECUDA);
    if (n_reads) {
        SeedArgs A{};
        A.ix = b0->view();
        A.io = (const IoBlock *)(ws + o_io);
        A.min_seeds = 1;
        A.max_occ = max_occ;
        A.ghits = (unsigned long long *)hits;
        A.ctr = ctr;
        A.r_begin = 0;
        A.r_end = ~0ull;
        A.bv = (const BatchView *)(ws + o_bv);
        A.n_bv = n_batches;
        A.n_hist = (uint32_t)T;
        A.div_magic = n_batches > 1 ? (uint32_t)(((1ull << 32) + n_batches - 1) / n_batches) : 0u;
        const bool smem_hist = T <= SMEM_HIST_MAX;
        const size_t smem = seed_smem_bytes<false, false>(smem_hist ? (uint32_t)T : 0);
        const uint64_t need = (n_reads + SEED_WARPS - 1) / SEED_WARPS;
        if (b0->hpc) rc = smem_hist ? launch_seed<true, false, true, true, true>(A, smem, need, s)
                                    : launch_seed<false, false, true, true, true>(A, smem, need, s);
        else rc = smem_hist ? launch_seed<true, false, true, false, true>(A, smem, need, s)
                            : launch_seed<false, false, true, false, true>(A, smem, need, s);
        if (rc) return fail(rc);
    }
    Counters h{};
    if (cudaMemcpyAsync(&h, ctr, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess) return fail(MT_ECUDA);
    dfree(ws, s);
    MT_CK(cudaStreamSynchronize(s));
    return status_of(h.err);
}

// Several genome shards' per-read location lists (device) merged by rank and decided: per-read
// outputs and the abundance profile (device pointers), as a single index's stage 3.
int mt::merge_decide(const mt_loc *lists, uint32_t R, const uint64_t *roff, uint64_t n_reads, uint32_t G,
                     const mt_classify_params *p, int32_t *taxon, uint8_t *nloc, mt_loc *locs, double *abundance,
                     cudaStream_t s) {
    const uint32_t tn = p->top_n;
    Carver c;
    const size_t o_ctr = c.take<Counters>(1), o_U = c.take<uint64_t>(G), o_M = c.take<double>(G);
    const size_t o_set = c.take<int32_t>(std::max<uint64_t>(n_reads * tn, 1));
    const size_t o_list = c.take<uint32_t>(std::max<uint64_t>(n_reads, 1));
    unsigned char *ws = nullptr;
    int rc = dalloc((void **)&ws, c.off + 256, s);
    if (rc) return rc;
    auto done = [&](int code) { dfree(ws, s); cudaStreamSynchronize(s); return code; };
    Counters *ctr = (Counters *)(ws + o_ctr);
    unsigned long long *U = (unsigned long long *)(ws + o_U);
    double *M = (double *)(ws + o_M);
    if (cudaMemsetAsync(ws, 0, o_set, s) != cudaSuccess) return done(MT_ECUDA);
    if (n_reads) {
        MergeArgs A;
        A.lists = lists; A.roff = roff; A.n_reads = n_reads;
        A.R = R; A.top_n = tn; A.e_abs = p->e_abs; A.e_permille = p->e_permille; A.G = G;
        A.hist = G <= SMEM_HIST_MAX;
        A.taxon = taxon; A.nloc = nloc; A.locs = locs; A.U = U;
        A.multi_set = (int32_t *)(ws + o_set); A.multi_list = (uint32_t *)(ws + o_list); A.ctr = ctr;
        const size_t smem = A.hist ? G * 8ull : 0;
        if (smem > 48 * 1024 && !cuda_ok(cudaFuncSetAttribute(k_merge_decide, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                             (int)smem), "k_merge_decide smem"))
            return done(MT_ECUDA);
        const unsigned grid = (unsigned)std::min<uint64_t>((n_reads + 255) / 256, (uint64_t)sm_count() * 8);
        k_merge_decide<<<grid, 256, smem, s>>>(A);
        if (!cuda_ok(cudaGetLastError(), "k_merge_decide")) return done(MT_ECUDA);
        k_multi<<<(unsigned)sm_count() * 4, 256, 0, s>>>(A.multi_list, ctr, A.multi_set, tn, U, M);
        if (!cuda_ok(cudaGetLastError(), "k_multi")) return done(MT_ECUDA);
    }
    k_abund<<<1, 1024, 0, s>>>(G, U, M, p->abund_cutoff, abundance);
    if (!cuda_ok(cudaGetLastError(), "k_abund")) return done(MT_ECUDA);
    return done(cuda_ok(cudaStreamSynchronize(s), "merge decide") ? MT_OK : MT_ECUDA);
}

int mt::check_classify_params(const mt_classify_params *p) { return check_params(p); }

// The containment cutoff over given counts (used by the partitioned-database query).
int mt::launch_mask(const uint64_t *hits, uint32_t G, uint32_t cont_num, uint32_t cont_den, uint8_t *keep,
                    cudaStream_t s) {
    k_mask<<<1, 1024, 0, s>>>((const unsigned long long *)hits, G, cont_num, cont_den, keep);
    MT_CK(cudaGetLastError());
    return MT_OK;
}

// ---- plans: preallocated workspace + captured CUDA graph ---------------------------------------------
struct mt_plan {
    const mt_index *ix = nullptr;
    mt_classify_params p{};
    uint64_t cap_reads = 0, cap_bases = 0;
    uint32_t max_len = 0, maxE = 0;
    Layout L{};
    unsigned char *ws = nullptr;
    IoBlock *h_io = nullptr;        // pinned
    Counters *h_ctr = nullptr;      // pinned
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cap_stream = nullptr;   // private stream the graph is captured on
    uint64_t calls = 0, launches = 0;
    // Host batches go up in chunks of reads on a copy stream, each seeded as it lands: chunk i
    // holds reads [chunk_r[i], chunk_r[i+1]) of the capacity (fixed, so one graph serves
    // every batch); the graph waits on chunk_ev[i], recorded each call after the chunk's copy
    // (or at once for device inputs).
    static constexpr uint32_t MAX_CHUNKS = 8;
    uint32_t n_chunks = 1;
    uint64_t chunk_r[MAX_CHUNKS + 1] = {};
    cudaEvent_t chunk_ev[MAX_CHUNKS] = {};
    cudaEvent_t ready = nullptr;
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t t_ev[2] = {};          // timing of a call's enqueue (stats), owned by the plan
};

extern "C" int mt_plan_create(const mt_index *ix, const mt_classify_params *p, uint64_t max_reads,
                              uint64_t max_bases, uint32_t max_read_len, mt_plan **out) {
    if (!out) return MT_EINVAL;
    *out = nullptr;
    if (!ix || ix->hpc || check_params(p) || max_reads == 0 || max_read_len == 0 || max_read_len > MT_MAX_READ_LEN)
        return MT_EINVAL;
    if (max_reads >= 0xFFFFFFFFull / MT_MAX_TOPN) return MT_EINVAL;
    const uint32_t maxE = edit_threshold(max_read_len, p->e_abs, p->e_permille);
    if (maxE > MT_MAX_E) return MT_EINVAL;
    mt_plan *pl = new mt_plan();
    pl->ix = ix;
    pl->p = *p;
    pl->cap_reads = max_reads;
    pl->cap_bases = max_bases;
    pl->max_len = max_read_len;
    pl->maxE = maxE;
    pl->L = plan_layout(ix, max_bases, max_reads, p->top_n, max_read_len, p->max_occ, true);
    cudaError_t e = alloc_fault() ? cudaErrorMemoryAllocation : cudaMalloc((void **)&pl->ws, pl->L.total);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete pl;
        return e == cudaErrorMemoryAllocation ? MT_ENOMEM : MT_ECUDA;
    }
    if (cudaMallocHost((void **)&pl->h_io, sizeof(IoBlock)) != cudaSuccess ||
        cudaMallocHost((void **)&pl->h_ctr, sizeof(Counters)) != cudaSuccess) {
        cudaFree(pl->ws);
        cudaFreeHost(pl->h_io);
        delete pl;
        return MT_ENOMEM;
    }
    // one chunk per 2^17 reads of capacity, at most MAX_CHUNKS (each chunk is one more seeding
    // launch, whose tail wave costs a little even when the reads are already on the device)
    pl->n_chunks = (uint32_t)std::min<uint64_t>(mt_plan::MAX_CHUNKS, std::max<uint64_t>(1, max_reads >> 17));
    for (uint32_t i = 0; i <= pl->n_chunks; i++) pl->chunk_r[i] = max_reads * i / pl->n_chunks;
    bool ok = cudaStreamCreateWithFlags(&pl->copy_stream, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&pl->ready, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreate(&pl->t_ev[0]) == cudaSuccess && cudaEventCreate(&pl->t_ev[1]) == cudaSuccess;
    for (uint32_t i = 0; ok && i < pl->n_chunks; i++)
        ok = cudaEventCreateWithFlags(&pl->chunk_ev[i], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        cuda_ok(cudaGetLastError(), "plan streams");
        mt_plan_destroy(pl);
        return MT_ECUDA;
    }
    *out = pl;
    return MT_OK;
}

extern "C" uint64_t mt_plan_device_bytes(const mt_plan *pl) { return pl ? pl->L.total : 0; }

extern "C" int mt_plan_classify(mt_plan *pl, const uint8_t *reads, uint64_t n_bases, const uint64_t *offsets,
                                uint64_t n_reads, int device_ptrs, void *stream, int32_t *taxon, uint8_t *nloc,
                                mt_loc *locs, uint64_t *genome_hits, double *abundance, mt_stats *stats) {
    if (!pl || !offsets || (!taxon && n_reads) || (!reads && n_bases)) return MT_EINVAL;
    if (n_reads > pl->cap_reads || n_bases > pl->cap_bases) return MT_EINVAL;
    Trace trace("mt_plan_classify");
    cudaStream_t s = (cudaStream_t)stream;
    const Layout &L = pl->L;
    const uint32_t G = pl->ix->G, top_n = pl->p.top_n;
    const bool host_io = !device_ptrs;
    auto P = [&](size_t off) { return (void *)(pl->ws + off); };
    if (stats) memset(stats, 0, sizeof(*stats));
    uint64_t off0 = 0;
    // reads with bad offsets or above the plan's read length are flagged by the seeding kernel
    // (MT_EINVAL after the call), so host offsets are not scanned here, except the chunk
    // boundaries, which bound the copies (non-decreasing offsets keep a read inside its chunk)
    if (host_io) {
        uint64_t prev = n_reads ? offsets[0] : 0;
        for (uint32_t i = 0; n_reads && i <= pl->n_chunks; i++) {
            const uint64_t o = offsets[std::min(pl->chunk_r[i], n_reads)];
            if (o < prev || o > n_bases) return MT_EINVAL;
            prev = o;
        }
        if (n_reads) off0 = offsets[0];
    } else if (n_reads) {
        MT_CK(cudaMemcpyAsync(&pl->h_ctr->stat[0], offsets, 8, cudaMemcpyDeviceToHost, s));
        MT_CK(cudaStreamSynchronize(s));
        off0 = pl->h_ctr->stat[0];
    }
    IoBlock &io = *pl->h_io;
    io.reads = reads; io.roff = offsets; io.n_reads = n_reads; io.n_bases = n_bases; io.off0 = off0;
    io.max_len = pl->max_len;
    io.taxon = taxon; io.nloc = nloc; io.locs = locs;
    if (host_io) {
        io.reads = (const uint8_t *)P(L.reads);
        io.roff = (const uint64_t *)P(L.roff);
        io.taxon = (int32_t *)P(L.taxon);
        io.nloc = (uint8_t *)P(L.nloc);
        io.locs = locs ? (mt_loc *)P(L.locs) : nullptr;
        MT_CK(cudaMemcpyAsync((void *)io.roff, offsets, (n_reads + 1) * 8, cudaMemcpyHostToDevice, s));
    }
    io.vec_ok = ((uintptr_t)io.reads & 15u) == 0;
    MT_CK(cudaMemcpyAsync(P(L.io), pl->h_io, sizeof(IoBlock), cudaMemcpyHostToDevice, s));
    if (host_io) {   // the reads' bytes, chunk by chunk, after what s has queued
        // (a single chunk goes up on s itself: nothing to overlap)
        cudaStream_t cs = pl->n_chunks > 1 ? pl->copy_stream : s;
        if (cs != s) {
            MT_CK(cudaEventRecord(pl->ready, s));
            MT_CK(cudaStreamWaitEvent(cs, pl->ready, 0));
        }
        for (uint32_t i = 0; i < pl->n_chunks; i++) {
            const uint64_t rb = std::min(pl->chunk_r[i], n_reads), re = std::min(pl->chunk_r[i + 1], n_reads);
            if (re > rb && offsets[re] > offsets[rb])
                MT_CK(cudaMemcpyAsync((uint8_t *)io.reads + offsets[rb], reads + offsets[rb], offsets[re] - offsets[rb],
                                      cudaMemcpyHostToDevice, cs));
            MT_CK(cudaEventRecord(pl->chunk_ev[i], cs));
        }
    } else {
        for (uint32_t i = 0; i < pl->n_chunks; i++) MT_CK(cudaEventRecord(pl->chunk_ev[i], s));
    }

    cudaEvent_t *ev = pl->t_ev;
    if (stats) MT_CK(cudaEventRecord(ev[0], s));
    EnqueueCtx ctx{pl->ix, &pl->p, &L, pl->ws, pl->cap_reads, pl->max_len, pl->maxE, false, nullptr, 0};
    ctx.n_chunks = pl->n_chunks;
    ctx.chunk_r = pl->chunk_r;
    ctx.chunk_ev = pl->chunk_ev;
    int rc = MT_OK;
    if (pl->calls == 0) {
        // the first call runs directly
        rc = enqueue_classify(ctx, s);
        pl->launches = ctx.launches;
    } else {
        if (!pl->exec) {
            // capture on the plan's own stream (the caller's may be the legacy default
            // stream, which cannot be captured); the graph is then launched on the caller's
            ctx.capturing = true;
            if (!pl->cap_stream) MT_CK(cudaStreamCreateWithFlags(&pl->cap_stream, cudaStreamNonBlocking));
            MT_CK(cudaStreamBeginCapture(pl->cap_stream, cudaStreamCaptureModeThreadLocal));
            rc = enqueue_classify(ctx, pl->cap_stream);
            cudaGraph_t g = nullptr;
            cudaError_t e = cudaStreamEndCapture(pl->cap_stream, &g);
            if (rc == MT_OK && !cuda_ok(e, "cudaStreamEndCapture")) rc = MT_ECUDA;
            if (rc == MT_OK && !cuda_ok(cudaGraphInstantiate(&pl->exec, g, 0), "cudaGraphInstantiate")) rc = MT_ECUDA;
            pl->graph = g;
            pl->launches = ctx.launches;
        }
        if (rc == MT_OK) MT_CK(cudaGraphLaunch(pl->exec, s));
    }
    if (rc) return rc;
    if (stats) MT_CK(cudaEventRecord(ev[1], s));
    cudaMemcpyKind kind = host_io ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    if (genome_hits) MT_CK(cudaMemcpyAsync(genome_hits, P(L.ghits), G * 8, kind, s));
    if (abundance) MT_CK(cudaMemcpyAsync(abundance, P(L.abund), G * 8, kind, s));
    if (host_io && n_reads) {
        MT_CK(cudaMemcpyAsync(taxon, io.taxon, n_reads * 4, cudaMemcpyDeviceToHost, s));
        if (nloc) MT_CK(cudaMemcpyAsync(nloc, io.nloc, n_reads, cudaMemcpyDeviceToHost, s));
        if (locs) MT_CK(cudaMemcpyAsync(locs, io.locs, n_reads * top_n * sizeof(mt_loc), cudaMemcpyDeviceToHost, s));
    }
    MT_CK(cudaMemcpyAsync(pl->h_ctr, P(L.ctr), sizeof(Counters), cudaMemcpyDeviceToHost, s));
    MT_CK(cudaStreamSynchronize(s));
    pl->calls++;
    const Counters h = *pl->h_ctr;
    fill_stats(stats, h, n_reads, L.total, pl->launches, nullptr);
    if (stats) {
        float ms = 0;
        cudaEventElapsedTime(&ms, ev[0], ev[1]);
        stats->ms_total = ms;
    }
    return status_of(h.err);
}

extern "C" void mt_plan_destroy(mt_plan *pl) {
    if (!pl) return;
    if (pl->exec) cudaGraphExecDestroy(pl->exec);
    if (pl->graph) cudaGraphDestroy(pl->graph);
    if (pl->cap_stream) cudaStreamDestroy(pl->cap_stream);
    if (pl->copy_stream) {
        cudaStreamSynchronize(pl->copy_stream);
        cudaStreamDestroy(pl->copy_stream);
    }
    for (uint32_t i = 0; i < mt_plan::MAX_CHUNKS; i++)
        if (pl->chunk_ev[i]) cudaEventDestroy(pl->chunk_ev[i]);
    if (pl->ready) cudaEventDestroy(pl->ready);
    for (cudaEvent_t e : pl->t_ev)
        if (e) cudaEventDestroy(e);
    cudaFree(pl->ws);
    cudaFreeHost(pl->h_io);
    cudaFreeHost(pl->h_ctr);
    delete pl;
}
