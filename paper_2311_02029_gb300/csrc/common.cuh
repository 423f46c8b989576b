// Device helpers shared by the GB300 kernels of the MetaTrinity hot path.
//
// Data layout in HBM (all built once per index, then read-only):
//   ref    : 2-bit packed genomes; base j of genome g at bits 2*(j%32) of word
//            gword[g] + j/32, gword[g] = (off[g] >> 5) + g (no overlap, one zero word slack)
//   table  : open-addressing hash table, power-of-two slots of 32 bytes = one DRAM sector:
//              w0 = (code + 1) | ninline << 62    (0 = empty slot)
//              ninline in 1..3 -> w1..w3 hold the occurrences inline
//              ninline == 0    -> w1 = count << 40 | offset into occ[]
//            slot of a key = top bits of (key * 0x9E3779B97F4A7C15) (Fibonacci hashing;
//            minimizer keys are biased towards small values, so their own top bits are not
//            used), linear probing.
//   occ    : every genome minimizer as genome << 33 | pos << 1 | strand, sorted by
//            (code, genome, pos)
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/mt.h"

#define MT_DEV __device__ __forceinline__

// error bits raised by kernels into a device word
enum : uint32_t {
    ERR_BAD_BASE = 1u << 0,
    ERR_BAD_OFFSETS = 1u << 1,
    ERR_READ_TOO_LONG = 1u << 2,
    ERR_BAD_PAIR = 1u << 3,
    ERR_PROBE_LIMIT = 1u << 4,
    ERR_SCRATCH = 1u << 5,
};

static constexpr uint64_t CODE_MASK62 = (1ull << 62) - 1;
static constexpr uint64_t EVEN_BITS = 0x5555555555555555ull;
static constexpr uint64_t OFF_MASK40 = (1ull << 40) - 1;
static constexpr uint32_t DIAG_BIAS = 1u << 11;   // > MT_MAX_READ_LEN: biased diagonals are >= 0

// Key of a k-mer code: the SplitMix64 finaliser (Steele, Lea & Flood, OOPSLA 2014). A
// bijection on 64-bit words, so distinct codes never collide.
MT_DEV uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

MT_DEV uint64_t slot_of(uint64_t key, uint32_t shift) {
    return (key * 0x9E3779B97F4A7C15ull) >> shift;
}

// Key filter of an index: one 64-bit block per key, picked by the top bits of another
// multiplicative hash; three bits from the key's low 18 bits (minimizer keys are small, so
// their low bits carry the entropy). A key in the index always passes; another passes with
// the blocks' fill rate cubed.
MT_DEV uint64_t filter_block(uint64_t key, uint32_t shift) {
    return (key * 0xD6E8FEB86659FD93ull) >> shift;
}
MT_DEV uint64_t filter_bits(uint64_t key) {
    return (1ull << (key & 63)) | (1ull << ((key >> 6) & 63)) | (1ull << ((key >> 12) & 63));
}

// ASCII -> 2-bit code (A0 C1 G2 T3); sets *bad for any other byte.
MT_DEV uint32_t base_code(uint32_t b, bool &bad) {
    uint32_t c = (b >> 1) & 3u;      // A->0 C->1 G->3 T->2
    c ^= (c >> 1);                    // swap G/T
    bad |= !(b == 'A' || b == 'C' || b == 'G' || b == 'T');
    return c;
}

// 32 bases starting at base `pos` of a packed array (pos >= 0; reads words pos/32, pos/32+1).
MT_DEV uint64_t get32(const uint64_t *s, uint32_t pos) {
    uint32_t wi = pos >> 5, sh = (pos & 31u) * 2u;
    uint64_t a = s[wi], b = s[wi + 1];
    return (a >> sh) | ((b << 1) << (63u - sh));
}

// Reverse the order of the 32 two-bit groups of a word.
MT_DEV uint64_t rev2(uint64_t x) {
    x = __brevll(x);
    return ((x >> 1) & EVEN_BITS) | ((x & EVEN_BITS) << 1);
}

// k-mer code at base i of a packed sequence: x holds bases i.. i+k-1 little-endian
// (base i in the low bits). Forward code reads the k-mer with its first base most
// significant; the reverse-complement code is x complemented (base i+t weighs 4^t).
MT_DEV void kmer_codes(uint64_t x, uint32_t k, uint64_t &fwd, uint64_t &rc) {
    const uint64_t mask = (k == 32) ? ~0ull : ((1ull << (2 * k)) - 1);
    x &= mask;
    rc = x ^ mask;
    fwd = rev2(x) >> (64 - 2 * k);
}

MT_DEV void canon(uint64_t fwd, uint64_t rc, uint32_t canonical, uint64_t &code, uint32_t &strand) {
    if (canonical && rc < fwd) { code = rc; strand = 1; }
    else { code = fwd; strand = 0; }
}

// Look a code up. Returns its occurrence count (0 = absent) and either the inline
// occurrences (o0..o2) or the offset of its list in occ[].
struct Lookup {
    uint32_t cnt;
    uint32_t ninline;
    uint64_t off;
    uint64_t o[3];
};

struct IndexView {
    const ulonglong2 *table;    // 2 x ulonglong2 per slot
    uint64_t slot_mask;
    uint32_t slot_shift;
    uint32_t G;
    const uint64_t *occ;
    const uint64_t *ref;        // packed genomes
    const uint64_t *gword;      // first word of genome g in ref
    const uint64_t *glen;       // genome lengths (bases)
    uint32_t k, w, canonical;
    uint32_t hk_db;             // diagonal bits of 32-bit match keys (0: keys need 64 bits)
};

MT_DEV Lookup probe(const IndexView &ix, uint64_t code, uint64_t key, uint32_t *err) {
    Lookup L;
    L.cnt = 0; L.ninline = 0; L.off = 0; L.o[0] = L.o[1] = L.o[2] = 0;
    uint64_t s = slot_of(key, ix.slot_shift);
    const uint64_t want = code + 1;
    for (uint64_t it = 0; it <= ix.slot_mask; it++) {
        ulonglong2 a = __ldg(&ix.table[2 * s]);
        if (a.x == 0) return L;
        if ((a.x & CODE_MASK62) == want) {
            uint32_t ni = (uint32_t)(a.x >> 62);
            if (ni == 0) {
                L.cnt = (uint32_t)(a.y >> 40);
                L.off = a.y & OFF_MASK40;
            } else {
                L.cnt = ni; L.ninline = ni;
                L.o[0] = a.y;
                if (ni > 1) {
                    ulonglong2 b = __ldg(&ix.table[2 * s + 1]);
                    L.o[1] = b.x; L.o[2] = b.y;
                }
            }
            return L;
        }
        s = (s + 1) & ix.slot_mask;
    }
    atomicOr(err, ERR_PROBE_LIMIT);
    return L;
}

MT_DEV uint64_t occ_at(const IndexView &ix, const Lookup &L, uint32_t t) {
    return L.ninline ? L.o[t] : __ldg(&ix.occ[L.off + t]);
}

// Seed-match key: genome << 34 | rel << 33 | (diag + DIAG_BIAS). Sorting these keys sorts
// matches by (genome, relative strand, diagonal).
MT_DEV uint64_t hit_key(uint64_t occ, uint32_t rpos, uint32_t rstrand, uint32_t n, uint32_t k) {
    uint64_t g = occ >> 33;
    int64_t gpos = (int64_t)((occ >> 1) & 0xFFFFFFFFull);
    uint32_t rel = (uint32_t)(occ & 1u) ^ rstrand;
    int64_t rp = rel ? (int64_t)(n - k - rpos) : (int64_t)rpos;
    int64_t diag = gpos - rp;
    return (g << 34) | ((uint64_t)rel << 33) | (uint64_t)(diag + DIAG_BIAS);
}
MT_DEV uint32_t hk_genome(uint64_t h) { return (uint32_t)(h >> 34); }
MT_DEV uint32_t hk_rel(uint64_t h) { return (uint32_t)((h >> 33) & 1u); }
MT_DEV int64_t hk_diag(uint64_t h) { return (int64_t)(h & ((1ull << 33) - 1)) - DIAG_BIAS; }

__host__ __device__ __forceinline__ uint32_t edit_threshold(uint32_t n, uint32_t e_abs, uint32_t e_permille) {
    return e_permille ? (uint32_t)(((uint64_t)n * e_permille) / 1000u) : e_abs;
}

// Per-call inputs and outputs of a classification, read by the kernels from device memory so
// that one captured CUDA graph serves every batch up to its capacity.
struct IoBlock {
    const uint8_t *reads;
    const uint64_t *roff;
    uint64_t n_reads, n_bases, off0;
    uint32_t vec_ok, max_len;
    int32_t *taxon;
    uint8_t *nloc;
    mt_loc *locs;
};

// Location record kept between the seeding and selection passes (16 bytes).
struct Cluster {
    uint64_t hkey;     // hit key of its first match (genome, rel, first diagonal)
    uint32_t seeds;
    uint32_t pad;      // seeding pass: the read's minimizer count (candidate order); else 0
};

// Word index of packed sequence i for base offsets relative to off0.
MT_DEV uint64_t seq_word(uint64_t off_i, uint64_t off0, uint64_t i) {
    return ((off_i - off0) >> 5) + i;
}

MT_DEV uint64_t umin64(uint64_t a, uint64_t b) { return a < b ? a : b; }

MT_DEV unsigned lane_id() { return threadIdx.x & 31u; }

template <typename T>
MT_DEV T warp_incl_scan(T v) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T u = __shfl_up_sync(0xffffffffu, v, o);
        if ((int)lane_id() >= o) v += u;
    }
    return v;
}
