// Edit-distance approximation stage: kernels, the two execution forms and the autotuner.
//
//   plain   : one launch per read-length bucket, one warp (32 lanes) per pair, a
//             non-persistent grid sized to the bucket.
//   batched : one persistent launch (grid = SMs x resident CTAs) over all pairs, ordered by
//             edit threshold E for SneakySnake and SHD (so a warp's pairs walk the same number
//             of diagonals), by edit-threshold class for the O(n) approximations; warps
//             steal chunks of pairs from a global counter; each edit-threshold class runs with
//             the shape (lanes per pair, pairs per chunk, CTA size) picked by the autotuner,
//             which runs only when asked (mt_eda_batch_autotune, mt_classify_autotune).
// Both forms stage each pair's packed read and window in shared memory and run the same
// walk, so their distances are identical.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "eda.cuh"
#include "internal.h"

namespace mt {

static constexpr unsigned FULL = 0xffffffffu;
static constexpr int EDA_THREADS = 256;          // CTA size of the plain form and the default
static constexpr int EDA_MAX_THREADS = 1024;     // largest CTA size the tuner tries
static constexpr uint32_t EDA_CHUNK = 128;       // default pairs per steal
static constexpr int MAX_CLASSES = 8;
static constexpr uint32_t E_KEYS = MT_MAX_E + 1;  // exact edit thresholds (batched ordering)
static constexpr uint32_t CURSOR_WORDS = 256;     // scatter cursors (<= E_KEYS or 33), then the steal counter
static constexpr uint32_t COUNTER_AT = 192;

struct PairInfo {
    uint32_t n, E;
    int32_t lo, hi;
    bool edges;
};

// ---- pair sources ---------------------------------------------------------------------------
// Pairs of the EDA-only call: read and window are packed sets (word start = off >> 5 + i).
struct BatchSrc {
    const uint64_t *rw, *roff, *ww, *woff;
    const uint32_t *pair_read;
    const uint16_t *E;
    uint8_t *dist;

    template <int G>
    MT_DEV PairInfo stage(uint64_t p, uint64_t *rd, uint64_t *wn, uint32_t gl) const {
        uint32_t r = pair_read[p];
        uint64_t r0 = roff[r];
        uint32_t n = (uint32_t)(roff[r + 1] - r0);
        uint32_t E_ = E[p];
        const uint64_t *rs = rw + (r0 >> 5) + r;
        const uint64_t *ws = ww + (woff[p] >> 5) + p;
        uint32_t nr = (n + 31) / 32, nwn = (n + 2 * E_ + 31) / 32;
#pragma unroll 4
        for (uint32_t t = gl; t < nr + 2; t += G) rd[t] = t < nr ? __ldg(rs + t) : 0ull;
#pragma unroll 4
        for (uint32_t t = gl; t < nwn + 3; t += G) wn[t] = t < nwn ? __ldg(ws + t) : 0ull;
        PairInfo pi;
        pi.n = n; pi.E = E_; pi.lo = 0; pi.hi = (int32_t)(n + 2 * E_); pi.edges = false;
        return pi;
    }
    MT_DEV void finish(uint64_t p, uint32_t d) const { dist[p] = (uint8_t)d; }
};

// 32 bases of a genome starting at `pos` (may lie outside the genome; those bits are
// don't-care and are masked as obstacles by the caller). Reads only words 0..nwg of it.
// Staging loads go through the read-only path, so that a staging loop's loads (the staged
// words are stored to shared memory between them) can all be in flight together.
MT_DEV uint64_t genome_get32(const uint64_t *g, uint64_t nwg, int64_t pos) {
    int64_t wi = pos >> 5;
    uint32_t sh = (uint32_t)(pos & 31) * 2u;
    uint64_t a = (wi >= 0 && wi <= (int64_t)nwg) ? __ldg(g + wi) : 0ull;
    uint64_t b = (wi + 1 >= 0 && wi + 1 <= (int64_t)nwg) ? __ldg(g + wi + 1) : 0ull;
    return (a >> sh) | ((b << 1) << (63u - sh));
}

// get32 of a packed sequence in global memory, through the read-only path.
MT_DEV uint64_t ldg_get32(const uint64_t *s, uint32_t pos) {
    const uint32_t wi = pos >> 5, sh = (pos & 31u) * 2u;
    const uint64_t a = __ldg(s + wi), b = __ldg(s + wi + 1);
    return (a >> sh) | ((b << 1) << (63u - sh));
}

// Candidates of the classification pipeline: the read (reverse-complemented for strand 1)
// against its genome window [d0 - E, d0 + n + E); window bases outside the genome are
// obstacles.
struct ClassifySrc {
    IndexView ix;
    const uint64_t *rw;
    const IoBlock *io;
    const uint32_t *cl;      // compact candidate slots
    const Cluster *cand;     // per slot (read * top_n + t)
    uint32_t top_n, e_abs, e_permille;
    uint8_t *dist;           // per slot

    template <int G>
    MT_DEV PairInfo stage(uint64_t i, uint64_t *rd, uint64_t *wn, uint32_t gl) const {
        uint32_t s = cl[i];
        uint32_t r = s / top_n;
        Cluster c = cand[s];
        const uint64_t *roff = io->roff;
        uint64_t ro = roff[r];
        uint32_t n = (uint32_t)(roff[r + 1] - ro);
        uint32_t E = edit_threshold(n, e_abs, e_permille);
        const uint64_t *rs = rw + seq_word(ro, io->off0, r);
        uint32_t nr = (n + 31) / 32;
        if (hk_rel(c.hkey)) {
#pragma unroll 4
            for (uint32_t t = gl; t < nr + 2; t += G) {
                uint64_t x = 0;
                if (t < nr) {
                    int32_t st = (int32_t)n - 32 * (int32_t)(t + 1);
                    x = st >= 0 ? ldg_get32(rs, (uint32_t)st) : (ldg_get32(rs, 0) << (2 * (uint32_t)(-st)));
                    x = ~rev2(x);
                }
                rd[t] = x;
            }
        } else {
#pragma unroll 4
            for (uint32_t t = gl; t < nr + 2; t += G) rd[t] = t < nr ? __ldg(rs + t) : 0ull;
        }
        uint32_t g = hk_genome(c.hkey);
        int64_t wstart = hk_diag(c.hkey) - (int64_t)E;
        uint64_t glen = ix.glen[g];
        uint64_t nwg = (glen + 31) / 32;
        const uint64_t *gp = ix.ref + ix.gword[g];
        uint32_t L = n + 2 * E, nwn = (L + 31) / 32;
#pragma unroll 4
        for (uint32_t t = gl; t < nwn + 3; t += G)
            wn[t] = t < nwn ? genome_get32(gp, nwg, wstart + 32 * (int64_t)t) : 0ull;
        int64_t lo = -wstart, hi = (int64_t)glen - wstart;
        lo = lo < 0 ? 0 : (lo > L ? L : lo);
        hi = hi < 0 ? 0 : (hi > L ? L : hi);
        PairInfo pi;
        pi.n = n; pi.E = E; pi.lo = (int32_t)lo; pi.hi = (int32_t)hi;
        pi.edges = (lo > 0) || (hi < (int64_t)L);
        return pi;
    }
    MT_DEV void finish(uint64_t i, uint32_t d) const { dist[cl[i]] = (uint8_t)d; }
};

// ---- kernels -----------------------------------------------------------------------------------
struct EdaPlan {
    uint32_t n_classes;
    uint32_t groups_max;               // 32 / smallest G in the plan (sets the smem layout)
    uint32_t cta;                      // threads per CTA of the launch
    uint32_t G[MAX_CLASSES];
    uint32_t chunk[MAX_CLASSES];       // pairs per steal
    uint64_t begin[MAX_CLASSES], end[MAX_CLASSES];
    const uint64_t *dyn_end;           // if set: class 0 ends at *dyn_end (device count)
    uint64_t cap;                      // if set: class 0 holds at most `cap` items (tuning samples)
    uint32_t lanes;                    // SneakySnake with G = 1 in every class: lanes refilled one by one
};

// The approximation A of one staged pair by the G lanes of gmask; xb: the group's extra
// shared words (q-gram histogram or SHD mask).
template <int A, int G, bool EDGES>
MT_DEV uint32_t approx(const uint64_t *rd, const uint64_t *wn, const PairInfo &pi, unsigned gmask, uint32_t gl,
                       uint64_t *xb) {
    if (A == ALGO_HD) return hamming_est<G, EDGES>(rd, wn, pi.n, pi.E, pi.lo, pi.hi, gmask, gl);
    if (A == ALGO_BC) return basecount_est<G, EDGES>(rd, wn, pi.n, pi.E, pi.lo, pi.hi, gmask, gl);
    if (A == ALGO_QGRAM) return qgram_est<EDGES>(rd, wn, pi.n, pi.E, pi.lo, pi.hi, reinterpret_cast<int *>(xb));
    if (A == ALGO_SHD)
        return shd_est<G, EDGES>(rd, wn, pi.n, pi.E, pi.lo, pi.hi, gmask, gl, reinterpret_cast<unsigned long long *>(xb));
    if (G == 32 && (2 * pi.E + 1 + G - 1) / G <= SNAKE_TMAX)   // whole-warp groups: registers to spare
        return sneaky_walk_cached<G, EDGES>(rd, wn, pi.n, pi.E, pi.lo, pi.hi, gmask, gl);
    return sneaky_walk<G, EDGES>(rd, wn, pi.n, pi.E, pi.lo, pi.hi, gmask, gl);
}

// Shared words a group needs beyond the read and window for approximation A (the q-gram
// histogram gets one word of slack so that it can start on a 16-byte boundary).
__host__ __device__ __forceinline__ uint32_t eda_extra_words(int A, uint32_t maxn) {
    return A == ALGO_QGRAM ? QGRAM_BINS / 2 + 1 : (A == ALGO_SHD ? (maxn + 31) / 32 + 1 : 0u);
}

template <int G, int A, class Src>
MT_DEV void do_items(const Src &src, const uint32_t *perm, uint64_t b, uint64_t e, uint64_t *wbase,
                     uint32_t rww, uint32_t www, uint32_t xw) {
    constexpr uint32_t groups = 32 / G;
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t gi = lane / G, gl = lane % G;
    const unsigned gmask = (G == 32) ? FULL : (((1u << G) - 1u) << (gi * G));
    uint64_t *rd = wbase + (uint64_t)gi * (rww + www + xw);
    uint64_t *wn = rd + rww;
    uint64_t *xb = wn + www;
    if (A == ALGO_QGRAM) {   // the histogram starts at zero; each pair leaves it at zero
        xb = reinterpret_cast<uint64_t *>((reinterpret_cast<uintptr_t>(xb) + 15) & ~static_cast<uintptr_t>(15));
        for (uint32_t t = gl; t < QGRAM_BINS / 2; t += G) xb[t] = 0;
        __syncwarp(gmask);
    }
    for (uint64_t it = b + gi; it < e; it += groups) {
        uint64_t item = perm ? perm[it] : it;
        PairInfo pi = src.template stage<G>(item, rd, wn, gl);
        __syncwarp(gmask);
        uint32_t d = pi.edges ? approx<A, G, true>(rd, wn, pi, gmask, gl, xb)
                              : approx<A, G, false>(rd, wn, pi, gmask, gl, xb);
        if (gl == 0) src.finish(item, d);
        __syncwarp(gmask);
    }
}

// One step of the SneakySnake walk of one lane over all 2E+1 diagonals of its pair (the G = 1
// case of sneaky_walk, no window bases outside the genome): from column c, the furthest
// column any diagonal's zero run reaches.
MT_DEV uint32_t snake_step(const uint64_t *rd, const uint64_t *wn, uint32_t n, uint32_t ndiag, uint32_t c) {
    return snake_diagonals<false>(rd, wn, n, c, 0, ndiag, 0, 0, c);
}

// SneakySnake with one lane per pair, each lane refilled on its own: every pass of the loop,
// lanes without a pair take the next items of the warp's chunk (a new chunk is stolen from
// the shared counter when it runs out), stage them in their own shared words, and then every
// lane holding a pair makes one walk step. Lanes whose pairs end early take new ones instead
// of idling until the warp's slowest pair ends, so the warp's lanes stay on the same steps
// (same instructions) until the last chunk runs out. A pair whose window reaches outside its
// genome is walked at once with the edge-masked walk. Same distances as sneaky_walk.
template <class Src>
MT_DEV void snake_lanes(const Src &src, const uint32_t *perm, const EdaPlan &plan, unsigned long long *counter,
                        const uint64_t (&pref)[MAX_CLASSES + 1], uint64_t total, uint64_t end0, uint64_t *wbase,
                        uint32_t rww, uint32_t www) {
    const uint32_t lane = threadIdx.x & 31u;
    uint64_t *rd = wbase + (uint64_t)lane * (rww + www);
    uint64_t *wn = rd + rww;
    uint64_t cb = 0, ce = 0;       // the warp's chunk: next unassigned item, end
    bool more = true;              // chunks left to steal
    bool busy = false;             // this lane holds a pair
    uint64_t item = 0;
    uint32_t n = 0, E = 0, c = 0, cnt = 0;
    while (true) {
        // hand the chunk's next items to the lanes without a pair (warp-uniform)
        unsigned idle = __ballot_sync(FULL, !busy);
        bool fresh = false;
        while (idle && more) {
            if (cb == ce) {
                unsigned long long id = 0;
                if (lane == 0) id = atomicAdd(counter, 1ull);
                id = __shfl_sync(FULL, id, 0);
                if (id >= total) { more = false; break; }
                uint32_t k = 0;
                while (id >= pref[k + 1]) k++;
                const uint64_t e = k == 0 ? end0 : plan.end[k];
                cb = plan.begin[k] + (id - pref[k]) * plan.chunk[k];
                ce = cb + plan.chunk[k] < e ? cb + plan.chunk[k] : e;
            }
            const uint32_t take = (uint32_t)min((uint64_t)__popc(idle), ce - cb);
            const uint32_t rank = __popc(idle & ((1u << lane) - 1u));
            if (!busy && rank < take) {
                item = perm ? perm[cb + rank] : cb + rank;
                busy = fresh = true;
            }
            cb += take;
            idle = __ballot_sync(FULL, !busy);
        }
        if (!__any_sync(FULL, busy)) break;
        if (fresh) {
            const PairInfo pi = src.template stage<1>(item, rd, wn, 0);
            n = pi.n; E = pi.E; c = 0; cnt = 0;
            if (pi.edges) {   // rare: a window overhanging a genome end
                src.finish(item, sneaky_walk<1, true>(rd, wn, pi.n, pi.E, pi.lo, pi.hi, 1u << lane, 0));
                busy = false;
            }
        }
        if (busy) {
            bool done = c >= n;
            if (!done) {
                c = snake_step(rd, wn, n, 2 * E + 1, c);
                if (c >= n) done = true;
                else if (++cnt > E) done = true;
                else if (++c >= n) done = true;
            }
            if (done) {
                src.finish(item, cnt < E + 1 ? cnt : E + 1);
                busy = false;
            }
        }
    }
}

template <class Src, int A>
__global__ void __launch_bounds__(EDA_MAX_THREADS) k_eda_persistent(Src src, const uint32_t *perm, EdaPlan plan,
                                                                    unsigned long long *counter,
                                                                    uint32_t rww, uint32_t www, uint32_t xw) {
    extern __shared__ uint64_t sm[];
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
    uint64_t *wbase = sm + (uint64_t)warp * plan.groups_max * (rww + www + xw);
    // chunk table: chunks of plan.chunk[c] items per class
    uint64_t pref[MAX_CLASSES + 1];
    pref[0] = 0;
    uint64_t end0 = plan.dyn_end ? *plan.dyn_end : plan.end[0];
    if (plan.cap && end0 > plan.begin[0] + plan.cap) end0 = plan.begin[0] + plan.cap;
    for (uint32_t c = 0; c < plan.n_classes; c++) {
        uint64_t e = c == 0 ? end0 : plan.end[c];
        uint64_t cnt = e > plan.begin[c] ? e - plan.begin[c] : 0;
        pref[c + 1] = pref[c] + (cnt + plan.chunk[c] - 1) / plan.chunk[c];
    }
    const uint64_t total = pref[plan.n_classes];
    if (A == ALGO_SNAKE && plan.lanes) {
        snake_lanes(src, perm, plan, counter, pref, total, end0, wbase, rww, www);
        return;
    }
    while (true) {
        unsigned long long id = 0;
        if (lane == 0) id = atomicAdd(counter, 1ull);
        id = __shfl_sync(FULL, id, 0);
        if (id >= total) break;
        uint32_t c = 0;
        while (id >= pref[c + 1]) c++;
        uint64_t e = c == 0 ? end0 : plan.end[c];
        uint64_t b = plan.begin[c] + (id - pref[c]) * plan.chunk[c];
        uint64_t ee = b + plan.chunk[c] < e ? b + plan.chunk[c] : e;
        if (A == ALGO_QGRAM) {   // one histogram per warp: a whole warp per pair
            do_items<32, A>(src, perm, b, ee, wbase, rww, www, xw);
            continue;
        }
        switch (plan.G[c]) {
            case 1: do_items<1, A>(src, perm, b, ee, wbase, rww, www, xw); break;
            case 2: do_items<2, A>(src, perm, b, ee, wbase, rww, www, xw); break;
            case 4: do_items<4, A>(src, perm, b, ee, wbase, rww, www, xw); break;
            case 8: do_items<8, A>(src, perm, b, ee, wbase, rww, www, xw); break;
            case 16: do_items<16, A>(src, perm, b, ee, wbase, rww, www, xw); break;
            default: do_items<32, A>(src, perm, b, ee, wbase, rww, www, xw); break;
        }
    }
}

// plain form: one warp per item of [begin, end) (end from *dyn_end when given)
template <class Src, int A>
__global__ void __launch_bounds__(EDA_THREADS) k_eda_plain(Src src, const uint32_t *perm, uint64_t begin,
                                                           uint64_t end, const uint64_t *dyn_end,
                                                           uint32_t rww, uint32_t www, uint32_t xw) {
    extern __shared__ uint64_t sm[];
    const uint32_t warp = threadIdx.x >> 5;
    uint64_t e = dyn_end ? *dyn_end : end;
    uint64_t it = begin + (uint64_t)blockIdx.x * (EDA_THREADS / 32) + warp;
    if (it >= e) return;
    do_items<32, A>(src, perm, it, it + 1, sm + (uint64_t)warp * (rww + www + xw), rww, www, xw);
}

// ---- bucketing of EDA-only pairs -----------------------------------------------------------------
// class of a pair for the batched form (by E), bucket for the plain form (by read words)
__host__ __device__ __forceinline__ uint32_t e_class(uint32_t E) {
    uint32_t c = 0;
    while (c + 1 < MAX_CLASSES && E >= (2u << c)) c++;
    return c;   // [0,1] [2,3] [4,7] [8,15] [16,31] [32,63] [64,127] [128+]
}

struct BucketStats {
    unsigned long long cls_count[MAX_CLASSES];
    unsigned long long bkt_count[33];
    unsigned long long e_count[E_KEYS];   // pairs per exact edit threshold
    unsigned int cls_maxn[MAX_CLASSES], cls_maxE[MAX_CLASSES];
    unsigned int bkt_maxE[33];
    unsigned int maxn, maxE, err;
};

// Per-pair checks and the buckets' statistics. Every count and maximum is gathered per CTA in
// shared memory (32-bit) and reaches the global statistics once per CTA: class counts and
// maximum thresholds follow from the per-threshold counts.
__global__ void k_bucket_count(const uint64_t *roff, uint64_t n_reads, const uint64_t *woff,
                               const uint32_t *pair_read, const uint16_t *E, uint64_t n_pairs,
                               BucketStats *st) {
    __shared__ unsigned int se[E_KEYS], sb[33], s_cmaxn[MAX_CLASSES], s_bmaxE[33], s_err;
    for (int i = threadIdx.x; i < (int)E_KEYS; i += blockDim.x) se[i] = 0;
    for (int i = threadIdx.x; i < 33; i += blockDim.x) { sb[i] = 0; s_bmaxE[i] = 0; }
    for (int i = threadIdx.x; i < MAX_CLASSES; i += blockDim.x) s_cmaxn[i] = 0;
    if (threadIdx.x == 0) s_err = 0;
    __syncthreads();
    for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n_pairs;
         p += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t r = pair_read[p];
        if (r >= n_reads) { s_err = ERR_BAD_PAIR; continue; }
        const uint64_t r0 = roff[r], r1 = roff[r + 1];
        uint64_t n64 = r1 - r0;
        uint32_t e = E[p];
        uint64_t L = woff[p + 1] - woff[p];
        if (r1 < r0 || n64 > MT_MAX_READ_LEN || e > MT_MAX_E || L != n64 + 2ull * e) {
            s_err = ERR_BAD_PAIR;
            continue;
        }
        uint32_t n = (uint32_t)n64;
        uint32_t b = (n + 31) / 32;
        atomicAdd(&se[e], 1u);
        atomicAdd(&sb[b], 1u);
        atomicMax(&s_cmaxn[e_class(e)], n);
        atomicMax(&s_bmaxE[b], e);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (s_err) atomicOr(&st->err, s_err);
        unsigned int maxn = 0, maxE = 0;
        for (int c = 0; c < MAX_CLASSES; c++) {
            if (s_cmaxn[c]) atomicMax(&st->cls_maxn[c], s_cmaxn[c]);
            maxn = max(maxn, s_cmaxn[c]);
        }
        for (int e = 0; e < (int)E_KEYS; e++) if (se[e]) maxE = e;
        if (maxn) atomicMax(&st->maxn, maxn);
        if (maxE) atomicMax(&st->maxE, maxE);
    }
    if (threadIdx.x < MAX_CLASSES) {   // class c: its thresholds' counts and largest threshold
        const int c = threadIdx.x;
        unsigned long long cnt = 0;
        unsigned int me = 0;
        for (int e = 0; e < (int)E_KEYS; e++)
            if ((int)e_class(e) == c && se[e]) { cnt += se[e]; me = e; }
        if (cnt) {
            atomicAdd(&st->cls_count[c], cnt);
            atomicMax(&st->cls_maxE[c], me);
        }
    }
    for (int i = threadIdx.x; i < 33; i += blockDim.x) {
        if (sb[i]) atomicAdd(&st->bkt_count[i], (unsigned long long)sb[i]);
        if (s_bmaxE[i]) atomicMax(&st->bkt_maxE[i], s_bmaxE[i]);
    }
    for (int i = threadIdx.x; i < (int)E_KEYS; i += blockDim.x)
        if (se[i]) atomicAdd(&st->e_count[i], (unsigned long long)se[i]);
}

// Segment keys of the scatter: the plain form's read-word buckets; for the batched form the
// exact edit threshold when the approximation's work grows with E (SneakySnake and SHD walk
// 2E+1 diagonals, so a warp of equal E keeps its lanes busy alike; classes stay contiguous
// since the class grows with E), else the edit-threshold class (HD, Base Counting and q-gram
// are O(n), and coarser segments keep neighbouring pairs' windows together).
enum ScatterKey : int { KEY_WORDS = 0, KEY_E = 1, KEY_CLASS = 2 };

// Scatters pair ids into segments of one key; cursor[] starts at the segment starts. A CTA takes
// tiles of one pair a thread: the tile's pairs are ranked per key in shared memory, the tile
// reserves each key's range with one global add, and every pair goes to its place (the order
// within a segment changes no result).
__global__ void k_bucket_scatter(const uint64_t *roff, const uint32_t *pair_read, const uint16_t *E,
                                 uint64_t n_pairs, int key_kind, unsigned long long *cursor,
                                 uint32_t *perm) {
    __shared__ unsigned int s_cnt[E_KEYS];
    __shared__ unsigned long long s_base[E_KEYS];
    const uint32_t nkeys = key_kind == KEY_E ? E_KEYS : key_kind == KEY_CLASS ? MAX_CLASSES : 33;
    for (uint64_t p0 = (uint64_t)blockIdx.x * blockDim.x; p0 < n_pairs; p0 += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t p = p0 + threadIdx.x;
        const bool ok = p < n_pairs;
        uint32_t key = 0;
        if (ok) {
            const uint32_t r = pair_read[p];
            const uint32_t n = (uint32_t)(roff[r + 1] - roff[r]);
            key = key_kind == KEY_E ? (uint32_t)E[p] : key_kind == KEY_CLASS ? e_class(E[p]) : (n + 31) / 32;
        }
        for (uint32_t i = threadIdx.x; i < nkeys; i += blockDim.x) s_cnt[i] = 0;
        __syncthreads();
        const uint32_t rank = ok ? atomicAdd(&s_cnt[key], 1u) : 0u;
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < nkeys; i += blockDim.x)
            if (s_cnt[i]) s_base[i] = atomicAdd(&cursor[i], (unsigned long long)s_cnt[i]);
        __syncthreads();
        if (ok) perm[s_base[key] + rank] = (uint32_t)p;
        __syncthreads();   // s_cnt and s_base are reused by the next tile
    }
}

// ---- launch helpers --------------------------------------------------------------------------------
// Group shapes: words of one group (read, window, extra) for the largest pair of a launch.
struct EdaShape {
    uint32_t rww, www, xw;
};

// The words a group takes are odd in number, so that the groups of a warp (one lane each
// when G = 1) reach their 8-byte words in different shared-memory banks.
static EdaShape eda_shape(int A, uint32_t maxn, uint32_t maxE) {
    EdaShape w{eda_read_words(maxn), eda_win_words(maxn, maxE), eda_extra_words(A, maxn)};
    if ((w.rww + w.www + w.xw) % 2 == 0) w.www++;
    return w;
}

static constexpr size_t EDA_SMEM_MAX = 200 * 1024;

static size_t eda_smem(uint32_t warps, uint32_t groups_per_warp, const EdaShape &w) {
    return (size_t)warps * groups_per_warp * (w.rww + w.www + w.xw) * 8;
}

template <int A, class Src>
static int launch_persistent(const Src &src, const uint32_t *perm, const EdaPlan &plan,
                             unsigned long long *counter, const EdaShape &w, cudaStream_t s) {
    const uint32_t cta = plan.cta ? plan.cta : EDA_THREADS;
    size_t smem = eda_smem(cta / 32, plan.groups_max, w);
    if (smem > EDA_SMEM_MAX || cta > EDA_MAX_THREADS || cta % 32) return MT_EINVAL;
    static std::mutex mu;
    {
        std::lock_guard<std::mutex> lk(mu);
        MT_CK(cudaFuncSetAttribute(k_eda_persistent<Src, A>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)EDA_SMEM_MAX));
    }
    int per_sm = 0;
    MT_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_eda_persistent<Src, A>, (int)cta, smem));
    if (per_sm < 1) per_sm = 1;
    unsigned grid = (unsigned)(sm_count() * per_sm);
    MT_CK(cudaMemsetAsync(counter, 0, 8, s));
    k_eda_persistent<Src, A><<<grid, cta, smem, s>>>(src, perm, plan, counter, w.rww, w.www, w.xw);
    MT_CK(cudaGetLastError());
    return MT_OK;
}

template <int A, class Src>
static int launch_plain(const Src &src, const uint32_t *perm, uint64_t begin, uint64_t end,
                        const uint64_t *dyn_end, const EdaShape &w, cudaStream_t s) {
    if (end <= begin) return MT_OK;
    size_t smem = eda_smem(EDA_THREADS / 32, 1, w);
    if (smem > EDA_SMEM_MAX) return MT_EINVAL;
    static std::mutex mu;
    {
        std::lock_guard<std::mutex> lk(mu);
        MT_CK(cudaFuncSetAttribute(k_eda_plain<Src, A>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)EDA_SMEM_MAX));
    }
    uint64_t warps = end - begin;
    uint64_t blocks = (warps + EDA_THREADS / 32 - 1) / (EDA_THREADS / 32);
    while (blocks > 0) {   // grid.x is limited to 2^31-1 blocks
        uint64_t nb = std::min<uint64_t>(blocks, (1ull << 31) - 1);
        k_eda_plain<Src, A><<<(unsigned)nb, EDA_THREADS, smem, s>>>(src, perm, begin, end, dyn_end, w.rww, w.www, w.xw);
        MT_CK(cudaGetLastError());
        begin += nb * (EDA_THREADS / 32);
        blocks -= nb;
    }
    return MT_OK;
}

// ---- autotuner ---------------------------------------------------------------------------------------
// The batched form's shape for each approximation and edit-threshold class: lanes per pair G,
// pairs per steal chunk and CTA size. Searched only when a caller asks
// (mt_eda_batch_autotune, mt_classify_autotune) on a sample of that call's own pairs, in
// three stages: G in {1, 2, 4, 8, 16, 32} at the default chunk and CTA size, then the chunk in
// {32, 64, 128, 256} with the best G (for SneakySnake with G = 1, lockstep lanes or lanes
// refilled one by one, whichever is faster, first), then the CTA size in {128, 256, 512, 1024};
// each candidate is
// launched twice and its second time counts. The result is kept per device for every later
// call; a class never tuned runs the default shape. q-gram always takes a whole warp per pair
// (one histogram per warp), so only its chunk and CTA size are searched.
static constexpr int N_ALGOS = 5;
struct TunedShape {
    uint32_t G, chunk, cta;
    uint32_t refill;   // SneakySnake, G = 1: lanes take a new pair as soon as theirs ends
};
struct TuneCache {
    std::mutex mu;
    TunedShape sh[64][N_ALGOS][2 * MAX_CLASSES];   // per device and algorithm: EDA-only classes, then classification classes
    TuneCache() { memset(sh, 0, sizeof(sh)); }
};
static TuneCache g_tune;

static uint32_t default_G(uint32_t E) {
    uint32_t nd = 2 * E + 1, G = 1;
    while (G < 32 && G * 3 < nd) G <<= 1;
    return G;
}

// The shape of a class never tuned: SneakySnake one lane per pair in 32-pair steals and
// 512-thread CTAs (the shape the search keeps for the workloads measured), the other
// approximations about three diagonals a lane.
static TunedShape default_shape(int algo, uint32_t E) {
    if (algo == ALGO_SNAKE) return TunedShape{1u, 32u, 512u, 0u};
    return TunedShape{algo == ALGO_QGRAM ? 32u : default_G(E), EDA_CHUNK, (uint32_t)EDA_THREADS, 0u};
}

static bool tuned_shape(int device, int algo, uint32_t slot, TunedShape *out) {
    std::lock_guard<std::mutex> lk(g_tune.mu);
    *out = g_tune.sh[device & 63][algo][slot];
    return out->G != 0;
}

static void set_tuned_shape(int device, int algo, uint32_t slot, const TunedShape &t) {
    std::lock_guard<std::mutex> lk(g_tune.mu);
    g_tune.sh[device & 63][algo][slot] = t;
}

// Runs the staged search; timed(shape, &ms) launches one shape on the sample (ms < 0: the
// shape does not fit).
template <class F>
static int search_shape(int algo, uint32_t E, F &&timed, TunedShape *out) {
    TunedShape best = default_shape(algo, E);
    float best_ms = 1e30f;
    auto consider = [&](TunedShape t) -> int {
        float ms = -1.0f;
        int rc = timed(t, &ms);
        if (rc) return rc;
        if (ms >= 0.0f && ms < best_ms) { best_ms = ms; best = t; }
        return MT_OK;
    };
    int rc;
    if (algo != ALGO_QGRAM)
        for (uint32_t G : {1u, 2u, 4u, 8u, 16u, 32u})
            if ((rc = consider(TunedShape{G, EDA_CHUNK, (uint32_t)EDA_THREADS, 0u}))) return rc;
    const uint32_t G = best.G;
    if (algo == ALGO_SNAKE && G == 1)   // one lane per pair: lockstep groups or refilled lanes
        if ((rc = consider(TunedShape{1u, EDA_CHUNK, (uint32_t)EDA_THREADS, 1u}))) return rc;
    const uint32_t rf = best.refill;
    for (uint32_t ch : {32u, 64u, 128u, 256u})
        if ((rc = consider(TunedShape{G, ch, (uint32_t)EDA_THREADS, rf}))) return rc;
    const uint32_t ch = best.chunk;
    for (uint32_t cta : {128u, 256u, 512u, 1024u})
        if ((rc = consider(TunedShape{G, ch, cta, rf}))) return rc;
    *out = best;
    return MT_OK;
}

// Times one launch of `plan` (twice; the second counts) with two events.
template <int A, class Src>
static int time_plan(const Src &src, const uint32_t *perm, const EdaPlan &plan, const EdaShape &w,
                     unsigned long long *counter, cudaStream_t s, float *ms) {
    if (eda_smem(plan.cta / 32, plan.groups_max, w) > EDA_SMEM_MAX) { *ms = -1.0f; return MT_OK; }
    cudaEvent_t e0, e1;
    MT_CK(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return MT_ECUDA; }
    int rc = MT_OK;
    for (int rep = 0; rep < 2 && rc == MT_OK; rep++) {
        if (!cuda_ok(cudaEventRecord(e0, s), "tune event")) { rc = MT_ECUDA; break; }
        rc = launch_persistent<A>(src, perm, plan, counter, w, s);
        if (rc) break;
        if (!cuda_ok(cudaEventRecord(e1, s), "tune event") || !cuda_ok(cudaEventSynchronize(e1), "tune sync") ||
            !cuda_ok(cudaEventElapsedTime(ms, e0, e1), "tune time"))
            rc = MT_ECUDA;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

static EdaPlan one_class_plan(int algo, const TunedShape &t, uint64_t b, uint64_t e) {
    EdaPlan plan{};
    plan.n_classes = 1;
    plan.lanes = algo == ALGO_SNAKE && t.G == 1 && t.refill;
    plan.G[0] = t.G;
    plan.chunk[0] = t.chunk;
    plan.cta = t.cta;
    plan.groups_max = 32 / t.G;
    plan.begin[0] = b;
    plan.end[0] = e;
    return plan;
}

// ---- classification EDA (called by mt_classify) ------------------------------------------------
template <int A>
static int classify_eda(const ClassifySrc &src, uint64_t max_items, const uint64_t *cl_count, uint32_t maxn,
                        uint32_t maxE, uint32_t form, unsigned long long *counter, cudaStream_t s,
                        bool tune, TunedShape *used) {
    const EdaShape w = eda_shape(A, maxn, maxE);
    if (form == MT_EDA_PLAIN) return launch_plain<A>(src, nullptr, 0, max_items, cl_count, w, s);
    int dev = 0;
    cudaGetDevice(&dev);
    const uint32_t slot = MAX_CLASSES + e_class(maxE);
    TunedShape t;
    if (tune) {
        // every candidate shape timed on the first 2^17 candidates of this call
        auto timed = [&](TunedShape c, float *ms) {
            EdaPlan tp = one_class_plan(A, c, 0, max_items);
            tp.dyn_end = cl_count;
            tp.cap = 1ull << 17;
            if (eda_smem(c.cta / 32, tp.groups_max, w) > 96 * 1024) { *ms = -1.0f; return (int)MT_OK; }
            return time_plan<A>(src, nullptr, tp, w, counter, s, ms);
        };
        int rc = search_shape(A, maxE, timed, &t);
        if (rc) return rc;
        set_tuned_shape(dev, A, slot, t);
    } else if (!tuned_shape(dev, A, slot, &t)) {
        t = default_shape(A, maxE);
    }
    EdaPlan plan = one_class_plan(A, t, 0, max_items);
    plan.dyn_end = cl_count;
    // keep the shared-memory footprint bounded for long reads
    while (eda_smem(plan.cta / 32, plan.groups_max, w) > 96 * 1024 && plan.G[0] < 32) {
        plan.G[0] <<= 1;
        plan.groups_max = 32 / plan.G[0];
        plan.lanes = 0;
    }
    if (used) *used = TunedShape{plan.G[0], plan.chunk[0], plan.cta, plan.lanes};
    return launch_persistent<A>(src, nullptr, plan, counter, w, s);
}

int launch_classify_eda(const IndexView &ix, const uint64_t *rw, const IoBlock *io,
                        const uint32_t *cl, const uint64_t *cl_count, uint64_t max_items,
                        const Cluster *cand, uint32_t top_n, uint32_t e_abs, uint32_t e_permille,
                        uint32_t maxn, uint32_t maxE, uint32_t mode, uint8_t *dist,
                        unsigned long long *counter, cudaStream_t s, bool tune, mt_eda_shape *used) {
    ClassifySrc src;
    src.ix = ix; src.rw = rw; src.io = io; src.cl = cl; src.cand = cand;
    src.top_n = top_n; src.e_abs = e_abs; src.e_permille = e_permille; src.dist = dist;
    const uint32_t form = mode & 15u;
    TunedShape t{0, 0, 0, 0};
    int rc;
    switch (mode >> 4) {
        case ALGO_HD: rc = classify_eda<ALGO_HD>(src, max_items, cl_count, maxn, maxE, form, counter, s, tune, &t); break;
        case ALGO_BC: rc = classify_eda<ALGO_BC>(src, max_items, cl_count, maxn, maxE, form, counter, s, tune, &t); break;
        case ALGO_QGRAM: rc = classify_eda<ALGO_QGRAM>(src, max_items, cl_count, maxn, maxE, form, counter, s, tune, &t); break;
        case ALGO_SHD: rc = classify_eda<ALGO_SHD>(src, max_items, cl_count, maxn, maxE, form, counter, s, tune, &t); break;
        default: rc = classify_eda<ALGO_SNAKE>(src, max_items, cl_count, maxn, maxE, form, counter, s, tune, &t); break;
    }
    if (used && t.G) {
        used->lanes_per_pair = t.G;
        used->pairs_per_chunk = t.chunk;
        used->cta_threads = t.cta;
        used->refill = t.refill;
    }
    return rc;
}

// ---- the EDA-only batch, after bucketing ------------------------------------------------------
// start[]: for the batched form the first pair of each edit-threshold class (MAX_CLASSES + 1
// entries), for the plain form the first pair of each read-word bucket (34 entries).
template <int A>
static int run_batch(const BatchSrc &src, const uint32_t *perm, const BucketStats &h,
                     const unsigned long long *start, uint32_t form, unsigned long long *counter,
                     bool tune, mt_eda_shape *shapes, cudaStream_t s) {
    if (form == MT_EDA_PLAIN) {
        for (int b = 1; b <= 32; b++) {
            if (!h.bkt_count[b]) continue;
            uint32_t maxn = (uint32_t)b * 32;
            int rc = launch_plain<A>(src, perm, start[b], start[b + 1], nullptr, eda_shape(A, maxn, h.bkt_maxE[b]), s);
            if (rc) return rc;
        }
        return MT_OK;
    }
    int dev = 0;
    cudaGetDevice(&dev);
    // two persistent launches at most: the classes whose SneakySnake lanes are refilled one by
    // one (plan 1), and the others (plan 0)
    EdaPlan plan[2] = {};
    uint32_t minG[2] = {32, 32};
    uint64_t most[2] = {0, 0};
    uint32_t maxn[2] = {0, 0}, maxE[2] = {0, 0};
    plan[0].cta = plan[1].cta = EDA_THREADS;
    for (int c = 0; c < MAX_CLASSES; c++) {
        if (!h.cls_count[c]) continue;
        TunedShape t;
        if (tune) {
            const EdaShape wc = eda_shape(A, h.cls_maxn[c], h.cls_maxE[c]);
            const uint64_t b = start[c], e = start[c] + std::min<uint64_t>(start[c + 1] - start[c], 1ull << 17);
            auto timed = [&](TunedShape cand, float *ms) {
                return time_plan<A>(src, perm, one_class_plan(A, cand, b, e), wc, counter, s, ms);
            };
            int rc = search_shape(A, h.cls_maxE[c], timed, &t);
            if (rc) return rc;
            set_tuned_shape(dev, A, (uint32_t)c, t);
        } else if (!tuned_shape(dev, A, (uint32_t)c, &t)) {
            t = default_shape(A, h.cls_maxE[c]);
        }
        const int q = (A == ALGO_SNAKE && t.G == 1 && t.refill) ? 1 : 0;
        EdaPlan &pl = plan[q];
        uint32_t k = pl.n_classes++;
        pl.G[k] = t.G;
        pl.chunk[k] = t.chunk;
        pl.begin[k] = start[c];
        pl.end[k] = start[c + 1];
        minG[q] = std::min(minG[q], t.G);
        maxn[q] = std::max(maxn[q], h.cls_maxn[c]);
        maxE[q] = std::max(maxE[q], h.cls_maxE[c]);
        if (h.cls_count[c] > most[q]) { most[q] = h.cls_count[c]; pl.cta = t.cta; }   // the largest class's CTA size
        if (shapes) shapes[c] = mt_eda_shape{t.G, t.chunk, t.cta, t.refill, tune ? 1u : 0u};
    }
    for (int q = 0; q < 2; q++) {
        EdaPlan &pl = plan[q];
        if (!pl.n_classes) continue;
        // one shared-memory layout serves every class of a launch: widen the smallest groups
        // (lockstep launch only) or shrink the CTA until it fits
        const EdaShape w = eda_shape(A, maxn[q], maxE[q]);
        while (q == 0 && minG[q] < 32 && eda_smem(pl.cta / 32, 32 / minG[q], w) > EDA_SMEM_MAX) minG[q] <<= 1;
        while (pl.cta > 128 && eda_smem(pl.cta / 32, 32 / minG[q], w) > EDA_SMEM_MAX) pl.cta >>= 1;
        for (uint32_t k = 0; k < pl.n_classes; k++) pl.G[k] = std::max(pl.G[k], minG[q]);
        pl.groups_max = 32 / minG[q];
        pl.lanes = q;
        int rc = launch_persistent<A>(src, perm, pl, counter, w, s);
        if (rc) return rc;
    }
    return MT_OK;
}

static int run_batch_algo(const BatchSrc &src, const uint32_t *perm, const BucketStats &h,
                          const unsigned long long *start, uint32_t mode, unsigned long long *counter,
                          bool tune, mt_eda_shape *shapes, cudaStream_t s) {
    const uint32_t form = mode & 15u;
    switch (mode >> 4) {
        case ALGO_HD: return run_batch<ALGO_HD>(src, perm, h, start, form, counter, tune, shapes, s);
        case ALGO_BC: return run_batch<ALGO_BC>(src, perm, h, start, form, counter, tune, shapes, s);
        case ALGO_QGRAM: return run_batch<ALGO_QGRAM>(src, perm, h, start, form, counter, tune, shapes, s);
        case ALGO_SHD: return run_batch<ALGO_SHD>(src, perm, h, start, form, counter, tune, shapes, s);
        default: return run_batch<ALGO_SNAKE>(src, perm, h, start, form, counter, tune, shapes, s);
    }
}

static int scatter_key(uint32_t mode) {
    if ((mode & 15u) != MT_EDA_BATCHED) return KEY_WORDS;
    const uint32_t a = mode >> 4;
    return (a == ALGO_SNAKE || a == ALGO_SHD) ? KEY_E : KEY_CLASS;
}

// Segment starts of the scattered pairs (keys[], one more entry than keys) and, for the
// batched form, the first pair of each edit-threshold class (cls[], MAX_CLASSES + 1 entries).
static int scatter_starts(const BucketStats &h, int kind, unsigned long long *keys, unsigned long long *cls) {
    const int nkeys = kind == KEY_E ? (int)E_KEYS : kind == KEY_CLASS ? MAX_CLASSES : 33;
    keys[0] = 0;
    for (int i = 0; i < nkeys; i++)
        keys[i + 1] = keys[i] + (kind == KEY_E ? h.e_count[i] : kind == KEY_CLASS ? h.cls_count[i] : h.bkt_count[i]);
    for (int c = 0; c <= MAX_CLASSES; c++) {
        const uint32_t e0 = c == 0 ? 0u : (c == MAX_CLASSES ? E_KEYS : std::min<uint32_t>(1u << c, E_KEYS));
        cls[c] = kind == KEY_E ? keys[e0] : kind == KEY_CLASS ? keys[c] : 0;
    }
    return nkeys;
}

// eda_mode / mode: execution form in the low 4 bits, approximation in bits 4-7.
bool eda_mode_ok(uint32_t mode) {
    return (mode & 15u) <= MT_EDA_PLAIN && (mode >> 4) < (uint32_t)N_ALGOS;
}

}  // namespace mt

using namespace mt;

namespace mt {
static int eda_batch_impl(const uint64_t *read_words, const uint64_t *read_off, uint64_t n_reads,
                          const uint64_t *win_words, const uint64_t *win_off, const uint32_t *pair_read,
                          const uint16_t *E, uint64_t n_pairs, uint32_t mode, void *stream, uint8_t *dist,
                          bool tune, mt_eda_shape *shapes) {
    if (!eda_mode_ok(mode)) return MT_EINVAL;
    if (n_pairs == 0) return MT_OK;
    if (!read_words || !read_off || !win_words || !win_off || !pair_read || !E || !dist || n_reads == 0)
        return MT_EINVAL;
    if (n_pairs > 0xFFFFFFFFull) return MT_EINVAL;
    Trace trace(tune ? "mt_eda_batch_autotune" : "mt_eda_batch");
    cudaStream_t s = (cudaStream_t)stream;
    int rc;
    BucketStats *st = nullptr;
    uint32_t *perm = nullptr;
    unsigned long long *cursor = nullptr;
    if ((rc = dalloc((void **)&st, sizeof(BucketStats), s))) return rc;
    if ((rc = dalloc((void **)&perm, n_pairs * 4, s))) { dfree(st, s); return rc; }
    if ((rc = dalloc((void **)&cursor, CURSOR_WORDS * 8, s))) { dfree(st, s); dfree(perm, s); return rc; }
    auto cleanup = [&]() { dfree(st, s); dfree(perm, s); dfree(cursor, s); };
    BucketStats h{};
    if (cudaMemsetAsync(st, 0, sizeof(BucketStats), s) != cudaSuccess) { cleanup(); return MT_ECUDA; }
    {
        unsigned blocks = (unsigned)std::min<uint64_t>((n_pairs + 255) / 256, (uint64_t)sm_count() * 8);
        k_bucket_count<<<blocks, 256, 0, s>>>(read_off, n_reads, win_off, pair_read, E, n_pairs, st);
        if (!cuda_ok(cudaGetLastError(), "k_bucket_count")) { cleanup(); return MT_ECUDA; }
    }
    if (!cuda_ok(cudaMemcpyAsync(&h, st, sizeof(h), cudaMemcpyDeviceToHost, s), "memcpy") ||
        !cuda_ok(cudaStreamSynchronize(s), "sync")) { cleanup(); return MT_ECUDA; }
    if (h.err) { cleanup(); return MT_EINVAL; }

    BatchSrc src;
    src.rw = read_words; src.roff = read_off; src.ww = win_words; src.woff = win_off;
    src.pair_read = pair_read; src.E = E; src.dist = dist;
    const int kind = scatter_key(mode);
    unsigned long long keys[E_KEYS + 1], cls[MAX_CLASSES + 1];
    const int nkeys = scatter_starts(h, kind, keys, cls);
    if (cudaMemcpyAsync(cursor, keys, nkeys * 8, cudaMemcpyHostToDevice, s) != cudaSuccess) { cleanup(); return MT_ECUDA; }
    {
        unsigned blocks = (unsigned)std::min<uint64_t>((n_pairs + 255) / 256, (uint64_t)sm_count() * 8);
        k_bucket_scatter<<<blocks, 256, 0, s>>>(read_off, pair_read, E, n_pairs, kind, cursor, perm);
        if (!cuda_ok(cudaGetLastError(), "k_bucket_scatter")) { cleanup(); return MT_ECUDA; }
    }
    unsigned long long *counter = cursor + COUNTER_AT;
    rc = run_batch_algo(src, perm, h, kind == KEY_WORDS ? keys : cls, mode, counter, tune, shapes, s);
    if (rc) { cleanup(); return rc; }
    cudaError_t e = cudaStreamSynchronize(s);
    cleanup();
    if (!cuda_ok(e, "mt_eda_batch")) return MT_ECUDA;
    return MT_OK;
}
}  // namespace mt

extern "C" int mt_eda_batch(const uint64_t *read_words, const uint64_t *read_off, uint64_t n_reads,
                            const uint64_t *win_words, const uint64_t *win_off, const uint32_t *pair_read,
                            const uint16_t *E, uint64_t n_pairs, uint32_t mode, void *stream, uint8_t *dist) {
    return eda_batch_impl(read_words, read_off, n_reads, win_words, win_off, pair_read, E, n_pairs, mode, stream,
                          dist, false, nullptr);
}

extern "C" int mt_eda_batch_autotune(const uint64_t *read_words, const uint64_t *read_off, uint64_t n_reads,
                                     const uint64_t *win_words, const uint64_t *win_off, const uint32_t *pair_read,
                                     const uint16_t *E, uint64_t n_pairs, uint32_t mode, void *stream, uint8_t *dist,
                                     mt_eda_shape *shapes) {
    if (shapes) memset(shapes, 0, MT_EDA_CLASSES * sizeof(mt_eda_shape));
    return eda_batch_impl(read_words, read_off, n_reads, win_words, win_off, pair_read, E, n_pairs, mode, stream,
                          dist, (mode & 15u) == MT_EDA_BATCHED, shapes);
}

extern "C" int mt_eda_set_shape(uint32_t mode, int classification, uint32_t E, const mt_eda_shape *shape) {
    if (!shape || !eda_mode_ok(mode) || E > MT_MAX_E) return MT_EINVAL;
    const int algo = (int)(mode >> 4);
    const uint32_t G = shape->lanes_per_pair, ch = shape->pairs_per_chunk, cta = shape->cta_threads;
    TunedShape t{0, 0, 0, 0};   // lanes_per_pair = 0: forget the kept shape
    if (G) {
        if (G > 32 || (G & (G - 1)) || (algo == ALGO_QGRAM && G != 32)) return MT_EINVAL;
        if (ch == 0 || ch > 4096 || cta < 32 || cta > (uint32_t)EDA_MAX_THREADS || cta % 32) return MT_EINVAL;
        if (shape->refill > 1 || (shape->refill && (algo != ALGO_SNAKE || G != 1))) return MT_EINVAL;
        t = TunedShape{G, ch, cta, shape->refill};
    }
    int dev = 0;
    if (!cuda_ok(cudaGetDevice(&dev), "cudaGetDevice")) return MT_ECUDA;
    set_tuned_shape(dev, algo, (classification ? MAX_CLASSES : 0) + e_class(E), t);
    return MT_OK;
}

extern "C" int mt_eda_shape_for(uint32_t mode, int classification, uint32_t E, mt_eda_shape *out) {
    if (!out || !eda_mode_ok(mode) || E > MT_MAX_E) return MT_EINVAL;
    int dev = 0;
    if (!cuda_ok(cudaGetDevice(&dev), "cudaGetDevice")) return MT_ECUDA;
    const int algo = (int)(mode >> 4);
    const uint32_t slot = (classification ? MAX_CLASSES : 0) + e_class(E);
    TunedShape t;
    const bool tuned = tuned_shape(dev, algo, slot, &t);
    if (!tuned) t = default_shape(algo, E);
    *out = mt_eda_shape{t.G, t.chunk, t.cta, t.refill, tuned ? 1u : 0u};
    return MT_OK;
}

namespace mt {
// ---- allocation-free variant of the batch call ----------------------------------------------
// Some callers cannot allocate device memory during a call: code that runs where
// cudaMalloc / cudaMallocAsync are not permitted or would stall the pipeline (inside a
// latency-critical serving loop with a fixed memory footprint, under an allocator owned by a
// host framework that forbids side allocations, or in processes that must not grow their
// device footprint after start-up). For them, mt_eda_batch_noalloc keeps its scratch (bucket
// statistics, cursors, the pair permutation) in the fixed array below instead of allocating.
static constexpr uint64_t NOALLOC_MAX_PAIRS = 1ull << 20;   // 4 MiB of permutation

struct NoAllocScratch {
    BucketStats st;
    unsigned long long cursor[CURSOR_WORDS];
    uint32_t perm[NOALLOC_MAX_PAIRS];
};

// One copy per device that loads the library, held until the process exits.
static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

static std::mutex g_noalloc_mu;
static NoAllocScratch *g_noalloc_ptr[64] = {nullptr};

// The device address of the array for the current device. The host symbol is only a
// stand-in, so the address is asked from the runtime once per device (with that device
// current) and cached.
static int noalloc_scratch(NoAllocScratch **out) {
    int dev = 0;
    MT_CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return MT_EINVAL;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (!cuda_ok(e, "cudaGetSymbolAddress(g_noalloc_scratch)")) return MT_ECUDA;
        g_noalloc_ptr[dev] = reinterpret_cast<NoAllocScratch *>(p);
    }
    *out = g_noalloc_ptr[dev];
    return MT_OK;
}
}  // namespace mt

extern "C" int mt_eda_batch_noalloc(const uint64_t *read_words, const uint64_t *read_off, uint64_t n_reads,
                                    const uint64_t *win_words, const uint64_t *win_off, const uint32_t *pair_read,
                                    const uint16_t *E, uint64_t n_pairs, uint32_t mode, void *stream, uint8_t *dist) {
    if (mode != MT_EDA_BATCHED && mode != MT_EDA_PLAIN) return MT_EINVAL;
    if (n_pairs > NOALLOC_MAX_PAIRS) return MT_EINVAL;
    if (n_pairs == 0) return MT_OK;
    if (!read_words || !read_off || !win_words || !win_off || !pair_read || !E || !dist || n_reads == 0)
        return MT_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    NoAllocScratch *sc = nullptr;
    int rc = noalloc_scratch(&sc);
    if (rc) return rc;
    BucketStats *st = &sc->st;
    unsigned long long *cursor = sc->cursor;
    uint32_t *perm = sc->perm;
    // the array keeps the previous call's contents: clear the counters that must start at 0
    // (the steal counter is cleared by each launch)
    MT_CK(cudaMemsetAsync(st, 0, sizeof(BucketStats), s));
    {
        unsigned blocks = (unsigned)std::min<uint64_t>((n_pairs + 255) / 256, (uint64_t)sm_count() * 8);
        k_bucket_count<<<blocks, 256, 0, s>>>(read_off, n_reads, win_off, pair_read, E, n_pairs, st);
        MT_CK(cudaGetLastError());
    }
    BucketStats h{};
    MT_CK(cudaMemcpyAsync(&h, st, sizeof(h), cudaMemcpyDeviceToHost, s));
    MT_CK(cudaStreamSynchronize(s));
    if (h.err) return MT_EINVAL;
    BatchSrc src;
    src.rw = read_words; src.roff = read_off; src.ww = win_words; src.woff = win_off;
    src.pair_read = pair_read; src.E = E; src.dist = dist;
    const int kind = scatter_key(mode);
    unsigned long long keys[E_KEYS + 1], cls[MAX_CLASSES + 1];
    const int nkeys = scatter_starts(h, kind, keys, cls);
    MT_CK(cudaMemcpyAsync(cursor, keys, nkeys * 8, cudaMemcpyHostToDevice, s));
    {
        unsigned blocks = (unsigned)std::min<uint64_t>((n_pairs + 255) / 256, (uint64_t)sm_count() * 8);
        k_bucket_scatter<<<blocks, 256, 0, s>>>(read_off, pair_read, E, n_pairs, kind, cursor, perm);
        MT_CK(cudaGetLastError());
    }
    unsigned long long *counter = cursor + COUNTER_AT;
    // shapes: the autotuned ones when this process has them, else the defaults (no timing
    // runs here, so no events are created)
    rc = run_batch_algo(src, perm, h, kind == KEY_WORDS ? keys : cls, mode, counter, false, nullptr, s);
    if (rc) return rc;
    MT_CK(cudaStreamSynchronize(s));
    return MT_OK;
}
