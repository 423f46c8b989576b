// Edit-distance approximation stage: kernels, the two execution forms and the autotuner.
//
//   plain   : one launch per read-length bucket, one warp (32 lanes) per pair, a
//             non-persistent grid sized to the bucket.
//   batched : one persistent launch (grid = SMs x resident CTAs) over all pairs, sorted by
//             edit-threshold class; warps steal chunks of 128 pairs from a global counter;
//             each class runs with the lanes-per-pair G (1..32) picked by the autotuner.
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
static constexpr int EDA_THREADS = 256;
static constexpr int MAX_CLASSES = 8;

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
        for (uint32_t t = gl; t < nr + 2; t += G) rd[t] = t < nr ? rs[t] : 0ull;
        for (uint32_t t = gl; t < nwn + 3; t += G) wn[t] = t < nwn ? ws[t] : 0ull;
        PairInfo pi;
        pi.n = n; pi.E = E_; pi.lo = 0; pi.hi = (int32_t)(n + 2 * E_); pi.edges = false;
        return pi;
    }
    MT_DEV void finish(uint64_t p, uint32_t d) const { dist[p] = (uint8_t)d; }
};

// 32 bases of a genome starting at `pos` (may lie outside the genome; those bits are
// don't-care and are masked as obstacles by the caller). Reads only words 0..nwg of it.
MT_DEV uint64_t genome_get32(const uint64_t *g, uint64_t nwg, int64_t pos) {
    int64_t wi = pos >> 5;
    uint32_t sh = (uint32_t)(pos & 31) * 2u;
    uint64_t a = (wi >= 0 && wi <= (int64_t)nwg) ? g[wi] : 0ull;
    uint64_t b = (wi + 1 >= 0 && wi + 1 <= (int64_t)nwg) ? g[wi + 1] : 0ull;
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
            for (uint32_t t = gl; t < nr + 2; t += G) {
                uint64_t x = 0;
                if (t < nr) {
                    int32_t st = (int32_t)n - 32 * (int32_t)(t + 1);
                    x = st >= 0 ? get32(rs, (uint32_t)st) : (get32(rs, 0) << (2 * (uint32_t)(-st)));
                    x = ~rev2(x);
                }
                rd[t] = x;
            }
        } else {
            for (uint32_t t = gl; t < nr + 2; t += G) rd[t] = t < nr ? rs[t] : 0ull;
        }
        uint32_t g = hk_genome(c.hkey);
        int64_t wstart = hk_diag(c.hkey) - (int64_t)E;
        uint64_t glen = ix.glen[g];
        uint64_t nwg = (glen + 31) / 32;
        const uint64_t *gp = ix.ref + ix.gword[g];
        uint32_t L = n + 2 * E, nwn = (L + 31) / 32;
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
    uint32_t G[MAX_CLASSES];
    uint64_t begin[MAX_CLASSES], end[MAX_CLASSES];
    const uint64_t *dyn_end;           // if set: class 0 ends at *dyn_end (device count)
    uint64_t cap;                      // if set: class 0 holds at most `cap` items (tuning samples)
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

template <class Src, int A>
__global__ void __launch_bounds__(EDA_THREADS) k_eda_persistent(Src src, const uint32_t *perm, EdaPlan plan,
                                                                unsigned long long *counter,
                                                                uint32_t rww, uint32_t www, uint32_t xw) {
    extern __shared__ uint64_t sm[];
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
    uint64_t *wbase = sm + (uint64_t)warp * plan.groups_max * (rww + www + xw);
    // chunk table: chunks of 128 items per class
    uint64_t pref[MAX_CLASSES + 1];
    pref[0] = 0;
    uint64_t end0 = plan.dyn_end ? *plan.dyn_end : plan.end[0];
    if (plan.cap && end0 > plan.begin[0] + plan.cap) end0 = plan.begin[0] + plan.cap;
    for (uint32_t c = 0; c < plan.n_classes; c++) {
        uint64_t e = c == 0 ? end0 : plan.end[c];
        uint64_t cnt = e > plan.begin[c] ? e - plan.begin[c] : 0;
        pref[c + 1] = pref[c] + (cnt + 127) / 128;
    }
    const uint64_t total = pref[plan.n_classes];
    while (true) {
        unsigned long long id = 0;
        if (lane == 0) id = atomicAdd(counter, 1ull);
        id = __shfl_sync(FULL, id, 0);
        if (id >= total) break;
        uint32_t c = 0;
        while (id >= pref[c + 1]) c++;
        uint64_t e = c == 0 ? end0 : plan.end[c];
        uint64_t b = plan.begin[c] + (id - pref[c]) * 128;
        uint64_t ee = b + 128 < e ? b + 128 : e;
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
    unsigned int cls_maxn[MAX_CLASSES], cls_maxE[MAX_CLASSES];
    unsigned int bkt_maxE[33];
    unsigned int maxn, maxE, err;
};

__global__ void k_bucket_count(const uint64_t *roff, uint64_t n_reads, const uint64_t *woff,
                               const uint32_t *pair_read, const uint16_t *E, uint64_t n_pairs,
                               BucketStats *st) {
    __shared__ unsigned long long sc[MAX_CLASSES], sb[33];
    for (int i = threadIdx.x; i < MAX_CLASSES; i += blockDim.x) sc[i] = 0;
    for (int i = threadIdx.x; i < 33; i += blockDim.x) sb[i] = 0;
    __syncthreads();
    for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n_pairs;
         p += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t r = pair_read[p];
        if (r >= n_reads) { atomicOr(&st->err, ERR_BAD_PAIR); continue; }
        uint64_t n64 = roff[r + 1] - roff[r];
        uint32_t e = E[p];
        uint64_t L = woff[p + 1] - woff[p];
        if (roff[r + 1] < roff[r] || n64 > MT_MAX_READ_LEN || e > MT_MAX_E || L != n64 + 2ull * e) {
            atomicOr(&st->err, ERR_BAD_PAIR);
            continue;
        }
        uint32_t n = (uint32_t)n64;
        uint32_t c = e_class(e), b = (n + 31) / 32;
        atomicAdd(&sc[c], 1ull);
        atomicAdd(&sb[b], 1ull);
        atomicMax(&st->cls_maxn[c], n);
        atomicMax(&st->cls_maxE[c], e);
        atomicMax(&st->bkt_maxE[b], e);
        atomicMax(&st->maxn, n);
        atomicMax(&st->maxE, e);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < MAX_CLASSES; i += blockDim.x)
        if (sc[i]) atomicAdd(&st->cls_count[i], sc[i]);
    for (int i = threadIdx.x; i < 33; i += blockDim.x)
        if (sb[i]) atomicAdd(&st->bkt_count[i], sb[i]);
}

// scatter pair ids into class (by_class=1) or bucket segments; cursor[] starts at the
// segment starts. Warp-aggregated per key.
__global__ void k_bucket_scatter(const uint64_t *roff, const uint32_t *pair_read, const uint16_t *E,
                                 uint64_t n_pairs, int by_class, unsigned long long *cursor,
                                 uint32_t *perm) {
    for (uint64_t p0 = (uint64_t)blockIdx.x * blockDim.x; p0 < n_pairs; p0 += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t p = p0 + threadIdx.x;
        bool ok = p < n_pairs;
        uint32_t key = 0xFFFFFFFFu;
        if (ok) {
            uint32_t r = pair_read[p];
            uint32_t n = (uint32_t)(roff[r + 1] - roff[r]);
            key = by_class ? e_class(E[p]) : (n + 31) / 32;
        }
        unsigned peers = __match_any_sync(FULL, key);
        uint32_t lane = threadIdx.x & 31u;
        uint32_t leader = __ffs(peers) - 1;
        unsigned long long base = 0;
        if (ok && lane == leader) base = atomicAdd(&cursor[key], (unsigned long long)__popc(peers));
        base = __shfl_sync(FULL, base, leader);
        if (ok) perm[base + __popc(peers & ((1u << lane) - 1))] = (uint32_t)p;
    }
}

// ---- launch helpers --------------------------------------------------------------------------------
// Group shapes: words of one group (read, window, extra) for the largest pair of a launch.
struct EdaShape {
    uint32_t rww, www, xw;
};

static EdaShape eda_shape(int A, uint32_t maxn, uint32_t maxE) {
    return EdaShape{eda_read_words(maxn), eda_win_words(maxn, maxE), eda_extra_words(A, maxn)};
}

static size_t eda_smem(uint32_t groups_per_warp, const EdaShape &w) {
    return (size_t)(EDA_THREADS / 32) * groups_per_warp * (w.rww + w.www + w.xw) * 8;
}

template <int A, class Src>
static int launch_persistent(const Src &src, const uint32_t *perm, const EdaPlan &plan,
                             unsigned long long *counter, const EdaShape &w, cudaStream_t s) {
    size_t smem = eda_smem(plan.groups_max, w);
    if (smem > 200 * 1024) return MT_EINVAL;
    static std::mutex mu;
    {
        std::lock_guard<std::mutex> lk(mu);
        MT_CK(cudaFuncSetAttribute(k_eda_persistent<Src, A>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    }
    int per_sm = 0;
    MT_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_eda_persistent<Src, A>, EDA_THREADS, smem));
    if (per_sm < 1) per_sm = 1;
    unsigned grid = (unsigned)(sm_count() * per_sm);
    MT_CK(cudaMemsetAsync(counter, 0, 8, s));
    k_eda_persistent<Src, A><<<grid, EDA_THREADS, smem, s>>>(src, perm, plan, counter, w.rww, w.www, w.xw);
    MT_CK(cudaGetLastError());
    return MT_OK;
}

template <int A, class Src>
static int launch_plain(const Src &src, const uint32_t *perm, uint64_t begin, uint64_t end,
                        const uint64_t *dyn_end, const EdaShape &w, cudaStream_t s) {
    if (end <= begin) return MT_OK;
    size_t smem = eda_smem(1, w);
    if (smem > 200 * 1024) return MT_EINVAL;
    static std::mutex mu;
    {
        std::lock_guard<std::mutex> lk(mu);
        MT_CK(cudaFuncSetAttribute(k_eda_plain<Src, A>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
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
// Lanes per pair for each approximation and edit-threshold class, picked by timing G in
// {1,2,4,8,16,32} on a sample of the class the first time the class is seen in this process
// (per device). The q-gram approximation always takes a whole warp (one histogram per warp).
static constexpr int N_ALGOS = 5;
struct TuneCache {
    std::mutex mu;
    int G[64][N_ALGOS][2 * MAX_CLASSES];   // per device and algorithm: EDA-only classes, then classification classes
    TuneCache() { memset(G, 0, sizeof(G)); }
};
static TuneCache g_tune;

static uint32_t default_G(uint32_t E) {
    uint32_t nd = 2 * E + 1, G = 1;
    while (G < 32 && G * 3 < nd) G <<= 1;
    return G;
}

static int tuned_G(int device, int algo, uint32_t cls, uint32_t *G) {
    if (algo == ALGO_QGRAM) { *G = 32; return 1; }
    std::lock_guard<std::mutex> lk(g_tune.mu);
    *G = (uint32_t)g_tune.G[device & 63][algo][cls];
    return *G != 0;
}

static void set_tuned_G(int device, int algo, uint32_t cls, uint32_t G) {
    std::lock_guard<std::mutex> lk(g_tune.mu);
    g_tune.G[device & 63][algo][cls] = (int)G;
}

template <int A, class Src>
static int autotune_class(const Src &src, const uint32_t *perm, uint64_t b, uint64_t e, uint32_t cls,
                          const EdaShape &w, unsigned long long *counter, cudaStream_t s, uint32_t *bestG) {
    uint64_t cnt = e - b;
    uint64_t sample = std::min<uint64_t>(cnt, 1ull << 17);
    cudaEvent_t e0, e1;
    MT_CK(cudaEventCreate(&e0));
    MT_CK(cudaEventCreate(&e1));
    float best = 1e30f;
    uint32_t bg = default_G(cls);
    const uint32_t cands[6] = {1, 2, 4, 8, 16, 32};
    for (int rep = 0; rep < 2; rep++) {   // first round warms up
        for (uint32_t G : cands) {
            EdaPlan plan{};
            plan.n_classes = 1;
            plan.groups_max = 32 / G;
            plan.G[0] = G;
            plan.begin[0] = b;
            plan.end[0] = b + sample;
            if (eda_smem(plan.groups_max, w) > 200 * 1024) continue;
            MT_CK(cudaEventRecord(e0, s));
            int rc = launch_persistent<A>(src, perm, plan, counter, w, s);
            if (rc) { cudaEventDestroy(e0); cudaEventDestroy(e1); return rc; }
            MT_CK(cudaEventRecord(e1, s));
            MT_CK(cudaEventSynchronize(e1));
            float ms = 0;
            MT_CK(cudaEventElapsedTime(&ms, e0, e1));
            if (rep == 1 && ms < best) { best = ms; bg = G; }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *bestG = bg;
    return MT_OK;
}

// ---- classification EDA (called by mt_classify) ------------------------------------------------
template <int A>
static int classify_eda(const ClassifySrc &src, uint64_t max_items, const uint64_t *cl_count, uint32_t maxn,
                        uint32_t maxE, uint32_t form, unsigned long long *counter, cudaStream_t s,
                        bool allow_tune) {
    const EdaShape w = eda_shape(A, maxn, maxE);
    if (form == MT_EDA_PLAIN) return launch_plain<A>(src, nullptr, 0, max_items, cl_count, w, s);
    int dev = 0;
    cudaGetDevice(&dev);
    const uint32_t slot = MAX_CLASSES + e_class(maxE);
    uint32_t G = 0;
    if (!tuned_G(dev, A, slot, &G) && !allow_tune) G = default_G(maxE);
    if (!G) {
        // time every lanes-per-pair choice on the first 2^17 candidates of this call
        cudaEvent_t e0, e1;
        MT_CK(cudaEventCreate(&e0));
        MT_CK(cudaEventCreate(&e1));
        float best = 1e30f;
        G = default_G(maxE);
        for (int rep = 0; rep < 2; rep++) {
            for (uint32_t g : {1u, 2u, 4u, 8u, 16u, 32u}) {
                EdaPlan tp{};
                tp.n_classes = 1; tp.G[0] = g; tp.groups_max = 32 / g;
                tp.begin[0] = 0; tp.end[0] = max_items; tp.dyn_end = cl_count; tp.cap = 1ull << 17;
                if (eda_smem(tp.groups_max, w) > 96 * 1024) continue;
                MT_CK(cudaEventRecord(e0, s));
                int rc = launch_persistent<A>(src, nullptr, tp, counter, w, s);
                if (rc) { cudaEventDestroy(e0); cudaEventDestroy(e1); return rc; }
                MT_CK(cudaEventRecord(e1, s));
                MT_CK(cudaEventSynchronize(e1));
                float ms = 0;
                MT_CK(cudaEventElapsedTime(&ms, e0, e1));
                if (rep == 1 && ms < best) { best = ms; G = g; }
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        set_tuned_G(dev, A, slot, G);
    }
    EdaPlan plan{};
    plan.n_classes = 1;
    plan.G[0] = G;
    plan.groups_max = 32 / G;
    plan.begin[0] = 0;
    plan.end[0] = max_items;
    plan.dyn_end = cl_count;
    // keep the shared-memory footprint bounded for long reads
    while (eda_smem(plan.groups_max, w) > 96 * 1024 && plan.G[0] < 32) {
        plan.G[0] <<= 1;
        plan.groups_max = 32 / plan.G[0];
    }
    return launch_persistent<A>(src, nullptr, plan, counter, w, s);
}

int launch_classify_eda(const IndexView &ix, const uint64_t *rw, const IoBlock *io,
                        const uint32_t *cl, const uint64_t *cl_count, uint64_t max_items,
                        const Cluster *cand, uint32_t top_n, uint32_t e_abs, uint32_t e_permille,
                        uint32_t maxn, uint32_t maxE, uint32_t mode, uint8_t *dist,
                        unsigned long long *counter, cudaStream_t s, bool allow_tune) {
    ClassifySrc src;
    src.ix = ix; src.rw = rw; src.io = io; src.cl = cl; src.cand = cand;
    src.top_n = top_n; src.e_abs = e_abs; src.e_permille = e_permille; src.dist = dist;
    const uint32_t form = mode & 15u;
    switch (mode >> 4) {
        case ALGO_HD: return classify_eda<ALGO_HD>(src, max_items, cl_count, maxn, maxE, form, counter, s, allow_tune);
        case ALGO_BC: return classify_eda<ALGO_BC>(src, max_items, cl_count, maxn, maxE, form, counter, s, allow_tune);
        case ALGO_QGRAM:
            return classify_eda<ALGO_QGRAM>(src, max_items, cl_count, maxn, maxE, form, counter, s, allow_tune);
        case ALGO_SHD: return classify_eda<ALGO_SHD>(src, max_items, cl_count, maxn, maxE, form, counter, s, allow_tune);
        default: return classify_eda<ALGO_SNAKE>(src, max_items, cl_count, maxn, maxE, form, counter, s, allow_tune);
    }
}

// ---- the EDA-only batch, after bucketing ------------------------------------------------------
template <int A>
static int run_batch(const BatchSrc &src, const uint32_t *perm, const BucketStats &h,
                     const unsigned long long *start, uint32_t form, unsigned long long *counter,
                     bool allow_tune, cudaStream_t s) {
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
    EdaPlan plan{};
    uint32_t minG = 32;
    for (int c = 0; c < MAX_CLASSES; c++) {
        if (!h.cls_count[c]) continue;
        uint32_t G = 0;
        if (!tuned_G(dev, A, c, &G)) {
            if (allow_tune) {
                int rc = autotune_class<A>(src, perm, start[c], start[c + 1], (uint32_t)c,
                                           eda_shape(A, h.cls_maxn[c], h.cls_maxE[c]), counter, s, &G);
                if (rc) return rc;
                set_tuned_G(dev, A, c, G);
            } else {
                G = default_G(h.cls_maxE[c]);
            }
        }
        uint32_t k = plan.n_classes++;
        plan.G[k] = G;
        plan.begin[k] = start[c];
        plan.end[k] = start[c + 1];
        minG = std::min(minG, G);
    }
    // one shared-memory layout serves every class: widen the smallest groups until it fits
    const EdaShape w = eda_shape(A, h.maxn, h.maxE);
    while (minG < 32 && eda_smem(32 / minG, w) > 200 * 1024) minG <<= 1;
    for (uint32_t k = 0; k < plan.n_classes; k++) plan.G[k] = std::max(plan.G[k], minG);
    plan.groups_max = 32 / minG;
    return launch_persistent<A>(src, perm, plan, counter, w, s);
}

static int run_batch_algo(const BatchSrc &src, const uint32_t *perm, const BucketStats &h,
                          const unsigned long long *start, uint32_t mode, unsigned long long *counter,
                          bool allow_tune, cudaStream_t s) {
    const uint32_t form = mode & 15u;
    switch (mode >> 4) {
        case ALGO_HD: return run_batch<ALGO_HD>(src, perm, h, start, form, counter, allow_tune, s);
        case ALGO_BC: return run_batch<ALGO_BC>(src, perm, h, start, form, counter, allow_tune, s);
        case ALGO_QGRAM: return run_batch<ALGO_QGRAM>(src, perm, h, start, form, counter, allow_tune, s);
        case ALGO_SHD: return run_batch<ALGO_SHD>(src, perm, h, start, form, counter, allow_tune, s);
        default: return run_batch<ALGO_SNAKE>(src, perm, h, start, form, counter, allow_tune, s);
    }
}

// eda_mode / mode: execution form in the low 4 bits, approximation in bits 4-7.
bool eda_mode_ok(uint32_t mode) {
    return (mode & 15u) <= MT_EDA_PLAIN && (mode >> 4) < (uint32_t)N_ALGOS;
}

}  // namespace mt

using namespace mt;

extern "C" int mt_eda_batch(const uint64_t *read_words, const uint64_t *read_off, uint64_t n_reads,
                            const uint64_t *win_words, const uint64_t *win_off, const uint32_t *pair_read,
                            const uint16_t *E, uint64_t n_pairs, uint32_t mode, void *stream, uint8_t *dist) {
    if (!eda_mode_ok(mode)) return MT_EINVAL;
    if (n_pairs == 0) return MT_OK;
    if (!read_words || !read_off || !win_words || !win_off || !pair_read || !E || !dist || n_reads == 0)
        return MT_EINVAL;
    if (n_pairs > 0xFFFFFFFFull) return MT_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    int rc;
    BucketStats *st = nullptr;
    uint32_t *perm = nullptr;
    unsigned long long *cursor = nullptr;
    if ((rc = dalloc((void **)&st, sizeof(BucketStats), s))) return rc;
    if ((rc = dalloc((void **)&perm, n_pairs * 4, s))) { dfree(st, s); return rc; }
    if ((rc = dalloc((void **)&cursor, 64 * 8, s))) { dfree(st, s); dfree(perm, s); return rc; }
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
    const int by_class = (mode & 15u) == MT_EDA_BATCHED;
    const int nkeys = by_class ? MAX_CLASSES : 33;
    std::vector<unsigned long long> start(nkeys + 1, 0);
    for (int i = 0; i < nkeys; i++) start[i + 1] = start[i] + (by_class ? h.cls_count[i] : h.bkt_count[i]);
    if (cudaMemcpyAsync(cursor, start.data(), nkeys * 8, cudaMemcpyHostToDevice, s) != cudaSuccess) { cleanup(); return MT_ECUDA; }
    {
        unsigned blocks = (unsigned)std::min<uint64_t>((n_pairs + 255) / 256, (uint64_t)sm_count() * 8);
        k_bucket_scatter<<<blocks, 256, 0, s>>>(read_off, pair_read, E, n_pairs, by_class, cursor, perm);
        if (!cuda_ok(cudaGetLastError(), "k_bucket_scatter")) { cleanup(); return MT_ECUDA; }
    }
    unsigned long long *counter = cursor + 48;
    rc = run_batch_algo(src, perm, h, start.data(), mode, counter, true, s);
    if (rc) { cleanup(); return rc; }
    cudaError_t e = cudaStreamSynchronize(s);
    cleanup();
    if (!cuda_ok(e, "mt_eda_batch")) return MT_ECUDA;
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
    unsigned long long cursor[64];
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
    const int by_class = mode == MT_EDA_BATCHED;
    const int nkeys = by_class ? MAX_CLASSES : 33;
    unsigned long long start[34] = {0};
    for (int i = 0; i < nkeys; i++) start[i + 1] = start[i] + (by_class ? h.cls_count[i] : h.bkt_count[i]);
    MT_CK(cudaMemcpyAsync(cursor, start, nkeys * 8, cudaMemcpyHostToDevice, s));
    {
        unsigned blocks = (unsigned)std::min<uint64_t>((n_pairs + 255) / 256, (uint64_t)sm_count() * 8);
        k_bucket_scatter<<<blocks, 256, 0, s>>>(read_off, pair_read, E, n_pairs, by_class, cursor, perm);
        MT_CK(cudaGetLastError());
    }
    unsigned long long *counter = cursor + 48;
    // lanes per pair: the autotuned value when this process has one, else the default (no
    // timing runs here, so no events are created)
    rc = run_batch_algo(src, perm, h, start, mode, counter, false, s);
    if (rc) return rc;
    MT_CK(cudaStreamSynchronize(s));
    return MT_OK;
}
