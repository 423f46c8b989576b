// Reference index on the device (Methods, "Reference Database Organisation and Index
// Construction & Querying"): every genome's (w,k)-minimizers, found by per-thread rolling
// windows over the 2-bit packed genomes, sorted by k-mer code (stable, so each code's
// occurrences stay in (genome, position) order), run-length encoded and inserted into an
// open-addressing table of 32-byte slots.
#include <cub/cub.cuh>

#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>

#include "internal.h"

namespace mt {

static thread_local std::string g_last_cuda_error;

void set_cuda_error(cudaError_t e, const char *what) {
    g_last_cuda_error = std::string(what) + ": " + cudaGetErrorString(e);
}

bool cuda_ok(cudaError_t e, const char *what) {
    if (e == cudaSuccess) return true;
    set_cuda_error(e, what);
    return false;
}

const char *last_cuda_error() { return g_last_cuda_error.c_str(); }

int sm_count() {
    static int cached = -1;
    int dev = 0;
    cudaGetDevice(&dev);
    if (cached < 0) {
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        cached = v > 0 ? v : 1;
    }
    return cached;
}

// Allocations left before an injected failure (-1: none injected).
static std::atomic<int64_t> g_fail_after{-1};

bool alloc_fault() {
    int64_t v = g_fail_after.load();
    while (v >= 0) {
        if (g_fail_after.compare_exchange_weak(v, v - 1)) return v == 0;
    }
    return false;
}

// The default pool of each device keeps freed blocks cached in this process; set once per
// device, the first time the library allocates there.
static std::mutex g_pool_mu;
static uint64_t g_pool_set[4] = {0, 0, 0, 0};   // bit d: device d's pool configured

static void configure_pool(int dev) {
    if (dev < 0 || dev >= 256) return;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (g_pool_set[dev >> 6] >> (dev & 63) & 1u) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    g_pool_set[dev >> 6] |= 1ull << (dev & 63);
}

int dalloc(void **p, size_t bytes, cudaStream_t s) {
    int dev = 0;
    cudaGetDevice(&dev);
    configure_pool(dev);
    *p = nullptr;
    if (alloc_fault()) return MT_ENOMEM;
    if (bytes == 0) bytes = 256;
    cudaError_t e = cudaMallocAsync(p, bytes, s);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return MT_ENOMEM;
    }
    if (!cuda_ok(e, "cudaMallocAsync")) return MT_ECUDA;
    return MT_OK;
}

void dfree(void *p, cudaStream_t s) {
    if (p) cudaFreeAsync(p, s);
}

}  // namespace mt

extern "C" void mt_inject_alloc_failure(int64_t n) { mt::g_fail_after.store(n < 0 ? -1 : n); }

extern "C" uint64_t mt_pool_used_bytes(void) {
    int dev = 0;
    cudaMemPool_t pool;
    uint64_t used = 0;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess)
        cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used);
    return used;
}

namespace mt {

// ---- 2-bit packing -----------------------------------------------------------------------
// One thread per output word: the sequence owning the word is found by binary search over
// the word starts (off[i]-off0 >> 5) + i, which increase strictly with i.
__global__ void k_pack_seqs(const uint8_t *__restrict__ seq, const uint64_t *__restrict__ off,
                            uint64_t n, uint64_t *__restrict__ words, uint64_t total_words,
                            uint64_t off0, uint32_t *err) {
    uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total_words) return;
    uint64_t lo = 0, hi = n + 1;   // find the largest i in [0, n] with start(i) <= t
    while (hi - lo > 1) {
        uint64_t mid = (lo + hi) >> 1;
        uint64_t sw = ((off[mid] - off0) >> 5) + mid;
        if (sw <= t) lo = mid; else hi = mid;
    }
    uint64_t i = lo;
    uint64_t sw = ((off[i] - off0) >> 5) + i;
    if (i >= n || t < sw) { words[t] = 0; return; }
    uint64_t j = t - sw;
    uint64_t len = off[i + 1] - off[i];
    if (j * 32 >= len) { words[t] = 0; return; }
    const uint8_t *p = seq + off[i] + j * 32;
    uint32_t m = (uint32_t)umin64(32, len - j * 32);
    uint64_t w = 0;
    bool bad = false;
    for (uint32_t b = 0; b < m; b++) w |= (uint64_t)base_code(p[b], bad) << (2 * b);
    if (bad) atomicOr(err, ERR_BAD_BASE);
    words[t] = w;
}

int launch_pack_seqs(const uint8_t *seq, const uint64_t *off, uint64_t n, uint64_t *words,
                     uint64_t total_words, uint32_t *err, cudaStream_t s) {
    if (total_words == 0) return MT_OK;
    // off0 = 0: word starts use the absolute base offsets (header convention)
    uint64_t blocks = (total_words + 255) / 256;
    k_pack_seqs<<<(unsigned)blocks, 256, 0, s>>>(seq, off, n, words, total_words, 0, err);
    MT_CK(cudaGetLastError());
    return MT_OK;
}

// ---- genome minimizers --------------------------------------------------------------------
struct Chunk {
    uint32_t g;
    uint32_t j0, j1;   // windows [j0, j1) of genome g
};

__device__ __forceinline__ void genome_kmer(const uint64_t *ref, uint64_t gw, uint64_t i,
                                            uint32_t k, uint32_t canonical, uint64_t &code,
                                            uint32_t &strand, uint64_t &key) {
    uint64_t pos = i;
    const uint64_t *base = ref + gw + (pos >> 5);
    uint32_t sh = (uint32_t)(pos & 31u) * 2u;
    uint64_t x = (base[0] >> sh) | ((base[1] << 1) << (63u - sh));
    uint64_t fwd, rc;
    kmer_codes(x, k, fwd, rc);
    canon(fwd, rc, canonical, code, strand);
    key = mix64(code);
}

// Sequential sliding-window minimum over windows [j0, j1) of one genome. Window j covers
// k-mers [j, j + w). The leftmost smallest key wins; a selected position is emitted once
// (selections never move backwards, so comparing with the previous window suffices).
// mode 0: count only; mode 1: write (code, occ) at out + base.
template <int MODE>
__device__ uint32_t chunk_minimizers(const uint64_t *ref, uint64_t gw, uint32_t g, uint32_t j0,
                                     uint32_t j1, uint32_t k, uint32_t w, uint32_t canonical,
                                     uint64_t *out_code, uint64_t *out_occ) {
    uint32_t start = j0 > 0 ? j0 - 1 : 0;
    uint64_t cur_code, cur_key;
    uint32_t cur_strand, cur_pos = start;
    genome_kmer(ref, gw, start, k, canonical, cur_code, cur_strand, cur_key);
    for (uint32_t t = start + 1; t < start + w; t++) {
        uint64_t c, kk; uint32_t s;
        genome_kmer(ref, gw, t, k, canonical, c, s, kk);
        if (kk < cur_key) { cur_key = kk; cur_code = c; cur_strand = s; cur_pos = t; }
    }
    uint32_t cnt = 0;
    uint32_t prev = 0xFFFFFFFFu;
    uint32_t jfirst = j0;
    if (j0 > 0) {
        prev = cur_pos;             // selection of window j0 - 1 (owned by the previous chunk)
        jfirst = j0;
    } else {
        if (MODE) { out_code[0] = cur_code; out_occ[0] = ((uint64_t)g << 33) | ((uint64_t)cur_pos << 1) | cur_strand; }
        cnt = 1;
        prev = cur_pos;
        jfirst = 1;
    }
    for (uint32_t j = jfirst; j < j1; j++) {
        uint32_t p = j + w - 1;
        if (cur_pos < j) {          // the minimum left the window: rescan it
            genome_kmer(ref, gw, j, k, canonical, cur_code, cur_strand, cur_key);
            cur_pos = j;
            for (uint32_t t = j + 1; t <= p; t++) {
                uint64_t c, kk; uint32_t s;
                genome_kmer(ref, gw, t, k, canonical, c, s, kk);
                if (kk < cur_key) { cur_key = kk; cur_code = c; cur_strand = s; cur_pos = t; }
            }
        } else {
            uint64_t c, kk; uint32_t s;
            genome_kmer(ref, gw, p, k, canonical, c, s, kk);
            if (kk < cur_key) { cur_key = kk; cur_code = c; cur_strand = s; cur_pos = p; }
        }
        if (cur_pos != prev) {
            if (MODE) {
                out_code[cnt] = cur_code;
                out_occ[cnt] = ((uint64_t)g << 33) | ((uint64_t)cur_pos << 1) | cur_strand;
            }
            cnt++;
            prev = cur_pos;
        }
    }
    return cnt;
}

__global__ void k_genome_min_count(const uint64_t *ref, const uint64_t *gword, const Chunk *ch,
                                   uint64_t n_chunks, uint32_t k, uint32_t w, uint32_t canonical,
                                   uint64_t *counts) {
    uint64_t c = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_chunks) return;
    Chunk q = ch[c];
    counts[c] = chunk_minimizers<0>(ref, gword[q.g], q.g, q.j0, q.j1, k, w, canonical, nullptr, nullptr);
}

// offs: the chunk's first output slot; counts (nullable): the number written, when offs are
// upper-bound slots (one per window plus one) to be compacted afterwards
__global__ void k_genome_min_write(const uint64_t *ref, const uint64_t *gword, const Chunk *ch,
                                   uint64_t n_chunks, uint32_t k, uint32_t w, uint32_t canonical,
                                   const uint64_t *offs, uint64_t *codes, uint64_t *occs, uint64_t *counts) {
    uint64_t c = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_chunks) return;
    Chunk q = ch[c];
    uint64_t o = offs[c];
    const uint32_t n = chunk_minimizers<1>(ref, gword[q.g], q.g, q.j0, q.j1, k, w, canonical, codes + o, occs + o);
    if (counts) counts[c] = n;
}

// packs every chunk's entries from its upper-bound slots to its place in chunk order (a warp
// per chunk)
__global__ void k_compact_chunks(uint64_t n_chunks, const uint64_t *ub, const uint64_t *cnt, const uint64_t *coff,
                                 const uint64_t *code_in, const uint64_t *occ_in, uint64_t *code_out,
                                 uint64_t *occ_out) {
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t lane = threadIdx.x & 31u;
    if (warp >= n_chunks) return;
    const uint64_t src = ub[warp], dst = coff[warp], n = cnt[warp];
    for (uint64_t i = lane; i < n; i += 32) {
        code_out[dst + i] = code_in[src + i];
        occ_out[dst + i] = occ_in[src + i];
    }
}

// ---- table insert -------------------------------------------------------------------------
__global__ void k_insert(const uint64_t *ucode, const uint32_t *ucount, const uint64_t *uoff,
                         const int64_t *n_keys_p, const uint64_t *occ, unsigned long long *table,
                         uint64_t mask, uint32_t shift, uint32_t *err) {
    uint64_t n_keys = (uint64_t)*n_keys_p;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_keys;
         i += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t code = ucode[i];
        uint32_t cnt = ucount[i];
        uint64_t off = uoff[i];
        uint32_t ni = cnt <= 3 ? cnt : 0;
        uint64_t w0 = (code + 1) | ((uint64_t)ni << 62);
        uint64_t s = slot_of(mix64(code), shift);
        bool done = false;
        for (uint64_t it = 0; it <= mask; it++) {
            unsigned long long prev = atomicCAS(&table[4 * s], 0ull, (unsigned long long)w0);
            if (prev == 0ull) {
                if (ni == 0) {
                    uint64_t c24 = cnt < (1u << 24) ? cnt : (1u << 24) - 1;
                    table[4 * s + 1] = (c24 << 40) | (off & OFF_MASK40);
                } else {
                    for (uint32_t t = 0; t < ni; t++) table[4 * s + 1 + t] = occ[off + t];
                }
                done = true;
                break;
            }
            s = (s + 1) & mask;
        }
        if (!done) atomicOr(err, ERR_PROBE_LIMIT);
    }
}

// ---- key filter -------------------------------------------------------------------------------
// One pass over the table: every stored key sets its three bits in its block. 8-16 bits a key
// (a power of two of blocks), so the filters of a few dozen batch indexes stay in L2.
__global__ void k_key_filter(const unsigned long long *table, uint64_t slots, uint64_t *filter, uint32_t shift) {
    for (uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; s < slots; s += (uint64_t)gridDim.x * blockDim.x) {
        const unsigned long long w0 = table[4 * s];
        if (!w0) continue;
        const uint64_t key = mix64((w0 & CODE_MASK62) - 1);
        atomicOr(reinterpret_cast<unsigned long long *>(&filter[filter_block(key, shift)]),
                 (unsigned long long)filter_bits(key));
    }
}

int build_key_filter(mt_index *ix, cudaStream_t s) {
    uint64_t blocks = 1024;
    while (blocks * 8 < ix->n_keys) blocks <<= 1;
    uint32_t lg = 0;
    while ((1ull << lg) < blocks) lg++;
    if (ix->d_filter) cudaFree(ix->d_filter);
    ix->d_filter = nullptr;
    MT_CK(cudaMalloc((void **)&ix->d_filter, blocks * 8));
    ix->filter_blocks = blocks;
    ix->filter_shift = 64 - lg;
    MT_CK(cudaMemsetAsync(ix->d_filter, 0, blocks * 8, s));
    const unsigned grid = (unsigned)std::min<uint64_t>((ix->slots + 255) / 256, (uint64_t)sm_count() * 8);
    k_key_filter<<<grid, 256, 0, s>>>((const unsigned long long *)ix->d_table, ix->slots, ix->d_filter, ix->filter_shift);
    MT_CK(cudaGetLastError());
    return MT_OK;
}

// ---- homopolymer compression (the containment index's seeds, minimap2's -H) ------------------
// Each run of one repeated byte in a sequence becomes one byte; runs never join across
// sequences. One block per sequence: count, then write in tiles of 4 bytes a thread with a
// block-wide scan of the kept counts.
static constexpr int HPC_THREADS = 256;

__global__ void __launch_bounds__(HPC_THREADS) k_hpc_count(const uint8_t *seq, const uint64_t *off,
                                                             uint64_t *cnt) {
    const uint64_t a = off[blockIdx.x], b = off[blockIdx.x + 1];
    uint64_t c = 0;
    for (uint64_t j = a + threadIdx.x; j < b; j += HPC_THREADS) c += (j == a || seq[j] != seq[j - 1]);
    typedef cub::BlockReduce<uint64_t, HPC_THREADS> Reduce;
    __shared__ typename Reduce::TempStorage tmp;
    const uint64_t tot = Reduce(tmp).Sum(c);
    if (threadIdx.x == 0) cnt[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(HPC_THREADS) k_hpc_write(const uint8_t *seq, const uint64_t *off,
                                                             const uint64_t *out_off, uint8_t *out) {
    const uint64_t a = off[blockIdx.x], b = off[blockIdx.x + 1];
    typedef cub::BlockScan<uint32_t, HPC_THREADS> Scan;
    __shared__ typename Scan::TempStorage tmp;
    uint64_t o = out_off[blockIdx.x];
    for (uint64_t t0 = a; t0 < b; t0 += 4 * HPC_THREADS) {
        const uint64_t j0 = t0 + 4ull * threadIdx.x;
        uint32_t keep = 0;
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const uint64_t j = j0 + q;
            if (j < b && (j == a || seq[j] != seq[j - 1])) keep |= 1u << q;
        }
        uint32_t pos, total;
        Scan(tmp).ExclusiveSum((uint32_t)__popc(keep), pos, total);
#pragma unroll
        for (int q = 0; q < 4; q++)
            if (keep & (1u << q)) out[o + pos++] = seq[j0 + q];
        o += total;
        __syncthreads();   // tmp is reused by the next tile
    }
}

}  // namespace mt

using namespace mt;

// ids: genome g of the index is genome ids[g] of the set (its bytes copied straight to the
// device, run by run of consecutive ids), or genome g itself when ids is null.
static int build_impl(const uint8_t *genomes, const uint64_t *offsets, const uint32_t *ids, uint32_t G,
                      const mt_index_params *p, cudaStream_t s, mt_index *ix) {
    auto src = [&](uint32_t g) { return ids ? ids[g] : g; };
    for (uint32_t g = 0; g < G; g++) {
        const uint64_t a = offsets[src(g)], b = offsets[src(g) + 1];
        if (b < a) return MT_EINVAL;
        if (b - a >= (1ull << 32)) return MT_EINVAL;
    }
    ix->G = G; ix->k = p->k; ix->w = p->w; ix->canonical = p->canonical ? 1 : 0;
    ix->hpc = (p->flags & MT_INDEX_HPC) ? 1 : 0;
    std::vector<uint64_t> hoff(G + 1, 0), hgword(G);
    for (uint32_t g = 0; g < G; g++) hoff[g + 1] = hoff[g] + (offsets[src(g) + 1] - offsets[src(g)]);
    uint64_t total = hoff[G];

    int rc = MT_OK;
    uint8_t *d_seq = nullptr;
    uint64_t *d_off = nullptr;
    uint32_t *d_err = nullptr;
    uint32_t h_err = 0;
    if ((rc = dalloc((void **)&d_seq, std::max<uint64_t>(total, 1), s))) return rc;
    if ((rc = dalloc((void **)&d_off, (G + 1) * 8, s))) return rc;
    if ((rc = dalloc((void **)&d_err, 4, s))) return rc;
    for (uint32_t g = 0; g < G && total;) {
        uint32_t e = g + 1;   // a run of genomes adjacent in the set
        while (e < G && offsets[src(e)] == offsets[src(e - 1) + 1]) e++;
        const uint64_t bytes = hoff[e] - hoff[g];
        if (bytes) MT_CK(cudaMemcpyAsync(d_seq + hoff[g], genomes + offsets[src(g)], bytes, cudaMemcpyHostToDevice, s));
        g = e;
    }
    MT_CK(cudaMemcpyAsync(d_off, hoff.data(), (G + 1) * 8, cudaMemcpyHostToDevice, s));
    if (ix->hpc) {   // the genomes are indexed in homopolymer-compressed form
        uint64_t *d_cnt = nullptr, *d_off2 = nullptr;
        uint8_t *d_seq2 = nullptr;
        if ((rc = dalloc((void **)&d_cnt, G * 8ull, s))) return rc;
        k_hpc_count<<<G, HPC_THREADS, 0, s>>>(d_seq, d_off, d_cnt);
        MT_CK(cudaGetLastError());
        std::vector<uint64_t> cnt(G);
        MT_CK(cudaMemcpyAsync(cnt.data(), d_cnt, G * 8ull, cudaMemcpyDeviceToHost, s));
        MT_CK(cudaStreamSynchronize(s));
        dfree(d_cnt, s);
        std::vector<uint64_t> hoff2(G + 1, 0);
        for (uint32_t g = 0; g < G; g++) hoff2[g + 1] = hoff2[g] + cnt[g];
        if ((rc = dalloc((void **)&d_seq2, std::max<uint64_t>(hoff2[G], 1), s))) return rc;
        if ((rc = dalloc((void **)&d_off2, (G + 1) * 8, s))) return rc;
        MT_CK(cudaMemcpyAsync(d_off2, hoff2.data(), (G + 1) * 8, cudaMemcpyHostToDevice, s));
        k_hpc_write<<<G, HPC_THREADS, 0, s>>>(d_seq, d_off, d_off2, d_seq2);
        MT_CK(cudaGetLastError());
        dfree(d_seq, s);
        dfree(d_off, s);
        d_seq = d_seq2;
        d_off = d_off2;
        hoff = hoff2;
        total = hoff2[G];
    }
    ix->total_bases = total;
    ix->h_glen.resize(G);
    for (uint32_t g = 0; g < G; g++) {
        ix->h_glen[g] = hoff[g + 1] - hoff[g];
        hgword[g] = (hoff[g] >> 5) + g;
    }
    ix->ref_words = (total >> 5) + G + 1;
    {   // 32-bit match keys (genome | strand | diagonal + bias) when they fit
        uint64_t max_len = 0;
        for (uint32_t g = 0; g < G; g++) max_len = std::max<uint64_t>(max_len, ix->h_glen[g]);
        uint32_t db = 1, gb = 1;
        while ((1ull << db) <= max_len + DIAG_BIAS + MT_MAX_E + 2) db++;
        while ((1ull << gb) < G) gb++;
        ix->hk_db = (gb + 1 + db <= 32) ? db : 0;
    }

    MT_CK(cudaMemsetAsync(d_err, 0, 4, s));
    MT_CK(cudaMalloc((void **)&ix->d_ref, ix->ref_words * 8));
    MT_CK(cudaMalloc((void **)&ix->d_gword, G * 8));
    MT_CK(cudaMalloc((void **)&ix->d_glen, G * 8));
    MT_CK(cudaMemcpyAsync(ix->d_gword, hgword.data(), G * 8, cudaMemcpyHostToDevice, s));
    MT_CK(cudaMemcpyAsync(ix->d_glen, ix->h_glen.data(), G * 8, cudaMemcpyHostToDevice, s));
    {
        uint64_t blocks = (ix->ref_words + 255) / 256;
        k_pack_seqs<<<(unsigned)blocks, 256, 0, s>>>(d_seq, d_off, G, ix->d_ref, ix->ref_words, 0, d_err);
        MT_CK(cudaGetLastError());
    }
    MT_CK(cudaMemcpyAsync(&h_err, d_err, 4, cudaMemcpyDeviceToHost, s));
    MT_CK(cudaStreamSynchronize(s));
    dfree(d_seq, s);
    dfree(d_off, s);
    if (h_err) { dfree(d_err, s); return MT_EINVAL; }

    // chunks of windows
    const uint32_t CH = 2048;
    std::vector<Chunk> chunks;
    for (uint32_t g = 0; g < G; g++) {
        uint64_t L = ix->h_glen[g];
        if (L < p->k) continue;
        uint64_t nk = L - p->k + 1;
        if (nk < p->w) continue;
        uint64_t nwin = nk - p->w + 1;
        for (uint64_t j = 0; j < nwin; j += CH)
            chunks.push_back(Chunk{g, (uint32_t)j, (uint32_t)std::min<uint64_t>(nwin, j + CH)});
    }
    uint64_t n_chunks = chunks.size();
    Chunk *d_ch = nullptr;
    uint64_t *d_cnt = nullptr, *d_coff = nullptr;
    if ((rc = dalloc((void **)&d_ch, std::max<uint64_t>(1, n_chunks) * sizeof(Chunk), s))) return rc;
    if ((rc = dalloc((void **)&d_cnt, (n_chunks + 1) * 8, s))) return rc;
    if ((rc = dalloc((void **)&d_coff, (n_chunks + 1) * 8, s))) return rc;
    if (n_chunks) MT_CK(cudaMemcpyAsync(d_ch, chunks.data(), n_chunks * sizeof(Chunk), cudaMemcpyHostToDevice, s));
    MT_CK(cudaMemsetAsync(d_cnt, 0, (n_chunks + 1) * 8, s));
    // One pass over the genomes when upper-bound staging (a window adds at most one position,
    // a chunk at most its windows plus one) fits in a quarter of the free memory and 32 GB:
    // chunks write at upper-bound slots and record their counts, then a compaction packs them
    // in chunk order. Otherwise the minimizers are found twice: counted, then written.
    std::vector<uint64_t> ub(n_chunks + 1, 0);
    for (uint64_t c = 0; c < n_chunks; c++) ub[c + 1] = ub[c] + (chunks[c].j1 - chunks[c].j0) + 1;
    size_t free_b = 0, total_b = 0;
    MT_CK(cudaMemGetInfo(&free_b, &total_b));
    const bool one_pass = n_chunks && ub[n_chunks] * 16 <= std::min<uint64_t>(free_b / 4, 32ull << 30);
    uint64_t *d_ub = nullptr, *d_ub_code = nullptr, *d_ub_occ = nullptr;
    if (one_pass) {
        if ((rc = dalloc((void **)&d_ub, (n_chunks + 1) * 8, s))) return rc;
        if ((rc = dalloc((void **)&d_ub_code, ub[n_chunks] * 8, s))) return rc;
        if ((rc = dalloc((void **)&d_ub_occ, ub[n_chunks] * 8, s))) return rc;
        MT_CK(cudaMemcpyAsync(d_ub, ub.data(), (n_chunks + 1) * 8, cudaMemcpyHostToDevice, s));
        k_genome_min_write<<<(unsigned)((n_chunks + 127) / 128), 128, 0, s>>>(
            ix->d_ref, ix->d_gword, d_ch, n_chunks, p->k, p->w, ix->canonical, d_ub, d_ub_code, d_ub_occ, d_cnt);
        MT_CK(cudaGetLastError());
    } else if (n_chunks) {
        k_genome_min_count<<<(unsigned)((n_chunks + 127) / 128), 128, 0, s>>>(
            ix->d_ref, ix->d_gword, d_ch, n_chunks, p->k, p->w, ix->canonical, d_cnt);
        MT_CK(cudaGetLastError());
    }
    void *d_tmp = nullptr;
    size_t tmp_bytes = 0;
    MT_CK(cub::DeviceScan::ExclusiveSum(nullptr, tmp_bytes, d_cnt, d_coff, (int64_t)(n_chunks + 1), s));
    if ((rc = dalloc(&d_tmp, tmp_bytes, s))) return rc;
    MT_CK(cub::DeviceScan::ExclusiveSum(d_tmp, tmp_bytes, d_cnt, d_coff, (int64_t)(n_chunks + 1), s));
    dfree(d_tmp, s);
    uint64_t n_occ = 0;
    MT_CK(cudaMemcpyAsync(&n_occ, d_coff + n_chunks, 8, cudaMemcpyDeviceToHost, s));
    MT_CK(cudaStreamSynchronize(s));
    ix->n_occ = n_occ;

    uint64_t *d_code[2] = {nullptr, nullptr}, *d_val[2] = {nullptr, nullptr};
    uint64_t nb = std::max<uint64_t>(1, n_occ) * 8;
    if ((rc = dalloc((void **)&d_code[0], nb, s))) return rc;
    if ((rc = dalloc((void **)&d_code[1], nb, s))) return rc;
    if ((rc = dalloc((void **)&d_val[0], nb, s))) return rc;
    MT_CK(cudaMalloc((void **)&d_val[1], nb));   // becomes the resident occurrence array
    if (one_pass) {
        k_compact_chunks<<<(unsigned)((n_chunks * 32 + 255) / 256), 256, 0, s>>>(
            n_chunks, d_ub, d_cnt, d_coff, d_ub_code, d_ub_occ, d_code[0], d_val[0]);
        MT_CK(cudaGetLastError());
        dfree(d_ub, s); dfree(d_ub_code, s); dfree(d_ub_occ, s);
    } else if (n_chunks) {
        k_genome_min_write<<<(unsigned)((n_chunks + 127) / 128), 128, 0, s>>>(
            ix->d_ref, ix->d_gword, d_ch, n_chunks, p->k, p->w, ix->canonical, d_coff,
            d_code[0], d_val[0], nullptr);
        MT_CK(cudaGetLastError());
    }
    dfree(d_ch, s); dfree(d_cnt, s); dfree(d_coff, s);

    // stable sort by code: each code's occurrences keep their (genome, position) order
    cub::DoubleBuffer<uint64_t> kb(d_code[0], d_code[1]), vb(d_val[0], d_val[1]);
    tmp_bytes = 0;
    int end_bit = (int)(2 * p->k);
    if (end_bit < 1) end_bit = 1;
    MT_CK(cub::DeviceRadixSort::SortPairs(nullptr, tmp_bytes, kb, vb, (int64_t)n_occ, 0, end_bit, s));
    if ((rc = dalloc(&d_tmp, tmp_bytes, s))) return rc;
    MT_CK(cub::DeviceRadixSort::SortPairs(d_tmp, tmp_bytes, kb, vb, (int64_t)n_occ, 0, end_bit, s));
    dfree(d_tmp, s);
    uint64_t *codes_sorted = kb.Current();
    uint64_t *occ_sorted = vb.Current();
    uint64_t *code_spare = kb.Alternate();
    uint64_t *occ_spare = vb.Alternate();

    // distinct codes and their run lengths / offsets
    uint64_t *d_ucode = code_spare;   // reuse the spare key buffer
    uint32_t *d_ucount = nullptr;
    uint64_t *d_uoff = nullptr;
    int64_t *d_nruns = nullptr;
    if ((rc = dalloc((void **)&d_ucount, std::max<uint64_t>(1, n_occ) * 4, s))) return rc;
    if ((rc = dalloc((void **)&d_uoff, std::max<uint64_t>(1, n_occ) * 8, s))) return rc;
    if ((rc = dalloc((void **)&d_nruns, 8, s))) return rc;
    MT_CK(cudaMemsetAsync(d_nruns, 0, 8, s));
    if (n_occ) {
        tmp_bytes = 0;
        MT_CK(cub::DeviceRunLengthEncode::Encode(nullptr, tmp_bytes, codes_sorted, d_ucode, d_ucount,
                                                 d_nruns, (int64_t)n_occ, s));
        if ((rc = dalloc(&d_tmp, tmp_bytes, s))) return rc;
        MT_CK(cub::DeviceRunLengthEncode::Encode(d_tmp, tmp_bytes, codes_sorted, d_ucode, d_ucount,
                                                 d_nruns, (int64_t)n_occ, s));
        dfree(d_tmp, s);
    }
    int64_t n_keys = 0;
    MT_CK(cudaMemcpyAsync(&n_keys, d_nruns, 8, cudaMemcpyDeviceToHost, s));
    MT_CK(cudaStreamSynchronize(s));
    ix->n_keys = (uint64_t)n_keys;
    if (n_keys) {
        tmp_bytes = 0;
        MT_CK(cub::DeviceScan::ExclusiveSum(nullptr, tmp_bytes, d_ucount, d_uoff, n_keys, s));
        if ((rc = dalloc(&d_tmp, tmp_bytes, s))) return rc;
        MT_CK(cub::DeviceScan::ExclusiveSum(d_tmp, tmp_bytes, d_ucount, d_uoff, n_keys, s));
        dfree(d_tmp, s);
    }

    // load factor <= 1/4 while the table stays within 16 GB (fewer warps wait on a second
    // probe), else <= 1/2
    uint64_t slots = 1024;
    while (slots < 4 * (uint64_t)n_keys) slots <<= 1;
    if (slots * 32 > (16ull << 30)) {
        slots = 1024;
        while (slots < 2 * (uint64_t)n_keys) slots <<= 1;
    }
    uint32_t lg = 0;
    while ((1ull << lg) < slots) lg++;
    ix->slots = slots;
    ix->slot_shift = 64 - lg;
    MT_CK(cudaMalloc((void **)&ix->d_table, slots * 32));
    MT_CK(cudaMemsetAsync(ix->d_table, 0, slots * 32, s));
    if (n_keys) {
        unsigned blocks = (unsigned)std::min<uint64_t>((n_keys + 255) / 256, 65535ull * 16);
        k_insert<<<blocks, 256, 0, s>>>(d_ucode, d_ucount, d_uoff, d_nruns, occ_sorted,
                                         (unsigned long long *)ix->d_table, slots - 1, ix->slot_shift, d_err);
        MT_CK(cudaGetLastError());
    }
    MT_CK(cudaMemcpyAsync(&h_err, d_err, 4, cudaMemcpyDeviceToHost, s));
    MT_CK(cudaStreamSynchronize(s));
    // keep the sorted occurrence array; release the rest
    if (occ_sorted == d_val[1]) {
        ix->d_occ = d_val[1];
        dfree(d_val[0], s);
    } else {
        // the sorted values ended in the pool buffer: move them to the resident one
        MT_CK(cudaMemcpyAsync(d_val[1], occ_sorted, nb, cudaMemcpyDeviceToDevice, s));
        ix->d_occ = d_val[1];
        dfree(d_val[0], s);
    }
    (void)occ_spare;
    dfree(d_code[0], s); dfree(d_code[1], s);
    dfree(d_ucount, s); dfree(d_uoff, s); dfree(d_nruns, s); dfree(d_err, s);
    if (!h_err && (rc = build_key_filter(ix, s))) return rc;
    MT_CK(cudaStreamSynchronize(s));
    if (h_err) return MT_ECUDA;
    ix->device_bytes = ix->ref_words * 8 + G * 16 + slots * 32 + nb + ix->filter_blocks * 8;
    return MT_OK;
}

static int build_checked(const uint8_t *genomes, const uint64_t *offsets, const uint32_t *ids, uint32_t n_genomes,
                         const mt_index_params *p, void *stream, mt_index **out) {
    if (!out) return MT_EINVAL;
    *out = nullptr;
    if (!genomes || !offsets || !p || n_genomes == 0 || n_genomes > MT_MAX_GENOMES) return MT_EINVAL;
    if (p->k < 1 || p->k > MT_MAX_K || p->w < 1 || p->w > MT_MAX_W || (p->flags & ~MT_INDEX_HPC) != 0) return MT_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    mt_index *ix = new mt_index();
    cudaGetDevice(&ix->device);
    int rc = build_impl(genomes, offsets, ids, n_genomes, p, s, ix);
    if (rc != MT_OK) {
        cudaStreamSynchronize(s);
        mt_free_index(ix);
        return rc;
    }
    *out = ix;
    return MT_OK;
}

extern "C" int mt_build_index(const uint8_t *genomes, const uint64_t *offsets, uint32_t n_genomes,
                              const mt_index_params *p, void *stream, mt_index **out) {
    Trace trace("mt_build_index");
    return build_checked(genomes, offsets, nullptr, n_genomes, p, stream, out);
}

extern "C" int mt_build_index_subset(const uint8_t *genomes, const uint64_t *offsets, uint32_t n_set,
                                     const uint32_t *ids, uint32_t n_ids, const mt_index_params *p, void *stream,
                                     mt_index **out) {
    if (out) *out = nullptr;
    if (!ids) return MT_EINVAL;
    for (uint32_t i = 0; i < n_ids; i++)
        if (ids[i] >= n_set) return MT_EINVAL;
    return build_checked(genomes, offsets, ids, n_ids, p, stream, out);
}

extern "C" const char *mt_last_cuda_error(void) { return mt::last_cuda_error(); }

extern "C" void mt_free_index(mt_index *ix) {
    if (!ix) return;
    cudaFree(ix->d_ref);
    cudaFree(ix->d_gword);
    cudaFree(ix->d_glen);
    cudaFree(ix->d_table);
    cudaFree(ix->d_occ);
    cudaFree(ix->d_filter);
    delete ix;
}

extern "C" int mt_index_get_info(const mt_index *ix, mt_index_info *info) {
    if (!ix || !info) return MT_EINVAL;
    info->n_genomes = ix->G;
    info->k = ix->k;
    info->w = ix->w;
    info->canonical = ix->canonical;
    info->total_bases = ix->total_bases;
    info->n_occ = ix->n_occ;
    info->n_keys = ix->n_keys;
    info->table_slots = ix->slots;
    info->device_bytes = ix->device_bytes;
    info->flags = ix->hpc ? MT_INDEX_HPC : 0u;
    info->pad = 0;
    return MT_OK;
}

extern "C" int mt_pack_seqs(const uint8_t *seq, const uint64_t *offsets, uint64_t n_seqs,
                            uint64_t *words, void *stream) {
    if (!seq || !offsets || !words) return MT_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    if (n_seqs == 0) return MT_OK;
    uint64_t last = 0;
    MT_CK(cudaMemcpyAsync(&last, offsets + n_seqs, 8, cudaMemcpyDeviceToHost, s));
    uint32_t *d_err = nullptr;
    int rc = dalloc((void **)&d_err, 4, s);
    if (rc) return rc;
    MT_CK(cudaMemsetAsync(d_err, 0, 4, s));
    MT_CK(cudaStreamSynchronize(s));
    uint64_t total_words = (last >> 5) + n_seqs + 1;
    rc = launch_pack_seqs(seq, offsets, n_seqs, words, total_words, d_err, s);
    uint32_t h_err = 0;
    if (rc == MT_OK) {
        MT_CK(cudaMemcpyAsync(&h_err, d_err, 4, cudaMemcpyDeviceToHost, s));
        MT_CK(cudaStreamSynchronize(s));
    }
    dfree(d_err, s);
    if (rc) return rc;
    return h_err ? MT_EINVAL : MT_OK;
}
