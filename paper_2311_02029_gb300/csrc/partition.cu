// One read batch against a reference database cut into batches (Methods, "Reference Database
// Organisation and Index Construction & Querying"; Evaluation Methodology).
//
// Stage 1 runs batch by batch with each batch's own index (the counting seeding kernel of
// mt_containment), or for all resident batches at once in one pass of that kernel that finds
// each read's minimizers once and looks them up in every batch's table; a genome keeps the
// highest count any batch gave it (one atomicMax per genome slot). The normalised cutoff then
// runs over the whole database, and stages 2-3 run against the subset index of the kept
// genomes (mt_classify_masked, every subset genome kept); the subset's genome ids are mapped
// back to global ids on the device. Between calls the query holds only the reads and
// n_genomes-sized vectors, so database batches can pass through device memory one at a time.
//
// Genome shards over ranks (mt_classify_genome_sharded, at the end of this file) reuse the
// query: each rank counts and maps against its own shard, and every rank merges all ranks'
// per-read locations by rank and decides them (merge_decide).
#include <algorithm>
#include <cstring>
#include <vector>

#include "internal.h"

namespace mt {

// highest count per global genome over the batches seen so far
__global__ void k_part_max(const unsigned long long *hits, const uint32_t *ids, uint32_t n, unsigned long long *H) {
    for (uint32_t l = blockIdx.x * blockDim.x + threadIdx.x; l < n; l += gridDim.x * blockDim.x)
        if (hits[l]) atomicMax(&H[ids[l]], hits[l]);
}

// subset genome ids -> global ids in the per-read outputs
__global__ void k_part_ids(uint64_t n_reads, uint32_t top_n, const uint32_t *ids, int32_t *taxon, mt_loc *locs) {
    const uint64_t n = n_reads * top_n;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        if (taxon && i < n_reads) {
            const int32_t t = taxon[i];
            if (t >= 0) taxon[i] = (int32_t)ids[t];
        }
        if (locs) {
            const int32_t g = locs[i].genome;
            if (g >= 0) locs[i].genome = (int32_t)ids[g];
        }
    }
}

__global__ void k_part_scatter(const double *a_sub, const uint32_t *ids, uint32_t n, double *a) {
    for (uint32_t l = blockIdx.x * blockDim.x + threadIdx.x; l < n; l += gridDim.x * blockDim.x) a[ids[l]] = a_sub[l];
}

// outputs of a query in which no genome was kept: no read maps
__global__ void k_part_empty(uint64_t n_reads, uint32_t top_n, int32_t *taxon, uint8_t *nloc, mt_loc *locs) {
    const uint64_t n = n_reads * top_n;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        if (i < n_reads) {
            taxon[i] = -1;
            if (nloc) nloc[i] = 0;
        }
        if (locs) {
            mt_loc L;
            memset(&L, 0, sizeof(L));
            L.genome = -1;
            locs[i] = L;
        }
    }
}

static unsigned grid_for(uint64_t n) {
    return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>((n + 255) / 256, (uint64_t)sm_count() * 4));
}

}  // namespace mt

using namespace mt;

struct mt_part {
    cudaStream_t s = nullptr;
    uint32_t G = 0;
    uint64_t n_reads = 0, n_bases = 0;
    bool host_io = false;
    const uint8_t *reads = nullptr;     // device
    const uint64_t *roff = nullptr;     // device
    unsigned char *mem = nullptr;       // H | keep | copies of host reads and offsets
    unsigned long long *H = nullptr;    // highest seed hits per global genome
    uint8_t *keep = nullptr;
    bool have_subset = false;
    std::vector<uint32_t> kept;         // kept global ids of the last cutoff, increasing
};

extern "C" int mt_part_create(uint32_t n_genomes, const uint8_t *reads, uint64_t n_bases, const uint64_t *offsets,
                              uint64_t n_reads, int device_ptrs, void *stream, mt_part **out) {
    if (!out) return MT_EINVAL;
    *out = nullptr;
    if (!n_genomes || !offsets || (!reads && n_bases)) return MT_EINVAL;
    mt_part *q = new mt_part;
    q->s = (cudaStream_t)stream;
    q->G = n_genomes;
    q->n_reads = n_reads;
    q->n_bases = n_bases;
    q->host_io = !device_ptrs;
    Carver c;
    const size_t o_H = c.take<uint64_t>(n_genomes), o_keep = c.take<uint8_t>(n_genomes);
    const size_t o_reads = q->host_io ? c.take<uint8_t>(std::max<uint64_t>(n_bases, 1)) : 0;
    const size_t o_off = q->host_io ? c.take<uint64_t>(n_reads + 1) : 0;
    int rc = dalloc((void **)&q->mem, c.off + 256, q->s);
    if (rc) { delete q; return rc; }
    q->H = (unsigned long long *)(q->mem + o_H);
    q->keep = q->mem + o_keep;
    auto fail = [&](int code) { mt_part_destroy(q); return code; };
    if (!cuda_ok(cudaMemsetAsync(q->H, 0, n_genomes * 8ull, q->s), "part H")) return fail(MT_ECUDA);
    if (q->host_io) {
        q->reads = q->mem + o_reads;
        q->roff = (const uint64_t *)(q->mem + o_off);
        if (n_bases && !cuda_ok(cudaMemcpyAsync((void *)q->reads, reads, n_bases, cudaMemcpyHostToDevice, q->s), "part reads"))
            return fail(MT_ECUDA);
        if (!cuda_ok(cudaMemcpyAsync((void *)q->roff, offsets, (n_reads + 1) * 8, cudaMemcpyHostToDevice, q->s), "part offsets"))
            return fail(MT_ECUDA);
    } else {
        q->reads = reads;
        q->roff = offsets;
    }
    if (!cuda_ok(cudaStreamSynchronize(q->s), "part create")) return fail(MT_ECUDA);
    *out = q;
    return MT_OK;
}

extern "C" void mt_part_destroy(mt_part *q) {
    if (!q) return;
    if (q->mem) {
        dfree(q->mem, q->s);
        cudaStreamSynchronize(q->s);
    }
    delete q;
}

extern "C" int mt_part_contain(mt_part *q, const mt_index *batch, const uint32_t *genome_ids, uint32_t max_occ) {
    if (!q || !batch || !genome_ids) return MT_EINVAL;
    const uint32_t Gb = batch->G;
    for (uint32_t l = 0; l < Gb; l++)
        if (genome_ids[l] >= q->G) return MT_EINVAL;
    Carver c;
    const size_t o_hits = c.take<uint64_t>(Gb), o_ids = c.take<uint32_t>(Gb);
    unsigned char *ws = nullptr;
    int rc = dalloc((void **)&ws, c.off + 256, q->s);
    if (rc) return rc;
    uint64_t *hits = (uint64_t *)(ws + o_hits);
    uint32_t *ids = (uint32_t *)(ws + o_ids);
    auto done = [&](int code) { dfree(ws, q->s); cudaStreamSynchronize(q->s); return code; };
    if (!cuda_ok(cudaMemcpyAsync(ids, genome_ids, Gb * 4ull, cudaMemcpyHostToDevice, q->s), "part ids"))
        return done(MT_ECUDA);
    rc = mt_containment(batch, q->reads, q->n_bases, q->roff, q->n_reads, max_occ, 1, 1, 1, q->s, hits, nullptr);
    if (rc) return done(rc);
    k_part_max<<<grid_for(Gb), 256, 0, q->s>>>((const unsigned long long *)hits, ids, Gb, q->H);
    if (!cuda_ok(cudaGetLastError(), "k_part_max")) return done(MT_ECUDA);
    q->have_subset = false;   // the counts changed: a new cutoff is due
    return done(cuda_ok(cudaStreamSynchronize(q->s), "part contain") ? MT_OK : MT_ECUDA);
}

extern "C" int mt_part_contain_batches(mt_part *q, const mt_index *const *batches, const uint32_t *const *genome_ids,
                                       uint32_t n_batches, uint32_t max_occ) {
    if (!q || (n_batches && (!batches || !genome_ids))) return MT_EINVAL;
    if (!n_batches) return MT_OK;
    uint64_t T = 0;
    for (uint32_t b = 0; b < n_batches; b++) {
        if (!batches[b] || !genome_ids[b]) return MT_EINVAL;
        for (uint32_t l = 0; l < batches[b]->G; l++)
            if (genome_ids[b][l] >= q->G) return MT_EINVAL;
        T += batches[b]->G;
    }
    if (T >= (1ull << 31)) return MT_EINVAL;
    // the batches' global ids one after another, like their counters
    std::vector<uint32_t> ids;
    ids.reserve(T);
    for (uint32_t b = 0; b < n_batches; b++) ids.insert(ids.end(), genome_ids[b], genome_ids[b] + batches[b]->G);
    Carver c;
    const size_t o_hits = c.take<uint64_t>(T), o_ids = c.take<uint32_t>(T);
    unsigned char *ws = nullptr;
    int rc = dalloc((void **)&ws, c.off + 256, q->s);
    if (rc) return rc;
    uint64_t *hits = (uint64_t *)(ws + o_hits);
    uint32_t *d_ids = (uint32_t *)(ws + o_ids);
    auto done = [&](int code) { dfree(ws, q->s); cudaStreamSynchronize(q->s); return code; };
    if (!cuda_ok(cudaMemcpyAsync(d_ids, ids.data(), T * 4, cudaMemcpyHostToDevice, q->s), "part ids"))
        return done(MT_ECUDA);
    // one pass per MULTI_MAX_INDEXES batches
    for (uint32_t b0 = 0, base = 0; b0 < n_batches; b0 += MULTI_MAX_INDEXES) {
        const uint32_t nb = std::min(n_batches - b0, MULTI_MAX_INDEXES);
        rc = contain_multi(batches + b0, nb, q->reads, q->n_bases, q->roff, q->n_reads, max_occ, hits + base, q->s);
        if (rc) return done(rc);
        for (uint32_t b = b0; b < b0 + nb; b++) base += batches[b]->G;
    }
    k_part_max<<<grid_for(T), 256, 0, q->s>>>((const unsigned long long *)hits, d_ids, (uint32_t)T, q->H);
    if (!cuda_ok(cudaGetLastError(), "k_part_max")) return done(MT_ECUDA);
    q->have_subset = false;
    return done(cuda_ok(cudaStreamSynchronize(q->s), "part contain") ? MT_OK : MT_ECUDA);
}

extern "C" int mt_part_subset(mt_part *q, uint32_t cont_num, uint32_t cont_den, uint8_t *keep, uint64_t *genome_hits,
                              uint32_t *kept, uint32_t *n_kept) {
    if (!q || cont_den == 0) return MT_EINVAL;
    int rc = launch_mask((const uint64_t *)q->H, q->G, cont_num, cont_den, q->keep, q->s);
    if (rc) return rc;
    std::vector<uint8_t> h(q->G);
    MT_CK(cudaMemcpyAsync(h.data(), q->keep, q->G, cudaMemcpyDeviceToHost, q->s));
    if (genome_hits)
        MT_CK(cudaMemcpyAsync(genome_hits, q->H, q->G * 8ull,
                              q->host_io ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, q->s));
    MT_CK(cudaStreamSynchronize(q->s));
    q->kept.clear();
    for (uint32_t g = 0; g < q->G; g++)
        if (h[g]) q->kept.push_back(g);
    q->have_subset = true;
    if (keep) memcpy(keep, h.data(), q->G);
    if (kept && !q->kept.empty()) memcpy(kept, q->kept.data(), q->kept.size() * 4);
    if (n_kept) *n_kept = (uint32_t)q->kept.size();
    return MT_OK;
}

extern "C" int mt_part_classify(mt_part *q, const mt_index *subset, const uint32_t *subset_ids, uint32_t n_subset,
                                const mt_classify_params *p, int32_t *taxon, uint8_t *nloc, mt_loc *locs,
                                double *abundance, mt_stats *stats) {
    if (!q || !p || !q->have_subset || (!taxon && q->n_reads)) return MT_EINVAL;
    if (p->top_n < 1 || p->top_n > MT_MAX_TOPN) return MT_EINVAL;
    if (n_subset != q->kept.size() || (n_subset && (!subset || !subset_ids))) return MT_EINVAL;
    if (n_subset && (subset->G != n_subset || subset->hpc)) return MT_EINVAL;
    for (uint32_t l = 0; l < n_subset; l++)
        if (subset_ids[l] != q->kept[l]) return MT_EINVAL;
    const uint32_t top_n = p->top_n;
    const uint64_t n = q->n_reads;
    const cudaMemcpyKind down = q->host_io ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;

    // device outputs: the caller's when the query is on device buffers, else scratch
    Carver c;
    const size_t o_ones = c.take<uint8_t>(std::max<uint32_t>(n_subset, 1));
    const size_t o_ids = c.take<uint32_t>(std::max<uint32_t>(n_subset, 1));
    const size_t o_asub = c.take<double>(std::max<uint32_t>(n_subset, 1));
    const size_t o_a = c.take<double>(q->G);
    const size_t o_tax = q->host_io ? c.take<int32_t>(std::max<uint64_t>(n, 1)) : 0;
    const size_t o_nloc = q->host_io ? c.take<uint8_t>(std::max<uint64_t>(n, 1)) : 0;
    const size_t o_locs = (q->host_io && locs) ? c.take<mt_loc>(std::max<uint64_t>(n * top_n, 1)) : 0;
    unsigned char *ws = nullptr;
    int rc = dalloc((void **)&ws, c.off + 256, q->s);
    if (rc) return rc;
    auto done = [&](int code) { dfree(ws, q->s); cudaStreamSynchronize(q->s); return code; };
    int32_t *d_tax = q->host_io ? (int32_t *)(ws + o_tax) : taxon;
    uint8_t *d_nloc = q->host_io ? (uint8_t *)(ws + o_nloc) : nloc;
    mt_loc *d_locs = q->host_io ? (locs ? (mt_loc *)(ws + o_locs) : nullptr) : locs;
    double *d_a = (double *)(ws + o_a);
    uint32_t *d_ids = (uint32_t *)(ws + o_ids);
    if (!cuda_ok(cudaMemsetAsync(d_a, 0, q->G * 8ull, q->s), "part abundance")) return done(MT_ECUDA);

    if (n_subset == 0) {
        if (stats) { memset(stats, 0, sizeof(*stats)); stats->n_reads = n; }
        if (n) {
            k_part_empty<<<grid_for(n * top_n), 256, 0, q->s>>>(n, top_n, d_tax, d_nloc, d_locs);
            if (!cuda_ok(cudaGetLastError(), "k_part_empty")) return done(MT_ECUDA);
        }
    } else {
        uint8_t *ones = ws + o_ones;
        double *a_sub = (double *)(ws + o_asub);
        if (!cuda_ok(cudaMemsetAsync(ones, 1, n_subset, q->s), "part ones") ||
            !cuda_ok(cudaMemcpyAsync(d_ids, subset_ids, n_subset * 4ull, cudaMemcpyHostToDevice, q->s), "part subset ids"))
            return done(MT_ECUDA);
        rc = mt_classify_masked(subset, q->reads, q->n_bases, q->roff, n, p, 1, q->s, ones, d_tax, d_nloc, d_locs,
                                nullptr, a_sub, stats);
        if (rc) return done(rc);
        if (n) {
            k_part_ids<<<grid_for(n * top_n), 256, 0, q->s>>>(n, top_n, d_ids, d_tax, d_locs);
            if (!cuda_ok(cudaGetLastError(), "k_part_ids")) return done(MT_ECUDA);
        }
        k_part_scatter<<<grid_for(n_subset), 256, 0, q->s>>>(a_sub, d_ids, n_subset, d_a);
        if (!cuda_ok(cudaGetLastError(), "k_part_scatter")) return done(MT_ECUDA);
        if (stats) stats->n_launches += n ? 2 : 1;
    }
    if (abundance && !cuda_ok(cudaMemcpyAsync(abundance, d_a, q->G * 8ull, down, q->s), "part abundance out"))
        return done(MT_ECUDA);
    if (q->host_io && n) {
        if (!cuda_ok(cudaMemcpyAsync(taxon, d_tax, n * 4, cudaMemcpyDeviceToHost, q->s), "part taxon") ||
            (nloc && !cuda_ok(cudaMemcpyAsync(nloc, d_nloc, n, cudaMemcpyDeviceToHost, q->s), "part nloc")) ||
            (locs && !cuda_ok(cudaMemcpyAsync(locs, d_locs, n * top_n * sizeof(mt_loc), cudaMemcpyDeviceToHost, q->s), "part locs")))
            return done(MT_ECUDA);
    }
    return done(cuda_ok(cudaStreamSynchronize(q->s), "part classify") ? MT_OK : MT_ECUDA);
}

extern "C" int mt_classify_partitioned(const mt_index *const *batches, const uint32_t *const *genome_ids,
                                       uint32_t n_batches, const uint8_t *genomes, const uint64_t *genome_offsets,
                                       uint32_t n_genomes, const mt_index_params *subset_params, const uint8_t *reads,
                                       uint64_t n_bases, const uint64_t *offsets, uint64_t n_reads,
                                       const mt_classify_params *p, int device_ptrs, void *stream, int32_t *taxon,
                                       uint8_t *nloc, mt_loc *locs, uint64_t *genome_hits, double *abundance,
                                       mt_stats *stats) {
    if ((n_batches && (!batches || !genome_ids)) || !genomes || !genome_offsets || !subset_params || !p)
        return MT_EINVAL;
    if (subset_params->flags & MT_INDEX_HPC) return MT_EINVAL;
    for (uint32_t g = 0; g < n_genomes; g++)
        if (genome_offsets[g + 1] < genome_offsets[g]) return MT_EINVAL;
    mt_part *q = nullptr;
    int rc = mt_part_create(n_genomes, reads, n_bases, offsets, n_reads, device_ptrs, stream, &q);
    if (rc) return rc;
    // one pass over the reads for all batches when they share their seeds' parameters
    bool same = n_batches > 0;
    for (uint32_t b = 0; b < n_batches && same; b++)
        same = batches[b] && batches[b]->k == batches[0]->k && batches[b]->w == batches[0]->w &&
               batches[b]->canonical == batches[0]->canonical && batches[b]->hpc == batches[0]->hpc;
    if (same) rc = mt_part_contain_batches(q, batches, genome_ids, n_batches, p->max_occ);
    else
        for (uint32_t b = 0; b < n_batches && !rc; b++) rc = mt_part_contain(q, batches[b], genome_ids[b], p->max_occ);
    std::vector<uint32_t> kept(n_genomes);
    uint32_t nk = 0;
    if (!rc) rc = mt_part_subset(q, p->cont_num, p->cont_den, nullptr, genome_hits, kept.data(), &nk);
    mt_index *sub = nullptr;   // the subset database: an index over the kept genomes, in kept order
    if (!rc && nk) rc = mt_build_index_subset(genomes, genome_offsets, n_genomes, kept.data(), nk, subset_params, stream, &sub);
    if (!rc) rc = mt_part_classify(q, sub, kept.data(), nk, p, taxon, nloc, locs, abundance, stats);
    if (sub) mt_free_index(sub);
    mt_part_destroy(q);
    return rc;
}

// ---- genome shards on separate devices (one process each) ---------------------------------------
// Every rank holds an index over its own genomes and sees every read. Exchanges, through the
// caller's functions: which genomes each rank holds (a sum, to refuse shards that overlap),
// the genome hits (a sum: each genome is counted by its one rank), and every rank's per-read
// top_n locations (an all-gather), which each rank merges by rank and decides.
extern "C" int mt_classify_genome_sharded(const mt_index *shard, const uint32_t *genome_ids, uint32_t n_genomes,
                                          uint32_t n_ranks, const uint8_t *reads, uint64_t n_bases,
                                          const uint64_t *offsets, uint64_t n_reads, const mt_classify_params *p,
                                          int device_ptrs, void *stream, mt_allreduce_fn allreduce,
                                          mt_allgather_fn allgather, void *ctx, int32_t *taxon, uint8_t *nloc,
                                          mt_loc *locs, uint64_t *genome_hits, double *abundance, mt_stats *stats) {
    // every check that can fail on one rank alone comes before the first exchange
    if (!shard || !genome_ids || !allreduce || !allgather || !offsets || n_genomes == 0 || n_ranks == 0 ||
        (!taxon && n_reads) || (!reads && n_bases))
        return MT_EINVAL;
    if (shard->hpc || check_classify_params(p)) return MT_EINVAL;
    if (n_reads >= 0xFFFFFFFFull / MT_MAX_TOPN) return MT_EINVAL;
    // increasing ids: the shard's own rank order (ties by genome) is then the global one
    for (uint32_t l = 0; l < shard->G; l++)
        if (genome_ids[l] >= n_genomes || (l && genome_ids[l] <= genome_ids[l - 1])) return MT_EINVAL;
    if (stats) memset(stats, 0, sizeof(*stats));
    cudaStream_t s = (cudaStream_t)stream;
    const uint32_t G = n_genomes, Gs = shard->G, tn = p->top_n;
    const uint64_t n = n_reads, per_rank = n * tn * sizeof(mt_loc);

    // 1. which genomes the ranks hold: each at most once
    std::vector<uint64_t> hold(G, 0);
    for (uint32_t l = 0; l < Gs; l++) hold[genome_ids[l]]++;
    if (allreduce(ctx, MT_XCHG_HOLDERS, hold.data(), G) != 0) return MT_EXCHANGE;
    for (uint32_t g = 0; g < G; g++)
        if (hold[g] > 1) return MT_EINVAL;

    mt_part *q = nullptr;
    int rc = mt_part_create(G, reads, n_bases, offsets, n_reads, device_ptrs, stream, &q);
    if (rc) return rc;
    Carver c;
    const size_t o_ids = c.take<uint32_t>(std::max<uint32_t>(Gs, 1)), o_keep = c.take<uint8_t>(std::max<uint32_t>(Gs, 1));
    const size_t o_tax = c.take<int32_t>(std::max<uint64_t>(n, 1)), o_nloc = c.take<uint8_t>(std::max<uint64_t>(n, 1));
    const size_t o_mine = c.take<mt_loc>(std::max<uint64_t>(n * tn, 1));
    const size_t o_all = c.take<mt_loc>(std::max<uint64_t>(n * tn * n_ranks, 1));
    const size_t o_out = c.take<mt_loc>(std::max<uint64_t>(n * tn, 1)), o_a = c.take<double>(G);
    unsigned char *ws = nullptr;
    if ((rc = dalloc((void **)&ws, c.off + 256, s))) { mt_part_destroy(q); return rc; }
    auto done = [&](int code) { dfree(ws, s); cudaStreamSynchronize(s); mt_part_destroy(q); return code; };
    uint32_t *d_ids = (uint32_t *)(ws + o_ids);
    uint8_t *d_keep = ws + o_keep;
    int32_t *d_tax = (int32_t *)(ws + o_tax);
    uint8_t *d_nloc = ws + o_nloc;
    mt_loc *d_mine = (mt_loc *)(ws + o_mine), *d_all = (mt_loc *)(ws + o_all), *d_out = (mt_loc *)(ws + o_out);
    double *d_a = (double *)(ws + o_a);

    // 2. stage 1 over this rank's genomes; the hits summed over the ranks; the cutoff
    if ((rc = mt_part_contain(q, shard, genome_ids, p->max_occ))) return done(rc);
    std::vector<uint64_t> H(G);
    if (!cuda_ok(cudaMemcpyAsync(H.data(), q->H, G * 8ull, cudaMemcpyDeviceToHost, s), "sharded hits") ||
        !cuda_ok(cudaStreamSynchronize(s), "sharded hits"))
        return done(MT_ECUDA);
    if (allreduce(ctx, MT_XCHG_GENOME_HITS, H.data(), G) != 0) return done(MT_EXCHANGE);
    if (!cuda_ok(cudaMemcpyAsync(q->H, H.data(), G * 8ull, cudaMemcpyHostToDevice, s), "sharded hits"))
        return done(MT_ECUDA);
    std::vector<uint8_t> keep(G);
    if ((rc = mt_part_subset(q, p->cont_num, p->cont_den, keep.data(), genome_hits, nullptr, nullptr))) return done(rc);

    // 3. stage 2 against this rank's kept genomes; locations in global ids
    std::vector<uint8_t> keep_mine(std::max<uint32_t>(Gs, 1));
    for (uint32_t l = 0; l < Gs; l++) keep_mine[l] = keep[genome_ids[l]];
    if (!cuda_ok(cudaMemcpyAsync(d_keep, keep_mine.data(), Gs, cudaMemcpyHostToDevice, s), "sharded keep") ||
        !cuda_ok(cudaMemcpyAsync(d_ids, genome_ids, Gs * 4ull, cudaMemcpyHostToDevice, s), "sharded ids"))
        return done(MT_ECUDA);
    rc = mt_classify_masked(shard, q->reads, q->n_bases, q->roff, n, p, 1, s, d_keep, d_tax, d_nloc, d_mine,
                            nullptr, nullptr, stats);
    if (rc) return done(rc);
    if (n) {
        k_part_ids<<<grid_for(n * tn), 256, 0, s>>>(n, tn, d_ids, nullptr, d_mine);
        if (!cuda_ok(cudaGetLastError(), "k_part_ids")) return done(MT_ECUDA);
    }

    // 4. every rank's locations, merged by rank and decided on every rank
    std::vector<unsigned char> mine(std::max<uint64_t>(per_rank, 1)), all(std::max<uint64_t>(per_rank * n_ranks, 1));
    if ((per_rank && !cuda_ok(cudaMemcpyAsync(mine.data(), d_mine, per_rank, cudaMemcpyDeviceToHost, s), "sharded locs")) ||
        !cuda_ok(cudaStreamSynchronize(s), "sharded locs"))
        return done(MT_ECUDA);
    if (allgather(ctx, MT_XCHG_LOCATIONS, mine.data(), per_rank, all.data()) != 0) return done(MT_EXCHANGE);
    if (per_rank && !cuda_ok(cudaMemcpyAsync(d_all, all.data(), per_rank * n_ranks, cudaMemcpyHostToDevice, s), "sharded all"))
        return done(MT_ECUDA);
    if ((rc = merge_decide(d_all, n_ranks, q->roff, n, G, p, d_tax, d_nloc, d_out, d_a, s))) return done(rc);

    const cudaMemcpyKind down = device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if ((n && !cuda_ok(cudaMemcpyAsync(taxon, d_tax, n * 4, down, s), "sharded taxon")) ||
        (n && nloc && !cuda_ok(cudaMemcpyAsync(nloc, d_nloc, n, down, s), "sharded nloc")) ||
        (n && locs && !cuda_ok(cudaMemcpyAsync(locs, d_out, n * tn * sizeof(mt_loc), down, s), "sharded out")) ||
        (abundance && !cuda_ok(cudaMemcpyAsync(abundance, d_a, G * 8ull, down, s), "sharded abundance")))
        return done(MT_ECUDA);
    return done(cuda_ok(cudaStreamSynchronize(s), "sharded") ? MT_OK : MT_ECUDA);
}
