/*
 * mt.h -- C ABI of the GB300 MetaTrinity hot path (seed -> count -> locate -> SneakySnake ->
 * abundance), after Gollwitzer et al., "MetaTrinity: Enabling Fast Metagenomic
 * Classification via Seed Counting and Edit Distance Approximation", arXiv 2311.02029.
 *
 * Conventions shared by every call:
 *  - Bases are upper-case ASCII A, C, G, T (Methods: the DNA alphabet). Any other byte,
 *    including N, makes a call fail with MT_EINVAL.
 *  - Sequence sets are one concatenated byte buffer plus uint64 offsets of length count+1
 *    (offsets[0] may be non-zero; sequence i is bytes [offsets[i], offsets[i+1])).
 *  - 2-bit packed sequences: base j of a sequence sits at bits 2*(j%32) .. 2*(j%32)+1 of
 *    word j/32 (codes A=0, C=1, G=2, T=3; unused high bits are zero). Sequence i of a set
 *    whose base offsets are off[] starts at word (off[i] >> 5) + i, so packed sets need
 *    (off[n] >> 5) + n + 1 words and no separate word-offset table.
 *  - Ownership: inputs are borrowed for the duration of the call; output buffers are owned
 *    by the caller; mt_index and mt_server objects are owned by the library until freed.
 *  - Errors: every call returns MT_OK (0) or a negative status (below). No call aborts the
 *    process; after an error the contents of output buffers are unspecified.
 *  - Streams: `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *    Calls that return results to the host synchronise that stream before returning.
 */
#ifndef MT_H_
#define MT_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------------------- */
#define MT_OK 0
#define MT_EINVAL (-1)      /* bad base, bad offsets, parameter out of range */
#define MT_ENOMEM (-2)      /* device or host allocation failed / over budget */
#define MT_ETIMEDOUT (-3)   /* a bounded wait ran out */
#define MT_ECUDA (-4)       /* a CUDA runtime error (see mt_last_cuda_error) */
#define MT_ECANCELED (-5)   /* a serving request was cancelled */
#define MT_EBUSY (-6)       /* a serving request is still in flight */
#define MT_EXCHANGE (-7)    /* the caller's allreduce of a sharded batch failed */
#define MT_EIO (-8)         /* a file could not be read or written, or is not a saved index */

/* ---- limits ---------------------------------------------------------------------------- */
#define MT_MAX_READ_LEN 1024u   /* bases per read (the paper targets short reads) */
#define MT_MAX_K 31u            /* k-mer length; codes use 2k <= 62 bits */
#define MT_MAX_W 64u            /* k-mers per minimizer window */
#define MT_MAX_E 127u           /* edit threshold; 2E+1 <= 255 diagonals */
#define MT_MAX_TOPN 8u          /* mapping locations kept per read */
#define MT_MAX_OCC_LIMIT 2048u  /* largest accepted max_occ */
#define MT_MAX_GENOMES (1u << 30)

typedef struct mt_index mt_index;     /* opaque device-resident reference index */
typedef struct mt_server mt_server;   /* opaque continuous-batching request loop */
typedef struct mt_plan mt_plan;       /* opaque preallocated classification with a CUDA graph */

/* Index parameters (Results, "Evaluation Methodology": minimap2 short-read seeds; the
 * paper's containment index uses k = 28, w = 18; the workloads here use k15/w10, k21/w11). */
typedef struct {
    uint32_t k;          /* k-mer length, 1..MT_MAX_K */
    uint32_t w;          /* consecutive k-mers per window, 1..MT_MAX_W */
    uint32_t canonical;  /* 1: a k-mer and its reverse complement share one code */
    uint32_t flags;      /* 0, or MT_INDEX_HPC */
} mt_index_params;

/* The index holds the minimizers of the homopolymer-compressed genomes (every run of one base
 * taken as a single base; minimap2's -H, which the paper's containment index uses with k = 28,
 * w = 18). Such an index counts seed hits for containment (mt_containment) only; its
 * positions are in compressed coordinates, so mt_classify refuses it. */
#define MT_INDEX_HPC 1u

/* Per-call classification parameters. Paper defaults in brackets. */
typedef struct {
    uint32_t e_abs;        /* edit threshold E in bases, used when e_permille == 0 */
    uint32_t e_permille;   /* E(n) = floor(n * e_permille / 1000)  [10% of the read length] */
    uint32_t min_seeds;    /* minimum seed hits per mapping location  [3] */
    uint32_t top_n;        /* locations per read kept for the approximation  [3] */
    uint32_t max_occ;      /* seeds with more occurrences are skipped  [1024] */
    uint32_t cont_num;     /* containment cutoff num/den on hits/max_hits  [1/10000] */
    uint32_t cont_den;
    uint32_t eda_mode;     /* execution form | approximation (below)  [SneakySnake, batched] */
    double abund_cutoff;   /* relative abundances below this are dropped  [1e-4] */
} mt_classify_params;

/* Edit-distance approximation of each candidate, eda_mode = form | approximation.
 * Execution forms (identical results):                                                    */
#define MT_EDA_BATCHED 0u  /* persistent work-stealing kernel, tuned (or default) group shape */
#define MT_EDA_PLAIN 1u    /* one warp per pair, one launch per length bucket */
/* Approximations (Table 1; the Discussion's O(n) count comparisons and O(nE) pigeonhole
 * filters). Each result is min(estimate, E + 1); a location is accepted iff it is <= E.
 * The paper gives no formulas for the last four; the readings implemented: HD, Base
 * Counting and q-gram compare the read with the window's central segment [E, E + n) (the
 * location's first diagonal), where a base outside the genome equals no read base.      */
#define MT_EDA_SNAKE (0u << 4)          /* SneakySnake over the 2E+1 diagonals [48] */
#define MT_EDA_HAMMING (1u << 4)        /* mismatches on the central segment [49] */
#define MT_EDA_BASE_COUNTING (2u << 4)  /* ceil(sum over bases |count difference| / 2) [46] */
#define MT_EDA_QGRAM (3u << 4)          /* ceil(q-gram profile distance / 2q), q = 5 [52] */
#define MT_EDA_SHD (4u << 4)            /* shifted Hamming: the 2E+1 diagonal mismatch masks,
                                           match runs of 1-2 between mismatches set to
                                           mismatches, AND-ed; set flags counted [50] */

/* One mapping location of a read (24 bytes). */
typedef struct {
    int64_t wstart;   /* reference window start, forward strand: first diagonal - E */
    int32_t genome;   /* genome index, -1 for an unused slot */
    uint32_t seeds;   /* seed hits of the location */
    uint8_t strand;   /* 1: the read matches the genome's reverse strand */
    uint8_t dist;     /* SneakySnake distance, capped at E + 1 (E + 1 = rejected) */
    uint8_t pad[6];
} mt_loc;

/* Optional per-call counters and stage times. The stage times are CUDA-event intervals
 * recorded on the call's stream around each stage's kernels. */
typedef struct {
    uint64_t n_reads;
    uint64_t n_minimizers;   /* read minimizers looked up */
    uint64_t n_hits;         /* seed matches (all genomes) */
    uint64_t n_candidates;   /* locations sent to the approximation */
    uint64_t n_accepted;     /* reads with a location at distance <= E */
    uint64_t n_multi;        /* accepted reads whose best distance is shared by >1 genome */
    uint64_t n_fallback;     /* reads re-mapped by the exact slow path (hit overflow) */
    uint64_t workspace_bytes;
    uint64_t n_ext_occ;      /* occurrences read from the occurrence array (not inline) */
    uint64_t n_stored;       /* location records written by the seeding pass */
    uint64_t n_launches;     /* kernels launched by the call */
    double ms_seed;          /* seeding, lookup, containment counts, locations */
    double ms_select;        /* containment mask, candidate selection, slow path */
    double ms_eda;           /* edit-distance approximation */
    double ms_profile;       /* per-read decision, multi-read split, abundances */
    double ms_total;         /* first to last kernel of the call */
    uint64_t err_bits;       /* device-side error flags of the call (0 when it succeeded) */
} mt_stats;

typedef struct {
    uint32_t n_genomes, k, w, canonical;
    uint64_t total_bases;
    uint64_t n_occ;          /* genome minimizers stored */
    uint64_t n_keys;         /* distinct minimizer codes */
    uint64_t table_slots;    /* open-addressing slots (power of two) */
    uint64_t device_bytes;   /* HBM held by the index */
    uint32_t flags;          /* the build's flags (MT_INDEX_HPC) */
    uint32_t pad;
} mt_index_info;

/* ---- general ---------------------------------------------------------------------------- */
const char *mt_strerror(int status);
/* Text of the last CUDA error seen by this thread (empty if none). */
const char *mt_last_cuda_error(void);
int mt_version(void);

/* ---- host-side fault injection and accounting, for tests (no counterpart in the paper) ----
 * mt_inject_alloc_failure(n): the next n device allocations of the library's calls succeed and
 * the one after fails as if the device were out of memory (the call returns MT_ENOMEM after
 * freeing what it took); n < 0 turns injection off (the default). Every later allocation
 * succeeds again once the injected failure has happened. Process-wide; it makes no GPU fault.
 * mt_pool_used_bytes(): bytes currently allocated from the current device's stream-ordered
 * pool by the library's calls and not yet freed (a call that returned holds none of them). */
void mt_inject_alloc_failure(int64_t n);
uint64_t mt_pool_used_bytes(void);

/* ---- index (Methods, "Reference Database Organisation and Index Construction &
 * Querying"): every genome's (w,k)-minimizers, key = SplitMix64 finaliser of the k-mer
 * code, held in HBM as an open-addressing table of 32-byte slots (one DRAM sector per
 * probe; up to three occurrences inline) plus an occurrence array sorted by
 * (code, genome, position). The 2-bit packed genomes stay resident for the
 * reference windows of the edit-distance approximation.
 *
 * genomes/offsets: HOST buffers, n_genomes sequences, each shorter than 2^32 bases.
 * stream: used for the build; the call returns after the build completes.
 * Errors: MT_EINVAL (bad base, k/w out of range, empty set), MT_ENOMEM, MT_ECUDA. */
int mt_build_index(const uint8_t *genomes, const uint64_t *offsets, uint32_t n_genomes,
                   const mt_index_params *params, void *stream, mt_index **out);
void mt_free_index(mt_index *ix);
/* mt_build_index over the genomes ids[0..n_ids) of a set of n_set genomes (genomes / offsets as
 * in mt_build_index, n_set + 1 offsets): genome i of the new index is genome ids[i] of the set.
 * The chosen genomes' bytes go to the device directly, without a host-side copy of the subset
 * (e.g. the subset database of a partitioned query). Errors: those of mt_build_index; MT_EINVAL
 * for NULL ids or an id >= n_set. */
int mt_build_index_subset(const uint8_t *genomes, const uint64_t *offsets, uint32_t n_set, const uint32_t *ids,
                          uint32_t n_ids, const mt_index_params *params, void *stream, mt_index **out);

/* ---- index persistence (Methods, "Index Construction & Querying": the index is built once
 * and queried many times, so building stays off the query path) ---------------------------
 * mt_save_index writes a built index to the file `path` (created or truncated; about the
 * index's device_bytes), copying through a pinned host buffer on `stream`. mt_load_index reads
 * such a file onto the current device into a new index (freed with mt_free_index), identical
 * in every query to the one saved. Files are native little-endian, with a checked header and a
 * trailer; a file of another shape, size or version is refused.
 * Errors: MT_EINVAL (NULL arguments), MT_EIO (open, read or write failed; not a saved index),
 * MT_ENOMEM / MT_ECUDA (device or pinned allocation, copies). On error *out is NULL. */
int mt_save_index(const mt_index *ix, const char *path, void *stream);
int mt_load_index(const char *path, void *stream, mt_index **out);
int mt_index_get_info(const mt_index *ix, mt_index_info *info);

/* ---- classification of one read batch (Fig. 1 stages 1-3; "The MetaTrinity Pipeline"):
 *  1. containment: minimizers of every read are looked up; hits are counted per genome
 *     over the whole batch; genome g is kept iff hits[g]/max(hits) > cont_num/cont_den;
 *  2. read mapping: per read, seed matches in kept genomes grouped into locations (one per
 *     genome, strand and diagonal band of width E); locations with < min_seeds seeds
 *     dropped, the top_n by seed count compared with SneakySnake against the reference
 *     window [first diagonal - E, first diagonal + n + E); locations at distance <= E are
 *     accepted;
 *  3. profiling: a read whose best accepted distance belongs to one genome is unique; one
 *     shared by several genomes is split in proportion to their unique counts (equally if
 *     they have none); relative abundances below abund_cutoff are dropped and the rest
 *     renormalised.
 * reads: a buffer of n_bases bytes; offsets: n_reads + 1 non-decreasing entries with
 *   offsets[n_reads] <= n_bases (read i is bytes [offsets[i], offsets[i+1]) of `reads`).
 * device_ptrs: 1 = reads, offsets and every output pointer are device pointers (the call
 *   still synchronises `stream` before returning, to report input errors); 0 = all are
 *   host pointers (copies are made on `stream`).
 * Outputs (any may be NULL except taxon, which may be NULL only when n_reads is 0):
 *   taxon[n_reads] (genome or -1);
 *   nloc[n_reads]; locs[n_reads * top_n] (unused slots have genome -1);
 *   genome_hits[n_genomes] (stage-1 counts); abundance[n_genomes]; stats.
 * Errors: MT_EINVAL (bad base, read longer than MT_MAX_READ_LEN, bad offsets, parameter
 *   out of range, an index built with MT_INDEX_HPC), MT_ENOMEM, MT_ECUDA. */
int mt_classify(const mt_index *ix, const uint8_t *reads, uint64_t n_bases,
                const uint64_t *offsets, uint64_t n_reads, const mt_classify_params *params,
                int device_ptrs, void *stream, int32_t *taxon, uint8_t *nloc, mt_loc *locs,
                uint64_t *genome_hits, double *abundance, mt_stats *stats);

/* Shape of the batched approximation kernel (MT_EDA_BATCHED) for one edit-threshold class
 * (classes: E in [0,1], [2,3], [4,7], [8,15], [16,31], [32,63], [64,127]). No counterpart in
 * the paper: the batching side of this library. */
#define MT_EDA_CLASSES 8u
typedef struct {
    uint32_t lanes_per_pair;    /* lanes of a warp working on one pair: 1, 2, 4, 8, 16 or 32 */
    uint32_t pairs_per_chunk;   /* pairs a warp takes from the shared counter at a time */
    uint32_t cta_threads;       /* threads per CTA of the persistent launch (128 .. 1024) */
    uint32_t refill;            /* SneakySnake, one lane per pair: 1 = a lane takes a new pair as
                                   soon as its own ends; 0 = the warp's lanes take pairs together */
    uint32_t tuned;             /* 1: kept in this process (an autotune call or mt_eda_set_shape); 0: the default */
} mt_eda_shape;

/* mt_classify that first times the batched approximation kernel's shapes on this batch's own
 * candidates (lanes per pair in {1,2,4,8,16,32}; with one lane per pair, lanes refilled one by
 * one or not; then pairs per chunk in {32,64,128,256}, then CTA size in {128,256,512,1024}; a
 * few dozen launches on at most 2^17 candidates) and keeps the
 * fastest for the batch's edit-threshold class on this device; the batch is then classified
 * with it (outputs and errors exactly as mt_classify). mt_classify, plans and the serving loop
 * never time anything themselves: they use the shape kept here, else the default. *shape
 * (nullable) receives the shape used. Only eda_mode's batched form is tuned. */
int mt_classify_autotune(const mt_index *ix, const uint8_t *reads, uint64_t n_bases,
                         const uint64_t *offsets, uint64_t n_reads, const mt_classify_params *params,
                         int device_ptrs, void *stream, int32_t *taxon, uint8_t *nloc, mt_loc *locs,
                         uint64_t *genome_hits, double *abundance, mt_stats *stats, mt_eda_shape *shape);

/* The shape the batched approximation kernel uses on this device for approximation `mode`
 * (form bits ignored), pairs of edit threshold E, in classification (classification = 1) or in
 * mt_eda_batch (0): the kept one if an autotune call chose it or mt_eda_set_shape set it
 * (tuned = 1), else the default (tuned = 0). Errors: MT_EINVAL, MT_ECUDA. */
int mt_eda_shape_for(uint32_t mode, int classification, uint32_t E, mt_eda_shape *out);
/* Keeps `shape` for the edit-threshold class of E (as an autotune call would), e.g. a shape
 * tuned in an earlier process and stored by the caller. Valid shapes: lanes_per_pair a power
 * of two up to 32 (32 for q-gram), pairs_per_chunk 1..4096, cta_threads a multiple of 32 up to
 * 1024, refill 0 or 1 (1 only for SneakySnake with one lane per pair); `tuned` is ignored.
 * lanes_per_pair = 0 forgets the kept shape (the class runs the default again). Every shape
 * gives the same distances. Errors: MT_EINVAL (an invalid shape or argument), MT_ECUDA. */
int mt_eda_set_shape(uint32_t mode, int classification, uint32_t E, const mt_eda_shape *shape);

/* ---- containment alone (Fig. 1 stage 1; "The MetaTrinity Pipeline") ------------------------
 * Seed hits per genome over the batch, counted with multiplicity for every minimizer of every
 * read that has at most max_occ occurrences, and the kept-genome mask
 * keep[g] = (hits[g] * cont_den > max_h hits[h] * cont_num). With an index built with
 * MT_INDEX_HPC the reads' minimizers are taken after homopolymer compression (the paper's
 * containment index: minimap2's -H, k = 28, w = 18). reads / offsets / device_ptrs as in
 * mt_classify; genome_hits[n_genomes] and keep[n_genomes] (keep may be NULL) are host or device
 * pointers like the inputs. Returns after synchronising `stream`.
 * Errors: MT_EINVAL (bad base, bad offsets, read longer than MT_MAX_READ_LEN, max_occ above
 * MT_MAX_OCC_LIMIT, cont_den 0), MT_ENOMEM, MT_ECUDA. */
int mt_containment(const mt_index *ix, const uint8_t *reads, uint64_t n_bases, const uint64_t *offsets,
                   uint64_t n_reads, uint32_t max_occ, uint32_t cont_num, uint32_t cont_den,
                   int device_ptrs, void *stream, uint64_t *genome_hits, uint8_t *keep);

/* mt_classify with a given kept-genome mask: read mapping and profiling (stages 2 and 3) over
 * the genomes g with keep[g] != 0 -- e.g. the mask mt_containment computes with a separate
 * containment index, the paper's subset database -- instead of the batch's own containment
 * cutoff (params->cont_num / cont_den are not used). genome_hits still reports this index's seed
 * hits. keep: n_genomes bytes, a host or device pointer like the inputs. Errors: those of
 * mt_classify; MT_EINVAL for a NULL keep. */
int mt_classify_masked(const mt_index *ix, const uint8_t *reads, uint64_t n_bases,
                       const uint64_t *offsets, uint64_t n_reads, const mt_classify_params *params,
                       int device_ptrs, void *stream, const uint8_t *keep, int32_t *taxon, uint8_t *nloc,
                       mt_loc *locs, uint64_t *genome_hits, double *abundance, mt_stats *stats);

/* ---- a reference database cut into batches (Methods, "Reference Database Organisation and
 * Index Construction & Querying"; Evaluation Methodology) --------------------------------------
 * The database is split into batches, each indexed on its own (built, saved, loaded and, when
 * one of its genomes changes, rebuilt without touching the others); a batch's genomes carry
 * global ids 0..n_genomes-1, and one genome may sit in several batches. One read batch is
 * classified against it in the paper's order:
 *  1. mt_part_contain, once per database batch (or mt_part_contain_batches for several resident
 *     batches at once): that batch's seed hits per genome over all the
 *     reads, with the batch's own repeat filter (max_occ counts occurrences in that batch); a
 *     genome keeps the highest count any batch gave it;
 *  2. mt_part_subset: the normalised cutoff over the whole database, keep[g] =
 *     (hits[g] * cont_den > max_h hits[h] * cont_num), and the list of kept genomes;
 *  3. the caller builds the subset database, an index over the kept genomes in that order
 *     (mt_build_index, any k / w, not MT_INDEX_HPC);
 *  4. mt_part_classify: read mapping and profiling (stages 2 and 3 of mt_classify) against the
 *     subset, all of whose genomes are kept; genome ids in the outputs are global ids.
 * Only the reads and a few n_genomes vectors stay on the device between the calls, so the
 * database batches can be loaded (mt_load_index), queried and freed one at a time: the
 * database need not fit in device memory, only one batch and the subset index.
 * All calls of a query run on its stream and return after synchronising it. */
typedef struct mt_part mt_part;   /* opaque: one read batch queried against a partitioned database */

/* Starts a query. reads / offsets / device_ptrs as in mt_classify; host inputs are copied to
 * the device here (the caller's buffers are free on return); device inputs are borrowed until
 * mt_part_destroy. n_genomes: global genome ids of the database, >= 1.
 * Errors: MT_EINVAL (NULL arguments, n_genomes 0), MT_ENOMEM, MT_ECUDA. */
int mt_part_create(uint32_t n_genomes, const uint8_t *reads, uint64_t n_bases, const uint64_t *offsets,
                   uint64_t n_reads, int device_ptrs, void *stream, mt_part **out);
/* Stage 1 for one database batch: genome_ids (host, batch's n_genomes entries, each <
 * n_genomes) are the global ids of the batch's genomes in index order. Any index kind,
 * including MT_INDEX_HPC (the paper's containment index).
 * Errors: MT_EINVAL (NULL arguments, an id out of range, max_occ above MT_MAX_OCC_LIMIT, bad
 * reads or offsets), MT_ENOMEM, MT_ECUDA. */
int mt_part_contain(mt_part *q, const mt_index *batch, const uint32_t *genome_ids, uint32_t max_occ);
/* Stage 1 for several resident database batches in one pass over the reads: each read's
 * minimizers are found once and looked up in every batch's table. Same counts as one
 * mt_part_contain per batch. genome_ids[b]: as in mt_part_contain for batches[b]. The batches
 * must share k, w, canonical and MT_INDEX_HPC.
 * Errors: those of mt_part_contain; MT_EINVAL for batches built with different seeds. */
int mt_part_contain_batches(mt_part *q, const mt_index *const *batches, const uint32_t *const *genome_ids,
                            uint32_t n_batches, uint32_t max_occ);
/* The cutoff over the counts gathered so far. Outputs (each may be NULL): keep[n_genomes] (host),
 * genome_hits[n_genomes] (the highest counts; host or device like the reads), kept (host,
 * n_genomes entries of room: the kept global ids, increasing) and *n_kept.
 * Errors: MT_EINVAL (NULL q, cont_den 0), MT_ECUDA. */
int mt_part_subset(mt_part *q, uint32_t cont_num, uint32_t cont_den, uint8_t *keep, uint64_t *genome_hits,
                   uint32_t *kept, uint32_t *n_kept);
/* Stages 2 and 3 against the subset index: subset_ids (host, n_subset entries) must be the kept
 * list of the last mt_part_subset, and subset an index over exactly those genomes in that
 * order (NULL when n_subset is 0: then no read maps). params as in mt_classify (cont_num /
 * cont_den unused). Outputs as in mt_classify, in global ids; abundance has n_genomes entries
 * (0 for genomes not kept); genome_hits is reported by mt_part_subset instead.
 * Errors: MT_EINVAL (mt_part_subset not called, a subset list or index that does not match
 * it, an MT_INDEX_HPC subset, bad params), MT_ENOMEM, MT_ECUDA. */
int mt_part_classify(mt_part *q, const mt_index *subset, const uint32_t *subset_ids, uint32_t n_subset,
                     const mt_classify_params *params, int32_t *taxon, uint8_t *nloc, mt_loc *locs,
                     double *abundance, mt_stats *stats);
void mt_part_destroy(mt_part *q);

/* The four steps in one call over resident database batches: batches[b] with global ids
 * genome_ids[b] (host arrays of each batch's n_genomes entries); genomes / genome_offsets (host,
 * n_genomes + 1 offsets) hold every genome by global id, for the subset index, which is built
 * with subset_params and freed before returning. Stage 1 uses params->max_occ and the cutoff
 * params->cont_num / cont_den. Outputs as in mt_classify (genome_hits: the highest counts).
 * Errors: those of the calls above and of mt_build_index. */
int mt_classify_partitioned(const mt_index *const *batches, const uint32_t *const *genome_ids, uint32_t n_batches,
                            const uint8_t *genomes, const uint64_t *genome_offsets, uint32_t n_genomes,
                            const mt_index_params *subset_params, const uint8_t *reads, uint64_t n_bases,
                            const uint64_t *offsets, uint64_t n_reads, const mt_classify_params *params,
                            int device_ptrs, void *stream, int32_t *taxon, uint8_t *nloc, mt_loc *locs,
                            uint64_t *genome_hits, double *abundance, mt_stats *stats);

/* ---- one batch sharded over several processes (ranks) -------------------------------------
 * Stages 1 and 3 are defined over the whole batch: the containment cutoff compares a genome's
 * hits with the largest hit count of the batch ("The MetaTrinity Pipeline", stage 1), and a
 * multi-mapped read is split by the batch's unique counts (Fig. 1, 3a-b). A batch cut into
 * shards, one per rank, therefore needs three element-wise sums over the ranks, which the
 * caller supplies as `allreduce`. The call runs the stages of its own shard and, at each
 * exchange point, copies a vector of n_genomes values to a host buffer and calls
 * allreduce(ctx, kind, buf, n_genomes); that must replace buf with the element-wise sum of
 * every rank's buf (all ranks make the same exchanges in the same order) and return 0:
 *   MT_XCHG_GENOME_HITS (uint64): seed hits per genome, before the containment cutoff;
 *   MT_XCHG_UNIQUE (uint64): uniquely mapped reads per genome, before the multi-mapped split;
 *   MT_XCHG_MULTI (double): multi-mapped read shares per genome, before the abundances.
 * Each rank then reports for its own reads exactly what mt_classify reports for them in the
 * whole batch; genome_hits and abundance are the whole batch's on every rank (abundance up to
 * the order in which doubles are summed). A rank with no reads still makes the call and
 * contributes zeros. Arguments are those of mt_classify plus allreduce (not NULL) and ctx
 * (passed through). The calls of one rank run on its own stream; the exchanges block the
 * calling host thread only.
 * Errors: those of mt_classify; a call that fails its argument checks returns before its first
 * exchange (the other ranks' allreduce must then fail on its own, e.g. by a time limit);
 * MT_EXCHANGE when allreduce returns non-zero (the call stops at that exchange). */
#define MT_XCHG_GENOME_HITS 0
#define MT_XCHG_UNIQUE 1
#define MT_XCHG_MULTI 2
#define MT_XCHG_HOLDERS 3     /* (uint64, mt_classify_genome_sharded) ranks holding each genome */
#define MT_XCHG_LOCATIONS 4   /* (bytes, all-gather, mt_classify_genome_sharded) per-read locations */
typedef int (*mt_allreduce_fn)(void *ctx, int kind, void *buf, uint64_t count);
/* recv (n_ranks * bytes) must receive every rank's send buffer (bytes each), in rank order. */
typedef int (*mt_allgather_fn)(void *ctx, int kind, const void *send, uint64_t bytes, void *recv);
int mt_classify_sharded(const mt_index *ix, const uint8_t *reads, uint64_t n_bases,
                        const uint64_t *offsets, uint64_t n_reads, const mt_classify_params *params,
                        int device_ptrs, void *stream, mt_allreduce_fn allreduce, void *ctx,
                        int32_t *taxon, uint8_t *nloc, mt_loc *locs, uint64_t *genome_hits,
                        double *abundance, mt_stats *stats);

/* ---- one read batch against genome shards held by several processes (ranks) ---------------
 * A database too large for one device, split by genome: rank r holds an index over its own
 * genomes (global ids genome_ids in index order, increasing, so that rank ties between genomes
 * break alike in a shard and in the database; the ranks' sets must be disjoint) and every
 * rank sees every read of the batch. The call, made by every rank with the same reads and
 * params, runs:
 *  1. allreduce(MT_XCHG_HOLDERS, n_genomes uint64: 1 for each genome this rank holds): a
 *     genome held twice makes every rank return MT_EINVAL;
 *  2. stage 1 over this rank's genomes; allreduce(MT_XCHG_GENOME_HITS) sums the hits (each
 *     genome counted by its one rank); the cutoff over the whole database;
 *  3. stage 2 (mt_classify_masked) against this rank's kept genomes: each read's top_n
 *     locations with their distances, in global ids;
 *  4. allgather(MT_XCHG_LOCATIONS, n_reads * top_n locations a rank) and, on every rank, each
 *     read's lists merged in rank order (seeds descending, then genome, strand, window start),
 *     the first top_n decided and profiled as by a single index.
 * With no key reaching the repeat filter (each rank filters by its own index) the outputs
 * equal mt_classify over one index of all genomes. Outputs (every rank, whole batch, global
 * genome ids) and reads / offsets / device_ptrs / stream as in mt_classify. The exchange
 * buffers are host memory; the calls block the calling host thread only.
 * Errors: those of mt_classify; MT_EINVAL (NULL allreduce / allgather, n_ranks 0, an id >=
 * n_genomes or ids not increasing, an MT_INDEX_HPC shard, overlapping shards); a call that
 * fails its argument checks
 * returns before its first exchange; MT_EXCHANGE when an exchange function returns non-zero. */
int mt_classify_genome_sharded(const mt_index *shard, const uint32_t *genome_ids, uint32_t n_genomes,
                               uint32_t n_ranks, const uint8_t *reads, uint64_t n_bases, const uint64_t *offsets,
                               uint64_t n_reads, const mt_classify_params *params, int device_ptrs, void *stream,
                               mt_allreduce_fn allreduce, mt_allgather_fn allgather, void *ctx, int32_t *taxon,
                               uint8_t *nloc, mt_loc *locs, uint64_t *genome_hits, double *abundance,
                               mt_stats *stats);

/* ---- taxonomic roll-up of a profile (Fig. 1, 3b; "Taxonomic Profile Generation") -----------
 * A taxonomy is a forest over n_nodes taxa given by parent[] (-1 for a root); genome g sits at
 * node genome_node[g]. node_abundance[v] = the sum of abundance[g] over the genomes whose node
 * is v or lies below v (genomes summed in index order). All pointers are HOST pointers; the
 * call uses no GPU. Errors: MT_EINVAL (a node index out of range, parent links with a cycle). */
int mt_profile_rollup(const double *abundance, uint32_t n_genomes, const uint32_t *genome_node,
                      const int32_t *parent, uint32_t n_nodes, double *node_abundance);
/* mt_profile_rollup on the device: abundance[n_genomes], genome_node[n_genomes], parent[n_nodes]
 * and node_abundance[n_nodes] are DEVICE pointers (e.g. the abundance vector of a device-buffer
 * mt_classify, which then needs no host pass); enqueued on `stream`, returns after
 * synchronising it. Each genome's abundance is added to the taxa on its path in parallel, so
 * the sums agree with mt_profile_rollup's up to the order of additions (within 1e-12 of 1).
 * Errors: MT_EINVAL (a node index out of range, parent links with a cycle; node_abundance is
 * then undefined), MT_ENOMEM, MT_ECUDA. */
int mt_profile_rollup_device(const double *abundance, uint32_t n_genomes, const uint32_t *genome_node,
                             const int32_t *parent, uint32_t n_nodes, double *node_abundance, void *stream);

/* ---- batched form with a captured CUDA graph ---------------------------------------------
 * A plan holds a preallocated workspace sized for batches of up to max_reads reads,
 * max_bases bases and reads of at most max_read_len bases, and the classification kernels
 * captured once into a CUDA graph. Every kernel reads the batch's pointers and sizes from a
 * small device block written per call, so the same graph serves every batch up to the
 * capacity: the first mt_plan_classify runs the kernels directly (and may autotune the
 * approximation), the second captures them on `stream` and every call after that replays the
 * graph. Results are identical to mt_classify with the same parameters.
 * Arguments of mt_plan_classify are those of mt_classify; batches above the capacity or with
 * a longer read fail with MT_EINVAL. A plan is used by one thread at a time. */
int mt_plan_create(const mt_index *ix, const mt_classify_params *params, uint64_t max_reads,
                   uint64_t max_bases, uint32_t max_read_len, mt_plan **out);
int mt_plan_classify(mt_plan *plan, const uint8_t *reads, uint64_t n_bases, const uint64_t *offsets,
                     uint64_t n_reads, int device_ptrs, void *stream, int32_t *taxon, uint8_t *nloc,
                     mt_loc *locs, uint64_t *genome_hits, double *abundance, mt_stats *stats);
/* Device bytes held by the plan (its workspace). */
uint64_t mt_plan_device_bytes(const mt_plan *plan);
void mt_plan_destroy(mt_plan *plan);

/* Device bytes that one mt_classify call with HOST buffers allocates for this batch shape
 * (workspace plus device staging of the inputs and outputs); max_read_len is the batch's
 * longest read (0: unknown, the bound min(n_bases, MT_MAX_READ_LEN) is used). The serving loop
 * charges exactly this figure against its HBM budget. 0 for invalid parameters. */
uint64_t mt_classify_workspace_bytes(const mt_index *ix, uint64_t n_bases, uint64_t n_reads,
                                     uint32_t max_read_len, const mt_classify_params *params);

/* ---- 2-bit packing (used by the seeding kernels; exposed for the EDA batch call) ---------
 * seq/offsets/words: DEVICE pointers. Writes sequence i at word (offsets[i] >> 5) + i;
 * words must hold (offsets[n_seqs] >> 5) + n_seqs + 1 entries. Errors: MT_EINVAL (non-ACGT
 * byte; checked after a stream synchronisation), MT_ECUDA. */
int mt_pack_seqs(const uint8_t *seq, const uint64_t *offsets, uint64_t n_seqs, uint64_t *words,
                 void *stream);

/* ---- edit-distance approximation stage alone (Table 1) ------------------------------------
 * Pair p compares read pair_read[p] (read_words: a packed set with base offsets read_off,
 * n_reads + 1 entries) with window p (win_words: a packed set with base offsets win_off,
 * n_pairs + 1 entries). Window length must equal the read length + 2 E[p]; E[p] <=
 * MT_MAX_E, read length <= MT_MAX_READ_LEN. dist[p] = the approximation of mode's
 * MT_EDA_* bits, min(estimate, E[p] + 1) (SneakySnake: obstacles; window bases all count as
 * genome bases here). All pointers are DEVICE pointers. mode = form | approximation, form
 * MT_EDA_BATCHED (one persistent work-stealing launch over the pairs ordered by E, each
 * edit-threshold class with its tuned or default shape) or MT_EDA_PLAIN (one launch per
 * read-length bucket, a warp per pair); both forms give identical dist. The call returns
 * after synchronising `stream`. Errors: MT_EINVAL (length mismatch, limits), MT_ENOMEM,
 * MT_ECUDA. */
int mt_eda_batch(const uint64_t *read_words, const uint64_t *read_off, uint64_t n_reads,
                 const uint64_t *win_words, const uint64_t *win_off, const uint32_t *pair_read,
                 const uint16_t *E, uint64_t n_pairs, uint32_t mode, void *stream, uint8_t *dist);

/* mt_eda_batch that, in the batched form, first times the shapes (as mt_classify_autotune) on
 * up to 2^17 pairs of every edit-threshold class in the batch, keeps the fastest per class on
 * this device for later mt_eda_batch calls, and then computes dist with them. shapes (nullable,
 * MT_EDA_CLASSES entries) receives each class's shape (zeros for classes not in the batch).
 * The plain form is computed as by mt_eda_batch, nothing timed. Errors: as mt_eda_batch. */
int mt_eda_batch_autotune(const uint64_t *read_words, const uint64_t *read_off, uint64_t n_reads,
                          const uint64_t *win_words, const uint64_t *win_off, const uint32_t *pair_read,
                          const uint16_t *E, uint64_t n_pairs, uint32_t mode, void *stream, uint8_t *dist,
                          mt_eda_shape *shapes);

/* ---- the same stage without any device allocation ----------------------------------------
 * No counterpart in the paper: an addition for callers that cannot allocate device memory
 * during a call (a serving loop with a fixed device footprint, a host framework that owns the
 * allocator, code that must not grow its footprint after start-up). Identical arguments,
 * layouts, limits and results as mt_eda_batch (all pointers DEVICE pointers), except:
 *  - its scratch is a fixed array of ~4 MiB in the library, one per device that loads the
 *    library, held until the process exits; n_pairs above 2^20 fails with MT_EINVAL;
 *  - the first call on a device looks up that array's device address (once per device, with
 *    the device current); make that first call before any stream capture;
 *  - every call uses the same array, so calls whose work overlaps on the GPU (other threads or
 *    streams) race and must be serialised by the caller;
 *  - mode is the SneakySnake forms only (MT_EDA_BATCHED or MT_EDA_PLAIN);
 *  - the batched form uses lanes per pair already tuned in this process, else a default; it
 *    times nothing itself.
 * It calls no cudaMalloc, cudaFree or other allocating routine. Returns after synchronising
 * `stream`. Errors: MT_EINVAL, MT_ECUDA. */
int mt_eda_batch_noalloc(const uint64_t *read_words, const uint64_t *read_off, uint64_t n_reads,
                         const uint64_t *win_words, const uint64_t *win_off, const uint32_t *pair_read,
                         const uint16_t *E, uint64_t n_pairs, uint32_t mode, void *stream, uint8_t *dist);

/* ---- continuous-batching serving loop over one resident index --------------------------
 * Requests (read batches) are admitted while a slot is free and their workspace fits in
 * hbm_budget bytes; admitted requests run concurrently on their own streams. Inputs are
 * HOST buffers borrowed until mt_server_poll reports completion. */
int mt_server_create(const mt_index *ix, uint64_t hbm_budget, int max_slots,
                     const mt_classify_params *params, mt_server **out);
int mt_server_submit(mt_server *s, const uint8_t *reads, uint64_t n_bases, const uint64_t *offsets,
                     uint64_t n_reads, int32_t *taxon, uint8_t *nloc, mt_loc *locs,
                     uint64_t *genome_hits, double *abundance, uint64_t *req_id);
/* Waits up to timeout_ms (0 = just check) for a request. Returns MT_OK when done (its
 * outputs are written), MT_EBUSY / MT_ETIMEDOUT while pending, or the request's error.
 * If latency_s != NULL it receives submit-to-completion seconds. The poll that reports a
 * final status (anything but MT_EBUSY / MT_ETIMEDOUT) releases the request: the server keeps
 * nothing of it afterwards, and its id is unknown to later polls and cancels (MT_EINVAL). */
int mt_server_poll(mt_server *s, uint64_t req_id, int timeout_ms, double *latency_s);
/* Cancels a request still in the queue: MT_OK (a later poll reports MT_ECANCELED), MT_EBUSY
 * when it is running or done but not yet polled, MT_EINVAL for an unknown or released id. */
int mt_server_cancel(mt_server *s, uint64_t req_id);
void mt_server_destroy(mt_server *s);

#ifdef __cplusplus
}
#endif
#endif /* MT_H_ */
