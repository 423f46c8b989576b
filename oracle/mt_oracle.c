/*
 * mt_oracle.c -- plain, slow, single-threaded CPU oracle of the MetaTrinity hot path.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing on the product path may call it: only the tests,
 * the smoke check of the build entry point and the benchmark's CPU-baseline / reference
 * legs load this file. It shares no code, header, table or constant generator with the
 * CUDA library; the two meet only in the seeded input generators.
 *
 * Every step follows the paper (Gollwitzer et al., "MetaTrinity", arXiv 2311.02029) in
 * its order, written for obviousness rather than speed:
 *   1. seeds: (w,k)-minimizers of reads and genomes     -- Results "Alignment-free
 *      read-mapping" (minimap2 minimizer seeds) and "Evaluation Methodology" (k, w).
 *   2. index: every genome's minimizers, looked up by k-mer code -- Methods
 *      "Reference Database Organisation and Index Construction & Querying".
 *   3. containment: per-genome seed-hit counts over the whole read set, normalised by
 *      the largest count and cut at 1e-4 -- "The MetaTrinity Pipeline" stage 1,
 *      "Evaluation Methodology" (normalised cutoff 0.0001), Fig. 1 (1a-d).
 *   4. mapping locations: per read, seed matches grouped into locations, locations with
 *      fewer than min_seeds seeds dropped, sorted by seed count, top 3 kept --
 *      Fig. 1 (2b-c), read-mapping "Evaluation Methodology", "Empirically Determined
 *      Parameters".
 *   5. edit-distance approximation: SneakySnake (Table 1, ref. [48]); pairs with an
 *      approximate distance <= E are kept -- Fig. 1 (2d), read-mapping "Evaluation
 *      Methodology".
 *   6. profiling: unique and multi-mapped reads to relative abundances, taxa below 0.01%
 *      dropped -- Fig. 1 (3a-b), "Taxonomic Profile Generation".
 * Where the paper is silent the readings listed in the design notes are taken (mixer,
 * leftmost-minimum tie, location clustering, rank tie-breaks, window edges, multi-read
 * split); each is marked "Reading:" below.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_EINVAL (-1)
#define OR_ENOMEM (-2)

/* ---- alphabet (Methods: the DNA alphabet A, C, G, T) ------------------------------ */
/* Reading: only upper-case A, C, G, T are accepted; anything else (including N) is an
 * invalid input. */
static int base_code(uint8_t b) {
    switch (b) {
        case 'A': return 0;
        case 'C': return 1;
        case 'G': return 2;
        case 'T': return 3;
        default: return -1;
    }
}

static int to_codes(const uint8_t *s, uint64_t n, uint8_t *out) {
    for (uint64_t i = 0; i < n; i++) {
        int c = base_code(s[i]);
        if (c < 0) return OR_EINVAL;
        out[i] = (uint8_t)c;
    }
    return OR_OK;
}

/* ---- k-mer key ---------------------------------------------------------------------
 * Reading: the paper relies on minimap2's internal hash; here the key of a k-mer is the
 * SplitMix64 finaliser (Steele, Lea & Flood, OOPSLA 2014) of its 2k-bit code. The
 * finaliser is a bijection on 64-bit words, so distinct k-mers never share a key. */
uint64_t or_mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

/* Minimizers of one sequence given as codes 0..3.
 * k-mer at i: fwd = sum_t c[i+t] 4^(k-1-t) (first base most significant); its reverse
 * complement rc = sum_t (3 - c[i+k-1-t]) 4^(k-1-t). Canonical: code = min(fwd, rc),
 * strand = (rc < fwd); otherwise code = fwd, strand = 0. For every window of w
 * consecutive k-mers the k-mer with the smallest key is selected (Reading: the leftmost
 * on a tie); the output is the set of selected positions in increasing order, each once.
 * A sequence with fewer than w k-mers has no minimizers. Any output pointer may be NULL.
 * Returns the number of minimizers, or OR_ENOMEM. */
static int64_t minimizers_of_codes(const uint8_t *c, uint64_t n, uint32_t k, uint32_t w,
                                   uint32_t canonical, uint64_t *o_code, uint64_t *o_key,
                                   uint64_t *o_pos, uint8_t *o_strand) {
    if (n < k) return 0;
    uint64_t nk = n - k + 1;
    if (nk < w) return 0;
    uint64_t *code = malloc(nk * sizeof(uint64_t));
    uint64_t *key = malloc(nk * sizeof(uint64_t));
    uint8_t *strand = malloc(nk);
    uint8_t *sel = calloc(nk, 1);
    if (!code || !key || !strand || !sel) {
        free(code); free(key); free(strand); free(sel);
        return OR_ENOMEM;
    }
    for (uint64_t i = 0; i < nk; i++) {
        uint64_t fwd = 0, rc = 0;
        for (uint32_t t = 0; t < k; t++) fwd = fwd * 4 + c[i + t];
        for (uint32_t t = 0; t < k; t++) rc = rc * 4 + (uint64_t)(3 - c[i + k - 1 - t]);
        if (canonical) {
            code[i] = rc < fwd ? rc : fwd;
            strand[i] = rc < fwd ? 1 : 0;
        } else {
            code[i] = fwd;
            strand[i] = 0;
        }
        key[i] = or_mix64(code[i]);
    }
    for (uint64_t j = 0; j + w <= nk; j++) {
        uint64_t best = j;
        for (uint64_t t = j + 1; t < j + w; t++)
            if (key[t] < key[best]) best = t;
        sel[best] = 1;
    }
    int64_t cnt = 0;
    for (uint64_t i = 0; i < nk; i++) {
        if (!sel[i]) continue;
        if (o_code) o_code[cnt] = code[i];
        if (o_key) o_key[cnt] = key[i];
        if (o_pos) o_pos[cnt] = i;
        if (o_strand) o_strand[cnt] = strand[i];
        cnt++;
    }
    free(code); free(key); free(strand); free(sel);
    return cnt;
}

/* Public: minimizers of an ASCII sequence. Output arrays must hold n entries.
 * Returns the count, OR_EINVAL for a non-ACGT base or bad k/w, or OR_ENOMEM. */
int64_t or_minimizers(const uint8_t *seq, uint64_t n, uint32_t k, uint32_t w, uint32_t canonical,
                      uint64_t *o_code, uint64_t *o_key, uint64_t *o_pos, uint8_t *o_strand) {
    if (k < 1 || k > 31 || w < 1) return OR_EINVAL;
    uint8_t *c = malloc(n ? n : 1);
    if (!c) return OR_ENOMEM;
    if (to_codes(seq, n, c) != OR_OK) { free(c); return OR_EINVAL; }
    int64_t r = minimizers_of_codes(c, n, k, w, canonical, o_code, o_key, o_pos, o_strand);
    free(c);
    return r;
}

/* ---- index (Methods, "Index Construction & Querying") ------------------------------
 * A plain multimap: every genome minimizer as (code, genome, position, strand), sorted by
 * (code, genome, position); a lookup is a binary search on the code. */
typedef struct {
    uint64_t code;
    uint32_t g;
    uint32_t pos;
    uint8_t strand;
} or_occ;

typedef struct {
    uint32_t k, w, canonical, G;
    uint64_t n_occ;
    or_occ *occ;
    uint8_t *codes;   /* genome bases as codes, concatenated */
    uint64_t *goff;   /* G + 1 offsets into codes */
} or_index;

static int occ_cmp(const void *a, const void *b) {
    const or_occ *x = a, *y = b;
    if (x->code != y->code) return x->code < y->code ? -1 : 1;
    if (x->g != y->g) return x->g < y->g ? -1 : 1;
    if (x->pos != y->pos) return x->pos < y->pos ? -1 : 1;
    return 0;
}

void or_free_index(or_index *ix) {
    if (!ix) return;
    free(ix->occ); free(ix->codes); free(ix->goff); free(ix);
}

/* Build the index of G genomes given as one ASCII buffer with G+1 offsets. Each genome
 * must be shorter than 2^32 bases. On failure returns NULL and sets *err. */
or_index *or_build_index(const uint8_t *seq, const uint64_t *off, uint32_t G, uint32_t k,
                         uint32_t w, uint32_t canonical, int *err) {
    *err = OR_OK;
    if (k < 1 || k > 31 || w < 1 || G == 0) { *err = OR_EINVAL; return NULL; }
    or_index *ix = calloc(1, sizeof(or_index));
    if (!ix) { *err = OR_ENOMEM; return NULL; }
    ix->k = k; ix->w = w; ix->canonical = canonical; ix->G = G;
    uint64_t total = off[G] - off[0];
    ix->codes = malloc(total ? total : 1);
    ix->goff = malloc((G + 1) * sizeof(uint64_t));
    if (!ix->codes || !ix->goff) { *err = OR_ENOMEM; or_free_index(ix); return NULL; }
    for (uint32_t g = 0; g <= G; g++) ix->goff[g] = off[g] - off[0];
    for (uint32_t g = 0; g < G; g++) {
        if (off[g + 1] < off[g] || off[g + 1] - off[g] >= (1ULL << 32)) {
            *err = OR_EINVAL; or_free_index(ix); return NULL;
        }
    }
    if (to_codes(seq + off[0], total, ix->codes) != OR_OK) {
        *err = OR_EINVAL; or_free_index(ix); return NULL;
    }
    /* count, then fill */
    uint64_t cap = 0;
    for (uint32_t g = 0; g < G; g++) cap += ix->goff[g + 1] - ix->goff[g];
    uint64_t *pos = malloc((cap ? cap : 1) * sizeof(uint64_t));
    uint64_t *code = malloc((cap ? cap : 1) * sizeof(uint64_t));
    uint8_t *strand = malloc(cap ? cap : 1);
    ix->occ = malloc((cap ? cap : 1) * sizeof(or_occ));
    if (!pos || !code || !strand || !ix->occ) {
        free(pos); free(code); free(strand);
        *err = OR_ENOMEM; or_free_index(ix); return NULL;
    }
    uint64_t n_occ = 0;
    for (uint32_t g = 0; g < G; g++) {
        uint64_t len = ix->goff[g + 1] - ix->goff[g];
        int64_t m = minimizers_of_codes(ix->codes + ix->goff[g], len, k, w, canonical, code, NULL,
                                        pos, strand);
        if (m < 0) { free(pos); free(code); free(strand); *err = (int)m; or_free_index(ix); return NULL; }
        for (int64_t i = 0; i < m; i++) {
            ix->occ[n_occ].code = code[i];
            ix->occ[n_occ].g = g;
            ix->occ[n_occ].pos = (uint32_t)pos[i];
            ix->occ[n_occ].strand = strand[i];
            n_occ++;
        }
    }
    free(pos); free(code); free(strand);
    ix->n_occ = n_occ;
    qsort(ix->occ, n_occ, sizeof(or_occ), occ_cmp);
    return ix;
}

uint64_t or_index_n_occ(const or_index *ix) { return ix->n_occ; }

/* Occurrences of a code: [*first, *first + count). */
static uint64_t lookup(const or_index *ix, uint64_t code, uint64_t *first) {
    uint64_t lo = 0, hi = ix->n_occ;
    while (lo < hi) {
        uint64_t mid = lo + (hi - lo) / 2;
        if (ix->occ[mid].code < code) lo = mid + 1; else hi = mid;
    }
    uint64_t e = lo;
    while (e < ix->n_occ && ix->occ[e].code == code) e++;
    *first = lo;
    return e - lo;
}

/* Public lookup for tests: number of occurrences of a code and, if out != NULL, their
 * (genome, position, strand) packed as g << 33 | pos << 1 | strand. */
uint64_t or_index_lookup(const or_index *ix, uint64_t code, uint64_t *out, uint64_t cap) {
    uint64_t first;
    uint64_t cnt = lookup(ix, code, &first);
    for (uint64_t i = 0; out && i < cnt && i < cap; i++) {
        const or_occ *o = &ix->occ[first + i];
        out[i] = ((uint64_t)o->g << 33) | ((uint64_t)o->pos << 1) | o->strand;
    }
    return cnt;
}

/* ---- stage 1: containment search ----------------------------------------------------
 * Seed every read, look each seed up, and add one to the genome of every occurrence.
 * Reading: hits are counted with multiplicity; a seed with more than max_occ occurrences
 * is skipped (the paper leaves minimap2's repeat filter unspecified). hits[] is added to,
 * so read sets can be counted in shards. */
int or_count_hits(const or_index *ix, const uint8_t *reads, const uint64_t *roff,
                  uint64_t n_reads, uint32_t max_occ, uint64_t *hits) {
    for (uint64_t r = 0; r < n_reads; r++) {
        uint64_t n = roff[r + 1] - roff[r];
        uint8_t *c = malloc(n ? n : 1);
        uint64_t *code = malloc((n ? n : 1) * sizeof(uint64_t));
        if (!c || !code) { free(c); free(code); return OR_ENOMEM; }
        if (to_codes(reads + roff[r], n, c) != OR_OK) { free(c); free(code); return OR_EINVAL; }
        int64_t m = minimizers_of_codes(c, n, ix->k, ix->w, ix->canonical, code, NULL, NULL, NULL);
        if (m < 0) { free(c); free(code); return (int)m; }
        for (int64_t i = 0; i < m; i++) {
            uint64_t first, cnt = lookup(ix, code[i], &first);
            if (cnt > max_occ) continue;
            for (uint64_t t = 0; t < cnt; t++) hits[ix->occ[first + t].g]++;
        }
        free(c); free(code);
    }
    return OR_OK;
}

/* Subset database: genome g is kept iff hits[g] / max_h > num / den, i.e. its normalised
 * seed-hit count surpasses the cutoff (strictly), computed in integers. Nothing is kept
 * when no genome has a hit. */
void or_keep(const uint64_t *hits, uint32_t G, uint32_t num, uint32_t den, uint8_t *keep) {
    uint64_t max_h = 0;
    for (uint32_t g = 0; g < G; g++) if (hits[g] > max_h) max_h = hits[g];
    for (uint32_t g = 0; g < G; g++) {
        unsigned __int128 lhs = (unsigned __int128)hits[g] * den;
        unsigned __int128 rhs = (unsigned __int128)max_h * num;
        keep[g] = (max_h > 0 && lhs > rhs) ? 1 : 0;
    }
}

/* ---- SneakySnake edit-distance approximation (Table 1, ref. [48]) --------------------
 * r: the read, n codes 0..3. W: the reference window of n + 2E codes; a code of 4 marks a
 * base outside the genome, which matches nothing. The neighbourhood map has one row per
 * diagonal d in [-E, E]: M[d][j] = 0 iff r[j] == W[E + j + d]. Starting at column 0, the
 * longest run of zeros beginning at the current column over all rows is followed, then the
 * obstacle after it is counted and stepped over; once more than E obstacles are counted
 * the pair is rejected. Returns min(obstacles, E + 1).
 * Reading: the whole map is walked at once (not the paper's hardware sub-matrices). */
uint32_t or_eda_codes(const uint8_t *r, uint32_t n, const uint8_t *W, uint32_t E) {
    uint32_t c = 0, cnt = 0;
    while (c < n) {
        uint32_t longest = 0;
        for (int64_t d = -(int64_t)E; d <= (int64_t)E; d++) {
            uint32_t run = 0;
            while (c + run < n && r[c + run] == W[(int64_t)E + (int64_t)(c + run) + d]) run++;
            if (run > longest) longest = run;
        }
        c += longest;
        if (c < n) {
            cnt++;
            c++;
            if (cnt > E) break;
        }
    }
    return cnt < E + 1 ? cnt : E + 1;
}

/* ---- the paper's other approximations on the same candidate (Table 1; the Discussion of
 * their cost: Base Counting and q-gram compare counts in O(n), HD and SHD follow the
 * pigeonhole principle in O(nE)). The paper gives no formulas; the readings taken:
 *  - HD, Base Counting and q-gram compare the read r with the window's central segment
 *    S = W[E, E + n), which starts at the location's first diagonal; a window code of 4
 *    (outside the genome) equals no read base;
 *  - SHD uses the 2E + 1 diagonals of SneakySnake's map.
 * Each returns min(estimate, E + 1); a pair is accepted iff the result is <= E. */

/* Hamming distance: the positions j with r[j] != S[j]. */
uint32_t or_hd_codes(const uint8_t *r, uint32_t n, const uint8_t *W, uint32_t E) {
    uint32_t cnt = 0;
    for (uint32_t j = 0; j < n; j++) cnt += r[j] != W[E + j];
    return cnt < E + 1 ? cnt : E + 1;
}

/* Base Counting: with c_r(b) and c_S(b) the number of bases b in r and in S (b = 4 only
 * in S), one edit changes sum_b |c_r(b) - c_S(b)| by at most 2, so ceil(sum / 2) is at most
 * the edit distance of r and S. */
uint32_t or_bc_codes(const uint8_t *r, uint32_t n, const uint8_t *W, uint32_t E) {
    int64_t cr[5] = {0, 0, 0, 0, 0}, cs[5] = {0, 0, 0, 0, 0};
    for (uint32_t j = 0; j < n; j++) {
        cr[r[j]]++;
        cs[W[E + j]]++;
    }
    int64_t sum = 0;
    for (int b = 0; b < 5; b++) sum += cr[b] > cs[b] ? cr[b] - cs[b] : cs[b] - cr[b];
    uint64_t est = (uint64_t)(sum + 1) / 2;
    return est < E + 1 ? (uint32_t)est : E + 1;
}

/* q-gram distance (Ukkonen's lemma): with P_r(g) and P_S(g) the occurrences of the q-long
 * string g in r and in S, one edit changes sum_g |P_r(g) - P_S(g)| by at most 2q, so
 * ceil(sum / 2q) is at most the edit distance of r and S. A q-gram of S holding an
 * out-of-genome base occurs in no read and adds 1 to the sum. n < q: no q-grams, 0.
 * q in [1, 8]; 0xFFFFFFFF otherwise or when out of memory. */
uint32_t or_qgram_q(const uint8_t *r, uint32_t n, const uint8_t *W, uint32_t E, uint32_t q) {
    if (q == 0 || q > 8) return 0xFFFFFFFFu;
    if (n < q) return 0;
    const size_t B = (size_t)1 << (2 * q);
    int64_t *P = calloc(B, sizeof(int64_t));
    if (!P) return 0xFFFFFFFFu;
    int64_t sum = 0;
    for (uint32_t j = 0; j + q <= n; j++) {
        size_t g = 0;
        for (uint32_t t = 0; t < q; t++) g |= (size_t)r[j + t] << (2 * t);
        P[g]++;
    }
    for (uint32_t j = 0; j + q <= n; j++) {
        size_t g = 0;
        int outside = 0;
        for (uint32_t t = 0; t < q; t++) {
            uint8_t b = W[E + j + t];
            if (b == 4) outside = 1;
            else g |= (size_t)b << (2 * t);
        }
        if (outside) sum++;
        else P[g]--;
    }
    for (size_t g = 0; g < B; g++) sum += P[g] < 0 ? -P[g] : P[g];
    free(P);
    uint64_t est = (uint64_t)(sum + 2 * q - 1) / (2 * q);
    return est < E + 1 ? (uint32_t)est : E + 1;
}

uint32_t or_qgram_codes(const uint8_t *r, uint32_t n, const uint8_t *W, uint32_t E) {
    return or_qgram_q(r, n, W, E, 5);
}

/* Shifted Hamming distance: for each diagonal d in [-E, E] the mismatch mask
 * H_d(j) = [r[j] != W[E + j + d]]; a run of one or two matches with a mismatch on both
 * sides is taken as a chance match and set to mismatches; the masks are AND-ed over the
 * diagonals and the mismatches left are counted. 0xFFFFFFFF when out of memory. */
uint32_t or_shd_codes(const uint8_t *r, uint32_t n, const uint8_t *W, uint32_t E) {
    uint8_t *F = malloc(n ? n : 1), *H = malloc(n ? n : 1);
    if (!F || !H) { free(F); free(H); return 0xFFFFFFFFu; }
    memset(F, 1, n ? n : 1);
    for (int64_t d = -(int64_t)E; d <= (int64_t)E; d++) {
        for (uint32_t j = 0; j < n; j++) H[j] = r[j] != W[(int64_t)E + (int64_t)j + d];
        uint32_t j = 0;
        while (j < n) {
            if (H[j]) { j++; continue; }
            uint32_t a = j;
            while (j < n && !H[j]) j++;            /* matches [a, j) */
            if (a > 0 && j < n && j - a <= 2)
                for (uint32_t t = a; t < j; t++) H[t] = 1;
        }
        for (uint32_t t = 0; t < n; t++) F[t] &= H[t];
    }
    uint32_t cnt = 0;
    for (uint32_t t = 0; t < n; t++) cnt += F[t];
    free(F); free(H);
    return cnt < E + 1 ? cnt : E + 1;
}

/* Approximation `algo` of one candidate: 0 SneakySnake, 1 HD, 2 Base Counting, 3 q-gram
 * (q = 5), 4 SHD; 0xFFFFFFFF for another algo. */
uint32_t or_approx_codes(uint32_t algo, const uint8_t *r, uint32_t n, const uint8_t *W, uint32_t E) {
    switch (algo) {
        case 0: return or_eda_codes(r, n, W, E);
        case 1: return or_hd_codes(r, n, W, E);
        case 2: return or_bc_codes(r, n, W, E);
        case 3: return or_qgram_codes(r, n, W, E);
        case 4: return or_shd_codes(r, n, W, E);
        default: return 0xFFFFFFFFu;
    }
}

/* ASCII wrappers: read of n bases, window of n + 2E bases (no out-of-genome bases).
 * Return 0xFFFFFFFF on a non-ACGT base. */
uint32_t or_approx_ascii(uint32_t algo, const uint8_t *read, uint32_t n, const uint8_t *win, uint32_t E) {
    uint8_t *r = malloc(n ? n : 1), *W = malloc(n + 2 * E ? n + 2 * E : 1);
    uint32_t out = 0xFFFFFFFFu;
    if (r && W && to_codes(read, n, r) == OR_OK && to_codes(win, n + 2 * E, W) == OR_OK)
        out = or_approx_codes(algo, r, n, W, E);
    free(r); free(W);
    return out;
}

uint32_t or_eda_ascii(const uint8_t *read, uint32_t n, const uint8_t *win, uint32_t E) {
    return or_approx_ascii(0, read, n, win, E);
}

/* A batch of read-versus-window pairs (the EDA stage alone): pair p compares read
 * pair_read[p] with window p, whose length must be that read's length + 2 E[p].
 * dist[p] = the approximation, or 0xFF for malformed input. */
int or_eda_batch(const uint8_t *read_seq, const uint64_t *read_off, const uint8_t *win_seq,
                 const uint64_t *win_off, const uint32_t *pair_read, const uint16_t *E,
                 uint64_t n_pairs, uint32_t algo, uint8_t *dist) {
    for (uint64_t p = 0; p < n_pairs; p++) {
        uint64_t r = pair_read[p];
        uint32_t n = (uint32_t)(read_off[r + 1] - read_off[r]);
        if (win_off[p + 1] - win_off[p] != (uint64_t)n + 2u * E[p]) { dist[p] = 0xFF; continue; }
        uint32_t d = or_approx_ascii(algo, read_seq + read_off[r], n, win_seq + win_off[p], E[p]);
        dist[p] = d == 0xFFFFFFFFu ? 0xFF : (uint8_t)d;
    }
    return OR_OK;
}

/* ---- stage 2: heuristic read mapping -------------------------------------------------- */
typedef struct { uint32_t g; uint8_t rel; int64_t diag; } or_hit;
typedef struct { uint32_t g; uint8_t rel; int64_t d0; uint32_t seeds; } or_cluster;

/* Output record of one mapping location (24 bytes). */
typedef struct {
    int64_t wstart;   /* window start on the genome's forward strand (d0 - E) */
    int32_t genome;   /* -1 for an empty slot */
    uint32_t seeds;   /* seed hits in the location */
    uint8_t strand;   /* 1: the read maps to the reverse strand */
    uint8_t dist;     /* approximate edit distance, capped at E + 1 */
    uint8_t pad[6];
} or_loc;

static int hit_cmp(const void *a, const void *b) {
    const or_hit *x = a, *y = b;
    if (x->g != y->g) return x->g < y->g ? -1 : 1;
    if (x->rel != y->rel) return x->rel < y->rel ? -1 : 1;
    if (x->diag != y->diag) return x->diag < y->diag ? -1 : 1;
    return 0;
}

/* Rank: seeds descending, then genome, strand and first diagonal ascending. */
static int cluster_cmp(const void *a, const void *b) {
    const or_cluster *x = a, *y = b;
    if (x->seeds != y->seeds) return x->seeds > y->seeds ? -1 : 1;
    if (x->g != y->g) return x->g < y->g ? -1 : 1;
    if (x->rel != y->rel) return x->rel < y->rel ? -1 : 1;
    if (x->d0 != y->d0) return x->d0 < y->d0 ? -1 : 1;
    return 0;
}

/* Reading: E(n) = e_abs, or floor(n * e_permille / 1000) when e_permille != 0. */
static uint32_t edit_threshold(uint64_t n, uint32_t e_abs, uint32_t e_permille) {
    return e_permille ? (uint32_t)((n * (uint64_t)e_permille) / 1000u) : e_abs;
}

/* Map reads [0, n_reads) against the kept genomes and decide each read.
 *  - seed matches: for read minimizer (rpos, rstrand) and occurrence (g, gpos, gstrand) in
 *    a kept genome, rel = rstrand xor gstrand, rpos' = rpos (rel 0) or n - k - rpos (rel 1),
 *    diag = gpos - rpos' (the read's start on the genome's forward strand);
 *  - Reading (mapping locations): matches sorted by (g, rel, diag) are grouped greedily: a
 *    location starts at the first unassigned match (diagonal d0) and takes every following
 *    match of the same (g, rel) with diag <= d0 + E; its seed count is its match count;
 *  - locations with fewer than min_seeds seeds are dropped; the rest are ranked by seeds
 *    (descending, ties by genome, strand, d0) and the first top_n are kept;
 *  - each kept location is compared with SneakySnake: the read (reverse-complemented when
 *    rel = 1) against the window [d0 - E, d0 + n + E) of its genome;
 *  - decision (Reading): locations with distance <= E are accepted; the read's taxon is the
 *    genome of the first accepted location (rank order) with the smallest distance, or -1;
 *    the read is unique when all accepted locations at that distance share one genome
 *    (U[g] += 1), and multi-mapped otherwise (its genomes go to multi[], -1 padded).
 * Outputs per read: taxon[r], nloc[r], locs[r*top_n ...], multi[r*top_n ...]. U[] is added
 * to. Returns OR_OK, OR_EINVAL (bad base / params) or OR_ENOMEM. */
int or_map_reads(const or_index *ix, const uint8_t *reads, const uint64_t *roff, uint64_t n_reads,
                 uint32_t max_occ, uint32_t e_abs, uint32_t e_permille, uint32_t min_seeds,
                 uint32_t top_n, uint32_t algo, const uint8_t *keep, int32_t *taxon, or_loc *locs,
                 uint8_t *nloc, int32_t *multi, uint64_t *U) {
    if (top_n < 1 || algo > 4) return OR_EINVAL;
    const uint32_t k = ix->k;
    for (uint64_t r = 0; r < n_reads; r++) {
        uint64_t n = roff[r + 1] - roff[r];
        uint32_t E = edit_threshold(n, e_abs, e_permille);
        for (uint32_t t = 0; t < top_n; t++) {
            or_loc *L = &locs[r * top_n + t];
            memset(L, 0, sizeof(*L));
            L->genome = -1;
            multi[r * top_n + t] = -1;
        }
        nloc[r] = 0;
        taxon[r] = -1;

        uint8_t *c = malloc(n ? n : 1);
        uint64_t *code = malloc((n ? n : 1) * sizeof(uint64_t));
        uint64_t *pos = malloc((n ? n : 1) * sizeof(uint64_t));
        uint8_t *strand = malloc(n ? n : 1);
        if (!c || !code || !pos || !strand) { free(c); free(code); free(pos); free(strand); return OR_ENOMEM; }
        if (to_codes(reads + roff[r], n, c) != OR_OK) { free(c); free(code); free(pos); free(strand); return OR_EINVAL; }
        int64_t m = minimizers_of_codes(c, n, k, ix->w, ix->canonical, code, NULL, pos, strand);
        if (m < 0) { free(c); free(code); free(pos); free(strand); return (int)m; }

        /* seed matches in kept genomes */
        uint64_t H = 0, cap = 16;
        or_hit *hits = malloc(cap * sizeof(or_hit));
        for (int64_t i = 0; i < m && hits; i++) {
            uint64_t first, cnt = lookup(ix, code[i], &first);
            if (cnt > max_occ) continue;
            for (uint64_t t = 0; t < cnt; t++) {
                const or_occ *o = &ix->occ[first + t];
                if (!keep[o->g]) continue;
                uint8_t rel = (uint8_t)(strand[i] ^ o->strand);
                int64_t rp = rel ? (int64_t)(n - k - pos[i]) : (int64_t)pos[i];
                if (H == cap) {
                    cap *= 2;
                    or_hit *nh = realloc(hits, cap * sizeof(or_hit));
                    if (!nh) { free(hits); hits = NULL; break; }
                    hits = nh;
                }
                hits[H].g = o->g;
                hits[H].rel = rel;
                hits[H].diag = (int64_t)o->pos - rp;
                H++;
            }
        }
        if (!hits) { free(c); free(code); free(pos); free(strand); return OR_ENOMEM; }
        qsort(hits, H, sizeof(or_hit), hit_cmp);

        /* greedy locations */
        or_cluster *cl = malloc((H ? H : 1) * sizeof(or_cluster));
        if (!cl) { free(hits); free(c); free(code); free(pos); free(strand); return OR_ENOMEM; }
        uint64_t Q = 0;
        for (uint64_t i = 0; i < H;) {
            uint64_t j = i + 1;
            while (j < H && hits[j].g == hits[i].g && hits[j].rel == hits[i].rel &&
                   hits[j].diag <= hits[i].diag + (int64_t)E)
                j++;
            if (j - i >= min_seeds) {
                cl[Q].g = hits[i].g;
                cl[Q].rel = hits[i].rel;
                cl[Q].d0 = hits[i].diag;
                cl[Q].seeds = (uint32_t)(j - i);
                Q++;
            }
            i = j;
        }
        qsort(cl, Q, sizeof(or_cluster), cluster_cmp);
        uint32_t nl = (uint32_t)(Q < top_n ? Q : top_n);

        /* edit-distance approximation of each kept location */
        uint8_t *rr = malloc(n ? n : 1);
        uint8_t *W = malloc(n + 2 * (uint64_t)E + 1);
        if (!rr || !W) { free(rr); free(W); free(cl); free(hits); free(c); free(code); free(pos); free(strand); return OR_ENOMEM; }
        for (uint32_t t = 0; t < nl; t++) {
            const or_cluster *q = &cl[t];
            int64_t wstart = q->d0 - (int64_t)E;
            const uint8_t *gc = ix->codes + ix->goff[q->g];
            int64_t glen = (int64_t)(ix->goff[q->g + 1] - ix->goff[q->g]);
            for (uint64_t x = 0; x < n + 2 * (uint64_t)E; x++) {
                int64_t gp = wstart + (int64_t)x;
                W[x] = (gp >= 0 && gp < glen) ? gc[gp] : 4;
            }
            for (uint64_t j = 0; j < n; j++) rr[j] = q->rel ? (uint8_t)(3 - c[n - 1 - j]) : c[j];
            uint32_t dist = or_approx_codes(algo, rr, (uint32_t)n, W, E);
            if (dist == 0xFFFFFFFFu) { free(rr); free(W); free(cl); free(hits); free(c); free(code); free(pos); free(strand); return OR_ENOMEM; }
            or_loc *L = &locs[r * top_n + t];
            L->wstart = wstart;
            L->genome = (int32_t)q->g;
            L->seeds = q->seeds;
            L->strand = q->rel;
            L->dist = (uint8_t)(dist > 255 ? 255 : dist);
        }
        nloc[r] = (uint8_t)nl;

        /* per-read decision */
        uint32_t best = E + 1;
        for (uint32_t t = 0; t < nl; t++) {
            uint32_t d = locs[r * top_n + t].dist;
            if (d <= E && d < best) best = d;
        }
        if (best <= E) {
            uint32_t ns = 0;
            for (uint32_t t = 0; t < nl; t++) {
                const or_loc *L = &locs[r * top_n + t];
                if (L->dist != best) continue;
                if (taxon[r] < 0) taxon[r] = L->genome;
                int seen = 0;
                for (uint32_t s = 0; s < ns; s++) if (multi[r * top_n + s] == L->genome) seen = 1;
                if (!seen) multi[r * top_n + ns++] = L->genome;
            }
            if (ns == 1) {
                U[multi[r * top_n]]++;
                multi[r * top_n] = -1;
            }
        }
        free(rr); free(W); free(cl); free(hits); free(c); free(code); free(pos); free(strand);
    }
    return OR_OK;
}

/* ---- stage 3: taxonomic profiling (Fig. 1 3a-b; "Taxonomic Profile Generation") -------
 * Reading (Metalign's profiler is not restated by the paper): a multi-mapped read with
 * genome set S adds U[g] / sum_{h in S} U[h] to M[g] for g in S, or 1/|S| to each when
 * that sum is 0 (U is final before the split). a[g] = (U[g] + M[g]) / sum over all genomes;
 * entries below the cutoff (0.01% = 1e-4) are zeroed and the rest renormalised. Abundance
 * is per read, without genome-length normalisation. All zeros when no read is classified. */
void or_abundance(const uint64_t *U, uint32_t G, const int32_t *multi, uint64_t n_reads,
                  uint32_t top_n, double cutoff, double *a) {
    double *M = calloc(G ? G : 1, sizeof(double));
    for (uint64_t r = 0; M && r < n_reads; r++) {
        const int32_t *S = multi + r * top_n;
        uint32_t ns = 0;
        while (ns < top_n && S[ns] >= 0) ns++;
        if (ns < 2) continue;
        uint64_t tot = 0;
        for (uint32_t s = 0; s < ns; s++) tot += U[S[s]];
        for (uint32_t s = 0; s < ns; s++)
            M[S[s]] += tot ? (double)U[S[s]] / (double)tot : 1.0 / (double)ns;
    }
    double sum = 0.0;
    for (uint32_t g = 0; g < G; g++) {
        a[g] = (double)U[g] + (M ? M[g] : 0.0);
        sum += a[g];
    }
    if (sum <= 0.0) {
        for (uint32_t g = 0; g < G; g++) a[g] = 0.0;
        free(M);
        return;
    }
    double kept = 0.0;
    for (uint32_t g = 0; g < G; g++) {
        a[g] /= sum;
        if (a[g] < cutoff) a[g] = 0.0;
        kept += a[g];
    }
    for (uint32_t g = 0; g < G && kept > 0.0; g++) a[g] /= kept;
    free(M);
}

uint32_t or_index_G(const or_index *ix) { return ix->G; }
uint32_t or_index_k(const or_index *ix) { return ix->k; }

/* Genome bases of the index as codes (for tests). */
const uint8_t *or_index_codes(const or_index *ix, uint32_t g, uint64_t *len) {
    *len = ix->goff[g + 1] - ix->goff[g];
    return ix->codes + ix->goff[g];
}

/* ---- the same index built on several host threads (verification runs only) ----------------
 * Identical contents to or_build_index: every genome's minimizers are found by the same
 * routine on a pool of threads, then the records are distributed into buckets by the top bits
 * of their code (bucket order = code order) and each bucket is sorted by (code, genome,
 * position) on the pool. Only the work is split; nothing is computed differently. */
#include <pthread.h>

typedef struct {
    const or_index *ix;
    uint32_t next_g;          /* shared work counter */
    pthread_mutex_t mu;
    uint64_t **pos;           /* per genome */
    uint64_t **code;
    uint8_t **strand;
    int64_t *cnt;
    int err;
} mt_job;

static void *mini_worker(void *arg) {
    mt_job *J = arg;
    const or_index *ix = J->ix;
    uint64_t scap = 0;
    uint64_t *spos = NULL, *scode = NULL;
    uint8_t *sst = NULL;
    for (;;) {
        pthread_mutex_lock(&J->mu);
        uint32_t g = J->next_g++;
        pthread_mutex_unlock(&J->mu);
        if (g >= ix->G) break;
        uint64_t len = ix->goff[g + 1] - ix->goff[g];
        uint64_t cap = len ? len : 1;
        if (cap > scap) {   /* thread scratch, then exact-size copies per genome */
            free(spos); free(scode); free(sst);
            spos = malloc(cap * sizeof(uint64_t));
            scode = malloc(cap * sizeof(uint64_t));
            sst = malloc(cap);
            scap = (spos && scode && sst) ? cap : 0;
        }
        if (!scap) { J->cnt[g] = OR_ENOMEM; continue; }
        int64_t m = minimizers_of_codes(ix->codes + ix->goff[g], len, ix->k, ix->w, ix->canonical,
                                        scode, NULL, spos, sst);
        J->cnt[g] = m;
        if (m <= 0) continue;
        J->pos[g] = malloc((uint64_t)m * sizeof(uint64_t));
        J->code[g] = malloc((uint64_t)m * sizeof(uint64_t));
        J->strand[g] = malloc((uint64_t)m);
        if (!J->pos[g] || !J->code[g] || !J->strand[g]) { J->cnt[g] = OR_ENOMEM; continue; }
        memcpy(J->pos[g], spos, (uint64_t)m * sizeof(uint64_t));
        memcpy(J->code[g], scode, (uint64_t)m * sizeof(uint64_t));
        memcpy(J->strand[g], sst, (uint64_t)m);
    }
    free(spos); free(scode); free(sst);
    return NULL;
}

typedef struct {
    or_occ *occ;
    uint64_t *bstart;         /* NB + 1 */
    uint32_t nb;
    uint32_t next_b;
    pthread_mutex_t mu;
} sort_job;

static void *sort_worker(void *arg) {
    sort_job *S = arg;
    for (;;) {
        pthread_mutex_lock(&S->mu);
        uint32_t b = S->next_b++;
        pthread_mutex_unlock(&S->mu);
        if (b >= S->nb) break;
        qsort(S->occ + S->bstart[b], S->bstart[b + 1] - S->bstart[b], sizeof(or_occ), occ_cmp);
    }
    return NULL;
}

or_index *or_build_index_threads(const uint8_t *seq, const uint64_t *off, uint32_t G, uint32_t k,
                                 uint32_t w, uint32_t canonical, uint32_t nthreads, int *err) {
    *err = OR_OK;
    if (k < 1 || k > 31 || w < 1 || G == 0 || nthreads < 1) { *err = OR_EINVAL; return NULL; }
    if (nthreads > 256) nthreads = 256;
    or_index *ix = calloc(1, sizeof(or_index));
    if (!ix) { *err = OR_ENOMEM; return NULL; }
    ix->k = k; ix->w = w; ix->canonical = canonical; ix->G = G;
    uint64_t total = off[G] - off[0];
    ix->codes = malloc(total ? total : 1);
    ix->goff = malloc((G + 1) * sizeof(uint64_t));
    if (!ix->codes || !ix->goff) { *err = OR_ENOMEM; or_free_index(ix); return NULL; }
    for (uint32_t g = 0; g <= G; g++) ix->goff[g] = off[g] - off[0];
    for (uint32_t g = 0; g < G; g++)
        if (off[g + 1] < off[g] || off[g + 1] - off[g] >= (1ULL << 32)) { *err = OR_EINVAL; or_free_index(ix); return NULL; }
    if (to_codes(seq + off[0], total, ix->codes) != OR_OK) { *err = OR_EINVAL; or_free_index(ix); return NULL; }

    mt_job J;
    memset(&J, 0, sizeof(J));
    J.ix = ix;
    pthread_mutex_init(&J.mu, NULL);
    J.pos = calloc(G, sizeof(uint64_t *));
    J.code = calloc(G, sizeof(uint64_t *));
    J.strand = calloc(G, sizeof(uint8_t *));
    J.cnt = calloc(G, sizeof(int64_t));
    pthread_t th[256];
    for (uint32_t t = 0; t < nthreads; t++) pthread_create(&th[t], NULL, mini_worker, &J);
    for (uint32_t t = 0; t < nthreads; t++) pthread_join(th[t], NULL);
    pthread_mutex_destroy(&J.mu);
    uint64_t n_occ = 0;
    for (uint32_t g = 0; g < G; g++) {
        if (J.cnt[g] < 0) *err = (int)J.cnt[g];
        else n_occ += (uint64_t)J.cnt[g];
    }
    /* buckets by the top 12 bits of the 2k-bit code */
    const uint32_t bits = 2 * k, shift = bits > 12 ? bits - 12 : 0, NB = 1u << (bits > 12 ? 12 : bits);
    uint64_t *bstart = calloc(NB + 1, sizeof(uint64_t));
    ix->occ = malloc((n_occ ? n_occ : 1) * sizeof(or_occ));
    if (*err == OR_OK && (!bstart || !ix->occ)) *err = OR_ENOMEM;
    if (*err == OR_OK) {
        for (uint32_t g = 0; g < G; g++)
            for (int64_t i = 0; i < J.cnt[g]; i++) bstart[(J.code[g][i] >> shift) + 1]++;
        for (uint32_t b = 0; b < NB; b++) bstart[b + 1] += bstart[b];
        uint64_t *cur = malloc(NB * sizeof(uint64_t));
        if (!cur) *err = OR_ENOMEM;
        else {
            memcpy(cur, bstart, NB * sizeof(uint64_t));
            for (uint32_t g = 0; g < G; g++)
                for (int64_t i = 0; i < J.cnt[g]; i++) {
                    or_occ *o = &ix->occ[cur[J.code[g][i] >> shift]++];
                    o->code = J.code[g][i];
                    o->g = g;
                    o->pos = (uint32_t)J.pos[g][i];
                    o->strand = J.strand[g][i];
                }
            free(cur);
        }
    }
    for (uint32_t g = 0; g < G; g++) { free(J.pos[g]); free(J.code[g]); free(J.strand[g]); }
    free(J.pos); free(J.code); free(J.strand); free(J.cnt);
    if (*err != OR_OK) { free(bstart); or_free_index(ix); return NULL; }
    ix->n_occ = n_occ;
    sort_job S;
    S.occ = ix->occ; S.bstart = bstart; S.nb = NB; S.next_b = 0;
    pthread_mutex_init(&S.mu, NULL);
    for (uint32_t t = 0; t < nthreads; t++) pthread_create(&th[t], NULL, sort_worker, &S);
    for (uint32_t t = 0; t < nthreads; t++) pthread_join(th[t], NULL);
    pthread_mutex_destroy(&S.mu);
    free(bstart);
    return ix;
}

/* ---- taxonomic roll-up (Fig. 1, 3b; "Taxonomic Profile Generation") --------------------
 * The abundance of taxon v is the sum of the abundances of the genomes that lie in v's
 * subtree: for every taxon and every genome, the genome counts when v is found on the path
 * from the genome's node to its root. Returns OR_EINVAL for an index out of range or a path
 * longer than the number of nodes (a cycle). */
int or_rollup(const double *a, uint32_t G, const uint32_t *genome_node, const int32_t *parent,
              uint32_t T, double *out) {
    for (uint32_t g = 0; g < G; g++)
        if (genome_node[g] >= T) return OR_EINVAL;
    for (uint32_t v = 0; v < T; v++)
        if (parent[v] < -1 || parent[v] >= (int64_t)T) return OR_EINVAL;
    for (uint32_t g = 0; g < G; g++) {          /* every genome's path reaches a root */
        int64_t u = genome_node[g];
        for (uint32_t steps = 0; u != -1; steps++) {
            if (steps >= T) return OR_EINVAL;
            u = parent[u];
        }
    }
    for (uint32_t v = 0; v < T; v++) {
        double s = 0.0;
        for (uint32_t g = 0; g < G; g++) {
            int64_t u = genome_node[g];
            uint32_t steps = 0;
            int below = 0;
            while (u != -1) {
                if (u == (int64_t)v) { below = 1; break; }
                u = parent[u];
                if (++steps > T) return OR_EINVAL;
            }
            if (below) s += a[g];
        }
        out[v] = s;
    }
    return OR_OK;
}

/* ---- homopolymer compression (the containment index's seeds: minimap2's -H, Results
 * "Evaluation Methodology", k = 28, w = 18) ------------------------------------------------
 * Every run of one repeated byte in a sequence becomes a single byte; runs never join across
 * sequences. out needs off[n] - off[0] bytes; out_off gets n + 1 offsets from 0. */
void or_hpc(const uint8_t *seq, const uint64_t *off, uint64_t n, uint8_t *out, uint64_t *out_off) {
    uint64_t o = 0;
    out_off[0] = 0;
    for (uint64_t i = 0; i < n; i++) {
        for (uint64_t j = off[i]; j < off[i + 1]; j++)
            if (j == off[i] || seq[j] != seq[j - 1]) out[o++] = seq[j];
        out_off[i + 1] = o;
    }
}
