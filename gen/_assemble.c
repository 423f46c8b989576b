/*
 * Window assembly for the synthetic read-versus-window pairs.
 *
 * Pure data generation: every random number (flank bases, edit positions, edit kinds,
 * substitute bases, window offsets) is drawn by the caller with numpy; this routine only
 * writes the edited read into its pre-filled random window. No classification or
 * edit-distance arithmetic lives here.
 */
#include <stdint.h>
#include <stdlib.h>

typedef struct { int32_t pos; uint8_t kind; uint8_t sub; } ev_t;

static int ev_cmp(const void *a, const void *b) {
    const ev_t *x = (const ev_t *)a, *y = (const ev_t *)b;
    if (x->pos != y->pos) return x->pos < y->pos ? -1 : 1;
    return (int)x->kind - (int)y->kind;
}

static const uint8_t ACGT[4] = {'A', 'C', 'G', 'T'};

static int code_of(uint8_t b) {
    switch (b) { case 'A': return 0; case 'C': return 1; case 'G': return 2; default: return 3; }
}

/* For pairs [0, n): window p (length wlen[p], at win + win_off[p]) already holds random
 * bases. Starting at column left[p], copy read pair_read[p] into it, applying the events
 * ev[ev_off[p] .. ev_off[p+1]): kind 0 = substitute (base += sub mod 4), 1 = insert (the
 * random base at the current column is kept before the read base), 2 = delete (skip the
 * read base). Copying stops at the window end. Returns 0. */
int gen_assemble(uint64_t n, const uint8_t *reads, const uint64_t *read_off,
                 const uint32_t *pair_read, const uint64_t *win_off, const int64_t *wlen,
                 const int64_t *left, const uint64_t *ev_off, const int32_t *ev_pos,
                 const uint8_t *ev_kind, const uint8_t *ev_sub, uint8_t *win) {
    ev_t buf[512];
    for (uint64_t p = 0; p < n; p++) {
        const uint8_t *r = reads + read_off[pair_read[p]];
        int64_t L = (int64_t)(read_off[pair_read[p] + 1] - read_off[pair_read[p]]);
        uint8_t *w = win + win_off[p];
        int64_t W = wlen[p];
        uint64_t e0 = ev_off[p], ne = ev_off[p + 1] - e0;
        if (ne > 512) ne = 512;
        for (uint64_t i = 0; i < ne; i++) {
            buf[i].pos = ev_pos[e0 + i]; buf[i].kind = ev_kind[e0 + i]; buf[i].sub = ev_sub[e0 + i];
        }
        qsort(buf, ne, sizeof(ev_t), ev_cmp);
        int64_t col = left[p];
        uint64_t e = 0;
        for (int64_t j = 0; j < L && col < W; j++) {
            int del = 0, sub = 0;
            while (e < ne && buf[e].pos == j) {
                if (buf[e].kind == 0) sub = (sub + buf[e].sub) & 3;
                else if (buf[e].kind == 1) col++;          /* keep one random base */
                else del = 1;
                e++;
            }
            if (del || col >= W) continue;
            w[col++] = sub ? ACGT[(code_of(r[j]) + sub) & 3] : r[j];
        }
    }
    return 0;
}
