/*
 * X-drop traceback oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * The paper's extension keeps three anti-diagonals and reports no path
 * (Sec. IV-A).  This file adds the alignment path of the best cell: the same
 * sweep as xdrop_oracle.c (linear gaps, every reading R1-R18 there), with
 * each anti-diagonal's evaluated cells kept, and a walk back from the best
 * cell to (0,0).  It shares no code, header or constant with the CUDA path
 * (nor with the other oracle files).
 *
 * Readings (in the design notes):
 *   T1 each live cell records the predecessor term that gave its score; when
 *      several give it, the diagonal wins, then the vertical move (i-1, j),
 *      then the horizontal one (i, j-1).
 *   T2 the path of an extension is the walk from its best cell back to
 *      (0,0) along the recorded predecessors; as operations: 'M' for a
 *      diagonal step (a match or a mismatch), 'I' for a vertical step (a
 *      base of a with none of b), 'D' for a horizontal step (a base of b with
 *      none of a), listed from (0,0) to the best cell.
 *   T3 a pair's alignment: the left extension's operations (the left
 *      extension runs on the reversed prefixes, so its walk from the best
 *      cell back to (0,0) lists them in the sequences' own order), k 'M'
 *      for the seed, then the right extension's operations; it spans
 *      [begA, endA) x [begB, endB).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define TB_OK 0
#define TB_INVALID 1
#define TB_NOMEM 2

static int64_t tmax(int64_t a, int64_t b) { return a > b ? a : b; }
static int64_t tmin(int64_t a, int64_t b) { return a < b ? a : b; }

/* the evaluated range of one anti-diagonal: score, liveness, predecessor */
typedef struct {
    int64_t lo, hi;          /* evaluated range (lo > hi: none) */
    int64_t tlo, thi;        /* trimmed live range stored for the next ones */
    int64_t *val;
    unsigned char *live, *dir;
} tb_diag_t;

static void tb_free(tb_diag_t *D, int64_t nd)
{
    for (int64_t d = 0; d < nd; ++d) { free(D[d].val); free(D[d].live); free(D[d].dir); }
    free(D);
}

static int tb_has(const tb_diag_t *e, int64_t i)
{
    return i >= e->tlo && i <= e->thi && e->live[i - e->lo];
}

/* One extension: best, its cell, cells, and the path as operations
 * ('M', 'I', 'D'; at most m + n of them) in ops[0 .. *nops). */
int oracle_xdrop_traceback(const uint8_t *a, int64_t m, const uint8_t *b, int64_t n,
                           int64_t match, int64_t mismatch, int64_t gap, int64_t X,
                           int64_t *best_out, int64_t *bi_out, int64_t *bj_out,
                           int64_t *cells_out, char *ops, int64_t *nops)
{
    const int64_t nd = m + n + 1;
    tb_diag_t *D = (tb_diag_t *)calloc((size_t)nd, sizeof(tb_diag_t));
    if (!D) return TB_NOMEM;
    /* d = 0: cell (0,0), score 0 */
    D[0].lo = D[0].hi = D[0].tlo = D[0].thi = 0;
    D[0].val = (int64_t *)malloc(sizeof(int64_t));
    D[0].live = (unsigned char *)malloc(1);
    D[0].dir = (unsigned char *)malloc(1);
    if (!D[0].val || !D[0].live || !D[0].dir) { tb_free(D, nd); return TB_NOMEM; }
    D[0].val[0] = 0; D[0].live[0] = 1; D[0].dir[0] = 0;
    int64_t best = 0, bi = 0, bj = 0, cells = 0, last_d = 0;
    for (int64_t d = 1; d < nd; ++d) {
        const tb_diag_t *p1 = &D[d - 1];
        const tb_diag_t *p2 = d >= 2 ? &D[d - 2] : NULL;
        int64_t rlo = tmax(p1->tlo, d - n), rhi = tmin(p1->thi + 1, m);
        if (rlo > rhi) break;
        tb_diag_t *cur = &D[d];
        const size_t w = (size_t)(rhi - rlo + 1);
        cur->lo = rlo; cur->hi = rhi;
        cur->val = (int64_t *)malloc(w * sizeof(int64_t));
        cur->live = (unsigned char *)calloc(w, 1);
        cur->dir = (unsigned char *)calloc(w, 1);
        if (!cur->val || !cur->live || !cur->dir) { tb_free(D, nd); return TB_NOMEM; }
        const int64_t thr = best - X;
        int any = 0;
        int64_t dmax = 0, dmax_i = 0, first = 0, last = 0;
        for (int64_t i = rlo; i <= rhi; ++i) {
            const int64_t j = d - i;
            int have = 0;
            unsigned char how = 0;
            int64_t s = 0, t;
            if (i > 0 && j > 0 && p2 && tb_has(p2, i - 1)) {       /* diagonal */
                s = p2->val[i - 1 - p2->lo] + (a[i - 1] == b[j - 1] ? match : mismatch);
                have = 1;
                how = 0;
            }
            if (i > 0 && tb_has(p1, i - 1)) {                       /* vertical */
                t = p1->val[i - 1 - p1->lo] + gap;
                if (!have || t > s) { s = t; how = 1; }
                have = 1;
            }
            if (j > 0 && tb_has(p1, i)) {                           /* horizontal */
                t = p1->val[i - p1->lo] + gap;
                if (!have || t > s) { s = t; how = 2; }
                have = 1;
            }
            const int is_live = have && !(s < thr);
            cur->val[i - rlo] = s;
            cur->live[i - rlo] = (unsigned char)is_live;
            cur->dir[i - rlo] = how;
            if (is_live) {
                if (!any || s > dmax) { dmax = s; dmax_i = i; }
                if (!any) first = i;
                last = i;
                any = 1;
            }
        }
        cells += rhi - rlo + 1;
        last_d = d;
        if (!any) { cur->tlo = 1; cur->thi = 0; break; }
        if (dmax > best) { best = dmax; bi = dmax_i; bj = d - dmax_i; }
        cur->tlo = first;
        cur->thi = last;
    }
    (void)last_d;
    /* walk back from the best cell (T2); ops come out last-first */
    int64_t k = 0, i = bi, j = bj;
    while (i + j > 0) {
        const tb_diag_t *e = &D[i + j];
        const unsigned char how = e->dir[i - e->lo];
        if (how == 0) { ops[k++] = 'M'; --i; --j; }
        else if (how == 1) { ops[k++] = 'I'; --i; }
        else { ops[k++] = 'D'; --j; }
    }
    for (int64_t x = 0; x < k / 2; ++x) { char c = ops[x]; ops[x] = ops[k - 1 - x]; ops[k - 1 - x] = c; }
    *nops = k;
    *best_out = best; *bi_out = bi; *bj_out = bj; *cells_out = cells;
    tb_free(D, nd);
    return TB_OK;
}

/* A seeded pair's alignment (T3): ops[0 .. *nops), at most lenA + lenB. */
int oracle_pair_traceback(const uint8_t *A, int64_t lenA, const uint8_t *B, int64_t lenB,
                          int64_t posA, int64_t posB, int64_t k, int64_t match,
                          int64_t mismatch, int64_t gap, int64_t X, char *ops, int64_t *nops)
{
    *nops = 0;
    if (k < 0 || posA < 0 || posB < 0 || posA + k > lenA || posB + k > lenB) return TB_INVALID;
    uint8_t *ra = (uint8_t *)malloc((size_t)posA + 1), *rb = (uint8_t *)malloc((size_t)posB + 1);
    if (!ra || !rb) { free(ra); free(rb); return TB_NOMEM; }
    for (int64_t t = 0; t < posA; ++t) ra[t] = A[posA - 1 - t];
    for (int64_t t = 0; t < posB; ++t) rb[t] = B[posB - 1 - t];
    int64_t bst, bi, bj, cl, nl = 0, nr = 0;
    /* left: the walk lists the reversed prefixes' path from the best cell
     * back to (0,0), i.e. the original order; undo the reversal done above */
    int e = oracle_xdrop_traceback(ra, posA, rb, posB, match, mismatch, gap, X, &bst, &bi, &bj,
                                   &cl, ops, &nl);
    free(ra); free(rb);
    if (e) return e;
    for (int64_t x = 0; x < nl / 2; ++x) { char c = ops[x]; ops[x] = ops[nl - 1 - x]; ops[nl - 1 - x] = c; }
    for (int64_t t = 0; t < k; ++t) ops[nl + t] = 'M';
    e = oracle_xdrop_traceback(A + posA + k, lenA - posA - k, B + posB + k, lenB - posB - k,
                               match, mismatch, gap, X, &bst, &bi, &bj, &cl, ops + nl + k, &nr);
    if (e) return e;
    *nops = nl + k + nr;
    return TB_OK;
}
