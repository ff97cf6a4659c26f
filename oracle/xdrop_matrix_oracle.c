/*
 * X-drop seed-extension oracle with a substitution matrix and affine gaps
 * -- TEST INFRASTRUCTURE ONLY.
 *
 * The paper scores DNA with match / mismatch and a linear gap (Sec. III-A)
 * and names protein alignment and other scoring schemes as future work
 * (Sec. VIII).  This file restates the paper's X-drop extension for any
 * alphabet of K letters (sequences given as letter codes 0..K-1) scored by
 * a K x K substitution matrix, with Gotoh's affine gaps (a gap of length L
 * scores gap_open + L * gap_extend; gap_open = 0 is the linear case).  The
 * anti-diagonal sweep, the X-drop rule, the band trimming, the best cell
 * and the cell count are the paper's, unchanged.  Only tests, the smoke
 * check and the benchmark's CPU baseline may load it; the library never
 * does, and it shares no code, header or table with the CUDA path (nor with
 * the other oracle files).
 *
 * Recurrence (terms whose predecessor does not exist are absent; a state
 * with no term is -infinity):
 *   E(i,j) = max(E(i,j-1) + e, H(i,j-1) + o + e)
 *   F(i,j) = max(F(i-1,j) + e, H(i-1,j) + o + e)
 *   H(i,j) = max(H(i-1,j-1) + M[a_i][b_j], E(i,j), F(i,j))
 *   H(0,0) = 0, E(0,0) = F(0,0) = -infinity.
 * Readings (as for the affine DNA oracle, with M in place of
 * match / mismatch):
 *   - X-drop acts on H; a pruned cell loses all three states.
 *   - a predecessor exists only in the stored (trimmed) range of its
 *     anti-diagonal and when live; the next range follows the first and
 *     last live H of the anti-diagonal.
 *   - best starts at 0 at (0,0), strict improvement, first anti-diagonal
 *     then smallest row on ties; cells = every evaluated cell for d >= 1.
 *   - the seed score is the sum of M over the seed's columns; a pair is
 *     left extension + seed + right extension, the left one on the
 *     reversed prefixes.
 *   Validation: 1 <= K <= 32; |M| <= 1000; -1000 <= o, e <= 0; 0 <= X <=
 *   2^29; letter codes < K; the seed inside both sequences; and
 *   max(max|M|, |o| + |e|) * (m + n) + X < 2^29 per pair.
 *
 * Arithmetic is int64 with an explicit existence flag per state.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

#define MX_OK 0
#define MX_INVALID 1
#define MX_NOMEM 2

typedef struct {
    int64_t best, bi, bj, cells;
} mx_ext_t;

typedef struct {
    int64_t score, left, right;
    int64_t begA, begB, endA, endB;
    int64_t cells;
    int64_t status;
} mx_pair_t;

static int64_t mx_max(int64_t a, int64_t b) { return a > b ? a : b; }
static int64_t mx_min(int64_t a, int64_t b) { return a < b ? a : b; }
static int64_t mx_abs(int64_t x) { return x < 0 ? -x : x; }

/* the three states of one anti-diagonal, indexed by row i */
typedef struct {
    int64_t *h, *e, *f;
    unsigned char *has_h, *has_e, *has_f, *live;
    int64_t lo, hi; /* stored range after trimming; lo > hi: empty */
} mx_diag_t;

static int mx_diag_alloc(mx_diag_t *a, int64_t rows)
{
    size_t n = (size_t)rows;
    a->h = (int64_t *)malloc(n * sizeof(int64_t));
    a->e = (int64_t *)malloc(n * sizeof(int64_t));
    a->f = (int64_t *)malloc(n * sizeof(int64_t));
    a->has_h = (unsigned char *)calloc(n, 1);
    a->has_e = (unsigned char *)calloc(n, 1);
    a->has_f = (unsigned char *)calloc(n, 1);
    a->live = (unsigned char *)calloc(n, 1);
    a->lo = 1;
    a->hi = 0;
    return a->h && a->e && a->f && a->has_h && a->has_e && a->has_f && a->live;
}

static void mx_diag_free(mx_diag_t *a)
{
    free(a->h); free(a->e); free(a->f);
    free(a->has_h); free(a->has_e); free(a->has_f); free(a->live);
}

static int mx_exists(const mx_diag_t *a, int64_t i)
{
    return i >= a->lo && i <= a->hi && a->live[i];
}

/* One extension of a[0..m-1] against b[0..n-1] (letter codes), matrix M
 * row-major K x K (M[x * K + y] scores letter x of a against y of b). */
int oracle_matrix_extend(const uint8_t *a, int64_t m, const uint8_t *b, int64_t n,
                         const int32_t *M, int64_t K, int64_t o, int64_t e, int64_t X,
                         mx_ext_t *out)
{
    mx_diag_t D[3];
    int ok = 1;
    for (int k = 0; k < 3; ++k) ok &= mx_diag_alloc(&D[k], m + 1);
    if (!ok) {
        for (int k = 0; k < 3; ++k) mx_diag_free(&D[k]);
        return MX_NOMEM;
    }
    D[0].h[0] = 0;
    D[0].has_h[0] = 1;
    D[0].live[0] = 1;
    D[0].lo = 0;
    D[0].hi = 0;
    int64_t best = 0, bi = 0, bj = 0, cells = 0;
    for (int64_t d = 1;; ++d) {
        mx_diag_t *cur = &D[d % 3], *p1 = &D[(d + 2) % 3], *p2 = &D[(d + 1) % 3];
        int64_t rlo = mx_max(p1->lo, d - n), rhi = mx_min(p1->hi + 1, m);
        if (rlo > rhi) break;
        int64_t thr = best - X;
        int any = 0;
        int64_t top = 0, top_i = 0, first = 0, last = 0;
        for (int64_t i = rlo; i <= rhi; ++i) {
            int64_t j = d - i, v;
            /* E from (i, j-1) on d-1 */
            int he = 0;
            int64_t ev = 0;
            if (j > 0 && mx_exists(p1, i)) {
                if (p1->has_e[i]) { ev = p1->e[i] + e; he = 1; }
                if (p1->has_h[i]) { v = p1->h[i] + o + e; ev = he ? mx_max(ev, v) : v; he = 1; }
            }
            /* F from (i-1, j) on d-1 */
            int hf = 0;
            int64_t fv = 0;
            if (i > 0 && mx_exists(p1, i - 1)) {
                if (p1->has_f[i - 1]) { fv = p1->f[i - 1] + e; hf = 1; }
                if (p1->has_h[i - 1]) { v = p1->h[i - 1] + o + e; fv = hf ? mx_max(fv, v) : v; hf = 1; }
            }
            /* H from (i-1, j-1) on d-2, or a gap state */
            int hh = 0;
            int64_t hv = 0;
            if (i > 0 && j > 0 && mx_exists(p2, i - 1) && p2->has_h[i - 1]) {
                hv = p2->h[i - 1] + M[(int64_t)a[i - 1] * K + b[j - 1]];
                hh = 1;
            }
            if (he) { hv = hh ? mx_max(hv, ev) : ev; hh = 1; }
            if (hf) { hv = hh ? mx_max(hv, fv) : fv; hh = 1; }
            int live = hh && !(hv < thr);
            cur->h[i] = hv; cur->e[i] = ev; cur->f[i] = fv;
            cur->has_h[i] = (unsigned char)(live && hh);
            cur->has_e[i] = (unsigned char)(live && he);
            cur->has_f[i] = (unsigned char)(live && hf);
            cur->live[i] = (unsigned char)live;
            if (live) {
                if (!any || hv > top) { top = hv; top_i = i; }
                if (!any) first = i;
                last = i;
                any = 1;
            }
        }
        cells += rhi - rlo + 1;
        if (!any) break;
        if (top > best) {
            best = top;
            bi = top_i;
            bj = d - top_i;
        }
        cur->lo = first;
        cur->hi = last;
    }
    out->best = best;
    out->bi = bi;
    out->bj = bj;
    out->cells = cells;
    for (int k = 0; k < 3; ++k) mx_diag_free(&D[k]);
    return MX_OK;
}

static int64_t mx_matrix_big(const int32_t *M, int64_t K)
{
    int64_t big = 0;
    for (int64_t t = 0; t < K * K; ++t) big = mx_max(big, mx_abs(M[t]));
    return big;
}

int oracle_matrix_params_valid(const int32_t *M, int64_t K, int64_t o, int64_t e, int64_t X)
{
    if (K < 1 || K > 32) return 0;
    if (mx_matrix_big(M, K) > 1000) return 0;
    if (o > 0 || e > 0 || o < -1000 || e < -1000) return 0;
    if (X < 0 || X > ((int64_t)1 << 29)) return 0;
    return 1;
}

int oracle_matrix_pair(const uint8_t *A, int64_t lenA, const uint8_t *B, int64_t lenB,
                       int64_t posA, int64_t posB, int64_t k, const int32_t *M, int64_t K,
                       int64_t o, int64_t e, int64_t X, mx_pair_t *r)
{
    memset(r, 0, sizeof(*r));
    r->status = MX_INVALID;
    if (!oracle_matrix_params_valid(M, K, o, e, X)) return MX_INVALID;
    if (lenA < 0 || lenB < 0 || lenA >= ((int64_t)1 << 31) || lenB >= ((int64_t)1 << 31))
        return MX_INVALID;
    if (k < 0 || posA < 0 || posB < 0 || posA + k > lenA || posB + k > lenB) return MX_INVALID;
    for (int64_t t = 0; t < lenA; ++t) if (A[t] >= K) return MX_INVALID;
    for (int64_t t = 0; t < lenB; ++t) if (B[t] >= K) return MX_INVALID;
    int64_t big = mx_max(mx_matrix_big(M, K), mx_abs(o) + mx_abs(e));
    if (big * (lenA + lenB) + X >= ((int64_t)1 << 29)) return MX_INVALID;

    int64_t seed = 0;
    for (int64_t t = 0; t < k; ++t) seed += M[(int64_t)A[posA + t] * K + B[posB + t]];

    mx_ext_t L, R;
    uint8_t *ra = (uint8_t *)malloc((size_t)posA + 1), *rb = (uint8_t *)malloc((size_t)posB + 1);
    if (!ra || !rb) { free(ra); free(rb); r->status = MX_NOMEM; return MX_NOMEM; }
    for (int64_t t = 0; t < posA; ++t) ra[t] = A[posA - 1 - t];
    for (int64_t t = 0; t < posB; ++t) rb[t] = B[posB - 1 - t];
    int e1 = oracle_matrix_extend(ra, posA, rb, posB, M, K, o, e, X, &L);
    free(ra); free(rb);
    int e2 = e1 ? e1 : oracle_matrix_extend(A + posA + k, lenA - posA - k, B + posB + k,
                                            lenB - posB - k, M, K, o, e, X, &R);
    if (e1 || e2) { r->status = MX_NOMEM; return MX_NOMEM; }
    r->left = L.best;
    r->right = R.best;
    r->score = L.best + seed + R.best;
    r->begA = posA - L.bi;
    r->begB = posB - L.bj;
    r->endA = posA + k + R.bi;
    r->endB = posB + k + R.bj;
    r->cells = L.cells + R.cells;
    r->status = MX_OK;
    return MX_OK;
}

typedef struct {
    const uint8_t *poolA, *poolB;
    const uint64_t *offA, *offB;
    const uint32_t *lenA, *lenB;
    uint32_t nA, nB;
    const uint32_t *seeds;
    const int32_t *Xs;
    const int32_t *M;
    int64_t K, o, e, X;
    int64_t n_pairs;
    mx_pair_t *out;
    int64_t next;
} mx_job_t;

static void *mx_worker(void *arg)
{
    mx_job_t *J = (mx_job_t *)arg;
    for (;;) {
        int64_t p = __atomic_fetch_add(&J->next, 1, __ATOMIC_RELAXED);
        if (p >= J->n_pairs) break;
        const uint32_t *s = J->seeds + 5 * p;
        mx_pair_t *r = J->out + p;
        if (s[0] >= J->nA || s[1] >= J->nB) {
            memset(r, 0, sizeof(*r));
            r->status = MX_INVALID;
            continue;
        }
        int64_t X = J->Xs ? (int64_t)J->Xs[p] : J->X;
        oracle_matrix_pair(J->poolA + J->offA[s[0]], J->lenA[s[0]], J->poolB + J->offB[s[1]],
                           J->lenB[s[1]], s[2], s[3], s[4], J->M, J->K, J->o, J->e, X, r);
    }
    return NULL;
}

/* Every pair over a thread pool; returns the number of threads used. */
int oracle_matrix_batch(const uint8_t *poolA, const uint64_t *offA, const uint32_t *lenA,
                        uint32_t nA, const uint8_t *poolB, const uint64_t *offB,
                        const uint32_t *lenB, uint32_t nB, const uint32_t *seeds, int64_t n_pairs,
                        const int32_t *M, int64_t K, int64_t o, int64_t e, int64_t X,
                        const int32_t *Xs, int nthreads, mx_pair_t *out)
{
    mx_job_t J;
    J.poolA = poolA; J.poolB = poolB; J.offA = offA; J.offB = offB;
    J.lenA = lenA; J.lenB = lenB; J.nA = nA; J.nB = nB; J.seeds = seeds; J.Xs = Xs;
    J.M = M; J.K = K; J.o = o; J.e = e; J.X = X;
    J.n_pairs = n_pairs; J.out = out; J.next = 0;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 1024) nthreads = 1024;
    pthread_t th[1024];
    int started = 0;
    for (int t = 1; t < nthreads; ++t)
        if (pthread_create(&th[started], NULL, mx_worker, &J) == 0) ++started;
    mx_worker(&J);
    for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
    return started + 1;
}
