/*
 * Affine-gap X-drop seed-extension oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * The paper's extension uses a linear gap score (Sec. III-A) and names
 * other scoring schemes as future work (Sec. VIII).  This file restates the
 * same X-drop extension for affine gaps: the three-state recurrence of
 * Gotoh (a gap of length L scores gap_open + L * gap_extend), with the
 * paper's anti-diagonal sweep, pruning rule and band trimming unchanged.
 * Only tests, the package's smoke check and the CPU baseline leg of the
 * benchmark may load it; the library never does.  It shares no code,
 * header, table or constant with the CUDA path (nor with xdrop_oracle.c).
 *
 * Recurrence (all terms that exist; a term whose predecessor does not exist
 * is absent; a state with no term is -infinity):
 *   E(i,j) = max(E(i,j-1) + e, H(i,j-1) + o + e)       gap in a (j advances)
 *   F(i,j) = max(F(i-1,j) + e, H(i-1,j) + o + e)       gap in b (i advances)
 *   H(i,j) = max(H(i-1,j-1) + (a_i == b_j ? match : mismatch), E(i,j), F(i,j))
 *   H(0,0) = 0, E(0,0) = F(0,0) = -infinity.
 * Readings (each is in the design notes; R-numbers are those of the linear
 * oracle, which carry over with "score" meaning H):
 *   A1  X-drop acts on H: a cell whose H < best - X is pruned, and all three
 *       of its states become -infinity (H >= E, F, so none of them could
 *       survive alone).
 *   A2  a predecessor (any of its states) exists only if its cell lies in
 *       the stored, trimmed range of its anti-diagonal and is live (R8);
 *       liveness and the range of the next anti-diagonal follow H.
 *   A3  best, its cell, the termination rule, the cells counted, the seed
 *       score and the combination of the two sides are those of the linear
 *       extension (R2-R5, R9-R13).
 *   Validation: |match|, |mismatch|, |gap_open|, |gap_extend| <= 1000,
 *   gap_open <= 0, gap_extend <= 0, mismatch <= match, 0 <= X <= 2^29, the
 *   seed inside both sequences, and
 *   max(|match|, |mismatch|, |gap_open| + |gap_extend|) * (m+n) + X < 2^29.
 *
 * Arithmetic is int64 with explicit existence flags per state.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

#define AFF_OK 0
#define AFF_INVALID 1
#define AFF_NOMEM 2

typedef struct {
    int64_t best, bi, bj, cells;
} aff_ext_t;

typedef struct {
    int64_t score, left, right;
    int64_t begA, begB, endA, endB;
    int64_t cells;
    int64_t status;
} aff_pair_t;

static int64_t amax(int64_t a, int64_t b) { return a > b ? a : b; }
static int64_t amin(int64_t a, int64_t b) { return a < b ? a : b; }
static int64_t aabs(int64_t x) { return x < 0 ? -x : x; }

/* one anti-diagonal: per row i the three states and whether each exists */
typedef struct {
    int64_t *h, *e, *f;
    unsigned char *hx, *ex, *fx;  /* state exists (is not -infinity) */
    unsigned char *live;
    int64_t lo, hi;               /* stored (trimmed) range; lo > hi: empty */
} antidiag_t;

static int ad_alloc(antidiag_t *a, int64_t rows)
{
    size_t n = (size_t)rows;
    a->h = (int64_t *)malloc(n * sizeof(int64_t));
    a->e = (int64_t *)malloc(n * sizeof(int64_t));
    a->f = (int64_t *)malloc(n * sizeof(int64_t));
    a->hx = (unsigned char *)calloc(n, 1);
    a->ex = (unsigned char *)calloc(n, 1);
    a->fx = (unsigned char *)calloc(n, 1);
    a->live = (unsigned char *)calloc(n, 1);
    a->lo = 1;
    a->hi = 0;
    return a->h && a->e && a->f && a->hx && a->ex && a->fx && a->live;
}

static void ad_free(antidiag_t *a)
{
    free(a->h); free(a->e); free(a->f);
    free(a->hx); free(a->ex); free(a->fx); free(a->live);
}

/* cell i of anti-diagonal a exists as a predecessor (A2) */
static int ad_has(const antidiag_t *a, int64_t i)
{
    return i >= a->lo && i <= a->hi && a->live[i];
}

int oracle_affine_extend(const uint8_t *a, int64_t m, const uint8_t *b, int64_t n,
                         int64_t match, int64_t mismatch, int64_t go, int64_t ge, int64_t X,
                         aff_ext_t *out)
{
    antidiag_t D[3];
    int k, ok = 1;
    for (k = 0; k < 3; ++k) ok &= ad_alloc(&D[k], m + 1);
    if (!ok) {
        for (k = 0; k < 3; ++k) ad_free(&D[k]);
        return AFF_NOMEM;
    }
    /* d = 0: cell (0,0), H = 0, no gap state */
    D[0].h[0] = 0; D[0].hx[0] = 1; D[0].ex[0] = 0; D[0].fx[0] = 0;
    D[0].live[0] = 1;
    D[0].lo = 0; D[0].hi = 0;
    /* d = -1 (slot 2): empty */
    D[2].lo = 1; D[2].hi = 0;

    int64_t best = 0, bi = 0, bj = 0, cells = 0;
    for (int64_t d = 1;; ++d) {
        antidiag_t *cur = &D[d % 3], *p1 = &D[(d - 1) % 3], *p2 = &D[(d + 1) % 3];
        int64_t rlo = amax(p1->lo, d - n);
        int64_t rhi = amin(p1->hi + 1, m);
        if (rlo > rhi) break;
        int64_t thr = best - X;
        int any = 0;
        int64_t dmax = 0, dmax_i = 0, first = 0, last = 0;
        for (int64_t i = rlo; i <= rhi; ++i) {
            int64_t j = d - i, t;
            /* E: from (i, j-1) on d-1 */
            int ex = 0;
            int64_t ev = 0;
            if (j > 0 && ad_has(p1, i)) {
                if (p1->ex[i]) { ev = p1->e[i] + ge; ex = 1; }
                if (p1->hx[i]) {
                    t = p1->h[i] + go + ge;
                    ev = ex ? amax(ev, t) : t;
                    ex = 1;
                }
            }
            /* F: from (i-1, j) on d-1 */
            int fx = 0;
            int64_t fv = 0;
            if (i > 0 && ad_has(p1, i - 1)) {
                if (p1->fx[i - 1]) { fv = p1->f[i - 1] + ge; fx = 1; }
                if (p1->hx[i - 1]) {
                    t = p1->h[i - 1] + go + ge;
                    fv = fx ? amax(fv, t) : t;
                    fx = 1;
                }
            }
            /* H: diagonal from (i-1, j-1) on d-2, or a gap state */
            int hx = 0;
            int64_t hv = 0;
            if (i > 0 && j > 0 && ad_has(p2, i - 1) && p2->hx[i - 1]) {
                hv = p2->h[i - 1] + (a[i - 1] == b[j - 1] ? match : mismatch);
                hx = 1;
            }
            if (ex) { hv = hx ? amax(hv, ev) : ev; hx = 1; }
            if (fx) { hv = hx ? amax(hv, fv) : fv; hx = 1; }
            int is_live = hx && !(hv < thr);     /* A1, strict as R5 */
            cur->h[i] = hv; cur->e[i] = ev; cur->f[i] = fv;
            cur->hx[i] = (unsigned char)(is_live && hx);
            cur->ex[i] = (unsigned char)(is_live && ex);
            cur->fx[i] = (unsigned char)(is_live && fx);
            cur->live[i] = (unsigned char)is_live;
            if (is_live) {
                if (!any || hv > dmax) { dmax = hv; dmax_i = i; }
                if (!any) first = i;
                last = i;
                any = 1;
            }
        }
        cells += rhi - rlo + 1;
        if (!any) break;
        if (dmax > best) {
            best = dmax;
            bi = dmax_i;
            bj = d - dmax_i;
        }
        cur->lo = first;
        cur->hi = last;
    }
    out->best = best;
    out->bi = bi;
    out->bj = bj;
    out->cells = cells;
    for (k = 0; k < 3; ++k) ad_free(&D[k]);
    return AFF_OK;
}

int oracle_affine_params_valid(int64_t match, int64_t mismatch, int64_t go, int64_t ge,
                               int64_t X)
{
    if (aabs(match) > 1000 || aabs(mismatch) > 1000 || aabs(go) > 1000 || aabs(ge) > 1000)
        return 0;
    if (go > 0 || ge > 0 || mismatch > match) return 0;
    if (X < 0 || X > ((int64_t)1 << 29)) return 0;
    return 1;
}

static int is_acgt(uint8_t c) { return c == 'A' || c == 'C' || c == 'G' || c == 'T'; }

/* one seeded pair, split and combined as the linear extension (A3) */
int oracle_affine_pair(const uint8_t *A, int64_t lenA, const uint8_t *B, int64_t lenB,
                       int64_t posA, int64_t posB, int64_t k, int64_t match, int64_t mismatch,
                       int64_t go, int64_t ge, int64_t X, aff_pair_t *r)
{
    memset(r, 0, sizeof(*r));
    r->status = AFF_INVALID;
    if (!oracle_affine_params_valid(match, mismatch, go, ge, X)) return AFF_INVALID;
    if (lenA < 0 || lenB < 0 || lenA >= ((int64_t)1 << 31) || lenB >= ((int64_t)1 << 31))
        return AFF_INVALID;
    if (k < 0 || posA < 0 || posB < 0 || posA + k > lenA || posB + k > lenB) return AFF_INVALID;
    for (int64_t t = 0; t < lenA; ++t) if (!is_acgt(A[t])) return AFF_INVALID;
    for (int64_t t = 0; t < lenB; ++t) if (!is_acgt(B[t])) return AFF_INVALID;
    int64_t big = amax(aabs(match), amax(aabs(mismatch), aabs(go) + aabs(ge)));
    if (big * (lenA + lenB) + X >= ((int64_t)1 << 29)) return AFF_INVALID;

    int64_t seed = 0;
    for (int64_t t = 0; t < k; ++t) seed += (A[posA + t] == B[posB + t]) ? match : mismatch;

    aff_ext_t L, R;
    uint8_t *ra = (uint8_t *)malloc((size_t)posA + 1), *rb = (uint8_t *)malloc((size_t)posB + 1);
    if (!ra || !rb) { free(ra); free(rb); r->status = AFF_NOMEM; return AFF_NOMEM; }
    for (int64_t t = 0; t < posA; ++t) ra[t] = A[posA - 1 - t];
    for (int64_t t = 0; t < posB; ++t) rb[t] = B[posB - 1 - t];
    int e1 = oracle_affine_extend(ra, posA, rb, posB, match, mismatch, go, ge, X, &L);
    free(ra); free(rb);
    int e2 = e1 ? e1 : oracle_affine_extend(A + posA + k, lenA - posA - k, B + posB + k,
                                            lenB - posB - k, match, mismatch, go, ge, X, &R);
    if (e1 || e2) { r->status = AFF_NOMEM; return AFF_NOMEM; }
    r->left = L.best;
    r->right = R.best;
    r->score = L.best + seed + R.best;
    r->begA = posA - L.bi;
    r->begB = posB - L.bj;
    r->endA = posA + k + R.bi;
    r->endB = posB + k + R.bj;
    r->cells = L.cells + R.cells;
    r->status = AFF_OK;
    return AFF_OK;
}

typedef struct {
    const uint8_t *poolA, *poolB;
    const uint64_t *offA, *offB;
    const uint32_t *lenA, *lenB;
    uint32_t nA, nB;
    const uint32_t *seeds;
    const int32_t *Xs;
    int64_t match, mismatch, go, ge, X;
    int64_t n_pairs;
    aff_pair_t *out;
    int64_t next;
} aff_job_t;

static void *aff_worker(void *arg)
{
    aff_job_t *J = (aff_job_t *)arg;
    for (;;) {
        int64_t p = __atomic_fetch_add(&J->next, 1, __ATOMIC_RELAXED);
        if (p >= J->n_pairs) break;
        const uint32_t *s = J->seeds + 5 * p;
        aff_pair_t *r = J->out + p;
        if (s[0] >= J->nA || s[1] >= J->nB) {
            memset(r, 0, sizeof(*r));
            r->status = AFF_INVALID;
            continue;
        }
        int64_t X = J->Xs ? (int64_t)J->Xs[p] : J->X;
        oracle_affine_pair(J->poolA + J->offA[s[0]], J->lenA[s[0]], J->poolB + J->offB[s[1]],
                           J->lenB[s[1]], s[2], s[3], s[4], J->match, J->mismatch, J->go, J->ge,
                           X, r);
    }
    return NULL;
}

int oracle_affine_batch(const uint8_t *poolA, const uint64_t *offA, const uint32_t *lenA,
                        uint32_t nA, const uint8_t *poolB, const uint64_t *offB,
                        const uint32_t *lenB, uint32_t nB, const uint32_t *seeds, int64_t n_pairs,
                        int64_t match, int64_t mismatch, int64_t go, int64_t ge, int64_t X,
                        const int32_t *Xs, int nthreads, aff_pair_t *out)
{
    aff_job_t J;
    J.poolA = poolA; J.poolB = poolB; J.offA = offA; J.offB = offB;
    J.lenA = lenA; J.lenB = lenB; J.nA = nA; J.nB = nB; J.seeds = seeds; J.Xs = Xs;
    J.match = match; J.mismatch = mismatch; J.go = go; J.ge = ge; J.X = X;
    J.n_pairs = n_pairs; J.out = out; J.next = 0;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 1024) nthreads = 1024;
    pthread_t th[1024];
    int started = 0;
    for (int t = 1; t < nthreads; ++t)
        if (pthread_create(&th[started], NULL, aff_worker, &J) == 0) ++started;
    aff_worker(&J);
    for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
    return started + 1;
}
