/*
 * X-drop seed-extension oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, obviously correct CPU restatement of the method of LOGAN
 * (Zeni et al., "LOGAN: High-Performance GPU-Based X-Drop Long-Read
 * Alignment").  Only tests, the package's smoke check and the CPU baseline
 * leg of the benchmark may load it; the library never does.  It shares no
 * code, header, table or constant with the CUDA path.
 *
 * Passages followed (section / equation / algorithm of the paper):
 *   - Sec. III-A, problem statement: best semi-global extension score over
 *     prefixes a_1..a_i and b_1..b_j.
 *   - Sec. III-A, cell recurrence: S(i,j) is the max of the diagonal
 *     predecessor plus match/mismatch (i>0, j>0) and the horizontal/vertical
 *     predecessors plus the gap score (j>0 / i>0).  Scores are signed values
 *     that are ADDED (match > 0, mismatch and gap <= 0).
 *   - Sec. III-A, X-drop rule: a cell whose score is below sigma - X, sigma
 *     the best score seen so far, becomes -infinity and is not used again;
 *     the -infinity cells at the ends of an anti-diagonal bound the next one.
 *   - Algorithm 1: anti-diagonal sweep with three rolling anti-diagonals,
 *     best initialised to 0, loop while the current anti-diagonal is not
 *     empty, return the best score.
 *   - Algorithm 2: per-cell update of one anti-diagonal.
 *   - Sec. IV-A: best is updated only after a whole anti-diagonal is done.
 *   - Sec. IV-B: each pair is split at the seed into a left and a right
 *     extension; the left one reads both sequences backwards.
 *
 * Readings where the paper is silent or garbled (each is in the design notes):
 *   R1  boundary cells S(i,0), S(0,j) are ordinary cells of the recurrence
 *       (only the vertical / horizontal term exists); X-drop applies to them.
 *   R2  best starts at 0 at cell (0,0); the empty extension is allowed.
 *   R3  best <- max(best, max over live cells of the anti-diagonal).
 *   R4  anti-diagonal d is pruned against best over anti-diagonals < d.
 *   R5  pruning is strict: S < best - X is dropped; S == best - X survives.
 *   R6  buffers rotate (d-2 <- d-1 <- d).
 *   R8  range of d: [max(lo', d-n), min(hi'+1, m)] where [lo', hi'] is the
 *       trimmed live range of d-1 (first..last live cell).  A predecessor
 *       outside the stored (trimmed) range of its anti-diagonal, or -inf,
 *       does not exist.  A cell with no existing predecessor is -inf.
 *   R9  the sweep runs over the whole (m+1)x(n+1) matrix and stops when an
 *       anti-diagonal has no live cell or its range is empty.
 *   R10 the best cell is the first anti-diagonal reaching the best score
 *       (strict improvement), smallest i on it.
 *   R11 result = left best + seed score + right best, with begin/end
 *       coordinates in the original sequences.
 *   R12 seed score = sum over the k seed columns of match/mismatch.
 *   R13 computed cells = every cell of every evaluated range for d >= 1,
 *       the pruned ones and the last (all pruned) anti-diagonal included.
 *   R14 a base outside A,C,G,T makes the pair invalid.
 *   Validation: |match|,|mismatch|,|gap| <= 1000, gap <= 0, mismatch <= match,
 *   0 <= X <= 2^29, seed inside both sequences, and
 *   max(|match|,|mismatch|,|gap|) * (m+n) + X < 2^29 for each pair.
 *
 * Arithmetic is int64 with explicit existence flags, independent of any
 * sentinel encoding of -infinity.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

#define ORACLE_OK 0
#define ORACLE_INVALID 1
#define ORACLE_NOMEM 2

typedef struct {
    int64_t best;   /* best extension score (>= 0) */
    int64_t bi;     /* cells of a consumed at the best cell */
    int64_t bj;     /* cells of b consumed at the best cell */
    int64_t cells;  /* computed cells (R13) */
} oracle_ext_t;

typedef struct {
    int64_t score, left, right;
    int64_t begA, begB, endA, endB;
    int64_t cells;
    int64_t status;
} oracle_pair_t;

static int64_t max64(int64_t a, int64_t b) { return a > b ? a : b; }
static int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }

static int is_base(uint8_t c) { return c == 'A' || c == 'C' || c == 'G' || c == 'T'; }

/*
 * One X-drop extension of a[0..m-1] against b[0..n-1] (Algorithm 1 with the
 * cell update of Algorithm 2 and the recurrence of Sec. III-A).
 * Anti-diagonal d holds cells (i, d-i); arrays are indexed by i.
 */
int oracle_xdrop_extend(const uint8_t *a, int64_t m, const uint8_t *b, int64_t n,
                        int64_t match, int64_t mismatch, int64_t gap, int64_t X,
                        oracle_ext_t *out)
{
    int64_t *val[3];
    unsigned char *live[3];
    int64_t lo[3], hi[3];
    int k;
    for (k = 0; k < 3; ++k) {
        val[k] = (int64_t *)malloc((size_t)(m + 1) * sizeof(int64_t));
        live[k] = (unsigned char *)calloc((size_t)(m + 1), 1);
        if (!val[k] || !live[k]) {
            for (; k >= 0; --k) { free(val[k]); free(live[k]); }
            return ORACLE_NOMEM;
        }
    }
    /* d = 0: the single cell (0,0) with score 0 (R2) */
    val[0][0] = 0;
    live[0][0] = 1;
    lo[0] = 0; hi[0] = 0;
    /* d = -1 (slot 2): empty range */
    lo[2] = 1; hi[2] = 0;

    int64_t best = 0, bi = 0, bj = 0, cells = 0;
    for (int64_t d = 1;; ++d) {
        int cur = (int)(d % 3), p1 = (int)((d - 1) % 3), p2 = (int)((d + 1) % 3);
        int64_t rlo = max64(lo[p1], d - n);       /* R8 */
        int64_t rhi = min64(hi[p1] + 1, m);
        if (rlo > rhi) break;                      /* R9: empty range */
        int64_t thr = best - X;                    /* R4: best over d' < d */
        int any = 0;
        int64_t dmax = 0, dmax_i = 0, first = 0, last = 0;
        for (int64_t i = rlo; i <= rhi; ++i) {
            int64_t j = d - i;
            int have = 0;
            int64_t s = 0, t;
            /* diagonal: S(i-1, j-1) on d-2, plus match / mismatch */
            if (i > 0 && j > 0 && i - 1 >= lo[p2] && i - 1 <= hi[p2] && live[p2][i - 1]) {
                s = val[p2][i - 1] + (a[i - 1] == b[j - 1] ? match : mismatch);
                have = 1;
            }
            /* vertical: S(i-1, j) on d-1, plus gap */
            if (i > 0 && i - 1 >= lo[p1] && i - 1 <= hi[p1] && live[p1][i - 1]) {
                t = val[p1][i - 1] + gap;
                s = have ? max64(s, t) : t;
                have = 1;
            }
            /* horizontal: S(i, j-1) on d-1, plus gap */
            if (j > 0 && i >= lo[p1] && i <= hi[p1] && live[p1][i]) {
                t = val[p1][i] + gap;
                s = have ? max64(s, t) : t;
                have = 1;
            }
            int is_live = have && !(s < thr);      /* R5 */
            val[cur][i] = s;
            live[cur][i] = (unsigned char)is_live;
            if (is_live) {
                if (!any || s > dmax) { dmax = s; dmax_i = i; }  /* R10 */
                if (!any) first = i;
                last = i;
                any = 1;
            }
        }
        cells += rhi - rlo + 1;                    /* R13 */
        if (!any) break;                           /* R9 */
        if (dmax > best) {                         /* R3, R10 */
            best = dmax;
            bi = dmax_i;
            bj = d - dmax_i;
        }
        lo[cur] = first;                           /* trim both ends */
        hi[cur] = last;
    }
    out->best = best;
    out->bi = bi;
    out->bj = bj;
    out->cells = cells;
    for (k = 0; k < 3; ++k) { free(val[k]); free(live[k]); }
    return ORACLE_OK;
}

static int64_t iabs64(int64_t x) { return x < 0 ? -x : x; }

int oracle_params_valid(int64_t match, int64_t mismatch, int64_t gap, int64_t X)
{
    if (iabs64(match) > 1000 || iabs64(mismatch) > 1000 || iabs64(gap) > 1000) return 0;
    if (gap > 0 || mismatch > match) return 0;
    if (X < 0 || X > ((int64_t)1 << 29)) return 0;
    return 1;
}

/*
 * One seeded pair (Sec. IV-B): right extension on A[posA+k..], B[posB+k..];
 * left extension on the reversed prefixes A[..posA-1], B[..posB-1]; the seed
 * columns in between score match/mismatch (R12); combined per R11.
 */
int oracle_pair(const uint8_t *A, int64_t lenA, const uint8_t *B, int64_t lenB,
                int64_t posA, int64_t posB, int64_t k,
                int64_t match, int64_t mismatch, int64_t gap, int64_t X,
                oracle_pair_t *r)
{
    memset(r, 0, sizeof(*r));
    r->status = ORACLE_INVALID;
    if (!oracle_params_valid(match, mismatch, gap, X)) return ORACLE_INVALID;
    if (lenA < 0 || lenB < 0 || lenA >= ((int64_t)1 << 31) || lenB >= ((int64_t)1 << 31))
        return ORACLE_INVALID;
    if (k < 0 || posA < 0 || posB < 0 || posA + k > lenA || posB + k > lenB) return ORACLE_INVALID;
    for (int64_t t = 0; t < lenA; ++t) if (!is_base(A[t])) return ORACLE_INVALID;
    for (int64_t t = 0; t < lenB; ++t) if (!is_base(B[t])) return ORACLE_INVALID;
    int64_t big = iabs64(match);
    if (iabs64(mismatch) > big) big = iabs64(mismatch);
    if (iabs64(gap) > big) big = iabs64(gap);
    if (big * (lenA + lenB) + X >= ((int64_t)1 << 29)) return ORACLE_INVALID;

    int64_t seed = 0;
    for (int64_t t = 0; t < k; ++t) seed += (A[posA + t] == B[posB + t]) ? match : mismatch;

    oracle_ext_t L, R;
    /* left: reversed prefixes */
    uint8_t *ra = (uint8_t *)malloc((size_t)posA + 1), *rb = (uint8_t *)malloc((size_t)posB + 1);
    if (!ra || !rb) { free(ra); free(rb); r->status = ORACLE_NOMEM; return ORACLE_NOMEM; }
    for (int64_t t = 0; t < posA; ++t) ra[t] = A[posA - 1 - t];
    for (int64_t t = 0; t < posB; ++t) rb[t] = B[posB - 1 - t];
    int e1 = oracle_xdrop_extend(ra, posA, rb, posB, match, mismatch, gap, X, &L);
    free(ra); free(rb);
    int e2 = e1 ? e1 : oracle_xdrop_extend(A + posA + k, lenA - posA - k, B + posB + k,
                                           lenB - posB - k, match, mismatch, gap, X, &R);
    if (e1 || e2) { r->status = ORACLE_NOMEM; return ORACLE_NOMEM; }

    r->left = L.best;
    r->right = R.best;
    r->score = L.best + seed + R.best;
    r->begA = posA - L.bi;
    r->begB = posB - L.bj;
    r->endA = posA + k + R.bi;
    r->endB = posB + k + R.bj;
    r->cells = L.cells + R.cells;
    r->status = ORACLE_OK;
    return ORACLE_OK;
}

/* ---- batch over a thread pool (each pair single-threaded) ---- */

typedef struct {
    const uint8_t *poolA, *poolB;
    const uint64_t *offA, *offB;
    const uint32_t *lenA, *lenB;
    uint32_t nA, nB;
    const uint32_t *seeds;   /* 5 x uint32 per pair: idxA idxB posA posB len */
    const int32_t *Xs;       /* nullable */
    int64_t match, mismatch, gap, X;
    int64_t n_pairs;
    oracle_pair_t *out;
    int64_t next;            /* shared work counter */
} batch_job_t;

static void *batch_worker(void *arg)
{
    batch_job_t *J = (batch_job_t *)arg;
    for (;;) {
        int64_t p = __atomic_fetch_add(&J->next, 1, __ATOMIC_RELAXED);
        if (p >= J->n_pairs) break;
        const uint32_t *s = J->seeds + 5 * p;
        oracle_pair_t *r = J->out + p;
        if (s[0] >= J->nA || s[1] >= J->nB) {
            memset(r, 0, sizeof(*r));
            r->status = ORACLE_INVALID;
            continue;
        }
        int64_t X = J->Xs ? (int64_t)J->Xs[p] : J->X;
        oracle_pair(J->poolA + J->offA[s[0]], J->lenA[s[0]], J->poolB + J->offB[s[1]],
                    J->lenB[s[1]], s[2], s[3], s[4], J->match, J->mismatch, J->gap, X, r);
    }
    return NULL;
}

/* Runs every pair; returns the number of threads used. */
int oracle_batch(const uint8_t *poolA, const uint64_t *offA, const uint32_t *lenA, uint32_t nA,
                 const uint8_t *poolB, const uint64_t *offB, const uint32_t *lenB, uint32_t nB,
                 const uint32_t *seeds, int64_t n_pairs, int64_t match, int64_t mismatch,
                 int64_t gap, int64_t X, const int32_t *Xs, int nthreads, oracle_pair_t *out)
{
    batch_job_t J;
    J.poolA = poolA; J.poolB = poolB; J.offA = offA; J.offB = offB;
    J.lenA = lenA; J.lenB = lenB; J.nA = nA; J.nB = nB; J.seeds = seeds; J.Xs = Xs;
    J.match = match; J.mismatch = mismatch; J.gap = gap; J.X = X;
    J.n_pairs = n_pairs; J.out = out; J.next = 0;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 1024) nthreads = 1024;
    pthread_t th[1024];
    int started = 0;
    for (int t = 1; t < nthreads; ++t)
        if (pthread_create(&th[started], NULL, batch_worker, &J) == 0) ++started;
    batch_worker(&J);
    for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
    return started + 1;
}
