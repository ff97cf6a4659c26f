// X-drop extension scored by a substitution matrix with affine gaps, one
// block per extension, band state in a device-memory ring.
//
// The paper's anti-diagonal sweep, X-drop rule and band trimming (Sec. III-A,
// Algorithms 1 and 2), with Gotoh's three states per cell and a K x K
// substitution matrix instead of match / mismatch (protein and other
// scoring schemes are the paper's future work, Sec. VIII):
//   E(i,j) = max(E(i,j-1) + e, H(i,j-1) + o + e)
//   F(i,j) = max(F(i-1,j) + e, H(i-1,j) + o + e)
//   H(i,j) = max(H(i-1,j-1) + M[a_i][b_j], E(i,j), F(i,j))
// A cell whose H < best - X is pruned with all three states.
//
// Layout: like the paper's V100 kernel (Sec. IV-B), the anti-diagonals live
// in device memory: each resident block owns a ring slot of six arrays of
// `cap` cells indexed by row i modulo cap -- H on d-2, d-1, d; E (updated in
// place: E(i, .) is read and written only by row i's cell); F on d-1 and d
// (F(i,j) reads row i-1).  256 threads sweep an anti-diagonal in strides;
// a block reduction gives the anti-diagonal's best H (smallest row on
// ties) and its first and last live rows; its barriers publish the writes.
// A band wider than cap - 2 rows ends the extension with LOGAN_ERANGE.
//
// Two users:
//  * logan_extend_batch_matrix: sequences of letter codes (one byte each,
//    values < K), any K <= 32; every extension runs here.
//  * the affine DNA path (logan_extend_batch_affine): its register windows
//    end at 512 rows; a band that outgrows them, or an X too large for their
//    keys, continues here on the 2-bit pools with the 4 x 4 match / mismatch
//    table, instead of ending with LOGAN_ERANGE.
#include <algorithm>
#include <climits>

#include "internal.h"
#include "../../include/logan.h"

namespace logan {

namespace {

constexpr uint32_t FULL = 0xffffffffu;
constexpr int kMxThreads = 256;
constexpr int kMxWarps = kMxThreads / 32;
constexpr int NEGM = -(1 << 30);  // -inf of the absolute scores
constexpr int kMaxK = 32;

struct MxRed {
    int mx, arg, first, last;
};

// max H, the smallest row reaching it, first and last live row over the
// block; every thread gets the result
__device__ __forceinline__ MxRed mx_block_reduce(MxRed v, MxRed* sh) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int mx = __reduce_max_sync(FULL, v.mx);
    int arg = __reduce_min_sync(FULL, v.mx == mx ? v.arg : INT_MAX);
    int first = __reduce_min_sync(FULL, v.first);
    int last = __reduce_max_sync(FULL, v.last);
    if (lane == 0) sh[w] = MxRed{mx, arg, first, last};
    __syncthreads();
    const MxRed p = lane < kMxWarps ? sh[lane] : MxRed{NEGM, INT_MAX, INT_MAX, -1};
    mx = __reduce_max_sync(FULL, p.mx);
    arg = __reduce_min_sync(FULL, p.mx == mx ? p.arg : INT_MAX);
    first = __reduce_min_sync(FULL, p.first);
    last = __reduce_max_sync(FULL, p.last);
    __syncthreads();  // sh is reused by the next anti-diagonal
    return MxRed{mx, arg, first, last};
}

// letter code of stream index q of an operand (2-bit words or bytes); the
// caller keeps q inside [0, len)
template <bool BYTES>
__device__ __forceinline__ uint32_t mx_code(const void* pool, int64_t pos, int dir, int64_t q) {
    const int64_t p = pos + (dir > 0 ? q : -q);
    if constexpr (BYTES) return static_cast<const uint8_t*>(pool)[p];
    else return code_at(static_cast<const uint32_t*>(pool), p);
}

struct MxArgs {
    const void* pa;  // pool of A: 2-bit words, or letter codes (bytes)
    const void* pb;
    const Item* items;
    ExtRes* ext;
    const uint32_t* queue;
    Counters* counters;
    int q;  // queue index in counters (every entry [0, tail) is taken)
    const int32_t* table;  // K x K, row = letter of a; nullptr: match / mismatch
    int K;
    int match, mismatch;
    int go, ge;
    int32_t* ring;  // per block: 6 * cap cells
    uint32_t cap;   // power of two
    int cells_level;  // counters->cells index credited with the cells
};

template <bool BYTES>
__device__ void mx_extend(const MxArgs& a, const Item& it, int32_t* R, const int* tab, ExtRes& r,
                          MxRed* sh) {
    const int dir = (it.flags & ITEM_LEFT) ? -1 : 1;
    const int m = int(it.m), n = int(it.n), X = it.X;
    const int mask = int(a.cap) - 1;
    int32_t* H0 = R;                 // d
    int32_t* H1 = R + a.cap;         // d-1
    int32_t* H2 = R + 2 * a.cap;     // d-2
    int32_t* E = R + 3 * a.cap;      // E on d-1, replaced by d
    int32_t* F1 = R + 4 * a.cap;     // F on d-1
    int32_t* F0 = R + 5 * a.cap;     // F on d
    if (threadIdx.x == 0) {
        H1[0] = 0;  // cell (0,0); it has no gap state
        E[0] = NEGM;
        F1[0] = NEGM;
    }
    __syncthreads();
    int lo1 = 0, hi1 = 0, lo2 = 1, hi2 = 0;
    int best = 0, bi = 0, bj = 0, status = 0;
    unsigned long long cells = 0ull;
    const int goe = a.go + a.ge;
    for (int d = 1;; ++d) {
        const int rlo = max(lo1, d - n), rhi = min(hi1 + 1, m);
        if (rlo > rhi) break;
        if (rhi - rlo + 2 > int(a.cap)) {
            status = LOGAN_ERANGE;
            break;
        }
        cells += (unsigned long long)(rhi - rlo + 1);
        const int T = best - X;
        MxRed v{NEGM, INT_MAX, INT_MAX, -1};
        for (int i = rlo + int(threadIdx.x); i <= rhi; i += kMxThreads) {
            const int j = d - i;
            const bool up = i > 0 && i - 1 >= lo1 && i - 1 <= hi1;
            const bool lf = j > 0 && i >= lo1 && i <= hi1;
            const bool dg = i > 0 && j > 0 && i - 1 >= lo2 && i - 1 <= hi2;
            const int hU = up ? H1[(i - 1) & mask] : NEGM;
            const int fU = up ? F1[(i - 1) & mask] : NEGM;
            const int hL = lf ? H1[i & mask] : NEGM;
            const int eL = lf ? E[i & mask] : NEGM;
            const int e = max(max(eL + a.ge, hL + goe), NEGM);
            const int f = max(max(fU + a.ge, hU + goe), NEGM);
            int h = max(e, f);
            if (dg) {
                const uint32_t ca = mx_code<BYTES>(a.pa, it.a_pos, dir, i - 1);
                const uint32_t cb = mx_code<BYTES>(a.pb, it.b_pos, dir, j - 1);
                h = max(h, H2[(i - 1) & mask] + tab[ca * uint32_t(a.K) + cb]);
            }
            const bool live = h >= T;
            H0[i & mask] = live ? h : NEGM;
            E[i & mask] = live ? e : NEGM;
            F0[i & mask] = live ? f : NEGM;
            if (live) {
                if (h > v.mx) {
                    v.mx = h;
                    v.arg = i;
                }
                v.first = min(v.first, i);
                v.last = i;
            }
        }
        const MxRed b = mx_block_reduce(v, sh);  // its barriers also publish the writes
        if (b.last < 0) break;
        if (b.mx > best) {
            best = b.mx;
            bi = b.arg;
            bj = d - b.arg;
        }
        lo2 = lo1;
        hi2 = hi1;
        lo1 = b.first;
        hi1 = b.last;
        int32_t* t = H2;
        H2 = H1;
        H1 = H0;
        H0 = t;
        t = F1;
        F1 = F0;
        F0 = t;
    }
    r.best = status ? 0 : best;
    r.bi = status ? 0 : bi;
    r.bj = status ? 0 : bj;
    r.status = status;
    r.cells = status ? 0ull : cells;
}

template <bool BYTES>
__global__ void __launch_bounds__(kMxThreads) k_mx_ring(MxArgs a) {
    __shared__ MxRed sh[kMxWarps];
    __shared__ int tab[kMaxK * kMaxK];
    __shared__ unsigned int s_slot;
    for (int t = threadIdx.x; t < a.K * a.K; t += kMxThreads)
        tab[t] = a.table ? a.table[t] : (t / a.K == t % a.K ? a.match : a.mismatch);
    int32_t* R = a.ring + size_t(blockIdx.x) * 6u * a.cap;
    for (;;) {
        if (threadIdx.x == 0) {
            const unsigned int s = atomicAdd(&a.counters->head[a.q], 1u);
            s_slot = s < a.counters->tail[a.q] ? s : ~0u;
        }
        __syncthreads();
        const unsigned int slot = s_slot;
        __syncthreads();
        if (slot == ~0u) break;
        const uint32_t id = a.queue[slot];
        const Item it = a.items[id];
        ExtRes r;
        mx_extend<BYTES>(a, it, R, tab, r, sh);
        if (threadIdx.x == 0) {
            a.ext[id] = r;
            atomicAdd(&a.counters->cells[a.cells_level], r.cells);
        }
        __syncthreads();
    }
}

// ---- the matrix call's own pre-processing ----

// per sequence: 1 if a letter code is >= K
__global__ void k_mx_validate(const uint8_t* __restrict__ pool, const uint64_t* __restrict__ off,
                              const uint32_t* __restrict__ len, uint32_t count, int K,
                              uint8_t* __restrict__ bad) {
    const uint32_t s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (s >= count) return;
    const uint8_t* p = pool + off[s];
    const uint32_t n = len[s];
    bool any = false;
    for (uint32_t t = lane; t < n; t += 32) any |= p[t] >= uint32_t(K);
    any = __any_sync(FULL, any);
    if (lane == 0) bad[s] = any ? 1 : 0;
}

struct MxPool {
    const uint8_t* bases;
    const uint64_t* off;
    const uint32_t* len;
    uint32_t count;
    const uint8_t* bad;
};

// items, seed score and per-pair status of every pair; runnable items are
// appended to queue 0
__global__ void k_mx_split(MxPool A, MxPool B, const uint32_t* __restrict__ seeds, uint32_t n_pairs,
                           const int32_t* __restrict__ table, int K, int64_t big, int32_t X,
                           const int32_t* __restrict__ Xs, Item* items, PairInfo* info, ExtRes* ext,
                           uint32_t* queue, Counters* counters) {
    const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_pairs) return;
    const uint32_t ia = seeds[5 * p], ib = seeds[5 * p + 1];
    const uint32_t posA = seeds[5 * p + 2], posB = seeds[5 * p + 3], k = seeds[5 * p + 4];
    const int32_t x = Xs ? Xs[p] : X;
    bool ok = ia < A.count && ib < B.count && x >= 0 && x <= kMaxX;
    uint32_t lenA = 0, lenB = 0;
    if (ok) {
        lenA = A.len[ia];
        lenB = B.len[ib];
        ok = !A.bad[ia] && !B.bad[ib] && lenA < (1u << 31) && lenB < (1u << 31) &&
             uint64_t(posA) + k <= lenA && uint64_t(posB) + k <= lenB &&
             big * (int64_t(lenA) + lenB) + x < kScoreRange;
    }
    const ExtRes zero = {0, 0, 0, 0, 0ull};
    ext[2 * p] = zero;
    ext[2 * p + 1] = zero;
    if (!ok) {
        const Item it = {0, 0, 0u, 0u, 0, ITEM_SKIP};
        items[2 * p] = it;
        items[2 * p + 1] = it;
        info[p] = PairInfo{0, LOGAN_EINVAL};
        return;
    }
    const int64_t offA = int64_t(A.off[ia]), offB = int64_t(B.off[ib]);
    int32_t seed = 0;
    for (uint32_t t = 0; t < k; ++t)
        seed += table[uint32_t(A.bases[offA + posA + t]) * uint32_t(K) + B.bases[offB + posB + t]];
    Item L, R;
    L.a_pos = offA + int64_t(posA) - 1;
    L.b_pos = offB + int64_t(posB) - 1;
    L.m = posA;
    L.n = posB;
    L.X = x;
    L.flags = ITEM_LEFT | ((posA == 0 && posB == 0) ? ITEM_SKIP : 0u);
    R.a_pos = offA + int64_t(posA) + k;
    R.b_pos = offB + int64_t(posB) + k;
    R.m = lenA - posA - k;
    R.n = lenB - posB - k;
    R.X = x;
    R.flags = (R.m == 0 && R.n == 0) ? ITEM_SKIP : 0u;
    items[2 * p] = L;
    items[2 * p + 1] = R;
    info[p] = PairInfo{seed, 0};
    if (!(L.flags & ITEM_SKIP)) queue[atomicAdd(&counters->tail[0], 1u)] = 2 * p;
    if (!(R.flags & ITEM_SKIP)) queue[atomicAdd(&counters->tail[0], 1u)] = 2 * p + 1;
}

__global__ void k_mx_reset(Counters* c) {
    const int t = threadIdx.x;
    if (t < kQueues) {
        c->head[t] = 0u;
        c->head2[t] = 0u;
        c->tail[t] = 0u;
        c->started[t] = 0u;
    }
    if (t <= kNumLevels) c->cells[t] = 0ull;
}

inline size_t mx_up(size_t v) { return (v + 255) / 256 * 256; }

struct MxLayout {
    size_t items, ext, info, queue, counters, badA, badB, table, ring, total;
    uint32_t slots;
};

MxLayout mx_layout(int num_sms, const logan_seqs_t* A, const logan_seqs_t* B, uint32_t n) {
    MxLayout L{};
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t at = off;
        off += mx_up(bytes);
        return at;
    };
    const size_t items = size_t(2) * n;
    L.items = take(items * sizeof(Item));
    L.ext = take(items * sizeof(ExtRes));
    L.info = take(size_t(n) * sizeof(PairInfo));
    L.queue = take(items * sizeof(uint32_t));
    L.counters = take(sizeof(Counters));
    L.badA = take(A->count);
    L.badB = take(B->count);
    L.table = take(sizeof(int32_t) * kMaxK * kMaxK);
    L.slots = uint32_t(std::max<size_t>(1, std::min<size_t>(size_t(num_sms) * 2, items)));
    L.ring = take(size_t(L.slots) * 6u * (size_t(1) << LOGAN_MATRIX_RING_LOG2) * sizeof(int32_t));
    L.total = off;
    return L;
}

}  // namespace

// the affine path's wide-band continuation: every entry of queue q, 2-bit
// pools, the 4 x 4 match / mismatch table
cudaError_t launch_affine_ring(const KernelArgs& ka, int q, int go, int ge, int grid,
                               cudaStream_t s) {
    if (grid <= 0) return cudaSuccess;
    MxArgs a;
    a.pa = ka.wa;
    a.pb = ka.wb;
    a.items = ka.items;
    a.ext = ka.ext;
    a.queue = ka.queues + size_t(q) * ka.qcap;
    a.counters = ka.counters;
    a.q = q;
    a.table = nullptr;
    a.K = 4;
    a.match = ka.sc.match;
    a.mismatch = ka.sc.mismatch;
    a.go = go;
    a.ge = ge;
    a.ring = ka.ring;
    // the workspace ring holds 3 * ring_cap cells per slot; six arrays fit
    // at half that width
    a.cap = ka.ring_cap / 2;
    a.cells_level = kNumLevels;
    k_mx_ring<false><<<grid, kMxThreads, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace logan

using namespace logan;

extern "C" int logan_matrix_workspace_size(const logan_ctx_t* ctx, const logan_seqs_t* seqsA,
                                           const logan_seqs_t* seqsB, uint32_t n_pairs,
                                           size_t* bytes) {
    if (!ctx || !seqsA || !seqsB || !bytes) return LOGAN_EINVAL;
    int64_t dev = 0;
    if (logan_get_option(const_cast<logan_ctx_t*>(ctx), LOGAN_OPT_DEVICE, &dev) != LOGAN_OK)
        return LOGAN_EINVAL;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, int(dev)) != cudaSuccess)
        return LOGAN_ECUDA;
    *bytes = mx_layout(sms, seqsA, seqsB, n_pairs).total;
    return LOGAN_OK;
}

extern "C" int logan_extend_batch_matrix(logan_ctx_t* ctx, const logan_seqs_t* seqsA,
                                         const logan_seqs_t* seqsB, const logan_seed_t* seeds,
                                         uint32_t n_pairs, const int32_t* matrix, int K,
                                         int32_t gap_open, int32_t gap_extend, int32_t X,
                                         const int32_t* X_per_pair, void* workspace,
                                         size_t ws_bytes, logan_result_t* out, void* stream) {
    if (!ctx || !seqsA || !seqsB || !matrix) return LOGAN_EINVAL;
    for (const logan_seqs_t* p : {seqsA, seqsB}) {
        if (p->packed2bit != 0) return LOGAN_EINVAL;  // letter codes, one byte each
        if (p->count && (!p->bases || !p->offsets || !p->lengths)) return LOGAN_EINVAL;
    }
    if (K < 1 || K > kMaxK) return LOGAN_EINVAL;
    if (gap_open > 0 || gap_extend > 0 || gap_open < -kMaxParam || gap_extend < -kMaxParam)
        return LOGAN_EINVAL;
    if (X < 0 || X > kMaxX) return LOGAN_EINVAL;
    int64_t big = int64_t(-gap_open) - gap_extend;
    for (int t = 0; t < K * K; ++t) {
        const int64_t v = matrix[t] < 0 ? -int64_t(matrix[t]) : matrix[t];
        if (v > kMaxParam) return LOGAN_EINVAL;
        big = std::max(big, v);
    }
    if (n_pairs == 0) return LOGAN_OK;
    if (!seeds || !out || !workspace || n_pairs > 0x7fffffffu) return LOGAN_EINVAL;
    if (reinterpret_cast<uintptr_t>(workspace) % 256) return LOGAN_EINVAL;
    int64_t dev = 0;
    if (logan_get_option(ctx, LOGAN_OPT_DEVICE, &dev) != LOGAN_OK) return LOGAN_EINVAL;
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) return LOGAN_ECUDA;
    if (prev != int(dev) && cudaSetDevice(int(dev)) != cudaSuccess) return LOGAN_ECUDA;
    int sms = 0;
    int rc = LOGAN_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, int(dev)) != cudaSuccess) {
        rc = LOGAN_ECUDA;
    } else {
        const MxLayout L = mx_layout(sms, seqsA, seqsB, n_pairs);
        char* ws = static_cast<char*>(workspace);
        if (ws_bytes < L.total) {
            rc = LOGAN_ENOMEM;
        } else {
            Item* items = reinterpret_cast<Item*>(ws + L.items);
            ExtRes* ext = reinterpret_cast<ExtRes*>(ws + L.ext);
            PairInfo* info = reinterpret_cast<PairInfo*>(ws + L.info);
            uint32_t* queue = reinterpret_cast<uint32_t*>(ws + L.queue);
            Counters* counters = reinterpret_cast<Counters*>(ws + L.counters);
            uint8_t* badA = reinterpret_cast<uint8_t*>(ws + L.badA);
            uint8_t* badB = reinterpret_cast<uint8_t*>(ws + L.badB);
            int32_t* table = reinterpret_cast<int32_t*>(ws + L.table);
            cudaError_t e = cudaMemcpyAsync(table, matrix, sizeof(int32_t) * K * K,
                                            cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess) {
                k_mx_reset<<<1, 32, 0, s>>>(counters);
                e = cudaGetLastError();
            }
            const bool same = seqsA->bases == seqsB->bases && seqsA->offsets == seqsB->offsets &&
                              seqsA->lengths == seqsB->lengths && seqsA->count == seqsB->count;
            if (e == cudaSuccess && seqsA->count) {
                k_mx_validate<<<(seqsA->count + 7) / 8, 256, 0, s>>>(
                    static_cast<const uint8_t*>(seqsA->bases), seqsA->offsets, seqsA->lengths,
                    seqsA->count, K, badA);
                e = cudaGetLastError();
            }
            if (e == cudaSuccess && seqsB->count && !same) {
                k_mx_validate<<<(seqsB->count + 7) / 8, 256, 0, s>>>(
                    static_cast<const uint8_t*>(seqsB->bases), seqsB->offsets, seqsB->lengths,
                    seqsB->count, K, badB);
                e = cudaGetLastError();
            }
            if (e == cudaSuccess) {
                const MxPool pa = {static_cast<const uint8_t*>(seqsA->bases), seqsA->offsets,
                                   seqsA->lengths, seqsA->count, badA};
                const MxPool pb = same ? MxPool{pa.bases, pa.off, pa.len, pa.count, badA}
                                       : MxPool{static_cast<const uint8_t*>(seqsB->bases),
                                                seqsB->offsets, seqsB->lengths, seqsB->count,
                                                badB};
                k_mx_split<<<(n_pairs + 255) / 256, 256, 0, s>>>(
                    pa, pb, reinterpret_cast<const uint32_t*>(seeds), n_pairs, table, K, big, X,
                    X_per_pair, items, info, ext, queue, counters);
                e = cudaGetLastError();
                if (e == cudaSuccess) {
                    MxArgs a;
                    a.pa = pa.bases;
                    a.pb = pb.bases;
                    a.items = items;
                    a.ext = ext;
                    a.queue = queue;
                    a.counters = counters;
                    a.q = 0;
                    a.table = table;
                    a.K = K;
                    a.match = 0;
                    a.mismatch = 0;
                    a.go = gap_open;
                    a.ge = gap_extend;
                    a.ring = reinterpret_cast<int32_t*>(ws + L.ring);
                    a.cap = 1u << LOGAN_MATRIX_RING_LOG2;
                    a.cells_level = 0;
                    k_mx_ring<true><<<L.slots, kMxThreads, 0, s>>>(a);
                    e = cudaGetLastError();
                }
                if (e == cudaSuccess) e = launch_combine(seeds, info, ext, n_pairs, out, s);
            }
            if (e != cudaSuccess) rc = LOGAN_ECUDA;
        }
    }
    if (prev >= 0 && prev != int(dev)) cudaSetDevice(prev);
    return rc;
}
