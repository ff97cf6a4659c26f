// Pre- and post-processing kernels of the batch pipeline:
//   pack     ASCII bases -> 2-bit words (same base positions)       HBM-bound
//   validate per-sequence input checks (bases, bounds)               HBM-bound
//   split    per pair: seed score, left/right extension items (Sec. IV-B)
//   bin      length/X binning into per-level work queues, longest first
//   combine  left best + seed score + right best, coordinates
#include <climits>

#include "internal.h"

namespace logan {

namespace {

// ASCII -> code with A0 C1 G2 T3: (c >> 1) & 3 maps A,C,T,G to 0,1,2,3;
// t ^ (t >> 1) swaps the last two.
__device__ __forceinline__ uint32_t ascii_code(uint32_t c) {
    const uint32_t t = (c >> 1) & 3u;
    return t ^ (t >> 1);
}

__global__ void k_pack(const uint8_t* __restrict__ in, uint64_t n_bases, uint32_t* __restrict__ out,
                       uint64_t n_words) {
    const uint64_t w = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (w >= n_words) return;
    const uint64_t b0 = w * 16u;
    uint32_t word = 0u;
    if (b0 + 16u <= n_bases && (reinterpret_cast<uintptr_t>(in) & 15u) == 0u) {
        const uint4 v = __ldg(reinterpret_cast<const uint4*>(in + b0));
        const uint32_t parts[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int b = 0; b < 4; ++b)
                word |= ascii_code((parts[q] >> (8 * b)) & 0xffu) << (2 * (4 * q + b));
    } else {
        for (int b = 0; b < 16; ++b)
            if (b0 + b < n_bases) word |= ascii_code(in[b0 + b]) << (2 * b);
    }
    out[w] = word;
}

// one warp per sequence
__global__ void k_validate(const uint8_t* __restrict__ bases, const uint64_t* __restrict__ off,
                           const uint32_t* __restrict__ len, uint32_t count, uint64_t pool_bases,
                           int ascii, uint8_t* __restrict__ bad) {
    const uint32_t s = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (s >= count) return;
    const uint64_t o = off[s];
    const uint32_t L = len[s];
    bool ok = L < (1u << 31) && o <= pool_bases && uint64_t(L) <= pool_bases - o;
    if (ok && ascii) {
        for (uint64_t t = lane; t < L; t += 32) {
            const uint8_t c = bases[o + t];
            ok &= (c == 'A') | (c == 'C') | (c == 'G') | (c == 'T');
        }
    }
    ok = __all_sync(0xffffffffu, ok);
    if (lane == 0) bad[s] = ok ? 0 : 1;
}

struct PoolView {
    const uint64_t* off;
    const uint32_t* len;
    const uint8_t* bad;
    const uint32_t* words;
    uint32_t count;
};

__global__ void k_split(PoolView A, PoolView B, const uint32_t* __restrict__ seeds,
                        uint32_t n_pairs, Scoring sc, int32_t X, const int32_t* __restrict__ Xs,
                        Item* __restrict__ items, PairInfo* __restrict__ info,
                        ExtRes* __restrict__ ext, int32_t* __restrict__ mig_slot) {
    const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_pairs) return;
    mig_slot[2 * p] = -1;
    mig_slot[2 * p + 1] = -1;
    const uint32_t idxA = seeds[5 * p], idxB = seeds[5 * p + 1];
    const uint32_t posA = seeds[5 * p + 2], posB = seeds[5 * p + 3], k = seeds[5 * p + 4];
    const int32_t x = Xs ? Xs[p] : X;
    bool ok = idxA < A.count && idxB < B.count && x >= 0 && x <= kMaxX;
    uint32_t lenA = 0, lenB = 0;
    int64_t offA = 0, offB = 0;
    if (ok) {
        lenA = A.len[idxA];
        lenB = B.len[idxB];
        offA = int64_t(A.off[idxA]);
        offB = int64_t(B.off[idxB]);
        ok = !A.bad[idxA] && !B.bad[idxB] && uint64_t(posA) + k <= lenA &&
             uint64_t(posB) + k <= lenB;
        const int64_t big = max(abs(sc.match), max(abs(sc.mismatch), abs(sc.gap)));
        ok = ok && big * (int64_t(lenA) + int64_t(lenB)) + x < kScoreRange;
    }
    const ExtRes zero = {0, 0, 0, 0, 0ull};
    if (!ok) {
        Item it = {0, 0, 0u, 0u, 0, ITEM_SKIP};
        items[2 * p] = it;
        items[2 * p + 1] = it;
        ext[2 * p] = zero;
        ext[2 * p + 1] = zero;
        info[p] = PairInfo{0, -22};  // LOGAN_EINVAL
        return;
    }
    int32_t seed = 0;
    for (uint32_t t = 0; t < k; ++t)
        seed += code_at(A.words, offA + posA + t) == code_at(B.words, offB + posB + t) ? sc.match
                                                                                       : sc.mismatch;
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
    ext[2 * p] = zero;
    ext[2 * p + 1] = zero;
    info[p] = PairInfo{seed, 0};
}

__device__ __forceinline__ int work_bucket(uint32_t m, uint32_t n) {
    const uint32_t w = m + n + 1u;
    const int lg = 31 - __clz(w);
    const int sub = lg >= 2 ? int((w >> (lg - 2)) & 3u) : 0;
    return min(kBuckets - 1, 4 * lg + sub);
}

// starting level of an item, or -1 when the X-class filter leaves it out
__device__ __forceinline__ int item_level(const Item& it, LevelTable table, int force, int maxl) {
    const int xc = x_class(it.X);
    int l = force >= 0 ? force : int(table.lv[xc]);
    if (it.X > kGroupMaxX && l < kWarpLevels) l = kWarpLevels;
    return min(l, maxl);
}

// queue of an item: its starting level, or that level's latency form for a
// long item
__device__ __forceinline__ int item_queue(const Item& it, LevelTable table, int force, int maxl) {
    const int l = item_level(it, table, force, maxl);
    if (l < kTwinLevels && uint64_t(it.m) + it.n >= table.long_min) return twin_queue(l);
    return l;
}

__global__ void k_bin_hist(const Item* __restrict__ items, uint32_t n, LevelTable table,
                           int force, int maxl, uint32_t* __restrict__ hist) {
    __shared__ uint32_t h[kQueues * kBuckets];
    for (int t = threadIdx.x; t < kQueues * kBuckets; t += blockDim.x) h[t] = 0u;
    __syncthreads();
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const Item it = items[i];
        if (it.flags & ITEM_SKIP) continue;
        const int q = item_queue(it, table, force, maxl);
        atomicAdd(&h[q * kBuckets + (kBuckets - 1 - work_bucket(it.m, it.n))], 1u);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < kQueues * kBuckets; t += blockDim.x)
        if (h[t]) atomicAdd(&hist[t], h[t]);
}

// one block of kBuckets threads: per queue exclusive scan of the bucket
// counts (longest bucket first) -> cursors; queue sizes -> counters (the
// fallback ring's queue gets no binned items)
__global__ void k_bin_scan(uint32_t* __restrict__ hist, Counters* __restrict__ c) {
    __shared__ uint32_t s[kBuckets];
    const int t = threadIdx.x;
    for (int l = 0; l < kQueues; ++l) {
        const uint32_t v = hist[l * kBuckets + t];
        s[t] = v;
        __syncthreads();
        for (int off = 1; off < kBuckets; off <<= 1) {
            const uint32_t a = t >= off ? s[t - off] : 0u;
            __syncthreads();
            s[t] += a;
            __syncthreads();
        }
        hist[l * kBuckets + t] = s[t] - v;  // exclusive prefix = cursor
        if (t == kBuckets - 1) {
            c->tail[l] = s[t];
            c->started[l] = s[t];
        }
        __syncthreads();
    }
    if (t < kQueues) {
        c->head[t] = 0u;
        c->head2[t] = 0u;
    }
    if (t <= kNumLevels) c->cells[t] = 0ull;
    if (t < kNumLevels) c->mig_used[t] = 0u;
}

__global__ void k_bin_scatter(const Item* __restrict__ items, uint32_t n, LevelTable table,
                              int force, int maxl, uint32_t* __restrict__ cursor,
                              uint32_t* __restrict__ queues, uint32_t qcap) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const Item it = items[i];
    if (it.flags & ITEM_SKIP) return;
    const int q = item_queue(it, table, force, maxl);
    const uint32_t pos = atomicAdd(&cursor[q * kBuckets + (kBuckets - 1 - work_bucket(it.m, it.n))], 1u);
    queues[size_t(q) * qcap + pos] = i;
}

__global__ void k_reset_counters(Counters* c, uint32_t first_items, int first_level) {
    const int t = threadIdx.x;
    if (t < kQueues) {
        c->head[t] = 0u;
        c->head2[t] = 0u;
        c->tail[t] = 0u;
        c->started[t] = 0u;  // the plain kernel takes items directly
    }
    if (t <= kNumLevels) c->cells[t] = 0ull;
    (void)first_items;
    (void)first_level;
    if (t < kNumLevels) c->mig_used[t] = 0u;
}

struct ResultOut {
    int32_t score, left, right, status;
    uint32_t begA, begB, endA, endB;
    unsigned long long cells;
};
static_assert(sizeof(ResultOut) == 40, "logan_result_t layout");

__global__ void k_combine(const uint32_t* __restrict__ seeds, const PairInfo* __restrict__ info,
                          const ExtRes* __restrict__ ext, uint32_t n_pairs, ResultOut* __restrict__ out) {
    const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_pairs) return;
    const PairInfo pi = info[p];
    const ExtRes L = ext[2 * p], R = ext[2 * p + 1];
    ResultOut r = {0, 0, 0, 0, 0u, 0u, 0u, 0u, 0ull};
    r.status = pi.status ? pi.status : (L.status ? L.status : R.status);
    if (r.status == 0) {
        const uint32_t posA = seeds[5 * p + 2], posB = seeds[5 * p + 3], k = seeds[5 * p + 4];
        r.left = L.best;
        r.right = R.best;
        r.score = L.best + pi.seed_score + R.best;
        r.begA = posA - uint32_t(L.bi);
        r.begB = posB - uint32_t(L.bj);
        r.endA = posA + k + uint32_t(R.bi);
        r.endB = posB + k + uint32_t(R.bj);
        r.cells = L.cells + R.cells;
    }
    out[p] = r;
}

inline unsigned int blocks_for(uint64_t n, unsigned int threads) {
    return unsigned((n + threads - 1) / threads);
}

}  // namespace

cudaError_t launch_pack(const PoolDev& p, uint32_t* words_out, cudaStream_t s) {
    const uint64_t n_words = (p.pool_bases + 15u) / 16u + 1u;
    k_pack<<<blocks_for(n_words, 256), 256, 0, s>>>(static_cast<const uint8_t*>(p.bases),
                                                     p.pool_bases, words_out, n_words);
    return cudaGetLastError();
}

cudaError_t launch_validate(const PoolDev& p, cudaStream_t s) {
    if (p.count == 0) return cudaSuccess;
    k_validate<<<blocks_for(p.count, 8), 256, 0, s>>>(static_cast<const uint8_t*>(p.bases), p.offsets,
                                                      p.lengths, p.count, p.pool_bases,
                                                      p.packed2bit ? 0 : 1, p.bad);
    return cudaGetLastError();
}

cudaError_t launch_split(const PoolDev& A, const PoolDev& B, const void* seeds, uint32_t n_pairs,
                         Scoring sc, int32_t X, const int32_t* Xs, Item* items, PairInfo* info,
                         ExtRes* ext, int32_t* mig_slot, cudaStream_t s) {
    if (n_pairs == 0) return cudaSuccess;
    PoolView a = {A.offsets, A.lengths, A.bad, A.words, A.count};
    PoolView b = {B.offsets, B.lengths, B.bad, B.words, B.count};
    k_split<<<blocks_for(n_pairs, 128), 128, 0, s>>>(a, b, static_cast<const uint32_t*>(seeds), n_pairs,
                                                     sc, X, Xs, items, info, ext, mig_slot);
    return cudaGetLastError();
}

cudaError_t launch_bin(const Item* items, uint32_t n_items, LevelTable table, int force_level,
                       uint32_t* hist, uint32_t* queues, uint32_t qcap, Counters* counters,
                       cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(hist, 0, sizeof(uint32_t) * kQueues * kBuckets, s);
    if (e != cudaSuccess) return e;
    const int maxl = table.max_level;
    if (n_items) {
        const unsigned int g = min(blocks_for(n_items, 256), 1024u);
        k_bin_hist<<<g, 256, 0, s>>>(items, n_items, table, force_level, maxl, hist);
    }
    k_bin_scan<<<1, kBuckets, 0, s>>>(hist, counters);
    if (n_items)
        k_bin_scatter<<<blocks_for(n_items, 256), 256, 0, s>>>(items, n_items, table, force_level,
                                                               maxl, hist, queues, qcap);
    return cudaGetLastError();
}

cudaError_t launch_reset_counters(Counters* c, uint32_t first_items, int first_level,
                                  cudaStream_t s) {
    k_reset_counters<<<1, 32, 0, s>>>(c, first_items, first_level);
    return cudaGetLastError();
}

cudaError_t launch_combine(const void* seeds, const PairInfo* info, const ExtRes* ext,
                           uint32_t n_pairs, void* out, cudaStream_t s) {
    if (n_pairs == 0) return cudaSuccess;
    k_combine<<<blocks_for(n_pairs, 256), 256, 0, s>>>(static_cast<const uint32_t*>(seeds), info,
                                                       ext, n_pairs, static_cast<ResultOut*>(out));
    return cudaGetLastError();
}

}  // namespace logan
