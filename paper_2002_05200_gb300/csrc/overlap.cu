// Many-to-many overlap seeding before the extension: the step that the
// paper's application (Sec. V) runs to find read pairs worth extending and
// a seed for each, and the adaptive threshold applied to the extension
// score.  The paper gives these steps in words only; the definitions here:
//   k-mer codes   base codes A0 C1 G2 T3; forward code of the k-mer at p =
//                 sum_t c[p+t] << 2t; reverse complement sum_t (3 - c[p+k-1-t])
//                 << 2t; canonical = the smaller, strand 1 when the reverse
//                 complement is strictly smaller (k <= 31)
//   reliable      min_freq <= occurrences of the canonical code <= max_freq
//   hits          two occurrences of a reliable k-mer in reads a < b:
//                 (a, b, strand_a ^ strand_b, pos_a, pos_b)
//   candidates    (a, b, o) with >= min_shared hits; the seed is the hit at
//                 index count / 2 in (pos_a, pos_b) order
//   threshold     keep when score * den >= ratio_num * L - delta * den, L the
//                 overlap the seed's diagonal implies
// Sorting runs on CUB radix sorts (library primitives; stable, so equal
// keys keep the order of their input); every other step is a kernel here.
#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_scan.cuh>
#include <cub/device/device_select.cuh>

#include <cstdint>
#include <vector>

#include "ctx_ext.h"
#include "internal.h"

#include "../../include/logan.h"

namespace logan {

namespace {

constexpr int kThreads = 256;

inline unsigned blocks_for(uint64_t n, unsigned t = kThreads) {
    return unsigned(std::min<uint64_t>((n + t - 1) / t, 1u << 20));
}

inline int bit_width(uint64_t v) {
    int b = 0;
    while (v >> b) ++b;
    return b;
}

// 2k bits of codes starting at pool position P (code of P in the low bits)
__device__ __forceinline__ uint64_t codes_at(const uint32_t* __restrict__ w, uint64_t P, int k) {
    const uint64_t i0 = P >> 4;
    const uint32_t sh = uint32_t(P & 15) * 2u;
    const uint64_t lo = uint64_t(__ldg(w + i0)) | (uint64_t(__ldg(w + i0 + 1)) << 32);
    uint64_t v = lo >> sh;
    if (sh && sh + 2u * k > 64u) v |= uint64_t(__ldg(w + i0 + 2)) << (64u - sh);
    return k == 32 ? v : (v & ((1ull << (2 * k)) - 1ull));
}

__device__ __forceinline__ uint64_t revcomp_code(uint64_t f, int k) {
    uint64_t v = __brevll(~f);
    v = ((v >> 1) & 0x5555555555555555ull) | ((v & 0x5555555555555555ull) << 1);
    return v >> (64 - 2 * k);
}

// k-mer positions per read (0 when the read is shorter than k)
__global__ void k_kmer_counts(const uint32_t* __restrict__ len, uint32_t n, int k,
                              uint64_t* __restrict__ cnt) {
    for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x)
        cnt[r] = len[r] >= uint32_t(k) ? uint64_t(len[r] - k + 1) : 0ull;
}

// one warp per read: (canonical code, read << 32 | pos << 1 | strand) at
// first[r] + pos, so the array is in (read, pos) order
__global__ void k_kmer_emit(const uint32_t* __restrict__ w, const uint64_t* __restrict__ off,
                            const uint32_t* __restrict__ len, uint32_t n, int k,
                            const uint64_t* __restrict__ first, uint64_t* __restrict__ keys,
                            uint64_t* __restrict__ vals) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t r = warp; r < n; r += nwarps) {
        if (len[r] < uint32_t(k)) continue;
        const uint32_t npos = len[r] - k + 1;
        for (uint32_t p = lane; p < npos; p += 32) {
            const uint64_t f = codes_at(w, off[r] + p, k);
            const uint64_t rc = revcomp_code(f, k);
            const uint64_t i = first[r] + p;
            keys[i] = rc < f ? rc : f;
            vals[i] = (uint64_t(r) << 32) | (uint64_t(p) << 1) | (rc < f ? 1ull : 0ull);
        }
    }
}

// 1 where a run of equal keys starts (flag[n] = 0 pads the scan)
__global__ void k_head_flags(const uint64_t* __restrict__ keys, uint64_t n,
                             uint64_t* __restrict__ flag) {
    for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i <= n;
         i += uint64_t(gridDim.x) * blockDim.x)
        flag[i] = (i < n && (i == 0 || keys[i] != keys[i - 1])) ? 1ull : 0ull;
}

// starts[rank[i]] = i for every run head i
__global__ void k_head_scatter(const uint64_t* __restrict__ flag, const uint64_t* __restrict__ rank,
                               uint64_t n, uint64_t* __restrict__ starts) {
    for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < n;
         i += uint64_t(gridDim.x) * blockDim.x)
        if (flag[i]) starts[rank[i]] = i;
}

// hits of a run of equal codes: pairs i < j from different reads (the run
// is in (read, pos) order, so read_i <= read_j); none outside the window
__global__ void k_run_hit_counts(const uint64_t* __restrict__ starts, uint64_t n_runs,
                                 uint64_t n, const uint64_t* __restrict__ vals, uint32_t fmin,
                                 uint32_t fmax, uint64_t* __restrict__ cnt) {
    for (uint64_t j = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; j < n_runs;
         j += uint64_t(gridDim.x) * blockDim.x) {
        const uint64_t s = starts[j], e = j + 1 < n_runs ? starts[j + 1] : n;
        const uint64_t f = e - s;
        uint64_t c = 0;
        if (f >= fmin && f <= fmax)
            for (uint64_t a = s; a < e; ++a)
                for (uint64_t b = a + 1; b < e; ++b)
                    c += (vals[a] >> 32) < (vals[b] >> 32) ? 1 : 0;
        cnt[j] = c;
    }
}

// hit key: read a, read b, o (pair and orientation); value: pos_a, pos_b
__global__ void k_run_hit_emit(const uint64_t* __restrict__ starts, uint64_t n_runs, uint64_t n,
                               const uint64_t* __restrict__ vals, uint32_t fmin, uint32_t fmax,
                               const uint64_t* __restrict__ at, int rb, int pb,
                               uint64_t* __restrict__ hk, uint64_t* __restrict__ hv) {
    for (uint64_t j = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; j < n_runs;
         j += uint64_t(gridDim.x) * blockDim.x) {
        const uint64_t s = starts[j], e = j + 1 < n_runs ? starts[j + 1] : n;
        const uint64_t f = e - s;
        if (f < fmin || f > fmax) continue;
        uint64_t o = at[j];
        for (uint64_t a = s; a < e; ++a)
            for (uint64_t b = a + 1; b < e; ++b) {
                const uint64_t ra = vals[a] >> 32, rb_ = vals[b] >> 32;
                if (ra >= rb_) continue;
                const uint64_t pa = (vals[a] >> 1) & 0x7fffffffull;
                const uint64_t pbv = (vals[b] >> 1) & 0x7fffffffull;
                const uint64_t ori = (vals[a] ^ vals[b]) & 1ull;
                hk[o] = (ra << (rb + 1)) | (rb_ << 1) | ori;
                hv[o] = (pa << pb) | pbv;
                ++o;
            }
    }
}

// per (a, b, o) segment of the sorted hits: its middle hit, kept when the
// segment has at least min_shared hits
__global__ void k_segment_pick(const uint64_t* __restrict__ starts, uint64_t n_seg, uint64_t n,
                               const uint64_t* __restrict__ hk, const uint64_t* __restrict__ hv,
                               int rb, int pb, uint32_t min_shared,
                               logan_candidate_t* __restrict__ cand, uint8_t* __restrict__ keep) {
    for (uint64_t j = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; j < n_seg;
         j += uint64_t(gridDim.x) * blockDim.x) {
        const uint64_t s = starts[j], e = j + 1 < n_seg ? starts[j + 1] : n;
        const uint64_t cnt = e - s, m = s + cnt / 2;
        const uint64_t key = hk[m], v = hv[m];
        logan_candidate_t c;
        c.a = uint32_t(key >> (rb + 1));
        c.b = uint32_t((key >> 1) & ((1ull << rb) - 1ull));
        c.o = uint32_t(key & 1ull);
        c.pos_a = uint32_t(v >> pb);
        c.pos_b = uint32_t(v & ((1ull << pb) - 1ull));
        c.count = uint32_t(cnt);
        cand[j] = c;
        keep[j] = cnt >= min_shared ? 1 : 0;
    }
}

// the reverse complement of every read, 16-base aligned after the forward
// pool's words: thread per output word
__global__ void k_revcomp_pool(const uint32_t* __restrict__ w, const uint64_t* __restrict__ off,
                               const uint32_t* __restrict__ len, uint32_t n,
                               const uint64_t* __restrict__ word_first, uint64_t fwd_words,
                               uint32_t* __restrict__ out, uint64_t* __restrict__ out_off) {
    for (uint32_t r = blockIdx.y; r < n; r += gridDim.y) {
        const uint64_t nw = (uint64_t(len[r]) + 15) / 16;
        if (blockIdx.x == 0 && threadIdx.x == 0) out_off[r] = (fwd_words + word_first[r]) * 16;
        for (uint64_t q = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; q < nw;
             q += uint64_t(gridDim.x) * blockDim.x) {
            uint32_t word = 0u;
            for (uint32_t t = 0; t < 16; ++t) {
                const uint64_t i = q * 16 + t;  // base i of the reverse complement
                if (i < len[r]) {
                    const uint32_t c = code_at(w, off[r] + len[r] - 1 - i);
                    word |= (3u - c) << (2 * t);
                }
            }
            out[fwd_words + word_first[r] + q] = word;
        }
    }
}

__global__ void k_overlap_seeds(const logan_candidate_t* __restrict__ c, uint64_t n,
                                const uint32_t* __restrict__ len, uint32_t n_reads, int k,
                                logan_seed_t* __restrict__ seeds) {
    for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < n;
         i += uint64_t(gridDim.x) * blockDim.x) {
        const logan_candidate_t x = c[i];
        logan_seed_t s;
        s.idxA = x.a;
        s.idxB = x.o ? n_reads + x.b : x.b;
        s.posA = x.pos_a;
        s.posB = x.o ? len[x.b] - x.pos_b - uint32_t(k) : x.pos_b;
        s.len = uint32_t(k);
        seeds[i] = s;
    }
}

__global__ void k_overlap_keep(const logan_result_t* __restrict__ res,
                               const logan_seed_t* __restrict__ seeds, uint64_t n,
                               const uint32_t* __restrict__ lenA, const uint32_t* __restrict__ lenB,
                               int64_t ratio_num, int64_t den, int64_t delta,
                               uint8_t* __restrict__ keep) {
    for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < n;
         i += uint64_t(gridDim.x) * blockDim.x) {
        const logan_seed_t s = seeds[i];
        const int64_t la = lenA[s.idxA], lb = lenB[s.idxB];
        const int64_t pa = s.posA, pbv = s.posB, k = s.len;
        const int64_t L = min(pa, pbv) + k + min(la - pa - k, lb - pbv - k);
        keep[i] = (res[i].status == 0 && int64_t(res[i].score) * den >= ratio_num * L - delta * den)
                      ? 1
                      : 0;
    }
}

// stream-ordered scratch that frees itself
struct Scratch {
    cudaStream_t s;
    cudaMemPool_t pool;  // the context's scratch pool (null: the default one)
    std::vector<void*> ptrs;
    bool ok = true;
    Scratch(cudaStream_t st, cudaMemPool_t p) : s(st), pool(p) {}
    template <typename T>
    T* get(size_t n) {
        void* p = nullptr;
        const size_t bytes = std::max<size_t>(n, 1) * sizeof(T);
        if (!ok || (pool ? cudaMallocFromPoolAsync(&p, bytes, pool, s)
                         : cudaMallocAsync(&p, bytes, s)) != cudaSuccess) {
            ok = false;
            return nullptr;
        }
        ptrs.push_back(p);
        return static_cast<T*>(p);
    }
    ~Scratch() {
        for (void* p : ptrs) cudaFreeAsync(p, s);
    }
};

// Start index of every run of equal keys in keys[0, n) (sorted); returns
// the number of runs (synchronises the stream), or -1 on failure.
int64_t run_heads(Scratch& sc, const uint64_t* keys, uint64_t n, uint64_t*& starts) {
    cudaStream_t s = sc.s;
    uint64_t* flag = sc.get<uint64_t>(n + 1);
    uint64_t* rank = sc.get<uint64_t>(n + 1);
    starts = sc.get<uint64_t>(n);
    size_t tb = 0;
    cub::DeviceScan::ExclusiveSum(nullptr, tb, flag, rank, n + 1, s);
    void* tmp = sc.get<char>(tb);
    if (!sc.ok) return -1;
    k_head_flags<<<blocks_for(n + 1), kThreads, 0, s>>>(keys, n, flag);
    cub::DeviceScan::ExclusiveSum(tmp, tb, flag, rank, n + 1, s);
    k_head_scatter<<<blocks_for(n), kThreads, 0, s>>>(flag, rank, n, starts);
    uint64_t nr = 0;
    if (cudaMemcpyAsync(&nr, rank + n, sizeof(uint64_t), cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return -1;
    return int64_t(nr);
}

}  // namespace

}  // namespace logan

using namespace logan;

extern "C" int logan_overlap_candidates(logan_ctx_t* ctx, const logan_seqs_t* reads, int k,
                                        uint32_t min_freq, uint32_t max_freq,
                                        uint32_t min_shared, logan_candidate_t* out,
                                        uint64_t capacity, uint64_t* n_found, void* stream) {
    if (!ctx || !reads || !n_found || k < 1 || k > 31 || min_freq < 2 || max_freq < min_freq ||
        max_freq > 1024 || min_shared < 1)
        return LOGAN_EINVAL;
    if (!reads->packed2bit || (reads->count && (!reads->bases || !reads->offsets || !reads->lengths)))
        return LOGAN_EINVAL;
    if (capacity && !out) return LOGAN_EINVAL;
    *n_found = 0;
    const uint32_t R = reads->count;
    if (R < 2) return LOGAN_OK;
    int64_t dev = 0;
    logan_get_option(ctx, LOGAN_OPT_DEVICE, &dev);
    int prev = 0;
    cudaGetDevice(&prev);
    if (prev != int(dev) && cudaSetDevice(int(dev)) != cudaSuccess) return LOGAN_ECUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const uint32_t* w = static_cast<const uint32_t*>(reads->bases);
    int rc = LOGAN_OK;
    {
        Scratch sc(s, ctx_scratch_pool(ctx));
        // 1. k-mer occurrences, (read, pos) order: first[r] = k-mers of
        // reads below r, first[R] = all of them
        uint64_t* cnt = sc.get<uint64_t>(R + 1);
        uint64_t* first = sc.get<uint64_t>(R + 1);
        size_t tb = 0;
        cub::DeviceScan::ExclusiveSum(nullptr, tb, cnt, first, R + 1, s);
        void* tmp = sc.get<char>(tb);
        if (!sc.ok) return LOGAN_ENOMEM;
        k_kmer_counts<<<blocks_for(R), kThreads, 0, s>>>(reads->lengths, R, k, cnt);
        cudaMemsetAsync(cnt + R, 0, sizeof(uint64_t), s);
        cub::DeviceScan::ExclusiveSum(tmp, tb, cnt, first, R + 1, s);
        uint64_t* nk_d = first + R;
        uint64_t nk = 0;
        cudaMemcpyAsync(&nk, nk_d, sizeof(uint64_t), cudaMemcpyDeviceToHost, s);
        if (cudaStreamSynchronize(s) != cudaSuccess) return LOGAN_ECUDA;
        if (nk < 2) return LOGAN_OK;
        uint64_t* keys = sc.get<uint64_t>(nk);
        uint64_t* vals = sc.get<uint64_t>(nk);
        uint64_t* keys2 = sc.get<uint64_t>(nk);
        uint64_t* vals2 = sc.get<uint64_t>(nk);
        if (!sc.ok) return LOGAN_ENOMEM;
        k_kmer_emit<<<blocks_for(uint64_t(R) * 32), kThreads, 0, s>>>(w, reads->offsets,
                                                                     reads->lengths, R, k, first,
                                                                     keys, vals);
        // 2. sort by code (stable: equal codes stay in (read, pos) order)
        size_t tsort = 0;
        cub::DeviceRadixSort::SortPairs(nullptr, tsort, keys, keys2, vals, vals2, nk, 0, 2 * k, s);
        void* tmp2 = sc.get<char>(tsort);
        if (!sc.ok) return LOGAN_ENOMEM;
        cub::DeviceRadixSort::SortPairs(tmp2, tsort, keys, keys2, vals, vals2, nk, 0, 2 * k, s);
        // 3. runs of equal codes
        uint64_t* starts = nullptr;
        const int64_t nrun_i = run_heads(sc, keys2, nk, starts);
        if (nrun_i < 0) return sc.ok ? LOGAN_ECUDA : LOGAN_ENOMEM;
        const uint64_t nrun = uint64_t(nrun_i);
        // 4. hits of the reliable runs
        uint64_t* hcnt = sc.get<uint64_t>(nrun + 1);
        uint64_t* hat = sc.get<uint64_t>(nrun + 1);
        if (!sc.ok) return LOGAN_ENOMEM;
        k_run_hit_counts<<<blocks_for(nrun), kThreads, 0, s>>>(starts, nrun, nk, vals2, min_freq,
                                                               max_freq, hcnt);
        cudaMemsetAsync(hcnt + nrun, 0, sizeof(uint64_t), s);
        size_t tscan = 0;
        cub::DeviceScan::ExclusiveSum(nullptr, tscan, hcnt, hat, nrun + 1, s);
        void* tmp4 = sc.get<char>(tscan);
        if (!sc.ok) return LOGAN_ENOMEM;
        cub::DeviceScan::ExclusiveSum(tmp4, tscan, hcnt, hat, nrun + 1, s);
        uint64_t nh = 0;
        cudaMemcpyAsync(&nh, hat + nrun, sizeof(uint64_t), cudaMemcpyDeviceToHost, s);
        if (cudaStreamSynchronize(s) != cudaSuccess) return LOGAN_ECUDA;
        if (nh == 0) return LOGAN_OK;
        uint32_t maxlen = 0;
        {
            std::vector<uint32_t> hl(R);
            cudaMemcpyAsync(hl.data(), reads->lengths, sizeof(uint32_t) * R, cudaMemcpyDeviceToHost, s);
            if (cudaStreamSynchronize(s) != cudaSuccess) return LOGAN_ECUDA;
            for (uint32_t v : hl) maxlen = std::max(maxlen, v);
        }
        const int rb = std::max(1, bit_width(R));
        const int pb = std::max(1, bit_width(maxlen));
        if (2 * rb + 1 > 64 || 2 * pb > 64) return LOGAN_EINVAL;
        uint64_t* hk = sc.get<uint64_t>(nh);
        uint64_t* hv = sc.get<uint64_t>(nh);
        uint64_t* hk2 = sc.get<uint64_t>(nh);
        uint64_t* hv2 = sc.get<uint64_t>(nh);
        if (!sc.ok) return LOGAN_ENOMEM;
        k_run_hit_emit<<<blocks_for(nrun), kThreads, 0, s>>>(starts, nrun, nk, vals2, min_freq,
                                                             max_freq, hat, rb, pb, hk, hv);
        // 5. order hits by (a, b, o), then (pos_a, pos_b): sort by position,
        // then stably by pair
        size_t t5 = 0;
        cub::DeviceRadixSort::SortPairs(nullptr, t5, hv, hv2, hk, hk2, nh, 0, 2 * pb, s);
        size_t t6 = 0;
        cub::DeviceRadixSort::SortPairs(nullptr, t6, hk2, hk, hv2, hv, nh, 0, 2 * rb + 1, s);
        void* tmp5 = sc.get<char>(std::max(t5, t6));
        if (!sc.ok) return LOGAN_ENOMEM;
        cub::DeviceRadixSort::SortPairs(tmp5, t5, hv, hv2, hk, hk2, nh, 0, 2 * pb, s);
        cub::DeviceRadixSort::SortPairs(tmp5, t6, hk2, hk, hv2, hv, nh, 0, 2 * rb + 1, s);
        // now hk / hv hold the hits in (a, b, o, pos_a, pos_b) order
        uint64_t* sstart = nullptr;
        const int64_t nseg_i = run_heads(sc, hk, nh, sstart);
        if (nseg_i < 0) return sc.ok ? LOGAN_ECUDA : LOGAN_ENOMEM;
        const uint64_t nseg = uint64_t(nseg_i);
        // 6. one candidate per segment, compacted in order
        logan_candidate_t* all = sc.get<logan_candidate_t>(nseg);
        uint8_t* keep = sc.get<uint8_t>(nseg);
        logan_candidate_t* kept = sc.get<logan_candidate_t>(nseg);
        uint64_t* nkept_d = sc.get<uint64_t>(1);
        if (!sc.ok) return LOGAN_ENOMEM;
        k_segment_pick<<<blocks_for(nseg), kThreads, 0, s>>>(sstart, nseg, nh, hk, hv, rb, pb,
                                                             min_shared, all, keep);
        size_t t8 = 0;
        cub::DeviceSelect::Flagged(nullptr, t8, all, keep, kept, nkept_d, nseg, s);
        void* tmp8 = sc.get<char>(t8);
        if (!sc.ok) return LOGAN_ENOMEM;
        cub::DeviceSelect::Flagged(tmp8, t8, all, keep, kept, nkept_d, nseg, s);
        uint64_t nkept = 0;
        cudaMemcpyAsync(&nkept, nkept_d, sizeof(uint64_t), cudaMemcpyDeviceToHost, s);
        if (cudaStreamSynchronize(s) != cudaSuccess) return LOGAN_ECUDA;
        *n_found = nkept;
        const uint64_t ncopy = std::min(nkept, capacity);
        if (ncopy)
            cudaMemcpyAsync(out, kept, sizeof(logan_candidate_t) * ncopy, cudaMemcpyDeviceToDevice,
                            s);
        if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess)
            rc = LOGAN_ECUDA;
    }
    if (prev != int(dev)) cudaSetDevice(prev);
    return rc;
}

extern "C" int logan_overlap_pool_words(logan_ctx_t* ctx, const logan_seqs_t* reads,
                                        uint64_t* words, void* stream) {
    if (!ctx || !reads || !words || !reads->packed2bit || (reads->count && !reads->lengths))
        return LOGAN_EINVAL;
    // the forward pool's words (with its spare word), then every reverse
    // complement 16-base aligned, then one spare word
    const uint32_t R = reads->count;
    std::vector<uint32_t> hl(R);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (R && (cudaMemcpyAsync(hl.data(), reads->lengths, sizeof(uint32_t) * R,
                              cudaMemcpyDeviceToHost, s) != cudaSuccess ||
              cudaStreamSynchronize(s) != cudaSuccess))
        return LOGAN_ECUDA;
    uint64_t tot = (reads->pool_bases + 15) / 16 + 1;
    for (uint32_t v : hl) tot += (uint64_t(v) + 15) / 16;
    *words = tot + 1;
    return LOGAN_OK;
}

extern "C" int logan_overlap_pool(logan_ctx_t* ctx, const logan_seqs_t* reads,
                                  uint32_t* words_out, uint64_t words_capacity,
                                  uint64_t* offsets_out, uint32_t* lengths_out,
                                  logan_seqs_t* pool_out, void* stream) {
    if (!ctx || !reads || !pool_out || !reads->packed2bit || !words_out || !offsets_out ||
        !lengths_out)
        return LOGAN_EINVAL;
    const uint32_t R = reads->count;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const uint64_t fwd = (reads->pool_bases + 15) / 16 + 1;
    std::vector<uint32_t> hl(R);
    if (R && (cudaMemcpyAsync(hl.data(), reads->lengths, sizeof(uint32_t) * R,
                              cudaMemcpyDeviceToHost, s) != cudaSuccess ||
              cudaStreamSynchronize(s) != cudaSuccess))
        return LOGAN_ECUDA;
    std::vector<uint64_t> wf(R);
    uint64_t tot = 0;
    for (uint32_t r = 0; r < R; ++r) {
        wf[r] = tot;
        tot += (uint64_t(hl[r]) + 15) / 16;
    }
    const uint64_t need = fwd + tot + 1;
    if (words_capacity < need) return LOGAN_ENOMEM;
    int rc = LOGAN_OK;
    {
        Scratch sc(s, ctx_scratch_pool(ctx));
        uint64_t* wfd = sc.get<uint64_t>(R);
        if (!sc.ok) return LOGAN_ENOMEM;
        if (R) cudaMemcpyAsync(wfd, wf.data(), sizeof(uint64_t) * R, cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(words_out, reads->bases, sizeof(uint32_t) * fwd, cudaMemcpyDeviceToDevice, s);
        cudaMemsetAsync(words_out + fwd + tot, 0, sizeof(uint32_t), s);
        if (R) {
            cudaMemcpyAsync(offsets_out, reads->offsets, sizeof(uint64_t) * R,
                            cudaMemcpyDeviceToDevice, s);
            cudaMemcpyAsync(lengths_out, reads->lengths, sizeof(uint32_t) * R,
                            cudaMemcpyDeviceToDevice, s);
            cudaMemcpyAsync(lengths_out + R, reads->lengths, sizeof(uint32_t) * R,
                            cudaMemcpyDeviceToDevice, s);
            dim3 grid(64, std::min<uint32_t>(R, 65535u));
            k_revcomp_pool<<<grid, 128, 0, s>>>(static_cast<const uint32_t*>(reads->bases),
                                                reads->offsets, reads->lengths, R, wfd, fwd,
                                                words_out, offsets_out + R);
        }
        // the host copies above read pageable host vectors: finish before they go
        if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess)
            rc = LOGAN_ECUDA;
    }
    pool_out->bases = words_out;
    pool_out->offsets = offsets_out;
    pool_out->lengths = lengths_out;
    pool_out->count = 2 * R;
    pool_out->packed2bit = 1;
    pool_out->pool_bases = (need - 1) * 16;
    return rc;
}

extern "C" int logan_overlap_seeds(logan_ctx_t* ctx, const logan_candidate_t* cands, uint64_t n,
                                   const logan_seqs_t* reads, int k, logan_seed_t* seeds,
                                   void* stream) {
    if (!ctx || !reads || (n && (!cands || !seeds)) || k < 1 || k > 31) return LOGAN_EINVAL;
    if (!n) return LOGAN_OK;
    k_overlap_seeds<<<blocks_for(n), kThreads, 0, static_cast<cudaStream_t>(stream)>>>(
        cands, n, reads->lengths, reads->count, k, seeds);
    return cudaGetLastError() == cudaSuccess ? LOGAN_OK : LOGAN_ECUDA;
}

extern "C" int logan_overlap_keep(logan_ctx_t* ctx, const logan_result_t* results,
                                  const logan_seed_t* seeds, uint64_t n,
                                  const logan_seqs_t* seqsA, const logan_seqs_t* seqsB,
                                  int64_t ratio_num, int64_t den, int64_t delta, uint8_t* keep,
                                  void* stream) {
    if (!ctx || !seqsA || !seqsB || den <= 0 || (n && (!results || !seeds || !keep)))
        return LOGAN_EINVAL;
    if (!n) return LOGAN_OK;
    k_overlap_keep<<<blocks_for(n), kThreads, 0, static_cast<cudaStream_t>(stream)>>>(
        results, seeds, n, seqsA->lengths, seqsB->lengths, ratio_num, den, delta, keep);
    return cudaGetLastError() == cudaSuccess ? LOGAN_OK : LOGAN_ECUDA;
}
