// Alignment paths of the batch's best cells (the paper keeps no traceback,
// Sec. IV-A; this adds one).  Readings:
//   T1 each live cell keeps the predecessor term that gave its score, the
//      diagonal first, then the vertical move (i-1, j), then the horizontal
//      one (i, j-1);
//   T2 an extension's path is the walk from its best cell back to (0,0);
//      operations M (diagonal), I (a base of A only: vertical), D (a base of
//      B only: horizontal);
//   T3 a pair's alignment is the left extension's path in the sequences'
//      order, k M for the seed, then the right extension's path.
//
// Three passes over the items of the batch, each item on one block of 256
// threads with its three anti-diagonals in a device-memory ring (the
// paper's layout, Sec. IV-B, as in the fallback kernel):
//   1 the sweep to the end: best cell, its anti-diagonal d*, and the words of
//     2-bit predecessor codes anti-diagonals 1..d* take (each one starts on a
//     16-cell word);
//   2 the sweep again up to d*, writing for every anti-diagonal its first
//     row, its first word and the codes of its cells (lanes OR 16 codes into
//     a word with shuffles);
//   3 one thread per pair walks both sides back and writes run-length codes
//     (length << 4 | op; op 0 = M, 1 = I, 2 = D).
// Same cell update and range rules as the extension kernels, so the best
// cells and cells equal theirs.
#include <cub/device/device_scan.cuh>

#include <climits>
#include <vector>

#include "internal.h"

#include "../../include/logan.h"

namespace logan {

namespace {

constexpr uint32_t FULL = 0xffffffffu;
constexpr int kTbThreads = 256;
constexpr int kTbWarps = kTbThreads / 32;

struct TbRed {
    int mx, arg, first, last;
};

__device__ __forceinline__ TbRed tb_reduce(TbRed v, TbRed* sh) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int mx = __reduce_max_sync(FULL, v.mx);
    int arg = __reduce_min_sync(FULL, v.mx == mx ? v.arg : INT_MAX);
    int first = __reduce_min_sync(FULL, v.first);
    int last = __reduce_max_sync(FULL, v.last);
    if (lane == 0) sh[w] = TbRed{mx, arg, first, last};
    __syncthreads();
    TbRed p = lane < kTbWarps ? sh[lane] : TbRed{NEG, INT_MAX, INT_MAX, -1};
    mx = __reduce_max_sync(FULL, p.mx);
    arg = __reduce_min_sync(FULL, p.mx == mx ? p.arg : INT_MAX);
    first = __reduce_min_sync(FULL, p.first);
    last = __reduce_max_sync(FULL, p.last);
    __syncthreads();
    return TbRed{mx, arg, first, last};
}

struct TbItem {  // pass 1 output per item
    int32_t best, bi, bj, status;
    uint64_t words;  // predecessor-code words of anti-diagonals 1..d*
    int32_t wide;    // the band outgrew the shared-memory ring: device-memory ring
    int32_t pad;
};

// anti-diagonals held in shared memory up to this width (3 x 2048 int32 =
// 24 KB per block); wider bands sweep again in the device-memory ring
constexpr int kSmemCap = 2048;
constexpr int TB_WIDE = 1;  // pass-1 status: retry in the device-memory ring

struct TbArgs {
    KernelArgs ka;      // pools, items, scoring, ring
    TbItem* info;       // per item
    const uint64_t* word_off;  // per item: first word of its codes
    const uint64_t* ad_off;    // per item: first entry of its anti-diagonal table
    uint32_t* codes;    // 2-bit predecessor codes
    int32_t* ad_rlo;    // per anti-diagonal: first evaluated row
    uint64_t* ad_word;  // per anti-diagonal: first word
    uint64_t n_words;   // size of codes (reads beyond it are refused)
};

// The sweep of one item; RECORD: up to d* with the codes written.
template <bool RECORD>
__device__ void tb_sweep(const TbArgs& t, uint32_t id, int32_t* R, int cap, TbRed* sh) {
    const KernelArgs& ka = t.ka;
    const Item it = ka.items[id];
    const int dir = (it.flags & ITEM_LEFT) ? -1 : 1;
    const int m = int(it.m), n = int(it.n), X = it.X;
    const int mask = cap - 1;
    int32_t* A0 = R;
    int32_t* A1 = R + cap;
    int32_t* A2 = R + 2 * cap;
    const int dstar = RECORD ? t.info[id].bi + t.info[id].bj : INT_MAX;
    if (threadIdx.x == 0) A1[0] = 0;
    __syncthreads();
    int lo1 = 0, hi1 = 0, lo2 = 1, hi2 = 0;
    int best = 0, bi = 0, bj = 0, status = 0;
    uint64_t words = 0, words_best = 0;
    uint64_t wbase = RECORD ? t.word_off[id] : 0;
    const uint64_t abase = RECORD ? t.ad_off[id] : 0;
    for (int d = 1; d <= dstar; ++d) {
        const int rlo = max(lo1, d - n), rhi = min(hi1 + 1, m);
        if (rlo > rhi) break;
        const int width = rhi - rlo + 1;
        if (width > cap) {
            status = cap < int(ka.ring_cap) ? TB_WIDE : LOGAN_ERANGE;
            break;
        }
        if (RECORD && threadIdx.x == 0) {
            t.ad_rlo[abase + d] = rlo;
            t.ad_word[abase + d] = wbase;
        }
        const int T = best - X;
        TbRed v{NEG, INT_MAX, INT_MAX, -1};
        // whole strides of the block so that every lane takes part in the
        // code packing
        for (int i0 = rlo; i0 <= rhi; i0 += kTbThreads) {
            const int i = i0 + int(threadIdx.x);
            uint32_t how = 0u;
            if (i <= rhi) {
                const int j = d - i;
                const int dg = (i > 0 && j > 0 && i - 1 >= lo2 && i - 1 <= hi2) ? A2[(i - 1) & mask] : NEG;
                const int up = (i > 0 && i - 1 >= lo1 && i - 1 <= hi1) ? A1[(i - 1) & mask] : NEG;
                const int lf = (j > 0 && i >= lo1 && i <= hi1) ? A1[i & mask] : NEG;
                int sub = ka.sc.mismatch;
                if (i > 0 && j > 0 &&
                    stream_code(ka.wa, it.a_pos, dir, it.m, i - 1) ==
                        stream_code(ka.wb, it.b_pos, dir, it.n, j - 1))
                    sub = ka.sc.match;
                const int sd = dg + sub, su = up + ka.sc.gap, sl = lf + ka.sc.gap;
                const int s = max(sd, max(su, sl));
                how = (sd == s) ? 0u : (su == s) ? 1u : 2u;  // T1
                const bool live = s >= T;
                A0[i & mask] = live ? s : NEG;
                if (live) {
                    if (s > v.mx) {
                        v.mx = s;
                        v.arg = i;
                    }
                    v.first = min(v.first, i);
                    v.last = i;
                }
            }
            if (RECORD) {
                // 16 codes per word: OR the half-warp's codes together
                uint32_t wv = how << (2 * (threadIdx.x & 15));
#pragma unroll
                for (int o = 8; o >= 1; o >>= 1) wv |= __shfl_xor_sync(FULL, wv, o);
                const int k = i0 - rlo + int(threadIdx.x);  // cell index in the anti-diagonal
                if ((threadIdx.x & 15) == 0 && k < width) t.codes[wbase + (k >> 4)] = wv;
            }
        }
        wbase += uint64_t(width + 15) >> 4;
        words += uint64_t(width + 15) >> 4;
        const TbRed b = tb_reduce(v, sh);
        if (b.last < 0) break;
        if (b.mx > best) {
            best = b.mx;
            bi = b.arg;
            bj = d - b.arg;
            words_best = words;
        }
        lo2 = lo1;
        hi2 = hi1;
        lo1 = b.first;
        hi1 = b.last;
        int32_t* tmp = A2;
        A2 = A1;
        A1 = A0;
        A0 = tmp;
    }
    if (!RECORD && threadIdx.x == 0) {
        TbItem r;
        r.best = status ? 0 : best;
        r.bi = status ? 0 : bi;
        r.bj = status ? 0 : bj;
        r.status = status;
        r.words = status ? 0 : words_best;
        r.wide = cap > kSmemCap ? 1 : 0;
        r.pad = 0;
        t.info[id] = r;
    }
}

template <bool RECORD>
__global__ void __launch_bounds__(kTbThreads) k_tb_sweep(TbArgs t) {
    __shared__ TbRed sh[kTbWarps];
    __shared__ int32_t sring[3 * kSmemCap];
    __shared__ int s_wide;
    int32_t* R = t.ka.ring + size_t(blockIdx.x) * 3u * t.ka.ring_cap;
    const int gcap = int(t.ka.ring_cap);
    for (uint32_t id = blockIdx.x; id < t.ka.n_items; id += gridDim.x) {
        const Item it = t.ka.items[id];
        if (it.flags & ITEM_SKIP) {
            if (!RECORD && threadIdx.x == 0) t.info[id] = TbItem{0, 0, 0, 0, 0ull, 0, 0};
            continue;
        }
        if (RECORD) {
            if (t.info[id].status || t.info[id].bi + t.info[id].bj == 0) continue;
            if (t.info[id].wide) tb_sweep<true>(t, id, R, gcap, sh);
            else tb_sweep<true>(t, id, sring, kSmemCap, sh);
        } else {
            const bool fits = gcap > kSmemCap;
            if (fits) tb_sweep<false>(t, id, sring, kSmemCap, sh);
            __syncthreads();
            if (threadIdx.x == 0) s_wide = !fits || t.info[id].status == TB_WIDE;
            __syncthreads();
            if (s_wide) tb_sweep<false>(t, id, R, gcap, sh);
        }
        __syncthreads();
    }
}

// per pair: run-length codes bound and the anti-diagonal table sizes
__global__ void k_tb_sizes(const TbItem* __restrict__ info, const PairInfo* __restrict__ pi,
                           const uint32_t* __restrict__ seeds, uint32_t n_pairs,
                           uint64_t* __restrict__ item_words, uint64_t* __restrict__ item_ads,
                           uint64_t* __restrict__ pair_codes) {
    for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < n_pairs;
         p += gridDim.x * blockDim.x) {
        uint64_t codes = 1;
        for (int s = 0; s < 2; ++s) {
            const TbItem x = info[2 * p + s];
            item_words[2 * p + s] = x.words;
            item_ads[2 * p + s] = uint64_t(x.bi + x.bj) + 1;
            codes += uint64_t(x.bi) + uint64_t(x.bj);
        }
        pair_codes[p] = codes + seeds[5 * p + 4];
    }
}

struct RleOut {
    uint32_t* out;
    uint64_t n;
    __device__ void put(uint32_t op, uint32_t len) {
        if (!len) return;
        if (n && (out[n - 1] & 15u) == op) out[n - 1] += len << 4;
        else out[n++] = (len << 4) | op;
    }
};

// predecessor code of cell (i, j); a cell outside the recorded tables reads
// as a diagonal step (it cannot occur on a walk from a best cell)
__device__ __forceinline__ uint32_t tb_code(const TbArgs& t, uint64_t abase, int i, int j) {
    const int d = i + j;
    const int k = i - t.ad_rlo[abase + d];
    if (k < 0) return 0u;
    const uint64_t w = t.ad_word[abase + d] + uint64_t(k >> 4);
    if (w >= t.n_words) return 0u;
    return (t.codes[w] >> (2 * (k & 15))) & 3u;
}

__global__ void k_tb_walk(TbArgs t, const PairInfo* __restrict__ pi,
                          const uint32_t* __restrict__ seeds, uint32_t n_pairs,
                          const uint64_t* __restrict__ op_start, uint32_t* __restrict__ ops,
                          uint32_t* __restrict__ op_count) {
    for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < n_pairs;
         p += gridDim.x * blockDim.x) {
        const TbItem L = t.info[2 * p], Rr = t.info[2 * p + 1];
        if (pi[p].status || L.status || Rr.status) {
            op_count[p] = 0;
            continue;
        }
        uint32_t* region = ops + op_start[p];
        RleOut o{region, 0};
        // left: the walk from the best cell back to (0,0) runs over the
        // reversed prefixes, i.e. in the sequences' own order
        {
            int i = L.bi, j = L.bj;
            const uint64_t ab = t.ad_off[2 * p];
            while (i + j > 0) {
                const uint32_t h = tb_code(t, ab, i, j);
                o.put(h, 1);
                if (h == 0) { --i; --j; } else if (h == 1) { --i; } else { --j; }
            }
        }
        o.put(0, seeds[5 * p + 4]);
        // right: the walk comes out last-first; write it downwards from the
        // region's end, then move it up behind the front part
        const uint64_t bound = uint64_t(L.bi) + L.bj + seeds[5 * p + 4] + Rr.bi + Rr.bj + 1;
        uint64_t tail = bound;  // codes in [tail, bound) read upwards are in order
        {
            int i = Rr.bi, j = Rr.bj;
            const uint64_t ab = t.ad_off[2 * p + 1];
            uint32_t cur = 3u, len = 0;
            while (i + j > 0) {
                const uint32_t h = tb_code(t, ab, i, j);
                if (h == cur) {
                    ++len;
                } else {
                    if (len) region[--tail] = (len << 4) | cur;
                    cur = h;
                    len = 1;
                }
                if (h == 0) { --i; --j; } else if (h == 1) { --i; } else { --j; }
            }
            if (len) region[--tail] = (len << 4) | cur;
        }
        for (uint64_t q = tail; q < bound; ++q) o.put(region[q] & 15u, region[q] >> 4);
        op_count[p] = uint32_t(o.n);
    }
}

struct TbScratch {
    cudaStream_t s;
    std::vector<void*> ptrs;
    bool ok = true;
    explicit TbScratch(cudaStream_t st) : s(st) {}
    template <typename T>
    T* get(size_t n) {
        void* p = nullptr;
        if (!ok || cudaMallocAsync(&p, std::max<size_t>(n, 1) * sizeof(T), s) != cudaSuccess) {
            ok = false;
            return nullptr;
        }
        ptrs.push_back(p);
        return static_cast<T*>(p);
    }
    ~TbScratch() {
        for (void* p : ptrs) cudaFreeAsync(p, s);
    }
};

// exclusive prefix of v[0, n) into out[0, n]; returns out[n] (synchronises)
bool tb_scan(TbScratch& sc, uint64_t* v, uint64_t n, uint64_t* out, uint64_t* total) {
    cudaMemsetAsync(v + n, 0, sizeof(uint64_t), sc.s);
    size_t tb = 0;
    cub::DeviceScan::ExclusiveSum(nullptr, tb, v, out, n + 1, sc.s);
    void* tmp = sc.get<char>(tb);
    if (!sc.ok) return false;
    cub::DeviceScan::ExclusiveSum(tmp, tb, v, out, n + 1, sc.s);
    return cudaMemcpyAsync(total, out + n, sizeof(uint64_t), cudaMemcpyDeviceToHost, sc.s) ==
               cudaSuccess &&
           cudaStreamSynchronize(sc.s) == cudaSuccess;
}

}  // namespace

namespace {

int run_traceback(int num_sms, const PoolDev& pa, const PoolDev& pb,
                  const logan_seed_t* seeds, uint32_t n_pairs, Scoring sc, int32_t X,
                  const int32_t* Xs, uint32_t ring_log2, uint32_t* ops, uint64_t capacity,
                  uint64_t* op_start, uint32_t* op_count, uint64_t* needed, cudaStream_t s) {
    TbScratch S(s);
    const uint32_t n_items = 2u * n_pairs;
    Item* items = S.get<Item>(n_items);
    PairInfo* info = S.get<PairInfo>(n_pairs);
    ExtRes* ext = S.get<ExtRes>(n_items);
    int32_t* mig = S.get<int32_t>(n_items);
    TbItem* tinfo = S.get<TbItem>(n_items);
    // 8 blocks of 256 threads fill an SM (24 KB of shared ring each)
    const int grid = int(std::min<uint32_t>(n_items, uint32_t(num_sms) * 8u));
    const uint32_t cap = 1u << ring_log2;
    int32_t* ring = S.get<int32_t>(size_t(grid) * 3u * cap);
    if (!S.ok) return LOGAN_ENOMEM;
    if (launch_split(pa, pb, seeds, n_pairs, sc, X, Xs, items, info, ext, mig, s) != cudaSuccess)
        return LOGAN_ECUDA;
    TbArgs t{};
    t.ka.wa = pa.words;
    t.ka.wb = pb.words;
    t.ka.items = items;
    t.ka.ext = ext;
    t.ka.ring = ring;
    t.ka.ring_cap = cap;
    t.ka.n_items = n_items;
    t.ka.sc = sc;
    t.info = tinfo;
    k_tb_sweep<false><<<grid, kTbThreads, 0, s>>>(t);
    uint64_t* iw = S.get<uint64_t>(n_items + 1);
    uint64_t* ia = S.get<uint64_t>(n_items + 1);
    uint64_t* pc = S.get<uint64_t>(n_pairs + 1);
    uint64_t* woff = S.get<uint64_t>(n_items + 1);
    uint64_t* aoff = S.get<uint64_t>(n_items + 1);
    if (!S.ok) return LOGAN_ENOMEM;
    k_tb_sizes<<<(n_pairs + 255) / 256, 256, 0, s>>>(tinfo, info,
                                                     reinterpret_cast<const uint32_t*>(seeds),
                                                     n_pairs, iw, ia, pc);
    uint64_t total_words = 0, total_ads = 0, total_codes = 0;
    if (!tb_scan(S, iw, n_items, woff, &total_words) || !tb_scan(S, ia, n_items, aoff, &total_ads) ||
        !tb_scan(S, pc, n_pairs, op_start, &total_codes))
        return S.ok ? LOGAN_ECUDA : LOGAN_ENOMEM;
    *needed = total_codes;
    if (capacity < total_codes) return LOGAN_ENOMEM;
    uint32_t* codes = S.get<uint32_t>(total_words);
    int32_t* ad_rlo = S.get<int32_t>(total_ads);
    uint64_t* ad_word = S.get<uint64_t>(total_ads);
    if (!S.ok) return LOGAN_ENOMEM;
    cudaMemsetAsync(ad_rlo, 0, sizeof(int32_t) * std::max<uint64_t>(total_ads, 1), s);
    cudaMemsetAsync(ad_word, 0, sizeof(uint64_t) * std::max<uint64_t>(total_ads, 1), s);
    t.word_off = woff;
    t.ad_off = aoff;
    t.codes = codes;
    t.ad_rlo = ad_rlo;
    t.ad_word = ad_word;
    t.n_words = total_words;
    k_tb_sweep<true><<<grid, kTbThreads, 0, s>>>(t);
    k_tb_walk<<<(n_pairs + 127) / 128, 128, 0, s>>>(t, info,
                                                    reinterpret_cast<const uint32_t*>(seeds),
                                                    n_pairs, op_start, ops, op_count);
    if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess)
        return LOGAN_ECUDA;
    return LOGAN_OK;
}

}  // namespace

}  // namespace logan

using namespace logan;

extern "C" int logan_traceback_batch(logan_ctx_t* ctx, const logan_seqs_t* A,
                                     const logan_seqs_t* B, const logan_seed_t* seeds,
                                     uint32_t n_pairs, int32_t match, int32_t mismatch,
                                     int32_t gap, int32_t X, const int32_t* X_per_pair,
                                     uint32_t* ops, uint64_t ops_capacity, uint64_t* op_start,
                                     uint32_t* op_count, uint64_t* ops_needed, void* stream) {
    auto bad = [](int32_t v) { return v > kMaxParam || v < -kMaxParam; };
    if (!ctx || !A || !B || !ops_needed || bad(match) || bad(mismatch) || bad(gap) || gap > 0 ||
        mismatch > match || X < 0 || X > kMaxX || n_pairs > 0x7fffffffu)
        return LOGAN_EINVAL;
    *ops_needed = 0;
    if (n_pairs == 0) return LOGAN_OK;
    if (!seeds || !op_start || !op_count || (ops_capacity && !ops)) return LOGAN_EINVAL;
    for (const logan_seqs_t* q : {A, B})
        if (q->packed2bit > 1 || (q->count && (!q->bases || !q->offsets || !q->lengths)))
            return LOGAN_EINVAL;
    int64_t dev = 0, ring_log2 = 16;
    logan_get_option(ctx, LOGAN_OPT_DEVICE, &dev);
    logan_get_option(ctx, LOGAN_OPT_RING_CAP, &ring_log2);
    int prev = 0;
    cudaGetDevice(&prev);
    if (prev != int(dev) && cudaSetDevice(int(dev)) != cudaSuccess) return LOGAN_ECUDA;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, int(dev));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const bool same = A->bases == B->bases && A->offsets == B->offsets &&
                      A->lengths == B->lengths && A->count == B->count &&
                      A->packed2bit == B->packed2bit && A->pool_bases == B->pool_bases;
    int rc = LOGAN_OK;
    {
        TbScratch S(s);
        auto pool = [&](const logan_seqs_t* q, PoolDev& d) {
            d = {q->bases, q->offsets, q->lengths, q->count, q->packed2bit, q->pool_bases,
                 static_cast<const uint32_t*>(q->bases), nullptr};
            uint8_t* badv = S.get<uint8_t>(q->count);
            uint32_t* words = q->packed2bit ? nullptr : S.get<uint32_t>((q->pool_bases + 15) / 16 + 1);
            if (!S.ok) return false;
            d.bad = badv;
            if (!q->packed2bit) {
                d.words = words;
                if (q->pool_bases && launch_pack(d, words, s) != cudaSuccess) return false;
            }
            return launch_validate(d, s) == cudaSuccess;
        };
        PoolDev pa, pb;
        if (!pool(A, pa) || (!same && !pool(B, pb))) {
            rc = S.ok ? LOGAN_ECUDA : LOGAN_ENOMEM;
        } else {
            if (same) pb = pa;
            rc = run_traceback(sms, pa, pb, seeds, n_pairs, Scoring{match, mismatch, gap}, X,
                               X_per_pair, uint32_t(ring_log2), ops, ops_capacity, op_start,
                               op_count, ops_needed, s);
        }
    }
    if (prev != int(dev)) cudaSetDevice(prev);
    return rc;
}
