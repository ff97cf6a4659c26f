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
// Steps:
//   1 the batch pipeline (logan_extend_batch) gives every extension its
//     best cell (bi, bj), hence its best anti-diagonal d* = bi + bj, and its
//     cells; its workspace keeps the packed sequences and the split items;
//   2 per extension the storage of its predecessor codes: every
//     anti-diagonal 1..d* starts on a 16-cell word, so cells / 16 + d* + 1
//     words suffice; scans give the offsets;
//   3 the sweep again up to d*, one warp per extension with its three
//     anti-diagonals in a shared-memory ring of 512 rows (a band that
//     outgrows it runs again on a block of 256 threads: 2048 rows in shared
//     memory, else a device-memory ring -- the paper's layout, Sec. IV-B),
//     writing for every anti-diagonal its first row, its first word and the
//     2-bit codes of its cells (16 lanes' codes ORed into a word by warp
//     reductions);
//   4 one thread per extension walks back from its best cell (run-length
//     codes, length << 4 | op; op 0 = M, 1 = I, 2 = D), one thread per pair
//     joins the left codes, the seed and the right codes.
// Same cell update and range rules as the extension kernels, so the sweep
// meets the same best cells.
#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_scan.cuh>

#include <algorithm>
#include <climits>
#include <vector>

#include "ctx_ext.h"
#include "internal.h"

#include "../../include/logan.h"

namespace logan {

namespace {

constexpr uint32_t FULL = 0xffffffffu;
constexpr int kTbThreads = 256;
constexpr int kTbWarps = kTbThreads / 32;

// ring arrays: 3 x 512 int32 per warp in shared memory (8 warps: 48 KB per
// block), 3 x 2048 per block of 256 threads (24 KB), else the device-memory
// ring; an array holds a band of up to its size - 2 rows
constexpr int kWarpCap = 512;
constexpr int kSmemCap = 2048;
constexpr int TB_WIDE = 1;       // status: retry in the device-memory ring
constexpr int TB_WARP_WIDE = 2;  // status: wide from the start, swept by a block
constexpr int TB_BOUND = 3;      // status: the codes outgrew the item's words (not expected)
constexpr int TB_OUTGREW = 4;    // status: outgrew a warp's ring, retry on a block

struct TbRed {
    int mx, first, last;
};

__device__ __forceinline__ TbRed tb_reduce(TbRed v, TbRed* sh) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int mx = __reduce_max_sync(FULL, v.mx);
    int first = __reduce_min_sync(FULL, v.first);
    int last = __reduce_max_sync(FULL, v.last);
    if (lane == 0) sh[w] = TbRed{mx, first, last};
    __syncthreads();
    TbRed p = lane < kTbWarps ? sh[lane] : TbRed{NEG, INT_MAX, -1};
    mx = __reduce_max_sync(FULL, p.mx);
    first = __reduce_min_sync(FULL, p.first);
    last = __reduce_max_sync(FULL, p.last);
    __syncthreads();
    return TbRed{mx, first, last};
}

struct TbItem {  // per item: its best cell and the recording sweep's status
    int32_t bi, bj, status;
    int32_t wide;  // swept by a block from the start (the warp sweep leaves it alone)
};

struct TbArgs {
    KernelArgs ka;             // pools, items, scoring, ring
    TbItem* info;              // per item
    const uint64_t* word_off;  // per item (+1): its words are [word_off[id], word_off[id + 1])
    const uint64_t* ad_off;    // per item: first entry of its anti-diagonal table
    uint32_t* codes;           // 2-bit predecessor codes
    int32_t* ad_rlo;           // per anti-diagonal: first evaluated row
    uint64_t* ad_word;         // per anti-diagonal: first word
    uint64_t n_words;          // size of codes (reads beyond it are refused)
    unsigned long long* cells; // nullable: cells of the completed sweeps
    const uint32_t* order;     // item ids, the most code words first
    unsigned int* next;        // pop cursors into order: [0] warps, [1] and [2] the block passes
};

// The sweep of one item up to its best anti-diagonal by TW threads (a warp,
// or the block of kTbThreads), writing the predecessor codes; the item's
// status gets 0, or a reason to retry in a wider ring.
template <int TW>
__device__ void tb_record(const TbArgs& t, uint32_t id, int32_t* R, int cap, TbRed* sh) {
    static_assert(TW == 32 || TW == kTbThreads, "a warp or the whole block");
    const int tid = TW == 32 ? int(threadIdx.x & 31u) : int(threadIdx.x);
    const KernelArgs& ka = t.ka;
    const Item it = ka.items[id];
    const int dir = (it.flags & ITEM_LEFT) ? -1 : 1;
    const int m = int(it.m), n = int(it.n), X = it.X;
    // code of stream index q: bits 2 (r + dir q) of the words from wp
    // (r + dir q may be negative: the shifts floor)
    const uint32_t* wpa = ka.wa + (it.a_pos >> 4);
    const uint32_t* wpb = ka.wb + (it.b_pos >> 4);
    const int ra = int(it.a_pos & 15), rb = int(it.b_pos & 15);
    const int mask = cap - 1;
    // Each ring array holds one anti-diagonal e at rows rlo_e - 1 .. rhi_e + 1:
    // the evaluated rows (NEG when pruned) and NEG at the two rows around
    // them.  Every predecessor that anti-diagonals e + 1 and e + 2 read lies
    // in that span (their ranges start at or above e's first live row and
    // end at most one row above e's last), so a missing predecessor reads
    // as NEG with no range test.
    int32_t* A0 = R;
    int32_t* A1 = R + cap;
    int32_t* A2 = R + 2 * cap;
    const int dstar = t.info[id].bi + t.info[id].bj;
    if (tid == 0) {
        A1[mask] = NEG;  // d = 0: rows -1, 0, 1
        A1[0] = 0;
        A1[1] = NEG;
        A2[mask] = NEG;  // d = -1: the diagonal reads of d = 1
        A2[0] = NEG;
    }
    if constexpr (TW == 32) __syncwarp();
    else __syncthreads();
    int lo1 = 0, hi1 = 0;
    int best = 0, status = 0;
    unsigned long long cells = 0;
    uint64_t wbase = t.word_off[id];
    const uint64_t wend = t.word_off[id + 1];
    const uint64_t abase = t.ad_off[id];
    for (int d = 1; d <= dstar; ++d) {
        const int rlo = max(lo1, d - n), rhi = min(hi1 + 1, m);
        if (rlo > rhi) break;
        const int width = rhi - rlo + 1;
        if (width + 2 > cap) {
            status = TW == 32 ? TB_OUTGREW : cap < int(ka.ring_cap) ? TB_WIDE : LOGAN_ERANGE;
            break;
        }
        const uint64_t nw = uint64_t(width + 15) >> 4;
        if (wbase + nw > wend) {
            status = TB_BOUND;
            break;
        }
        if (tid == 0) {
            t.ad_rlo[abase + d] = rlo;
            t.ad_word[abase + d] = wbase;
            A0[(rlo - 1) & mask] = NEG;
            A0[(rhi + 1) & mask] = NEG;
        }
        cells += unsigned(width);
        const int T = best - X;
        TbRed v{NEG, INT_MAX, -1};
        // whole strides of the unit so that every lane takes part in the
        // code packing
        for (int i0 = rlo; i0 <= rhi; i0 += TW) {
            const int i = i0 + tid;
            uint32_t how = 0u;
            if (i <= rhi) {
                const int j = d - i;
                const int dg = A2[(i - 1) & mask];
                const int up = A1[(i - 1) & mask];
                const int lf = A1[i & mask];
                int sub = ka.sc.mismatch;
                if (i > 0 && j > 0) {  // (a diagonal step exists: both bases are in range)
                    const int ta = ra + dir * (i - 1), tb = rb + dir * (j - 1);
                    const uint32_t ca = __ldg(wpa + (ta >> 4)) >> (uint32_t(ta & 15) * 2u);
                    const uint32_t cb = __ldg(wpb + (tb >> 4)) >> (uint32_t(tb & 15) * 2u);
                    if (((ca ^ cb) & 3u) == 0u) sub = ka.sc.match;
                }
                const int sd = dg + sub, su = up + ka.sc.gap, sl = lf + ka.sc.gap;
                const int s = max(sd, max(su, sl));
                how = (sd == s) ? 0u : (su == s) ? 1u : 2u;  // T1
                const bool live = s >= T;
                A0[i & mask] = live ? s : NEG;
                if (live) {
                    v.mx = max(v.mx, s);
                    v.first = min(v.first, i);
                    v.last = i;
                }
            }
            // 16 codes per word: each half-warp's codes ORed together
            const uint32_t mine = how << (2u * uint32_t(tid & 15));
            const uint32_t wlo = __reduce_or_sync(FULL, (tid & 16) ? 0u : mine);
            const uint32_t whi = __reduce_or_sync(FULL, (tid & 16) ? mine : 0u);
            const int k = i0 - rlo + tid;  // cell index in the anti-diagonal
            if ((tid & 15) == 0 && k < width) t.codes[wbase + (k >> 4)] = (tid & 16) ? whi : wlo;
        }
        wbase += nw;
        TbRed b;
        if constexpr (TW == 32) {
            b.mx = __reduce_max_sync(FULL, v.mx);
            b.first = __reduce_min_sync(FULL, v.first);
            b.last = __reduce_max_sync(FULL, v.last);
            __syncwarp();  // anti-diagonal d written and d-2 read by every lane
        } else {
            b = tb_reduce(v, sh);
        }
        if (b.last < 0) break;
        best = max(best, b.mx);
        lo1 = b.first;
        hi1 = b.last;
        int32_t* tmp = A2;
        A2 = A1;
        A1 = A0;
        A0 = tmp;
    }
    if (tid == 0) {
        t.info[id].status = status;
        if (t.cells && status == 0) atomicAdd(t.cells, cells);
    }
}

// The recording sweep, one item per warp; warps pop the items, the largest
// first, so that the sweep does not end on a few warps holding several long
// items each while the rest of the GPU idles.
__global__ void __launch_bounds__(kTbThreads) k_tb_record_warp(TbArgs t) {
    __shared__ int32_t wring[kTbWarps][3 * kWarpCap];
    const int w = int(threadIdx.x >> 5);
    for (;;) {
        unsigned int slot = 0u;
        if ((threadIdx.x & 31u) == 0u) slot = atomicAdd(&t.next[0], 1u);
        slot = __shfl_sync(FULL, slot, 0);
        if (slot >= t.ka.n_items) break;
        const uint32_t id = t.order[slot];
        const TbItem x = t.info[id];
        if (x.wide || x.status || x.bi + x.bj == 0) continue;
        tb_record<32>(t, id, wring[w], kWarpCap, nullptr);
        __syncwarp();
    }
}

// The items of status `which`, one per block: 2048 rows in shared memory,
// else the block's slice of the device-memory ring.  Two passes: the items
// wide from the start (TB_WARP_WIDE, beside the warp sweep, which leaves
// them alone), then those that outgrew a warp's ring (TB_OUTGREW).
__global__ void __launch_bounds__(kTbThreads) k_tb_record_block(TbArgs t, int which, int cursor) {
    __shared__ TbRed sh[kTbWarps];
    __shared__ int32_t sring[3 * kSmemCap];
    __shared__ int s_wide;
    __shared__ unsigned int s_slot;
    int32_t* R = t.ka.ring + size_t(blockIdx.x) * 3u * t.ka.ring_cap;
    const int gcap = int(t.ka.ring_cap);
    for (;;) {
        if (threadIdx.x == 0) s_slot = atomicAdd(&t.next[cursor], 1u);
        __syncthreads();
        const unsigned int slot = s_slot;
        __syncthreads();
        if (slot >= t.ka.n_items) break;
        const uint32_t id = t.order[slot];
        if (t.info[id].status != which) continue;
        const bool fits = gcap > kSmemCap;
        if (fits) tb_record<kTbThreads>(t, id, sring, kSmemCap, sh);
        __syncthreads();
        if (threadIdx.x == 0) s_wide = !fits || t.info[id].status == TB_WIDE;
        __syncthreads();
        if (s_wide) tb_record<kTbThreads>(t, id, R, gcap, sh);
        __syncthreads();
    }
}

// Per item from the extension's results: best cell, status and sizes (code
// words, anti-diagonal table entries); per pair the run-length codes bound.
__global__ void k_tb_prepare(const Item* __restrict__ items, const ExtRes* __restrict__ ext,
                             const PairInfo* __restrict__ pi,
                             const uint32_t* __restrict__ seeds, uint32_t n_pairs,
                             TbItem* __restrict__ info, uint64_t* __restrict__ item_words,
                             uint64_t* __restrict__ item_ads, uint64_t* __restrict__ pair_codes) {
    for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < n_pairs;
         p += gridDim.x * blockDim.x) {
        uint64_t codes = 1;
        for (int s = 0; s < 2; ++s) {
            const uint32_t id = 2 * p + s;
            const ExtRes e = ext[id];
            const int32_t st = pi[p].status ? pi[p].status : e.status;
            TbItem x{st ? 0 : e.bi, st ? 0 : e.bj, st, 0};
            const uint64_t dstar = uint64_t(x.bi) + uint64_t(x.bj);
            // a sweep of at most m + n anti-diagonals whose cells average
            // more than kWarpCap / 2 per anti-diagonal is swept by a block
            // from the start (a warp would outgrow its ring)
            const Item it = items[id];
            if (!st && dstar &&
                uint64_t(e.cells) > uint64_t(kWarpCap / 2) * (uint64_t(it.m) + uint64_t(it.n))) {
                x.status = TB_WARP_WIDE;
                x.wide = 1;
            }
            info[id] = x;
            // anti-diagonals 1..d* hold at most the extension's cells, each
            // starting on a word
            item_words[id] = dstar ? uint64_t(e.cells) / 16u + dstar + 1u : 0u;
            item_ads[id] = dstar + 1u;
            codes += dstar;
        }
        pair_codes[p] = codes + seeds[5 * p + 4];
    }
}

__global__ void k_tb_iota(uint32_t* __restrict__ ids, uint32_t n) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) ids[i] = i;
}

// predecessor code of the cell in row i of the anti-diagonal whose table
// entry is (rlo, word); a cell outside the recorded words reads as a
// diagonal step (it cannot occur on a walk from a best cell)
__device__ __forceinline__ uint32_t tb_code(const TbArgs& t, int rlo, uint64_t word, int i) {
    const int k = i - rlo;
    if (k < 0) return 0u;
    const uint64_t w = word + uint64_t(k >> 4);
    if (w >= t.n_words) return 0u;
    return (t.codes[w] >> (2 * (k & 15))) & 3u;
}

// One thread per extension walks from its best cell back to (0,0).  The
// left extension's walk lists its operations in the sequences' order and
// goes to the front of the pair's region; the right one's come out
// last-first and go downwards from the region's end.  side_n gets the
// left's code count and the right's first code.
__global__ void k_tb_walk(TbArgs t, const uint32_t* __restrict__ seeds, uint32_t n_pairs,
                          const uint64_t* __restrict__ op_start, uint32_t* __restrict__ ops,
                          uint64_t* __restrict__ side_n) {
    const uint32_t n_items = 2u * n_pairs;
    for (uint32_t id = blockIdx.x * blockDim.x + threadIdx.x; id < n_items;
         id += gridDim.x * blockDim.x) {
        const uint32_t p = id >> 1;
        const bool right = (id & 1u) != 0u;
        const TbItem x = t.info[id];
        const TbItem o = t.info[id ^ 1u];
        if (x.status || o.status) continue;
        uint32_t* region = ops + op_start[p];
        const TbItem& L = right ? o : x;
        const TbItem& Rr = right ? x : o;
        const uint64_t bound = uint64_t(L.bi) + L.bj + seeds[5 * p + 4] + Rr.bi + Rr.bj + 1;
        uint64_t at = right ? bound : 0;
        int i = x.bi, d = x.bi + x.bj;
        const uint64_t ab = t.ad_off[id];
        uint32_t cur = 3u, len = 0;
        if (d > 0) {
            int rlo = t.ad_rlo[ab + d];
            uint64_t word = t.ad_word[ab + d];
            while (d > 0) {
                // the table entries of both possible next anti-diagonals load
                // alongside this step's code
                const int d1 = d - 1, d2 = max(d - 2, 0);
                const int r1 = t.ad_rlo[ab + d1], r2 = t.ad_rlo[ab + d2];
                const uint64_t w1 = t.ad_word[ab + d1], w2 = t.ad_word[ab + d2];
                const uint32_t h = tb_code(t, rlo, word, i);
                if (h == cur) {
                    ++len;
                } else {
                    if (len) {
                        if (right) region[--at] = (len << 4) | cur;
                        else region[at++] = (len << 4) | cur;
                    }
                    cur = h;
                    len = 1;
                }
                if (h == 0u) {
                    --i;
                    d = d2;
                    rlo = r2;
                    word = w2;
                } else {
                    i -= h == 1u ? 1 : 0;
                    d = d1;
                    rlo = r1;
                    word = w1;
                }
            }
        }
        if (len) {
            if (right) region[--at] = (len << 4) | cur;
            else region[at++] = (len << 4) | cur;
        }
        side_n[id] = at;
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

// Per pair: the left codes, k M for the seed, then the right codes moved up
// behind them (runs that meet merge).
__global__ void k_tb_join(const TbItem* __restrict__ info, const uint32_t* __restrict__ seeds,
                          uint32_t n_pairs, const uint64_t* __restrict__ op_start,
                          uint32_t* __restrict__ ops, const uint64_t* __restrict__ side_n,
                          uint32_t* __restrict__ op_count) {
    for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < n_pairs;
         p += gridDim.x * blockDim.x) {
        const TbItem L = info[2 * p], Rr = info[2 * p + 1];
        if (L.status || Rr.status) {
            op_count[p] = 0;
            continue;
        }
        uint32_t* region = ops + op_start[p];
        RleOut o{region, side_n[2 * p]};
        o.put(0, seeds[5 * p + 4]);
        const uint64_t bound = uint64_t(L.bi) + L.bj + seeds[5 * p + 4] + Rr.bi + Rr.bj + 1;
        for (uint64_t q = side_n[2 * p + 1]; q < bound; ++q) o.put(region[q] & 15u, region[q] >> 4);
        op_count[p] = uint32_t(o.n);
    }
}

struct TbScratch {
    cudaStream_t s;
    cudaMemPool_t pool;  // the context's scratch pool (null: the default one)
    std::vector<void*> ptrs;
    bool ok = true;
    // a second stream and its fork / join events, for the concurrent sweeps
    cudaStream_t aux = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    TbScratch(cudaStream_t st, cudaMemPool_t p) : s(st), pool(p) {
        ok = cudaStreamCreateWithFlags(&aux, cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&join, cudaEventDisableTiming) == cudaSuccess;
    }
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
    ~TbScratch() {
        // (after an error between the fork and the join, aux may still run)
        if (aux) cudaStreamSynchronize(aux);
        for (void* p : ptrs) cudaFreeAsync(p, s);
        if (join) cudaEventDestroy(join);
        if (fork) cudaEventDestroy(fork);
        if (aux) cudaStreamDestroy(aux);
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

// CUDA events around the steps of one timed call (LOGAN_OPT_TIMING)
struct TbClock {
    enum { START, EXT_END, REC_START, REC_END, END, N };
    cudaEvent_t ev[N] = {};
    bool on = false;
    uint32_t launches = 0;  // kernels of this library launched by the call
    uint64_t words = 0;
    unsigned long long* dcells = nullptr;  // device counter of recorded cells
    explicit TbClock(bool timing) {
        if (!timing) return;
        on = true;
        for (auto& e : ev)
            if (cudaEventCreate(&e) != cudaSuccess) on = false;
    }
    void mark(int k, cudaStream_t s) {
        if (on && cudaEventRecord(ev[k], s) != cudaSuccess) on = false;
    }
    // the elapsed times, once the stream has synchronised
    bool read(logan_traceback_stats_t* st) const {
        if (!on) return false;
        auto ms = [&](int a, int b, float* out) {
            return cudaEventElapsedTime(out, ev[a], ev[b]) == cudaSuccess;
        };
        *st = logan_traceback_stats_t{};
        st->code_words = words;
        st->launches = launches;
        unsigned long long c = 0;
        if (!dcells || cudaMemcpy(&c, dcells, sizeof(c), cudaMemcpyDeviceToHost) != cudaSuccess)
            return false;
        st->record_cells = c;
        return ms(START, EXT_END, &st->sweep_ms) && ms(REC_START, REC_END, &st->record_ms) &&
               ms(REC_END, END, &st->walk_ms) && ms(START, END, &st->total_ms);
    }
    ~TbClock() {
        for (auto& e : ev)
            if (e) cudaEventDestroy(e);
    }
};

int run_traceback(int num_sms, const ExtensionViews& v, const logan_seed_t* seeds,
                  uint32_t n_pairs, Scoring sc, uint32_t ring_log2, uint32_t* ops,
                  uint64_t capacity, uint64_t* op_start, uint32_t* op_count, uint64_t* needed,
                  cudaStream_t s, TbScratch& S, TbClock& clk) {
    const uint32_t n_items = 2u * n_pairs;
    const uint32_t* sd = reinterpret_cast<const uint32_t*>(seeds);
    TbItem* tinfo = S.get<TbItem>(n_items);
    uint64_t* iw = S.get<uint64_t>(n_items + 1);
    uint64_t* ia = S.get<uint64_t>(n_items + 1);
    uint64_t* pc = S.get<uint64_t>(n_pairs + 1);
    uint64_t* woff = S.get<uint64_t>(n_items + 1);
    uint64_t* aoff = S.get<uint64_t>(n_items + 1);
    uint64_t* side_n = S.get<uint64_t>(n_items);
    if (!S.ok) return LOGAN_ENOMEM;
    k_tb_prepare<<<(n_pairs + 255) / 256, 256, 0, s>>>(v.items, v.ext, v.info, sd, n_pairs,
                                                       tinfo, iw, ia, pc);
    ++clk.launches;
    uint64_t total_words = 0, total_ads = 0, total_codes = 0;
    if (!tb_scan(S, iw, n_items, woff, &total_words) || !tb_scan(S, ia, n_items, aoff, &total_ads) ||
        !tb_scan(S, pc, n_pairs, op_start, &total_codes))
        return S.ok ? LOGAN_ECUDA : LOGAN_ENOMEM;
    *needed = total_codes;
    if (capacity < total_codes) return LOGAN_ENOMEM;
    // 8 blocks of 256 threads fill an SM (24 KB of shared ring each)
    const int grid = int(std::min<uint32_t>(n_items, uint32_t(num_sms) * 8u));
    const int wgrid = int(std::min<uint32_t>((n_items + kTbWarps - 1) / kTbWarps,
                                             uint32_t(num_sms) * 4u));
    const uint32_t cap = 1u << ring_log2;
    int32_t* ring = S.get<int32_t>(size_t(grid) * 3u * cap);
    uint32_t* codes = S.get<uint32_t>(total_words);
    int32_t* ad_rlo = S.get<int32_t>(total_ads);
    uint64_t* ad_word = S.get<uint64_t>(total_ads);
    if (clk.on) clk.dcells = S.get<unsigned long long>(1);
    if (!S.ok) return LOGAN_ENOMEM;
    // the recording sweeps pop the items the most code words first
    uint32_t* ids = S.get<uint32_t>(n_items);
    uint32_t* order = S.get<uint32_t>(n_items);
    uint64_t* keys = S.get<uint64_t>(n_items);
    unsigned int* next = S.get<unsigned int>(3);
    size_t sort_bytes = 0;
    cub::DeviceRadixSort::SortPairsDescending(nullptr, sort_bytes, iw, keys, ids, order,
                                              int(n_items), 0, 64, s);
    void* sort_tmp = S.get<char>(sort_bytes);
    if (!S.ok) return LOGAN_ENOMEM;
    k_tb_iota<<<(n_items + 255) / 256, 256, 0, s>>>(ids, n_items);
    ++clk.launches;
    if (cub::DeviceRadixSort::SortPairsDescending(sort_tmp, sort_bytes, iw, keys, ids, order,
                                                  int(n_items), 0, 64, s) != cudaSuccess)
        return LOGAN_ECUDA;
    cudaMemsetAsync(next, 0, 3 * sizeof(unsigned int), s);
    cudaMemsetAsync(ad_rlo, 0, sizeof(int32_t) * std::max<uint64_t>(total_ads, 1), s);
    cudaMemsetAsync(ad_word, 0, sizeof(uint64_t) * std::max<uint64_t>(total_ads, 1), s);
    if (clk.dcells) cudaMemsetAsync(clk.dcells, 0, sizeof(unsigned long long), s);
    TbArgs t{};
    t.ka.wa = v.wa;
    t.ka.wb = v.wb;
    t.ka.items = v.items;
    t.ka.ring = ring;
    t.ka.ring_cap = cap;
    t.ka.n_items = n_items;
    t.ka.sc = sc;
    t.info = tinfo;
    t.word_off = woff;
    t.ad_off = aoff;
    t.codes = codes;
    t.ad_rlo = ad_rlo;
    t.ad_word = ad_word;
    t.n_words = total_words;
    t.cells = clk.dcells;
    t.order = order;
    t.next = next;
    clk.mark(TbClock::REC_START, s);
    // the block sweep of the items wide from the start runs beside the warp
    // sweep (it holds a few SMs for long, the warp sweep fills the rest); the
    // block sweep of the items that outgrew a warp's ring follows both
    if (cudaEventRecord(S.fork, s) != cudaSuccess || cudaStreamWaitEvent(S.aux, S.fork, 0) != cudaSuccess)
        return LOGAN_ECUDA;
    k_tb_record_block<<<grid, kTbThreads, 0, s>>>(t, TB_WARP_WIDE, 1);
    k_tb_record_warp<<<wgrid, kTbThreads, 0, S.aux>>>(t);
    if (cudaEventRecord(S.join, S.aux) != cudaSuccess || cudaStreamWaitEvent(s, S.join, 0) != cudaSuccess)
        return LOGAN_ECUDA;
    k_tb_record_block<<<grid, kTbThreads, 0, s>>>(t, TB_OUTGREW, 2);
    clk.mark(TbClock::REC_END, s);
    k_tb_walk<<<(n_items + 127) / 128, 128, 0, s>>>(t, sd, n_pairs, op_start, ops, side_n);
    k_tb_join<<<(n_pairs + 127) / 128, 128, 0, s>>>(tinfo, sd, n_pairs, op_start, ops, side_n,
                                                    op_count);
    clk.mark(TbClock::END, s);
    clk.launches += 5;
    clk.words = total_words;
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
    int64_t dev = 0, ring_log2 = 16, timing = 0;
    logan_get_option(ctx, LOGAN_OPT_DEVICE, &dev);
    logan_get_option(ctx, LOGAN_OPT_RING_CAP, &ring_log2);
    logan_get_option(ctx, LOGAN_OPT_TIMING, &timing);
    int prev = 0;
    cudaGetDevice(&prev);
    if (prev != int(dev) && cudaSetDevice(int(dev)) != cudaSuccess) return LOGAN_ECUDA;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, int(dev));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int rc = LOGAN_OK;
    {
        TbClock clk(timing != 0);
        TbScratch S(s, ctx_scratch_pool(ctx));
        size_t ws_bytes = 0;
        rc = logan_workspace_size(ctx, A, B, n_pairs, &ws_bytes);
        char* ws = rc == LOGAN_OK ? S.get<char>(ws_bytes) : nullptr;
        logan_result_t* res = S.get<logan_result_t>(n_pairs);
        if (rc == LOGAN_OK && !S.ok) rc = LOGAN_ENOMEM;
        // step 1: the batch pipeline (best cells, cells, packed pools, items)
        clk.mark(TbClock::START, s);
        if (rc == LOGAN_OK)
            rc = logan_extend_batch(ctx, A, B, seeds, n_pairs, match, mismatch, gap, X,
                                    X_per_pair, ws, ws_bytes, res, stream);
        clk.mark(TbClock::EXT_END, s);
        if (rc == LOGAN_OK) {
            ExtensionViews v;
            extension_views(ctx, A, B, n_pairs, ws, &v);
            clk.launches += v.launches;
            rc = run_traceback(sms, v, seeds, n_pairs, Scoring{match, mismatch, gap},
                               uint32_t(ring_log2), ops, ops_capacity, op_start, op_count,
                               ops_needed, s, S, clk);
        }
        if (rc == LOGAN_OK && clk.on) {
            TracebackTiming* tt = ctx_traceback_timing(ctx);
            tt->valid = clk.read(&tt->last);
        }
    }
    if (prev != int(dev)) cudaSetDevice(prev);
    return rc;
}

extern "C" int logan_traceback_last_stats(logan_ctx_t* ctx, logan_traceback_stats_t* stats) {
    if (!ctx || !stats) return LOGAN_EINVAL;
    const TracebackTiming* tt = ctx_traceback_timing(ctx);
    if (!tt->valid) return LOGAN_EINVAL;
    *stats = tt->last;
    return LOGAN_OK;
}
