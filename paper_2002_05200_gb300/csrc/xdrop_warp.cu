// X-drop extension with one warp per extension and the band held in
// registers (window levels 0..4: 32 lanes x C cells, C = 1, 2, 4, 8, 16).
//
// Method (paper Sec. III-A recurrence, X-drop rule; Algorithm 1 sweep;
// Algorithm 2 cell update; Sec. IV-A parallel max reduction):
//   anti-diagonal d holds cells (i, d-i).  Lane l owns cells
//   i = base + l*C + k (k < C) of a window [base, base + 32C) that slides up
//   in whole lanes.  The three rolling anti-diagonals (d-2, d-1, d) are
//   three register arrays that swap roles every step (the loop is unrolled
//   three times), so no value moves in memory:
//     up   = S(i-1, j)   on d-1: own register k-1, or lane l-1's C-1 (shuffle)
//     left = S(i, j-1)   on d-1: own register k
//     diag = S(i-1, j-1) on d-2: own register k-1, or lane l-1's C-1 (shuffle)
//   Base codes are 2-bit: a' codes of a lane's cells are fixed while the
//   window stays put; b' codes shift one cell per anti-diagonal (a 2C-bit
//   shift register per lane, fed by one code fetch in lane 0).
//   Per step: the warp max is one __reduce_max_sync; live cells are a
//   ballot, whose first/last set lanes give the trimmed band (Algorithm 1's
//   trims from both ends); the best cell's row is a second ballot, only on
//   steps that improve the best score.
//   A band that outgrows the window is handed to the next, wider level,
//   which recomputes the extension from the start (results are identical;
//   the work of the narrow attempt is lost).
#include "internal.h"

namespace logan {

namespace {

constexpr uint32_t FULL = 0xffffffffu;

struct ExtArgs {
    const uint32_t* wa;
    const uint32_t* wb;
    int64_t apos, bpos;
    int adir, bdir;
    int m, n, X;
    int match, mismatch, gap;
};

struct WState {
    int base, lo, hi, d;
    int best, bi, bj;
    unsigned long long cells;
    uint32_t aw, bw;
    bool overflow;
};

__device__ __forceinline__ uint32_t a_code(const ExtArgs& e, int64_t q) {
    return stream_code(e.wa, e.apos, e.adir, uint32_t(e.m), q);
}
__device__ __forceinline__ uint32_t b_code(const ExtArgs& e, int64_t q) {
    return stream_code(e.wb, e.bpos, e.bdir, uint32_t(e.n), q);
}

// One anti-diagonal step.  Q2 = d-2, Q1 = d-1 on entry; O receives d.
// Returns true when the extension ends (no live cell, empty range, or the
// band left the window -- then st.overflow is set).
template <int C>
__device__ __forceinline__ bool warp_step(const ExtArgs& e, WState& st, int (&Q2)[C],
                                          int (&Q1)[C], int (&O)[C]) {
    constexpr int W = 32 * C;
    constexpr uint32_t MASK2C = (C >= 16) ? 0xffffffffu : ((1u << (2 * C)) - 1u);
    const int lane = threadIdx.x & 31;
    const int rlo = max(st.lo, st.d - e.n);
    const int rhi = min(st.hi + 1, e.m);
    if (rlo > rhi) return true;
    if (rhi >= st.base + W) {
        // slide the window up by s whole lanes, keeping row rlo-1 (the
        // predecessor row of the lowest computed cell) inside it
        const int s = (rlo - 1 - st.base) / C;
        if (s <= 0 || rhi >= st.base + s * C + W) {
            st.overflow = true;
            return true;
        }
#pragma unroll
        for (int k = 0; k < C; ++k) {
            Q2[k] = __shfl_down_sync(FULL, Q2[k], s);
            Q1[k] = __shfl_down_sync(FULL, Q1[k], s);
        }
        uint32_t aw = __shfl_down_sync(FULL, st.aw, s);
        uint32_t bw = __shfl_down_sync(FULL, st.bw, s);
        st.base += s * C;
        if (lane >= 32 - s) {
            const int i0 = st.base + lane * C;
            aw = 0u;
            bw = 0u;
#pragma unroll
            for (int k = 0; k < C; ++k) {
                Q2[k] = NEG;
                Q1[k] = NEG;
                aw |= a_code(e, int64_t(i0) + k - 1) << (2 * k);
                // b' codes as of anti-diagonal d-1: index (d-1) - i - 1
                bw |= b_code(e, int64_t(st.d) - 2 - (i0 + k)) << (2 * k);
            }
        }
        st.aw = aw;
        st.bw = bw;
    }
    st.cells += (unsigned long long)(rhi - rlo + 1);
    // advance the b' shift register to anti-diagonal d
    uint32_t carry = (__shfl_up_sync(FULL, st.bw, 1) >> (2 * (C - 1))) & 3u;
    if (lane == 0) carry = b_code(e, int64_t(st.d) - st.base - 1);
    st.bw = ((st.bw << 2) | carry) & MASK2C;
    int upc = __shfl_up_sync(FULL, Q1[C - 1], 1);
    int dgc = __shfl_up_sync(FULL, Q2[C - 1], 1);
    if (lane == 0) {
        upc = NEG;
        dgc = NEG;
    }
    const uint32_t x = st.aw ^ st.bw;
    const uint32_t eq = ~(x | (x >> 1));  // bit 2k set iff cell k's bases match
    const int i0 = st.base + lane * C;
    const int kmin = rlo - i0, kmax = rhi - i0;
    const int T = st.best - e.X;
    int lmax = NEG;
    uint32_t bits = 0u;
#pragma unroll
    for (int k = 0; k < C; ++k) {
        const int up = k ? Q1[k - 1] : upc;
        const int dg = k ? Q2[k - 1] : dgc;
        const int sub = ((eq >> (2 * k)) & 1u) ? e.match : e.mismatch;
        int s = __viaddmax_s32(max(up, Q1[k]), e.gap, dg + sub);
        const bool live = (k >= kmin) & (k <= kmax) & (s >= T);
        s = live ? s : NEG;
        O[k] = s;
        lmax = max(lmax, s);
        bits |= live ? (1u << k) : 0u;
    }
    const uint32_t vote = __ballot_sync(FULL, bits != 0u);
    if (vote == 0u) return true;
    const int wmax = __reduce_max_sync(FULL, lmax);
    if (wmax > st.best) {
        uint32_t eb = 0u;
#pragma unroll
        for (int k = 0; k < C; ++k) eb |= (O[k] == wmax) ? (1u << k) : 0u;
        const uint32_t ev = __ballot_sync(FULL, eb != 0u);
        const int L = __ffs(ev) - 1;
        const int kk = __ffs(__shfl_sync(FULL, eb, L)) - 1;
        st.best = wmax;
        st.bi = st.base + L * C + kk;
        st.bj = st.d - st.bi;
    }
    const int fl = __ffs(vote) - 1, ll = 31 - __clz(vote);
    const uint32_t fb = __shfl_sync(FULL, bits, fl), lb = __shfl_sync(FULL, bits, ll);
    st.lo = st.base + fl * C + __ffs(fb) - 1;
    st.hi = st.base + ll * C + 31 - __clz(lb);
    st.d += 1;
    return false;
}

template <int C>
__device__ __forceinline__ bool warp_extend(const ExtArgs& e, ExtRes& r) {
    const int lane = threadIdx.x & 31;
    int P0[C], P1[C], P2[C];
#pragma unroll
    for (int k = 0; k < C; ++k) {
        P0[k] = NEG;
        P1[k] = NEG;
        P2[k] = NEG;
    }
    if (lane == 0) P1[0] = 0;  // S(0,0) = 0 on anti-diagonal 0
    WState st;
    st.base = 0;
    st.lo = 0;
    st.hi = 0;
    st.d = 1;
    st.best = 0;
    st.bi = 0;
    st.bj = 0;
    st.cells = 0ull;
    st.overflow = false;
    st.aw = 0u;
    st.bw = 0u;
#pragma unroll
    for (int k = 0; k < C; ++k) st.aw |= a_code(e, int64_t(lane) * C + k - 1) << (2 * k);
    for (;;) {
        if (warp_step<C>(e, st, P0, P1, P2)) break;
        if (warp_step<C>(e, st, P1, P2, P0)) break;
        if (warp_step<C>(e, st, P2, P0, P1)) break;
    }
    r.best = st.best;
    r.bi = st.bi;
    r.bj = st.bj;
    r.status = 0;
    r.cells = st.cells;
    return st.overflow;
}

__device__ __forceinline__ ExtArgs make_args(const KernelArgs& ka, const Item& it) {
    ExtArgs e;
    e.wa = ka.wa;
    e.wb = ka.wb;
    e.apos = it.a_pos;
    e.bpos = it.b_pos;
    e.adir = (it.flags & ITEM_LEFT) ? -1 : 1;
    e.bdir = e.adir;
    e.m = int(it.m);
    e.n = int(it.n);
    e.X = it.X;
    e.match = ka.sc.match;
    e.mismatch = ka.sc.mismatch;
    e.gap = ka.sc.gap;
    return e;
}

// Runs one item at `level` with this warp; escalates on overflow.
template <int C>
__device__ __forceinline__ void warp_run_item(const KernelArgs& ka, uint32_t id, int level) {
    const Item it = ka.items[id];
    const ExtArgs e = make_args(ka, it);
    ExtRes r;
    const bool ovf = warp_extend<C>(e, r);
    if ((threadIdx.x & 31) == 0) {
        if (ovf) {
            const int nl = level + 1 <= int(ka.max_level) ? level + 1 : kNumLevels;
            const unsigned int t = atomicAdd(&ka.counters->tail[nl], 1u);
            ka.queues[size_t(nl) * ka.qcap + t] = id;
        } else {
            ka.ext[id] = r;
            atomicAdd(&ka.counters->cells[level], r.cells);
        }
    }
}

template <int C>
__global__ void __launch_bounds__(128) k_warp_persistent(KernelArgs ka, int level) {
    const int lane = threadIdx.x & 31;
    const unsigned int count = ka.counters->tail[level];
    const uint32_t* q = ka.queues + size_t(level) * ka.qcap;
    for (;;) {
        unsigned int slot = 0u;
        if (lane == 0) slot = atomicAdd(&ka.counters->head[level], 1u);
        slot = __shfl_sync(FULL, slot, 0);
        if (slot >= count) break;
        warp_run_item<C>(ka, q[slot], level);
    }
}

template <int C>
__global__ void __launch_bounds__(128) k_warp_plain(KernelArgs ka, int level) {
    const uint32_t wid = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (wid >= ka.n_items) return;
    if (ka.items[wid].flags & ITEM_SKIP) return;
    warp_run_item<C>(ka, wid, level);
}

}  // namespace

cudaError_t launch_warp_level_persistent(int level, const KernelArgs& ka, int grid,
                                         cudaStream_t s) {
    switch (level) {
        case 0: k_warp_persistent<1><<<grid, 128, 0, s>>>(ka, level); break;
        case 1: k_warp_persistent<2><<<grid, 128, 0, s>>>(ka, level); break;
        case 2: k_warp_persistent<4><<<grid, 128, 0, s>>>(ka, level); break;
        case 3: k_warp_persistent<8><<<grid, 128, 0, s>>>(ka, level); break;
        case 4: k_warp_persistent<16><<<grid, 128, 0, s>>>(ka, level); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_warp_level_plain(int level, const KernelArgs& ka, cudaStream_t s) {
    const unsigned int grid = (ka.n_items + 3u) / 4u;
    if (grid == 0) return cudaSuccess;
    switch (level) {
        case 0: k_warp_plain<1><<<grid, 128, 0, s>>>(ka, level); break;
        case 1: k_warp_plain<2><<<grid, 128, 0, s>>>(ka, level); break;
        case 2: k_warp_plain<4><<<grid, 128, 0, s>>>(ka, level); break;
        case 3: k_warp_plain<8><<<grid, 128, 0, s>>>(ka, level); break;
        case 4: k_warp_plain<16><<<grid, 128, 0, s>>>(ka, level); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

int warp_level_blocks_per_sm(int level) {
    int n = 0;
    cudaError_t e = cudaErrorInvalidValue;
    switch (level) {
        case 0: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_warp_persistent<1>, 128, 0); break;
        case 1: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_warp_persistent<2>, 128, 0); break;
        case 2: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_warp_persistent<4>, 128, 0); break;
        case 3: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_warp_persistent<8>, 128, 0); break;
        case 4: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_warp_persistent<16>, 128, 0); break;
        default: break;
    }
    return e == cudaSuccess ? n : 0;
}

}  // namespace logan
