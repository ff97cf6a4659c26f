// X-drop extension with a multi-warp unit per extension (window level 6:
// 128 threads x 16 rows, level 7: 512 threads x 8 rows, in registers).
// Level 6 runs here in its 32-bit form; when a call's scores fit 16 bits it
// runs packed in one warp instead (xdrop_group16.cu).
//
// Same cell update as the G-lane kernels (paper Sec. III-A recurrence and
// X-drop rule, Algorithm 2), with the anti-diagonal split across warps as in
// the paper's segmented scheme (Sec. IV-A), except that every segment is
// resident at once: thread t of the unit owns cells i = base + t*C + k.
// Across warp boundaries the neighbour values travel through shared memory:
// each warp's last lane publishes its top cell of every anti-diagonal and
// its top b' code; the warp partials (max, first/last live row, best row)
// are combined after one block barrier per anti-diagonal (the shared-memory
// partials of Sec. IV-A).  A window slide moves whole threads through a
// shared-memory exchange (rare: the band moves about half a cell per step).
#include <climits>

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

__device__ __forceinline__ uint32_t a_code(const ExtArgs& e, int64_t q) {
    return stream_code(e.wa, e.apos, e.adir, uint32_t(e.m), q);
}
__device__ __forceinline__ uint32_t b_code(const ExtArgs& e, int64_t q) {
    return stream_code(e.wb, e.bpos, e.bdir, uint32_t(e.n), q);
}

template <int C, int NW>
struct CtaSmem {
    int4 part[2][NW];          // per warp: max, first live row, last live row, best row
    int top[3][NW];            // per warp: top cell of anti-diagonal d (index d % 3)
    uint32_t btop[2][NW];      // per warp: b' codes of the top lane (index d % 2)
    int xbuf[(2 * C + 2) * NW * 32];  // window-slide exchange, [field][thread]
    unsigned int slot;
    int mslot;
};

struct CState {
    int base, lo, hi, d;
    int best, bi, bj;
    unsigned long long cells;
    unsigned long long cells0;  // cells computed before this level (resumed items)
    uint32_t aw, bw;
    bool overflow;
    bool migrated;
    // for saving the band on overflow
    const KernelArgs* ka;
    uint32_t item;
    int level;
};

__device__ __forceinline__ int mod3(int v) { return v % 3; }

template <int C, int NW>
__device__ __forceinline__ bool cta_step(const ExtArgs& e, CState& st, CtaSmem<C, NW>& sm,
                                         int (&Q2)[C], int (&Q1)[C], int (&O)[C]) {
    constexpr int NT = NW * 32, W = NT * C;
    constexpr uint32_t MASK2C = (C >= 16) ? 0xffffffffu : ((1u << (2 * C)) - 1u);
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const int d = st.d;
    const int rlo = max(st.lo, d - e.n);
    const int rhi = min(st.hi + 1, e.m);
    if (rlo > rhi) return true;
    if (rhi >= st.base + W) {
        const int s = (rlo - 1 - st.base) / C;
        if (s <= 0 || rhi >= st.base + s * C + W) {
            // save rows [base, base + W) of d-1 and d-2 for the next level
            if (t == 0) sm.mslot = mig_alloc(*st.ka, st.level);
            __syncthreads();
            const int32_t slot = sm.mslot;
            if (slot >= 0) {
                int32_t* rec = mig_record(*st.ka, slot);
#pragma unroll
                for (int k = 0; k < C; ++k) {
                    rec[kMigHeader + t * C + k] = Q1[k];
                    rec[kMigHeader + W + t * C + k] = Q2[k];
                }
                if (t == 0) {
                    rec[MIG_KIND] = MIG_ABSOLUTE;
                    rec[MIG_ROWS] = W;
                    rec[MIG_D] = d;
                    rec[MIG_BASE] = st.base;
                    rec[MIG_LO] = st.lo;
                    rec[MIG_HI] = st.hi;
                    rec[MIG_BEST] = st.best;
                    rec[MIG_BI] = st.bi;
                    rec[MIG_BJ] = st.bj;
                    rec[MIG_CELLS_LO] = int32_t(uint32_t(st.cells));
                    rec[MIG_CELLS_HI] = int32_t(uint32_t(st.cells >> 32));
                    rec[MIG_LEVEL] = st.level;
                    st.ka->mig_slot[st.item] = slot;
                }
            }
            st.migrated = slot >= 0;
            st.overflow = true;
            return true;
        }
#pragma unroll
        for (int k = 0; k < C; ++k) {
            sm.xbuf[k * NT + t] = Q2[k];
            sm.xbuf[(C + k) * NT + t] = Q1[k];
        }
        sm.xbuf[(2 * C) * NT + t] = int(st.aw);
        sm.xbuf[(2 * C + 1) * NT + t] = int(st.bw);
        __syncthreads();
        st.base += s * C;
        const int src = t + s;
        if (src < NT) {
#pragma unroll
            for (int k = 0; k < C; ++k) {
                Q2[k] = sm.xbuf[k * NT + src];
                Q1[k] = sm.xbuf[(C + k) * NT + src];
            }
            st.aw = uint32_t(sm.xbuf[(2 * C) * NT + src]);
            st.bw = uint32_t(sm.xbuf[(2 * C + 1) * NT + src]);
        } else {
            const int i0 = st.base + t * C;
            st.aw = 0u;
            st.bw = 0u;
#pragma unroll
            for (int k = 0; k < C; ++k) {
                Q2[k] = NEG;
                Q1[k] = NEG;
                st.aw |= a_code(e, int64_t(i0) + k - 1) << (2 * k);
                st.bw |= b_code(e, int64_t(d) - 2 - (i0 + k)) << (2 * k);
            }
        }
        if (lane == 31) {
            sm.top[mod3(d + 2)][w] = Q1[C - 1];  // anti-diagonal d-1
            sm.top[mod3(d + 1)][w] = Q2[C - 1];  // anti-diagonal d-2
            sm.btop[(d + 1) & 1][w] = st.bw;     // codes as of d-1
        }
        __syncthreads();
    }
    st.cells += (unsigned long long)(rhi - rlo + 1);
    // advance b' codes to anti-diagonal d
    uint32_t below = __shfl_up_sync(FULL, st.bw, 1);
    if (lane == 0) below = w > 0 ? sm.btop[(d + 1) & 1][w - 1] : 0u;
    uint32_t carry = (below >> (2 * (C - 1))) & 3u;
    if (t == 0) carry = b_code(e, int64_t(d) - st.base - 1);
    st.bw = ((st.bw << 2) | carry) & MASK2C;
    if (lane == 31) sm.btop[d & 1][w] = st.bw;
    int upc = __shfl_up_sync(FULL, Q1[C - 1], 1);
    int dgc = __shfl_up_sync(FULL, Q2[C - 1], 1);
    if (lane == 0) {
        upc = w > 0 ? sm.top[mod3(d + 2)][w - 1] : NEG;
        dgc = w > 0 ? sm.top[mod3(d + 1)][w - 1] : NEG;
    }
    const uint32_t x = st.aw ^ st.bw;
    const uint32_t eq = ~(x | (x >> 1));
    const int i0 = st.base + t * C;
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
    if (lane == 31) sm.top[mod3(d)][w] = O[C - 1];
    const uint32_t vote = __ballot_sync(FULL, bits != 0u);
    const int wmax = __reduce_max_sync(FULL, lmax);
    int first = INT_MAX, last = -1, arg = INT_MAX;
    if (vote) {
        const int fl = __ffs(vote) - 1, ll = 31 - __clz(vote);
        const uint32_t fb = __shfl_sync(FULL, bits, fl), lb = __shfl_sync(FULL, bits, ll);
        first = st.base + (w * 32 + fl) * C + __ffs(fb) - 1;
        last = st.base + (w * 32 + ll) * C + 31 - __clz(lb);
        if (wmax > st.best) {
            uint32_t eb = 0u;
#pragma unroll
            for (int k = 0; k < C; ++k) eb |= (O[k] == wmax) ? (1u << k) : 0u;
            const uint32_t ev = __ballot_sync(FULL, eb != 0u);
            const int L = __ffs(ev) - 1;
            arg = st.base + (w * 32 + L) * C + __ffs(__shfl_sync(FULL, eb, L)) - 1;
        }
    }
    if (lane == 0) sm.part[d & 1][w] = make_int4(vote ? wmax : NEG, first, last, arg);
    __syncthreads();
    const int4 p = lane < NW ? sm.part[d & 1][lane] : make_int4(NEG, INT_MAX, -1, INT_MAX);
    const int bmax = __reduce_max_sync(FULL, p.x);
    const int bfirst = __reduce_min_sync(FULL, p.y);
    const int blast = __reduce_max_sync(FULL, p.z);
    if (blast < 0) return true;  // no live cell on d
    if (bmax > st.best) {
        const int barg = __reduce_min_sync(FULL, p.x == bmax ? p.w : INT_MAX);
        st.best = bmax;
        st.bi = barg;
        st.bj = d - barg;
    }
    st.lo = bfirst;
    st.hi = blast;
    st.d = d + 1;
    return false;
}

template <int C, int NW>
__device__ bool cta_extend(const KernelArgs& ka, uint32_t id, int level, const ExtArgs& e,
                           ExtRes& r, unsigned long long& cells_here, CtaSmem<C, NW>& sm) {
    constexpr int NT = NW * 32;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    int P0[C], P1[C], P2[C];
    CState st;
    st.ka = &ka;
    st.item = id;
    st.level = level;
    st.overflow = false;
    st.migrated = false;
    st.aw = 0u;
    st.bw = 0u;
    const int32_t slot = ka.mig_slot[id];
    const int32_t* rec = slot >= 0 ? mig_record(ka, slot) : nullptr;
    if (rec) {
        // resume a band saved by a narrower level
        const bool rel = rec[MIG_KIND] == MIG_RELATIVE;
        const int rows = rec[MIG_ROWS];
        const int T1 = rec[MIG_T1], T2 = rec[MIG_T2];
        st.d = rec[MIG_D];
        st.base = rec[MIG_BASE];
        st.lo = rec[MIG_LO];
        st.hi = rec[MIG_HI];
        st.best = rec[MIG_BEST];
        st.bi = rec[MIG_BI];
        st.bj = rec[MIG_BJ];
        st.cells = (unsigned long long)uint32_t(rec[MIG_CELLS_LO]) |
                   ((unsigned long long)uint32_t(rec[MIG_CELLS_HI]) << 32);
        const int i0 = st.base + t * C;
#pragma unroll
        for (int k = 0; k < C; ++k) {
            const int rr = t * C + k;
            int v1 = rr < rows ? rec[kMigHeader + rr] : NEG;
            int v2 = rr < rows ? rec[kMigHeader + rows + rr] : NEG;
            if (rel) {
                v1 = (rr < rows && v1 >= 0) ? v1 + T1 : NEG;
                v2 = (rr < rows && v2 >= 0) ? v2 + T2 : NEG;
            }
            P1[k] = v1;
            P0[k] = v2;
            P2[k] = NEG;
            st.aw |= a_code(e, int64_t(i0) + k - 1) << (2 * k);
            st.bw |= b_code(e, int64_t(st.d) - 2 - (i0 + k)) << (2 * k);
        }
        (void)NT;
    } else {
#pragma unroll
        for (int k = 0; k < C; ++k) {
            P0[k] = NEG;
            P1[k] = NEG;
            P2[k] = NEG;
        }
        if (t == 0) P1[0] = 0;
        st.base = 0;
        st.lo = 0;
        st.hi = 0;
        st.d = 1;
        st.best = 0;
        st.bi = 0;
        st.bj = 0;
        st.cells = 0ull;
#pragma unroll
        for (int k = 0; k < C; ++k) st.aw |= a_code(e, int64_t(t) * C + k - 1) << (2 * k);
    }
    st.cells0 = st.cells;
    if (lane == 31) {
        sm.top[mod3(st.d + 2)][w] = P1[C - 1];  // d-1
        sm.top[mod3(st.d + 1)][w] = P0[C - 1];  // d-2
        sm.btop[(st.d + 1) & 1][w] = st.bw;     // codes as of d-1
    }
    __syncthreads();
    for (;;) {
        if (cta_step<C, NW>(e, st, sm, P0, P1, P2)) break;
        if (cta_step<C, NW>(e, st, sm, P1, P2, P0)) break;
        if (cta_step<C, NW>(e, st, sm, P2, P0, P1)) break;
    }
    r.best = st.best;
    r.bi = st.bi;
    r.bj = st.bj;
    r.status = 0;
    r.cells = st.cells;
    // cells computed here (none are kept when a band restarts elsewhere)
    cells_here = (!st.overflow || st.migrated) ? st.cells - st.cells0 : 0ull;
    return st.overflow;
}

template <int C, int NW>
__global__ void __launch_bounds__(NW * 32)
    k_cta_persistent(KernelArgs ka, int level, int queue, int phase) {
    __shared__ CtaSmem<C, NW> sm;
    const bool plain = phase == PHASE_PLAIN;
    const bool twin = queue != level;  // (no latency forms at these levels)
    const uint32_t* q = ka.queues + size_t(queue) * ka.qcap;
    for (;;) {
        if (threadIdx.x == 0) {
            if (plain) {
                const unsigned int s = atomicAdd(&ka.counters->head[level], 1u);
                sm.slot = s < ka.n_items ? s : ~0u;
            } else {
                sm.slot = pop_slot(ka.counters, queue, phase);
            }
        }
        __syncthreads();
        const unsigned int slot = sm.slot;
        __syncthreads();
        if (slot == ~0u) break;
        const uint32_t id = plain ? slot : q[slot];
        const Item it = ka.items[id];
        if (it.flags & ITEM_SKIP) continue;
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
        ExtRes r;
        unsigned long long cells_here = 0ull;
        const bool ovf = cta_extend<C, NW>(ka, id, level, e, r, cells_here, sm);
        if (threadIdx.x == 0) {
            if (cells_here) atomicAdd(&ka.counters->cells[level], cells_here);
            if (ovf) {
                const int nq = escalate_queue(ka, level, twin);
                const unsigned int tl = atomicAdd(&ka.counters->tail[nq], 1u);
                ka.queues[size_t(nq) * ka.qcap + tl] = id;
            } else {
                ka.ext[id] = r;
            }
        }
        __syncthreads();
    }
}

}  // namespace

cudaError_t launch_cta_level(int level, const KernelArgs& ka, int grid, int phase,
                             cudaStream_t s) {
    switch (level) {
        case 6: k_cta_persistent<16, 4><<<grid, 128, 0, s>>>(ka, level, level, phase); break;
        case 7: k_cta_persistent<8, 16><<<grid, 512, 0, s>>>(ka, level, level, phase); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

int cta_level_blocks_per_sm(int level) {
    int n = 0;
    cudaError_t e = cudaErrorInvalidValue;
    switch (level) {
        case 6: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_cta_persistent<16, 4>, 128, 0); break;
        case 7: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_cta_persistent<8, 16>, 512, 0); break;
        default: break;
    }
    return e == cudaSuccess ? n : 0;
}

}  // namespace logan
