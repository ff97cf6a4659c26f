// Fallback X-drop extension for bands wider than every register window.
//
// This is the paper's own layout (Sec. IV-B: the three anti-diagonals live
// in device memory, one block per alignment, segments of blockDim cells,
// Sec. IV-A): each resident block owns one ring slot of three arrays of
// ring_cap cells, indexed by row i modulo ring_cap, and sweeps an
// anti-diagonal in strides of 256 threads.  It is slow but has no width
// limit below ring_cap; a wider band ends the extension with LOGAN_ERANGE.
#include <climits>

#include "internal.h"

namespace logan {

namespace {

constexpr uint32_t FULL = 0xffffffffu;
constexpr int kRingThreads = 256;
constexpr int kRingWarps = kRingThreads / 32;

struct Red {
    int mx, arg, first, last;
};

// Block-wide reduction: max score, smallest row reaching it, min first live
// row, max last live row.  Ends with every thread holding the result.
__device__ __forceinline__ Red block_reduce(Red v, Red* sh) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int mx = __reduce_max_sync(FULL, v.mx);
    int arg = __reduce_min_sync(FULL, v.mx == mx ? v.arg : INT_MAX);
    int first = __reduce_min_sync(FULL, v.first);
    int last = __reduce_max_sync(FULL, v.last);
    if (lane == 0) sh[w] = Red{mx, arg, first, last};
    __syncthreads();
    Red p = lane < kRingWarps ? sh[lane] : Red{NEG, INT_MAX, INT_MAX, -1};
    mx = __reduce_max_sync(FULL, p.mx);
    arg = __reduce_min_sync(FULL, p.mx == mx ? p.arg : INT_MAX);
    first = __reduce_min_sync(FULL, p.first);
    last = __reduce_max_sync(FULL, p.last);
    __syncthreads();  // sh is reused by the next call
    return Red{mx, arg, first, last};
}

__device__ void ring_extend(const KernelArgs& ka, const Item& it, int32_t* R, ExtRes& r,
                            Red* sh) {
    const int dir = (it.flags & ITEM_LEFT) ? -1 : 1;
    const int m = int(it.m), n = int(it.n), X = it.X;
    const int mask = int(ka.ring_cap) - 1;
    int32_t* A0 = R;                   // anti-diagonal d
    int32_t* A1 = R + ka.ring_cap;     // d-1
    int32_t* A2 = R + 2 * ka.ring_cap; // d-2
    if (threadIdx.x == 0) A1[0] = 0;   // S(0,0)
    __syncthreads();
    int lo1 = 0, hi1 = 0, lo2 = 1, hi2 = 0;
    int best = 0, bi = 0, bj = 0, status = 0;
    unsigned long long cells = 0ull;
    for (int d = 1;; ++d) {
        const int rlo = max(lo1, d - n), rhi = min(hi1 + 1, m);
        if (rlo > rhi) break;
        if (rhi - rlo + 1 > int(ka.ring_cap)) {
            status = -34;  // LOGAN_ERANGE
            break;
        }
        cells += (unsigned long long)(rhi - rlo + 1);
        const int T = best - X;
        Red v{NEG, INT_MAX, INT_MAX, -1};
        for (int i = rlo + int(threadIdx.x); i <= rhi; i += kRingThreads) {
            const int j = d - i;
            const int dg = (i > 0 && j > 0 && i - 1 >= lo2 && i - 1 <= hi2) ? A2[(i - 1) & mask] : NEG;
            const int up = (i > 0 && i - 1 >= lo1 && i - 1 <= hi1) ? A1[(i - 1) & mask] : NEG;
            const int lf = (j > 0 && i >= lo1 && i <= hi1) ? A1[i & mask] : NEG;
            int sub = ka.sc.mismatch;
            if (i > 0 && j > 0 &&
                stream_code(ka.wa, it.a_pos, dir, it.m, i - 1) ==
                    stream_code(ka.wb, it.b_pos, dir, it.n, j - 1))
                sub = ka.sc.match;
            int s = max(dg + sub, max(up, lf) + ka.sc.gap);
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
        const Red b = block_reduce(v, sh);  // its barriers also publish A0
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
        int32_t* tmp = A2;
        A2 = A1;
        A1 = A0;
        A0 = tmp;
    }
    r.best = status ? 0 : best;
    r.bi = status ? 0 : bi;
    r.bj = status ? 0 : bj;
    r.status = status;
    r.cells = status ? 0ull : cells;
}

__global__ void __launch_bounds__(kRingThreads) k_ring(KernelArgs ka) {
    __shared__ Red sh[kRingWarps];
    __shared__ unsigned int s_slot;
    int32_t* R = ka.ring + size_t(blockIdx.x) * 3u * ka.ring_cap;
    const uint32_t* q = ka.queues + size_t(kNumLevels) * ka.qcap;
    for (;;) {
        if (threadIdx.x == 0) s_slot = pop_slot(ka.counters, kNumLevels, PHASE_ESCALATED);
        __syncthreads();
        const unsigned int slot = s_slot;
        __syncthreads();
        if (slot == ~0u) break;
        const uint32_t id = q[slot];
        const Item it = ka.items[id];
        ExtRes r;
        ring_extend(ka, it, R, r, sh);
        if (threadIdx.x == 0) {
            ka.ext[id] = r;
            atomicAdd(&ka.counters->cells[kNumLevels], r.cells);
        }
        __syncthreads();
    }
}

}  // namespace

cudaError_t launch_ring(const KernelArgs& ka, int grid, cudaStream_t s) {
    if (grid <= 0) return cudaSuccess;
    k_ring<<<grid, kRingThreads, 0, s>>>(ka);
    return cudaGetLastError();
}

}  // namespace logan
