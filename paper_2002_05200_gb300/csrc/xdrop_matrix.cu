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
//    values < K), any K <= 32; extensions run first in register windows of
//    64 .. 512 rows (k_mx_group below), and only bands that outgrow them, or
//    an X too large for their keys, come here.
//  * the affine DNA path (logan_extend_batch_affine): its register windows
//    end at 512 rows; a band that outgrows them, or an X too large for their
//    keys, continues here on the 2-bit pools with the 4 x 4 match / mismatch
//    table, instead of ending with LOGAN_ERANGE.
#include <algorithm>
#include <climits>

#include "ctx_ext.h"
#include "internal.h"
#include "packed16.cuh"
#include "../../include/logan.h"

namespace logan {

namespace {

// (FULL, the packed keys and reductions: packed16.cuh)
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
    const uint32_t* queue;   // the ring's queue
    Counters* counters;
    int q;  // the ring's queue index in counters (every entry [0, tail) is taken)
    uint32_t* queues;        // register levels: queue l at queues + l * qcap
    uint32_t qcap;
    const int32_t* table;  // K x K, row = letter of a; nullptr: match / mismatch
    int K;
    int match, mismatch;
    int go, ge;
    int32_t* ring;  // per block: 6 * cap cells
    uint32_t cap;   // power of two
    int cells_level;  // counters->cells index credited with the cells
    int sub_min;      // the table's smallest entry (packed windows)
    int one;          // 1 at run time: additions as multiply-adds (FMA pipe)
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

// ---- register windows for letter codes: several extensions per warp ----
//
// The affine register kernel's layout (xdrop_affine.cu) for letter codes:
// a unit of G lanes x C rows per extension (lane g owns rows base + g*C + k
// of a window that slides up in whole lanes), H on d-2 / d-1 / d in three
// rotating register arrays, E and F updated in place (rows in descending
// order), keys (H - T) * W + (W-1-row) for the best and its tie-break.  The
// letters of a lane's rows are bytes, four to a word; the b' letters shift
// up one row per anti-diagonal (a funnel shift per word, the lane below's
// top letter carried in); the substitution is one shared-memory load of the
// K x K table per cell.  A band that outgrows the window restarts at the next
// level; after the widest it continues in the ring kernel above.

constexpr int kMxLevels = 4;         // 64, 128, 256, 512 rows
constexpr int kMxRingQueue = kMxLevels;
constexpr int32_t kMxGroupMaxX = (1 << 20) - 4096;  // keys need (X + 1000) * W < 2^31

template <int G, int C>
struct MGroup {
    static constexpr int W = G * C;
    static constexpr int LOG2W = W == 64 ? 6 : W == 128 ? 7 : W == 256 ? 8 : 9;
    static constexpr int PREFETCH = 4 * G;  // b' letters a unit holds
    static_assert(C % 4 == 0 && (1 << LOG2W) == W, "shape");
};

struct MState {
    int base, lo, hi, d;
    int best, bi, bj;
    int m, n, X;
    unsigned long long cells;
    uint32_t c32;  // cells of the current loop iteration, folded into cells at its top
    int64_t apos, bpos;
    int dir;
    int q0;
    uint32_t bpre;
    uint32_t item;
    bool active, done, overflow;
};

// letter of stream index q (0 outside [0, len))
__device__ __forceinline__ uint32_t mx_letter(const uint8_t* __restrict__ pool, int64_t pos,
                                              int dir, int len, int64_t q) {
    if (q < 0 || q >= len) return 0u;
    return pool[pos + (dir > 0 ? q : -q)];
}

// letters of stream indices q .. q+3, q in the low byte
__device__ __forceinline__ uint32_t mx_letters4(const uint8_t* __restrict__ pool, int64_t pos,
                                                int dir, int len, int64_t q) {
    return mx_letter(pool, pos, dir, len, q) | (mx_letter(pool, pos, dir, len, q + 1) << 8) |
           (mx_letter(pool, pos, dir, len, q + 2) << 16) | (mx_letter(pool, pos, dir, len, q + 3) << 24);
}

template <int G, int C>
__device__ __forceinline__ void mg_init(const MxArgs& a, MState& u, uint32_t id, int gl,
                                        int (&H2)[C], int (&H1)[C], int (&E)[C], int (&F)[C],
                                        uint32_t (&aw)[C / 4], uint32_t (&bw)[C / 4]) {
    const Item it = a.items[id];
    const uint8_t* pa = static_cast<const uint8_t*>(a.pa);
    const uint8_t* pb = static_cast<const uint8_t*>(a.pb);
    u.item = id;
    u.apos = it.a_pos;
    u.bpos = it.b_pos;
    u.dir = (it.flags & ITEM_LEFT) ? -1 : 1;
    u.m = int(it.m);
    u.n = int(it.n);
    u.X = it.X;
    u.base = u.lo = u.hi = 0;
    u.d = 1;
    u.best = u.bi = u.bj = 0;
    u.cells = 0ull;
    u.q0 = 0;
    u.bpre = mx_letters4(pb, u.bpos, u.dir, u.n, 4 * gl);
#pragma unroll
    for (int k = 0; k < C; ++k) H2[k] = H1[k] = E[k] = F[k] = NEGM;
#pragma unroll
    for (int w = 0; w < C / 4; ++w) {
        aw[w] = mx_letters4(pa, u.apos, u.dir, u.m, int64_t(gl) * C + 4 * w - 1);
        bw[w] = 0u;
    }
    if (gl == 0) H1[0] = 0;  // cell (0,0): no gap state
    u.active = true;
    u.done = false;
    u.overflow = false;
}

__device__ __forceinline__ void mg_finish(const MxArgs& a, const MState& u, int level, int gl) {
    if (gl != 0) return;
    if (u.overflow) {
        // the next window, after the widest the ring
        const int nq = level + 1 < kMxLevels ? level + 1 : kMxRingQueue;
        const unsigned int t = atomicAdd(&a.counters->tail[nq], 1u);
        a.queues[size_t(nq) * a.qcap + t] = u.item;
        return;
    }
    ExtRes r;
    r.best = u.best;
    r.bi = u.bi;
    r.bj = u.bj;
    r.status = 0;
    r.cells = u.cells;
    a.ext[u.item] = r;
    atomicAdd(&a.counters->cells[level], u.cells);
}

template <int G, int C>
__device__ __forceinline__ void mg_prepare(const MxArgs& a, MState& u, int gl, int (&H2)[C],
                                           int (&H1)[C], int (&E)[C], int (&F)[C],
                                           uint32_t (&aw)[C / 4], uint32_t (&bw)[C / 4]) {
    using Gr = MGroup<G, C>;
    const uint8_t* pa = static_cast<const uint8_t*>(a.pa);
    const uint8_t* pb = static_cast<const uint8_t*>(a.pb);
    const int rlo = max(u.lo, u.d - u.n);
    const int top = min(u.hi + 3, u.m);
    const bool need = u.active && top >= u.base + Gr::W;
    if (__any_sync(FULL, need)) {
        const int s = need ? (rlo - 1 - u.base) / C : 0;
        const bool ovf = need && (s <= 0 || top >= u.base + s * C + Gr::W);
        const int sh = (need && !ovf) ? s : 0;
#pragma unroll
        for (int k = 0; k < C; ++k) {
            H2[k] = __shfl_down_sync(FULL, H2[k], sh, G);
            H1[k] = __shfl_down_sync(FULL, H1[k], sh, G);
            E[k] = __shfl_down_sync(FULL, E[k], sh, G);
            F[k] = __shfl_down_sync(FULL, F[k], sh, G);
        }
#pragma unroll
        for (int w = 0; w < C / 4; ++w) {
            aw[w] = __shfl_down_sync(FULL, aw[w], sh, G);
            bw[w] = __shfl_down_sync(FULL, bw[w], sh, G);
        }
        u.base += sh * C;
        if (sh > 0 && gl >= G - sh) {
            const int i0 = u.base + gl * C;
#pragma unroll
            for (int k = 0; k < C; ++k) H2[k] = H1[k] = E[k] = F[k] = NEGM;
#pragma unroll
            for (int w = 0; w < C / 4; ++w) {
                aw[w] = mx_letters4(pa, u.apos, u.dir, u.m, int64_t(i0) + 4 * w - 1);
                // b' letters as of anti-diagonal d-1: index (d-1) - i - 1, row order
                uint32_t v = 0u;
#pragma unroll
                for (int t = 0; t < 4; ++t)
                    v |= mx_letter(pb, u.bpos, u.dir, u.n, int64_t(u.d) - 2 - (i0 + 4 * w + t))
                         << (8 * t);
                bw[w] = v;
            }
        }
        if (ovf) {
            u.active = false;
            u.done = true;
            u.overflow = true;
        }
    }
    const int q = u.d - u.base - 1;  // the next three steps read q .. q+2
    const bool refill = u.active && (q < u.q0 || q + 2 >= u.q0 + Gr::PREFETCH);
    if (__any_sync(FULL, refill)) {
        if (refill) {
            u.q0 = q;
            u.bpre = mx_letters4(pb, u.bpos, u.dir, u.n, int64_t(q) + 4 * gl);
        }
    }
}

template <int G>
__device__ __forceinline__ int mg_unit_max(int v) {
    if constexpr (G == 32) {
        return __reduce_max_sync(FULL, v);
    } else {
#pragma unroll
        for (int o = G / 2; o >= 1; o >>= 1) v = max(v, __shfl_xor_sync(FULL, v, o, G));
        return v;
    }
}

// one anti-diagonal of every unit of the warp: H2 / H1 = H on d-2 / d-1, HO
// receives H on d; E and F on d-1 are replaced by those of d
template <int G, int C>
__device__ __forceinline__ void mg_step(const MxArgs& a, const int* tab, MState& u, int gl,
                                        int unit, const int (&H2)[C], const int (&H1)[C],
                                        int (&HO)[C], int (&E)[C], int (&F)[C],
                                        const uint32_t (&aw)[C / 4], uint32_t (&bw)[C / 4]) {
    using Gr = MGroup<G, C>;
    const int rlo = max(u.lo, u.d - u.n);
    const int rhi = min(u.hi + 1, u.m);
    const bool run = u.active && rlo <= rhi;
    // b' letters move up one row; window row 0 takes stream index d - base - 1
    const int qq = u.d - u.base - 1 - u.q0;
    const uint32_t pre = __shfl_sync(FULL, u.bpre, unit * G + ((qq >> 2) & (G - 1)));
    const uint32_t front = (pre >> (8u * uint32_t(qq & 3))) & 0xffu;
    uint32_t carry = __shfl_up_sync(FULL, bw[C / 4 - 1], 1, G);
    carry = gl == 0 ? (front << 24) : carry;
#pragma unroll
    for (int w = C / 4 - 1; w >= 1; --w) bw[w] = __funnelshift_l(bw[w - 1], bw[w], 8);
    bw[0] = __funnelshift_l(carry, bw[0], 8);
    int h1c = __shfl_up_sync(FULL, H1[C - 1], 1, G);
    int f1c = __shfl_up_sync(FULL, F[C - 1], 1, G);
    int h2c = __shfl_up_sync(FULL, H2[C - 1], 1, G);
    if (gl == 0) h1c = f1c = h2c = NEGM;
    const int T = u.best - u.X;
    const int goe = a.go + a.ge;
    const int one = a.one;
    const int i0 = u.base + gl * C;
    const int k0 = __viaddmin_s32_relu(rlo, -i0, C);
    const int k1 = __viaddmin_s32_relu(rhi, 1 - i0, C);
    const uint32_t rb = __funnelshift_lc(~0u, 0u, k1) & ~__funnelshift_lc(~0u, 0u, k0);
    const uint32_t kbase = uint32_t(C - 1) - uint32_t(T) * uint32_t(Gr::W);
    int lkey = -1;
    uint32_t bits = 0u;
#pragma unroll
    for (int k = C - 1; k >= 0; --k) {  // descending: F[k-1] still holds d-1
        const int uh = k ? H1[k - 1] : h1c;
        const int uf = k ? F[k - 1] : f1c;
        const int dg = k ? H2[k - 1] : h2c;
        // the additions as multiply-adds with a run-time 1 (FMA pipe), the
        // maxima 3-input DPX (ALU pipe)
        const int e = __vimax3_s32(E[k] * one + a.ge, H1[k] * one + goe, NEGM);
        const int f = __vimax3_s32(uf * one + a.ge, uh * one + goe, NEGM);
        const uint32_t la = (aw[k >> 2] >> (8 * (k & 3))) & 0xffu;
        const uint32_t lb = (bw[k >> 2] >> (8 * (k & 3))) & 0xffu;
        const int h = __vimax3_s32(dg * one + tab[la * uint32_t(a.K) + lb], e, f);
        const bool live = ((rb >> k) & 1u) && h >= T;
        HO[k] = live ? h : NEGM;
        E[k] = live ? e : NEGM;
        F[k] = live ? f : NEGM;
        // live: 0 <= h - T <= X + max entry, so the key stays below 2^31
        lkey = max(lkey, live ? int(uint32_t(h) * uint32_t(Gr::W) + (kbase - uint32_t(k))) : -1);
        bits = (bits << 1) | (live ? 1u : 0u);
    }
    if constexpr (C >= 16) {  // (the 16-row lanes are short of registers)
        if (run) u.cells += (unsigned long long)(rhi - rlo + 1);
    } else {
        u.c32 += run ? uint32_t(rhi - rlo + 1) : 0u;
    }
    const int wkey = mg_unit_max<G>(lkey >= 0 ? lkey + (G - 1 - gl) * C : -1);
    int rfirst, rlast;
    if constexpr (G == 32) {
        rfirst = __reduce_min_sync(FULL, bits ? gl * C + (__ffs(bits) - 1) : Gr::W);
        rlast = __reduce_max_sync(FULL, bits ? gl * C + (31 - __clz(bits)) : -1);
    } else {
        const uint32_t vote = __ballot_sync(FULL, bits != 0u);
        const uint32_t uvv = (vote >> (unit * G)) & ((1u << G) - 1u);
        const int fl = uvv ? __ffs(uvv) - 1 : 0, ll = uvv ? 31 - __clz(uvv) : 0;
        const uint32_t fb = __shfl_sync(FULL, bits, unit * G + fl);
        const uint32_t lb = __shfl_sync(FULL, bits, unit * G + ll);
        rfirst = uvv ? fl * C + (__ffs(fb) - 1) : Gr::W;
        rlast = uvv ? ll * C + (31 - __clz(lb)) : -1;
    }
    // the anti-diagonal's outcome: it advances when it had a range and a live
    // cell, else the extension ends here
    if constexpr (C >= 16) {  // (branches: the 16-row lanes are short of registers)
        if (run && rlast >= 0) {
            const int hmax = T + (wkey >> Gr::LOG2W);
            if (hmax > u.best) {
                u.best = hmax;
                u.bi = u.base + Gr::W - 1 - (wkey & (Gr::W - 1));
                u.bj = u.d - u.bi;
            }
            u.lo = u.base + rfirst;
            u.hi = u.base + rlast;
        } else if (u.active) {
            u.active = false;
            u.done = true;
        }
        u.d += 1;
        return;
    }
    const bool adv = run && rlast >= 0;
    const int hmax = T + (wkey >> Gr::LOG2W);
    const bool imp = adv && hmax > u.best;  // strict: the first anti-diagonal reaching it
    const int r = u.base + Gr::W - 1 - (wkey & (Gr::W - 1));
    u.bi = imp ? r : u.bi;
    u.bj = imp ? u.d - r : u.bj;
    u.best = imp ? hmax : u.best;
    u.lo = adv ? u.base + rfirst : u.lo;
    u.hi = adv ? u.base + rlast : u.hi;
    u.done = u.done || (u.active && !adv);
    u.active = u.active && adv;
    u.d += 1;
}

template <int G, int C>
__global__ void __launch_bounds__(128, C >= 16 ? 3 : 4) k_mx_group(MxArgs a, int level) {
    __shared__ int tab[kMaxK * kMaxK];
    for (int t = threadIdx.x; t < a.K * a.K; t += blockDim.x) tab[t] = a.table[t];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int gl = lane % G, unit = lane / G;
    const uint32_t* q = a.queues + size_t(level) * a.qcap;
    int P0[C], P1[C], P2[C], E[C], F[C];
    uint32_t aw[C / 4], bw[C / 4];
#pragma unroll
    for (int k = 0; k < C; ++k) P0[k] = P1[k] = P2[k] = E[k] = F[k] = NEGM;
#pragma unroll
    for (int w = 0; w < C / 4; ++w) aw[w] = bw[w] = 0u;
    MState u;
    u.active = u.done = u.overflow = false;
    u.item = 0u;
    u.m = u.n = 0;
    u.base = u.lo = u.hi = 0;
    u.d = 1;
    u.best = u.bi = u.bj = 0;
    u.X = 0;
    u.cells = 0ull;
    u.apos = u.bpos = 0;
    u.dir = 1;
    u.q0 = 0;
    u.bpre = 0u;
    u.c32 = 0u;
    bool exhausted = false;
    bool first_wave = true;  // the warp's first pop takes static slots
    for (;;) {
        if constexpr (C < 16) {
            u.cells += u.c32;
            u.c32 = 0u;
        }
        if (__any_sync(FULL, u.done || (!u.active && !exhausted))) {
            if (u.done) {
                mg_finish(a, u, level, gl);
                u.done = false;
            }
            const bool need = !u.active && !exhausted;
            uint32_t id = 0xffffffffu;
            const uint32_t want = __ballot_sync(FULL, need && gl == 0);
            if (want) {
                // levels run one after another, so a level's queue is complete
                unsigned int limit = 0u;
                const unsigned int slot = pop_unit_slot<G>(a.counters, level, PHASE_WHOLE, want,
                                                           lane, unit, first_wave, limit);
                if (need && slot < limit) id = q[slot];
            }
            if (need) {
                if (id != 0xffffffffu) mg_init<G, C>(a, u, id, gl, P0, P1, E, F, aw, bw);
                else exhausted = true;
            }
        }
        if (!__any_sync(FULL, u.active)) break;
        mg_prepare<G, C>(a, u, gl, P0, P1, E, F, aw, bw);
        mg_step<G, C>(a, tab, u, gl, unit, P0, P1, P2, E, F, aw, bw);
        mg_step<G, C>(a, tab, u, gl, unit, P1, P2, P0, E, F, aw, bw);
        mg_step<G, C>(a, tab, u, gl, unit, P2, P0, P1, E, F, aw, bw);
    }
}

#define LOGAN_MX_LEVELS(X) X(0, 8, 8) X(1, 16, 8) X(2, 32, 8) X(3, 32, 16)

cudaError_t launch_mx_level(int level, const MxArgs& a, int grid, cudaStream_t s) {
    switch (level) {
#define CASE(L, G, C) case L: k_mx_group<G, C><<<grid, 128, 0, s>>>(a, L); break;
        LOGAN_MX_LEVELS(CASE)
#undef CASE
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

int mx_level_blocks(int level) {
    int n = 0;
    cudaError_t e = cudaErrorInvalidValue;
    switch (level) {
#define CASE(L, G, C) \
    case L: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_mx_group<G, C>, 128, 0); break;
        LOGAN_MX_LEVELS(CASE)
#undef CASE
        default: break;
    }
    return e == cudaSuccess ? std::max(1, n) : 1;
}

// ---- packed register windows: two rows per 32-bit register ----
//
// The packed affine windows (xdrop_affine16.cu) for letter codes: units of G
// lanes x 32 rows, register h of a lane holding rows h and h + 16 as 16-bit
// keys 32768 + 128*u + (31 - k) (DEAD = 16384), H on d-2 / d-1 / d in three
// rotating arrays, E and F in place with the registers in descending order.
// A lane keeps its rows' letters as 16-bit halves too: A16[h] = a' letters of
// rows (h, h + 16), B16[h] = their b' letters, which move up one register per
// anti-diagonal (register 0 takes the row below: a byte permute, plus one
// shuffle from the lower lane).  The substitution of a pair of cells is
// A16[h] * K + B16[h] (both table indices in one multiply-add) and two 16-bit
// loads of the table, kept in shared memory as 128 (M[x][y] - min M): the
// diagonal term is H(d-2) + 128 (min M + T_{d-2} - T_d) - 1 + that entry,
// which the bounds below keep inside [0, 65536) with no carry between
// halves.  The host runs a window packed only when
//   128*(Xmax + 2*max(max M,0) + |go| + |ge| + 2) + 31 <= 32767   and
//   128*(|min M| + |go| + 2*|ge| + 2*max(max M,0) + 2) <= 16383
// (the packed affine windows' bounds with max M and min M for match and
// mismatch); a band that outgrows a window restarts at the next.

struct M16 {
    int base, lo, hi, d;
    int best, T, T1, T2;
    int bi, bj;
    int m, n, X;
    unsigned long long cells;
    uint32_t c32;  // cells of the current loop iteration, folded into cells at its top
    int64_t apos, bpos;
    int dir;
    int q0;
    uint32_t bpre;  // this lane's 4 prefetched b' letters: q0 + 4g ...
    uint32_t item;
    bool active, done, overflow;
};

// letters of rows (h, h+16), h < 16, of the 32 rows from stream index q
// (row r: index q + r, or q - r for the b' stream read backwards), as halves
template <bool BACK>
__device__ __forceinline__ void m16_letters(const uint8_t* __restrict__ pool, int64_t pos, int dir,
                                            int len, int64_t q, uint32_t (&L)[16]) {
#pragma unroll
    for (int h = 0; h < 16; ++h) {
        const int64_t q0 = BACK ? q - h : q + h;
        const int64_t q1 = BACK ? q - h - 16 : q + h + 16;
        L[h] = mx_letter(pool, pos, dir, len, q0) | (mx_letter(pool, pos, dir, len, q1) << 16);
    }
}

template <int G>
__device__ __forceinline__ void m16_init(const MxArgs& a, M16& u, uint32_t id, int gl,
                                         uint32_t (&H2)[16], uint32_t (&H1)[16], uint32_t (&E)[16],
                                         uint32_t (&F)[16], uint32_t (&A16)[16], uint32_t (&B16)[16]) {
    const Item it = a.items[id];
    const uint8_t* pa = static_cast<const uint8_t*>(a.pa);
    const uint8_t* pb = static_cast<const uint8_t*>(a.pb);
    u.item = id;
    u.apos = it.a_pos;
    u.bpos = it.b_pos;
    u.dir = (it.flags & ITEM_LEFT) ? -1 : 1;
    u.m = int(it.m);
    u.n = int(it.n);
    u.X = it.X;
    u.base = u.lo = u.hi = 0;
    u.d = 1;
    u.best = 0;
    u.T = u.T1 = u.T2 = -it.X;
    u.bi = u.bj = 0;
    u.cells = 0ull;
    u.q0 = 0;
    u.bpre = mx_letters4(pb, u.bpos, u.dir, u.n, 4 * gl);
#pragma unroll
    for (int h = 0; h < 16; ++h) {
        H2[h] = H1[h] = E[h] = F[h] = DEAD2;
        B16[h] = 0u;
    }
    // S(0,0) = 0 relative to T_0 = -X, window row 0; it has no gap state
    if (gl == 0) H1[0] = (DEAD2 & 0xffff0000u) | live_key(it.X, 0);
    // row r needs a' index base + g*32 + r - 1
    m16_letters<false>(pa, u.apos, u.dir, u.m, int64_t(gl) * 32 - 1, A16);
    u.active = true;
    u.done = false;
    u.overflow = false;
}

// result, next window or the ring of a finished unit (leader lane)
__device__ __forceinline__ void m16_finish(const MxArgs& a, const M16& u, int level, int gl) {
    if (gl != 0) return;
    if (u.overflow) {
        const int nq = level + 1 < kMxLevels ? level + 1 : kMxRingQueue;
        const unsigned int t = atomicAdd(&a.counters->tail[nq], 1u);
        a.queues[size_t(nq) * a.qcap + t] = u.item;
        return;
    }
    ExtRes r;
    r.best = u.best;
    r.bi = u.bi;
    r.bj = u.bj;
    r.status = 0;
    r.cells = u.cells;
    a.ext[u.item] = r;
    atomicAdd(&a.counters->cells[level], u.cells);
}

// Loop top: slide by half-lanes so that the next three steps fit (a band that
// cannot overflows), keep the b' prefetch covering them.
template <int G>
__device__ __forceinline__ void m16_prepare(const MxArgs& a, M16& u, int gl, uint32_t (&H2)[16],
                                            uint32_t (&H1)[16], uint32_t (&E)[16],
                                            uint32_t (&F)[16], uint32_t (&A16)[16],
                                            uint32_t (&B16)[16]) {
    constexpr int W = P16<G, 1>::W;
    const uint8_t* pa = static_cast<const uint8_t*>(a.pa);
    const uint8_t* pb = static_cast<const uint8_t*>(a.pb);
    const int rlo = max(u.lo, u.d - u.n);
    const int top = min(u.hi + 3, u.m);
    const bool need = u.active && top >= u.base + W;
    if (__any_sync(FULL, need)) {
        const int s = need ? (rlo - 1 - u.base) / 16 : 0;
        const bool ovf = need && (s <= 0 || top >= u.base + s * 16 + W);
        const int sh = (need && !ovf) ? s : 0;  // half-lanes to drop
        const int t = sh >> 1;
        const bool odd = (sh & 1) != 0;
        const bool lo_ok = 2 * gl + sh < 2 * G;
        const bool hi_ok = 2 * gl + sh + 1 < 2 * G;
        const uint32_t keep = (lo_ok ? 0x0000ffffu : 0u) | (hi_ok ? 0xffff0000u : 0u);
        // keys: an odd shift moves rows k + 16 to k (code + 16) and the next
        // lane's rows k to k + 16 (code - 16); letters move as they are
        const uint32_t rebase = odd ? 16u - (16u << 16) : 0u;
        auto slide = [&](uint32_t& r, bool key) {
            uint32_t x = __shfl_down_sync(FULL, r, t, G);
            const uint32_t y = __shfl_down_sync(FULL, r, t + 1, G);
            if (odd) x = __byte_perm(x, y, 0x5432);
            if (sh > 0) r = key ? (((x + rebase) & keep) | (DEAD2 & ~keep)) : x;
        };
#pragma unroll
        for (int h = 0; h < 16; ++h) {
            slide(H2[h], true);
            slide(H1[h], true);
            slide(E[h], true);
            slide(F[h], true);
            slide(A16[h], false);
            slide(B16[h], false);
        }
        if (sh > 0) {
            u.base += 16 * sh;
            if (!(lo_ok && hi_ok)) {
                // rows new to the window: letters from memory (b' as of d-1)
                const int64_t i0 = int64_t(u.base) + int64_t(gl) * 32;
                m16_letters<false>(pa, u.apos, u.dir, u.m, i0 - 1, A16);
                m16_letters<true>(pb, u.bpos, u.dir, u.n, int64_t(u.d) - 2 - i0, B16);
            }
        }
        if (ovf) {
            u.active = false;
            u.done = true;
            u.overflow = true;
        }
    }
    const int q = u.d - u.base - 1;  // the next three steps read q .. q+2
    const bool refill = u.active && (q < u.q0 || q + 2 >= u.q0 + 4 * G);
    if (__any_sync(FULL, refill)) {
        if (refill) {
            u.q0 = q;
            u.bpre = mx_letters4(pb, u.bpos, u.dir, u.n, int64_t(q) + 4 * gl);
        }
    }
}

// One anti-diagonal of every unit of the warp (H2 = d-2, H1 = d-1, O = d;
// E, F on d-1 replaced by d; B16 moves to d's letters).
template <int G>
__device__ __forceinline__ void m16_step(const MxArgs& a, const uint16_t* tab, M16& u, int gl,
                                         int unit, const uint32_t (&H2)[16],
                                         const uint32_t (&H1)[16], uint32_t (&O)[16],
                                         uint32_t (&E)[16], uint32_t (&F)[16],
                                         const uint32_t (&A16)[16], uint32_t (&B16)[16]) {
    constexpr int W = P16<G, 1>::W;
    const int rlo = max(u.lo, u.d - u.n);
    const int rhi = min(u.hi + 1, u.m);
    const bool run = u.active && rlo <= rhi;
    // b' letters move up one row; window row 0 takes stream index d - base - 1
    const int qq = u.d - u.base - 1 - u.q0;
    const uint32_t pre = __shfl_sync(FULL, u.bpre, unit * G + ((qq >> 2) & (G - 1)));
    const uint32_t front = (pre >> (8u * uint32_t(qq & 3))) & 0xffu;
    uint32_t bb = __shfl_up_sync(FULL, B16[15], 1, G);
    uint32_t b0 = __byte_perm(bb, B16[15], 0x5432);  // (lower lane's row 31, own row 15)
    b0 = gl == 0 ? ((b0 & 0xffff0000u) | front) : b0;
#pragma unroll
    for (int h = 15; h >= 1; --h) B16[h] = B16[h - 1];
    B16[0] = b0;
    // the row below register 0: lower lane's row 31, own row 15; the lower
    // lane's row 31 has code 0 where row 0 expects code 32: +32 on the low half
    uint32_t xu = __shfl_up_sync(FULL, H1[15], 1, G);
    uint32_t xd = __shfl_up_sync(FULL, H2[15], 1, G);
    uint32_t xf = __shfl_up_sync(FULL, F[15], 1, G);
    xu = gl == 0 ? DEAD2 : xu;
    xd = gl == 0 ? DEAD2 : xd;
    xf = gl == 0 ? DEAD2 : xf;
    const uint32_t one = uint32_t(a.one);
    const uint32_t U0 = __byte_perm(xu, H1[15], 0x5432) * one + 32u;
    const uint32_t D0 = __byte_perm(xd, H2[15], 0x5432) * one + 32u;
    const uint32_t F0 = __byte_perm(xf, F[15], 0x5432) * one + 32u;
    const int gE = (a.ge + u.T1 - u.T) * KS;
    const int gH = (a.go + a.ge + u.T1 - u.T) * KS;
    const uint32_t GE = uint32_t(gE) * 0x10001u;
    const uint32_t GH = uint32_t(gH) * 0x10001u;
    const uint32_t GEu = uint32_t(gE - 1) * 0x10001u;
    const uint32_t GHu = uint32_t(gH - 1) * 0x10001u;
    const uint32_t SM = uint32_t((a.sub_min + u.T2 - u.T) * KS - 1) * 0x10001u;
    const uint32_t K = uint32_t(a.K);
    const int i0 = u.base + gl * 32;
    const int k0 = __viaddmin_s32_relu(rlo, -i0, 32);
    const int k1 = __viaddmin_s32_relu(rhi, 1 - i0, 32);
    const uint32_t rb = __funnelshift_lc(~0u, 0u, k1) & ~__funnelshift_lc(~0u, 0u, k0);
    uint32_t L = 0u;
    uint32_t lk1 = 0u;
#pragma unroll
    for (int h = 15; h >= 0; --h) {  // descending: F[h-1] still holds d-1
        const uint32_t hu = h ? H1[h - 1] : U0;
        const uint32_t fu = h ? F[h - 1] : F0;
        const uint32_t dg = h ? H2[h - 1] : D0;
        const uint32_t e = __vimax3_u16x2(E[h] * one + GE, H1[h] * one + GH, 0u);
        const uint32_t f = __vimax3_u16x2(fu * one + GEu, hu * one + GHu, 0u);
        // both cells' table indices, a' letter * K + b' letter, in one
        const uint32_t idx = A16[h] * K + B16[h];
        const uint32_t sub = __byte_perm(uint32_t(tab[idx & 0xffffu]), uint32_t(tab[idx >> 16]),
                                         0x5410);
        const uint32_t t2 = sub * one + (dg * one + SM);
        const uint32_t v = __vimax3_u16x2(t2, e, f);
        const uint32_t x = v & (rb << (15 - h) & 0x80008000u);
        const uint32_t mk = sign_mask16(x);  // 0xffff per live half
        O[h] = (v & mk) | (DEAD2 & ~mk);
        E[h] = (e & mk) | (DEAD2 & ~mk);
        F[h] = (f & mk) | (DEAD2 & ~mk);
        L |= mk & (0x10001u << h);
    }
#pragma unroll
    for (int h = 0; h < 16; h += 2) lk1 = __vimax3_u16x2(lk1, O[h], O[h + 1]);
    const uint32_t lkey = max(lk1 & 0xffffu, lk1 >> 16);
    const uint32_t fkey = lkey >= LIVE ? (((lkey - LIVE) >> LOG2KS) << P16<G, 1>::LOG2W) |
                                             uint32_t(W - 32 - gl * 32) + (lkey & 31u)
                                       : 0u;
    const int fr = __ffs(L) - 1, lr = 31 - __clz(L);
    const uint32_t flw = L ? (uint32_t(W - (gl * 32 + fr)) | (uint32_t(gl * 32 + lr + 1) << 16)) : 0u;
    const uint32_t wkey = unit_max_u32<G>(fkey);
    const uint32_t fl = unit_max_u16x2<G>(flw);
    u.c32 += run ? uint32_t(rhi - rlo + 1) : 0u;
    const bool adv = run && fl != 0u;
    const int umax = int(wkey >> P16<G, 1>::LOG2W);
    const bool imp = adv && umax > u.X;  // S > best  <=>  S - T_d > X
    const int r = W - 1 - int(wkey & uint32_t(W - 1));
    const int best = imp ? u.T + umax : u.best;
    u.bi = imp ? u.base + r : u.bi;
    u.bj = imp ? u.d - (u.base + r) : u.bj;
    u.best = best;
    const int T = u.T, T1 = u.T1;
    u.T2 = adv ? T1 : u.T2;
    u.T1 = adv ? T : T1;
    u.T = adv ? best - u.X : T;
    u.lo = adv ? u.base + (W - int(fl & 0xffffu)) : u.lo;
    u.hi = adv ? u.base + int(fl >> 16) - 1 : u.hi;
    u.done = u.done || (u.active && !adv);
    u.active = u.active && adv;
    u.d += 1;
}

template <int G>
__global__ void __launch_bounds__(128, 2) k_mx16(MxArgs a, int level) {
    __shared__ uint16_t tab[kMaxK * kMaxK];
    // 128 (M[x][y] - min M): 16-bit, non-negative under the host's bounds
    for (int t = threadIdx.x; t < a.K * a.K; t += blockDim.x)
        tab[t] = uint16_t((a.table[t] - a.sub_min) * KS);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int gl = lane % G, unit = lane / G;
    const uint32_t* q = a.queues + size_t(level) * a.qcap;
    uint32_t P0[16], P1[16], P2[16], E[16], F[16], A16[16], B16[16];
#pragma unroll
    for (int h = 0; h < 16; ++h) {
        P0[h] = P1[h] = P2[h] = E[h] = F[h] = DEAD2;
        A16[h] = B16[h] = 0u;
    }
    M16 u;
    u.active = u.done = u.overflow = false;
    u.item = 0u;
    u.m = u.n = 0;
    u.base = u.lo = u.hi = 0;
    u.d = 1;
    u.best = u.bi = u.bj = 0;
    u.T = u.T1 = u.T2 = 0;
    u.X = 0;
    u.cells = 0ull;
    u.c32 = 0u;
    u.apos = u.bpos = 0;
    u.dir = 1;
    u.q0 = 0;
    u.bpre = 0u;
    bool exhausted = false;
    for (;;) {
        u.cells += u.c32;
        u.c32 = 0u;
        if (__any_sync(FULL, u.done || (!u.active && !exhausted))) {
            if (u.done) {
                m16_finish(a, u, level, gl);
                u.done = false;
            }
            const bool need = !u.active && !exhausted;
            uint32_t id = 0xffffffffu;
            const uint32_t want = __ballot_sync(FULL, need && gl == 0);
            if (want) {
                const int leader = __ffs(want) - 1;
                // levels run one after another, so a level's queue is complete
                unsigned int first = 0u, limit = 0u;
                if (lane == leader) {
                    first = atomicAdd(&a.counters->head[level], unsigned(__popc(want)));
                    limit = a.counters->tail[level];
                }
                first = __shfl_sync(FULL, first, leader);
                limit = __shfl_sync(FULL, limit, leader);
                const unsigned int slot = first + unsigned(__popc(want & ((1u << (unit * G)) - 1u)));
                if (need && slot < limit) id = q[slot];
            }
            if (need) {
                if (id != 0xffffffffu) m16_init<G>(a, u, id, gl, P0, P1, E, F, A16, B16);
                else exhausted = true;
            }
        }
        if (!__any_sync(FULL, u.active)) break;
        m16_prepare<G>(a, u, gl, P0, P1, E, F, A16, B16);
        m16_step<G>(a, tab, u, gl, unit, P0, P1, P2, E, F, A16, B16);
        m16_step<G>(a, tab, u, gl, unit, P1, P2, P0, E, F, A16, B16);
        m16_step<G>(a, tab, u, gl, unit, P2, P0, P1, E, F, A16, B16);
    }
}

// matrix level -> G of its packed form (one 32-row lane; level 0, 64 rows,
// has none)
#define LOGAN_MX16_LEVELS(X) X(1, 4) X(2, 8) X(3, 16)

bool mx16_level(int level) {
    switch (level) {
#define CASE(L, G) case L: return true;
        LOGAN_MX16_LEVELS(CASE)
#undef CASE
        default: return false;
    }
}

cudaError_t launch_mx16_level(int level, const MxArgs& a, int grid, cudaStream_t s) {
    switch (level) {
#define CASE(L, G) case L: k_mx16<G><<<grid, 128, 0, s>>>(a, L); break;
        LOGAN_MX16_LEVELS(CASE)
#undef CASE
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

int mx16_level_blocks(int level) {
    int n = 0;
    cudaError_t e = cudaErrorInvalidValue;
    switch (level) {
#define CASE(L, G) \
    case L: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_mx16<G>, 128, 0); break;
        LOGAN_MX16_LEVELS(CASE)
#undef CASE
        default: break;
    }
    return e == cudaSuccess ? std::max(1, n) : 1;
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
                           uint32_t* queues, uint32_t qcap, Counters* counters) {
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
    // the narrowest register window first; an X too large for its keys
    // goes straight to the ring
    const int q = x > kMxGroupMaxX ? kMxRingQueue : 0;
    uint32_t* queue = queues + size_t(q) * qcap;
    if (!(L.flags & ITEM_SKIP)) queue[atomicAdd(&counters->tail[q], 1u)] = 2 * p;
    if (!(R.flags & ITEM_SKIP)) queue[atomicAdd(&counters->tail[q], 1u)] = 2 * p + 1;
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
    L.queue = take(size_t(kMxLevels + 1) * items * sizeof(uint32_t));
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
    MxArgs a{};
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
    a.queues = nullptr;
    a.qcap = 0;
    a.ring = ka.ring;
    // the workspace ring holds 6 * ring_cap cells per slot
    a.cap = ka.ring_cap;
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
    int32_t sub_min = matrix[0], sub_max = matrix[0];
    for (int t = 0; t < K * K; ++t) {
        const int64_t v = matrix[t] < 0 ? -int64_t(matrix[t]) : matrix[t];
        if (v > kMaxParam) return LOGAN_EINVAL;
        big = std::max(big, v);
        sub_min = std::min(sub_min, matrix[t]);
        sub_max = std::max(sub_max, matrix[t]);
    }
    // windows of 128-512 rows run packed (two 16-bit cells per register) when
    // the scores provably fit (see the packed kernel); with per-pair X the
    // call does not know the largest X, and keeps the 32-bit windows
    uint32_t packed = 0u;
    int64_t opt_packed = 1;
    logan_get_option(ctx, LOGAN_OPT_PACKED16, &opt_packed);
    if (opt_packed && !X_per_pair) {
        const int64_t mp = std::max<int64_t>(sub_max, 0);
        const int64_t am = sub_min < 0 ? -int64_t(sub_min) : sub_min;
        const int64_t ao = -int64_t(gap_open), ae = -int64_t(gap_extend);
        constexpr int64_t S = 128;  // score scale of the packed keys
        if (S * (int64_t(X) + 2 * mp + ao + ae + 2) + 31 <= 32767 &&
            S * (am + ao + 2 * ae + 2 * mp + 2) <= 16383)
            for (int l = 0; l < kMxLevels; ++l)
                if (mx16_level(l)) packed |= 1u << l;
    }
    ctx_set_matrix_packed(ctx, packed);
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
                const uint32_t qcap = 2u * n_pairs;
                k_mx_split<<<(n_pairs + 255) / 256, 256, 0, s>>>(
                    pa, pb, reinterpret_cast<const uint32_t*>(seeds), n_pairs, table, K, big, X,
                    X_per_pair, items, info, ext, queue, qcap, counters);
                e = cudaGetLastError();
                if (e == cudaSuccess) {
                    MxArgs a{};
                    a.pa = pa.bases;
                    a.pb = pb.bases;
                    a.items = items;
                    a.ext = ext;
                    a.queues = queue;
                    a.qcap = qcap;
                    a.queue = queue + size_t(kMxRingQueue) * qcap;
                    a.counters = counters;
                    a.q = kMxRingQueue;
                    a.table = table;
                    a.K = K;
                    a.match = 0;
                    a.mismatch = 0;
                    a.go = gap_open;
                    a.ge = gap_extend;
                    a.ring = reinterpret_cast<int32_t*>(ws + L.ring);
                    a.cap = 1u << LOGAN_MATRIX_RING_LOG2;
                    a.cells_level = kMxRingQueue;
                    // register windows of 64 .. 512 rows, narrowest first,
                    // then the ring for what outgrew them
                    a.sub_min = sub_min;
                    a.one = 1;
                    for (int l = 0; l < kMxLevels && e == cudaSuccess; ++l)
                        e = ((packed >> l) & 1u)
                                ? launch_mx16_level(l, a, sms * mx16_level_blocks(l), s)
                                : launch_mx_level(l, a, sms * mx_level_blocks(l), s);
                    if (e == cudaSuccess) {
                        k_mx_ring<true><<<L.slots, kMxThreads, 0, s>>>(a);
                        e = cudaGetLastError();
                    }
                }
                if (e == cudaSuccess) e = launch_combine(seeds, info, ext, n_pairs, out, s);
            }
            if (e != cudaSuccess) rc = LOGAN_ECUDA;
        }
    }
    if (prev >= 0 && prev != int(dev)) cudaSetDevice(prev);
    return rc;
}
