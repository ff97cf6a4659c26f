// X-drop extension with affine gaps (a gap of length L scores
// gap_open + L * gap_extend): the paper's anti-diagonal sweep, pruning rule
// and band trimming (Sec. III-A recurrence and X-drop rule, Algorithm 1,
// Algorithm 2, Sec. IV-A reductions) applied to Gotoh's three states per cell
//   E(i,j) = max(E(i,j-1) + e, H(i,j-1) + o + e)      (i, j-1) on d-1
//   F(i,j) = max(F(i-1,j) + e, H(i-1,j) + o + e)      (i-1, j) on d-1
//   H(i,j) = max(H(i-1,j-1) + sub, E(i,j), F(i,j))    (i-1, j-1) on d-2
// A cell whose H < best - X is pruned with all three of its states.
//
// Units of G lanes x C rows as in the linear kernels (lane g owns rows
// base + g*C + k of a window that slides up in whole lanes), absolute
// scores with -inf = NEGA.  H on d-2 / d-1 / d lives in three register
// arrays that rotate roles (the loop is unrolled three times); E and F are
// updated in place, rows in descending order: E(i,j) reads its own row on
// d-1 and F(i,j) the row below, which is not yet overwritten.  (A six-step
// unroll with two E / F arrays each stalled on instruction fetch.)  Keys
// (H - T_d) * W + (W - 1 - row) give the best and its tie-break in one max.
// Levels: 64 rows (8 lanes x 8, four extensions per warp), 128 (8 x 16,
// four per warp), 256 (16 x 16, two per warp) and 512 (32 x 16); an item
// starts at the level its X class maps to, a band that outgrows a window
// restarts at the next one, and one outgrowing 512 rows (or an X too large
// for the keys) continues in the device-memory ring kernel of
// xdrop_matrix.cu, which has no width limit below the workspace ring.
#include "internal.h"

#include "../../include/logan.h"

namespace logan {

namespace {

constexpr uint32_t FULL = 0xffffffffu;
constexpr int NEGA = -(1 << 30);  // -inf of the absolute scores

template <int G, int C>
struct AGroup {
    static constexpr int W = G * C;
    static constexpr int LOG2W = W == 64 ? 6 : W == 128 ? 7 : W == 256 ? 8 : W == 512 ? 9 : 10;
    static constexpr uint32_t MASK2C = (C >= 16) ? 0xffffffffu : ((1u << (2 * C)) - 1u);
    static constexpr int PREFETCH = 16 * G;  // b' codes held by a unit
    static constexpr int UNROLL = 3;         // steps per loop iteration
    static_assert(C <= 16 && C % 2 == 0, "a lane's row codes fit one word");
    static_assert((1 << LOG2W) == W, "window must be a power of two");
};

struct AState {
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
    uint32_t aw, bw;  // a' / b' codes of the lane's rows, row k at bits 2k
};

template <int G, int C>
__device__ __forceinline__ void a_init(const KernelArgs& ka, AState& u, uint32_t id, int gl,
                                       int (&H2)[C], int (&H1)[C], int (&E1)[C], int (&F1)[C]) {
    // H2, H1: H on d-2, d-1; E1, F1: E, F on d-1
    const Item it = ka.items[id];
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
    u.bpre = stream_codes16(ka.wb, u.bpos, u.dir, u.n, 16 * gl);
    u.aw = 0u;
    u.bw = 0u;
#pragma unroll
    for (int k = 0; k < C; ++k) {
        H2[k] = NEGA;
        H1[k] = NEGA;
        E1[k] = NEGA;
        F1[k] = NEGA;
        u.aw |= stream_code(ka.wa, u.apos, u.dir, uint32_t(u.m), int64_t(gl) * C + k - 1) << (2 * k);
    }
    if (gl == 0) H1[0] = 0;  // cell (0,0) on anti-diagonal 0; no gap state there
    u.active = true;
    u.done = false;
    u.overflow = false;
}

// result, next window or LOGAN_ERANGE of a finished unit (leader lane)
__device__ __forceinline__ void a_finish(const KernelArgs& ka, const AState& u, int level,
                                         int gl, int n_levels) {
    if (gl != 0) return;
    ExtRes r;
    r.best = 0;
    r.bi = 0;
    r.bj = 0;
    r.status = 0;
    r.cells = 0ull;
    if (u.overflow) {
        // the next window, or after the widest one the device-memory ring
        // (queue kWarpLevels, which also holds the items whose X is too
        // large for these keys)
        const int nq = level + 1 < n_levels ? level + 1 : kWarpLevels;
        const unsigned int t = atomicAdd(&ka.counters->tail[nq], 1u);
        ka.queues[size_t(nq) * ka.qcap + t] = u.item;
        return;
    } else {
        r.best = u.best;
        r.bi = u.bi;
        r.bj = u.bj;
        r.cells = u.cells;
    }
    ka.ext[u.item] = r;
}

// loop top: slide the window so that the next UNROLL steps fit, keep the b'
// prefetch covering them; a band that cannot fit overflows
template <int G, int C>
__device__ __forceinline__ void a_prepare(const KernelArgs& ka, AState& u, int gl, int (&H2)[C],
                                          int (&H1)[C], int (&E1)[C], int (&F1)[C]) {
    using Gr = AGroup<G, C>;
    const int rlo = max(u.lo, u.d - u.n);
    const int top = min(u.hi + Gr::UNROLL, u.m);
    const bool need = u.active && top >= u.base + Gr::W;
    if (__any_sync(FULL, need)) {
        const int s = need ? (rlo - 1 - u.base) / C : 0;
        const bool ovf = need && (s <= 0 || top >= u.base + s * C + Gr::W);
        const int sh = (need && !ovf) ? s : 0;
#pragma unroll
        for (int k = 0; k < C; ++k) {
            H2[k] = __shfl_down_sync(FULL, H2[k], sh, G);
            H1[k] = __shfl_down_sync(FULL, H1[k], sh, G);
            E1[k] = __shfl_down_sync(FULL, E1[k], sh, G);
            F1[k] = __shfl_down_sync(FULL, F1[k], sh, G);
        }
        u.aw = __shfl_down_sync(FULL, u.aw, sh, G);
        u.bw = __shfl_down_sync(FULL, u.bw, sh, G);
        u.base += sh * C;
        if (sh > 0 && gl >= G - sh) {
            const int i0 = u.base + gl * C;
            u.aw = 0u;
            u.bw = 0u;
#pragma unroll
            for (int k = 0; k < C; ++k) {
                H2[k] = NEGA;
                H1[k] = NEGA;
                E1[k] = NEGA;
                F1[k] = NEGA;
                u.aw |= stream_code(ka.wa, u.apos, u.dir, uint32_t(u.m), int64_t(i0) + k - 1)
                        << (2 * k);
                // b' codes as of anti-diagonal d-1: index (d-1) - i - 1
                u.bw |= stream_code(ka.wb, u.bpos, u.dir, uint32_t(u.n),
                                    int64_t(u.d) - 2 - (i0 + k))
                        << (2 * k);
            }
        }
        if (ovf) {
            u.active = false;
            u.done = true;
            u.overflow = true;
        }
    }
    const int q = u.d - u.base - 1;  // the next UNROLL steps read q .. q+UNROLL-1
    const bool refill = u.active && (q < u.q0 || q + Gr::UNROLL - 1 >= u.q0 + Gr::PREFETCH);
    if (__any_sync(FULL, refill)) {
        if (refill) {
            u.q0 = q;
            u.bpre = stream_codes16(ka.wb, u.bpos, u.dir, u.n, q + 16 * gl);
        }
    }
}

template <int G>
__device__ __forceinline__ int a_unit_max(int v) {
    if constexpr (G == 32) {
        return __reduce_max_sync(FULL, v);
    } else {
#pragma unroll
        for (int o = G / 2; o >= 1; o >>= 1) v = max(v, __shfl_xor_sync(FULL, v, o, G));
        return v;
    }
}

// One anti-diagonal of every unit of the warp: H2 = H on d-2, H1 = H on
// d-1, HO receives H on d; EF: E and F on d-1, replaced by those of d.
template <int G, int C>
__device__ __forceinline__ void a_step(const KernelArgs& ka, int go, int ge, AState& u, int gl,
                                       int unit, const int (&H2)[C], const int (&H1)[C],
                                       int (&HO)[C], int (&E)[C], int (&F)[C]) {
    using Gr = AGroup<G, C>;
    const int rlo = max(u.lo, u.d - u.n);
    const int rhi = min(u.hi + 1, u.m);
    const bool run = u.active && rlo <= rhi;
    // b' shift register: lane 0 takes stream index d - base - 1
    const int qq = u.d - u.base - 1 - u.q0;
    const uint32_t pre = __shfl_sync(FULL, u.bpre, unit * G + ((qq >> 4) & (G - 1)));
    const uint32_t front = (pre >> (uint32_t(qq & 15) * 2u)) & 3u;
    uint32_t carry = (__shfl_up_sync(FULL, u.bw, 1, G) >> (2 * (C - 1))) & 3u;
    carry = gl == 0 ? front : carry;
    u.bw = ((u.bw << 2) | carry) & Gr::MASK2C;
    // the row below the lane: H and F on d-1 (for F), H on d-2 (diagonal)
    int h1c = __shfl_up_sync(FULL, H1[C - 1], 1, G);
    int f1c = __shfl_up_sync(FULL, F[C - 1], 1, G);
    int h2c = __shfl_up_sync(FULL, H2[C - 1], 1, G);
    if (gl == 0) h1c = f1c = h2c = NEGA;
    const uint32_t x = u.aw ^ u.bw;
    const uint32_t eq = ~(x | (x >> 1));  // bit 2k set iff row k's bases match
    const int T = u.best - u.X;           // prune below (best over d' < d) - X
    const int goe = go + ge;
    const int i0 = u.base + gl * C;
    const int k0 = __viaddmin_s32_relu(rlo, -i0, C);     // clamp(rlo - i0, 0, C)
    const int k1 = __viaddmin_s32_relu(rhi, 1 - i0, C);  // clamp(rhi + 1 - i0, 0, C)
    const uint32_t rb = __funnelshift_lc(~0u, 0u, k1) & ~__funnelshift_lc(~0u, 0u, k0);
    // the additions are multiply-adds with a run-time 1 and the substitution
    // score is picked by a multiply (the row's match flag moved to the sign
    // bit, then the high word of a product with 1), so that they run on the
    // FMA pipe beside the ALU pipe's maxima and selects
    const int one = ka.one;
    const int dsub = ka.sc.mismatch - ka.sc.match;
    // key = (h - T) * W + (C-1-k) = h * W + kbase - k, in wrapping unsigned
    // arithmetic (h * W alone can exceed 32 bits; the key itself cannot)
    const uint32_t kbase = uint32_t(C - 1) - uint32_t(T) * uint32_t(Gr::W);
    const uint32_t wscale = uint32_t(one) * uint32_t(Gr::W);
    int lkey = -1;
    uint32_t bits = 0u;  // bit k: row k live
#pragma unroll
    for (int k = C - 2; k >= 0; k -= 2) {
        int key[2];
#pragma unroll
        for (int hh = 1; hh >= 0; --hh) {
            const int kk = k + hh;  // descending: F[kk-1] still holds d-1
            const int uh = kk ? H1[kk - 1] : h1c;
            const int uf = kk ? F[kk - 1] : f1c;
            const int dg = kk ? H2[kk - 1] : h2c;
            const int e = __vimax3_s32(E[kk] * one + ge, H1[kk] * one + goe, NEGA);
            const int f = __vimax3_s32(uf * one + ge, uh * one + goe, NEGA);
            const int y = __mulhi(int(eq * ka.pw[kk]), one);  // -1 on a match, else 0
            const int t = y * dsub + (dg * one + ka.sc.mismatch);
            const int h = __vimax3_s32(t, e, f);
            const bool live = ((rb >> kk) & 1u) && h >= T;
            HO[kk] = live ? h : NEGA;
            E[kk] = live ? e : NEGA;
            F[kk] = live ? f : NEGA;
            // live: 0 <= h - T <= X + match, so the key stays below 2^31
            key[hh] = live ? int(uint32_t(h) * wscale + (kbase - uint32_t(kk))) : -1;
            bits = (bits << 1) | (live ? 1u : 0u);
        }
        lkey = __vimax3_s32(lkey, key[0], key[1]);
    }
    u.c32 += run ? uint32_t(rhi - rlo + 1) : 0u;
    const int wkey = a_unit_max<G>(lkey >= 0 ? lkey + (G - 1 - gl) * C : -1);
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
    // the anti-diagonal's outcome, without branches: it advances when it had
    // a range and a live cell, else the extension ends here
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
__global__ void __launch_bounds__(128, 4) k_affine(KernelArgs ka, int go, int ge, int level,
                                                int n_levels) {
    const int lane = threadIdx.x & 31;
    const int gl = lane % G, unit = lane / G;
    const uint32_t* q = ka.queues + size_t(level) * ka.qcap;
    int P0[C], P1[C], P2[C], E[C], F[C];
#pragma unroll
    for (int k = 0; k < C; ++k) P0[k] = P1[k] = P2[k] = E[k] = F[k] = NEGA;
    AState u;
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
    u.bpre = u.aw = u.bw = 0u;
    u.c32 = 0u;
    bool exhausted = false;
    for (;;) {
        u.cells += u.c32;
        u.c32 = 0u;
        if (__any_sync(FULL, u.done || (!u.active && !exhausted))) {
            if (u.done) {
                a_finish(ka, u, level, gl, n_levels);
                u.done = false;
            }
            const bool need = !u.active && !exhausted;
            uint32_t id = 0xffffffffu;
            const uint32_t want = __ballot_sync(FULL, need && gl == 0);
            if (want) {
                const int leader = __ffs(want) - 1;
                // levels run one after another, so a level's queue (its
                // binned items, then those escalated into it) is complete
                unsigned int first = 0u, limit = 0u;
                if (lane == leader) {
                    first = atomicAdd(&ka.counters->head[level], unsigned(__popc(want)));
                    limit = ka.counters->tail[level];
                }
                first = __shfl_sync(FULL, first, leader);
                limit = __shfl_sync(FULL, limit, leader);
                const unsigned int slot = first + unsigned(__popc(want & ((1u << (unit * G)) - 1u)));
                if (need && slot < limit) id = q[slot];
            }
            if (need) {
                // the roles are P0 = d-2, P1 = d-1 at the loop top
                if (id != 0xffffffffu) a_init<G, C>(ka, u, id, gl, P0, P1, E, F);
                else exhausted = true;
            }
        }
        if (!__any_sync(FULL, u.active)) break;
        a_prepare<G, C>(ka, u, gl, P0, P1, E, F);
        a_step<G, C>(ka, go, ge, u, gl, unit, P0, P1, P2, E, F);
        a_step<G, C>(ka, go, ge, u, gl, unit, P1, P2, P0, E, F);
        a_step<G, C>(ka, go, ge, u, gl, unit, P2, P0, P1, E, F);
        // roles are back to P0 = d-2, P1 = d-1
    }
}

#define LOGAN_AFFINE_LEVELS(X) X(0, 8, 8) X(1, 8, 16) X(2, 16, 16) X(3, 32, 16)
constexpr int kAffineLevels = 4;

}  // namespace

int affine_levels() { return kAffineLevels; }

int affine_blocks_per_sm(int level) {
    int n = 0;
    cudaError_t e = cudaErrorInvalidValue;
    switch (level) {
#define CASE(L, G, C) \
    case L: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_affine<G, C>, 128, 0); break;
        LOGAN_AFFINE_LEVELS(CASE)
#undef CASE
        default: break;
    }
    return e == cudaSuccess ? n : 0;
}

cudaError_t launch_affine_level(int level, const KernelArgs& ka, int go, int ge, int grid,
                                cudaStream_t s) {
    switch (level) {
#define CASE(L, G, C) \
    case L: k_affine<G, C><<<grid, 128, 0, s>>>(ka, go, ge, level, kAffineLevels); break;
        LOGAN_AFFINE_LEVELS(CASE)
#undef CASE
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace logan
