// X-drop extension with affine gaps, two band rows per 32-bit register
// (16-bit SIMD), for the affine window levels of 128, 256 and 512 rows when
// the call's scores provably fit 16 bits.
//
// Method: Gotoh's three states per cell under the paper's anti-diagonal
// sweep, X-drop rule and band trimming (Sec. III-A, Algorithms 1 and 2;
// other scoring schemes are the paper's future work, Sec. VIII) -- the
// computation of the 32-bit affine kernel (xdrop_affine.cu), with the same
// results.  Layout and keys as the packed linear kernel (xdrop_group16.cu,
// packed16.cuh): lane g of a unit of G lanes owns window rows g*32 + k,
// register h holds rows h and h + 16, a live value is the key
// 32768 + 128*u + (31 - k) with u = S - T_d (T_d = best_{<d} - X), DEAD =
// 16384.  H on d-2 / d-1 / d lives in three register arrays that rotate;
// E and F on d-1 are replaced in place by d, registers in descending order
// (F reads the register below, not yet overwritten).  Per register, both
// halves at once, every candidate re-based onto the cell's own row code
// and onto T_d:
//   e = max(E(d-1) + ge', H(d-1) + goe')               same row
//   f = max(F(d-1) + ge' - 1, H(d-1) + goe' - 1)       the row below (code + 1)
//   h = max(H(d-2) + sm + bonus, e, f)                  the diagonal (code + 1)
// with ge' = 128 (ge + T_{d-1} - T_d), goe' = 128 (go + ge + T_{d-1} - T_d),
// sm = 128 (mismatch + T_{d-2} - T_d) - 1, bonus = 128 (match - mismatch) on
// a match; the additions are 32-bit multiply-adds (FMA pipe), the maxima
// 3-input 16-bit DPX instructions.
//
// Pruning: a cell whose H is below the threshold or outside the
// anti-diagonal's range stores DEAD in all three states (the oracle's rule:
// a pruned cell keeps no gap state).  A live cell keeps its E and F as
// computed even when they are below the threshold: along the E and F paths
// every offset is non-positive (gap extension, the threshold's rise), so
// such a value stays below 32768 -- dead as a key, never deciding a live H
// -- and the maximum with the H term keeps it at or above DEAD + goe' - 1,
// so it never leaves [0, 65536).  The host enables this kernel only when
//   128*(Xmax + 2*max(match,0) + |go| + |ge| + 2) + 31 <= 32767   and
//   128*(|mismatch| + |go| + 2*|ge| + 2*max(match,0) + 2) <= 16383,
// which keeps every half inside [0, 65536) through every addition.
//
// A band that outgrows the window restarts at the next level (no band-state
// records), after the widest in the device-memory ring, as in the 32-bit
// affine kernel; slides move the four arrays by half-lanes (16 rows).
#include "packed16.cuh"

namespace logan {

namespace {

template <int G>
using PA = P16<G, 1>;

template <int G>
__device__ __forceinline__ void a16_init(const KernelArgs& ka, S16<1>& u, uint32_t id, int gl,
                                         uint32_t (&H2)[16], uint32_t (&H1)[16],
                                         uint32_t (&E)[16], uint32_t (&F)[16]) {
    const Item it = ka.items[id];
    u.item = id;
    u.apos = it.a_pos;
    u.bpos = it.b_pos;
    u.dir = (it.flags & ITEM_LEFT) ? -1 : 1;
    u.m = int(it.m);
    u.n = int(it.n);
    u.X = it.X;
    u.base = 0;
    u.lo = 0;
    u.hi = 0;
    u.d = 1;
    u.best = 0;
    u.T = -it.X;
    u.T1 = -it.X;
    u.T2 = -it.X;
    u.bi = 0;
    u.bj = 0;
    u.cells = 0ull;
    u.q0 = 0;
    u.bpre = b_codes16_of(ka, u, 16 * gl);
#pragma unroll
    for (int h = 0; h < 16; ++h) H2[h] = H1[h] = E[h] = F[h] = DEAD2;
    // S(0,0) = 0 relative to T_0 = -X, window row 0; it has no gap state
    if (gl == 0) H1[0] = (DEAD2 & 0xffff0000u) | live_key(it.X, 0);
    load_a_planes(ka, u, gl);
    u.b0[0] = 0u;
    u.b1[0] = 0u;
    u.active = true;
    u.done = false;
    u.overflow = false;
}

// result, next window or the ring of a finished unit (leader lane)
__device__ __forceinline__ void a16_finish(const KernelArgs& ka, const S16<1>& u, int level,
                                           int gl, int n_levels) {
    if (gl != 0) return;
    if (u.overflow) {
        const int nq = level + 1 < n_levels ? level + 1 : kWarpLevels;
        const unsigned int t = atomicAdd(&ka.counters->tail[nq], 1u);
        ka.queues[size_t(nq) * ka.qcap + t] = u.item;
        return;
    }
    ExtRes r;
    r.best = u.best;
    r.bi = u.bi;
    r.bj = u.bj;
    r.status = 0;
    r.cells = u.cells;
    ka.ext[u.item] = r;
}

// Loop top: slide the window by half-lanes so that the next three steps
// fit (a band that cannot fit overflows), keep the b' prefetch covering
// them.  H2 = d-2, H1 = d-1, E and F on d-1.
template <int G>
__device__ __forceinline__ void a16_prepare(const KernelArgs& ka, S16<1>& u, int gl,
                                            uint32_t (&H2)[16], uint32_t (&H1)[16],
                                            uint32_t (&E)[16], uint32_t (&F)[16]) {
    constexpr int W = PA<G>::W;
    const int rlo = max(u.lo, u.d - u.n);
    const int top = min(u.hi + 3, u.m);  // highest row the next three steps can reach
    const bool need = u.active && top >= u.base + W;
    if (__any_sync(FULL, need)) {
        // keep row rlo - 1 (a predecessor of the lowest cell) in the window
        const int s = need ? (rlo - 1 - u.base) / 16 : 0;
        const bool ovf = need && (s <= 0 || top >= u.base + s * 16 + W);
        const int sh = (need && !ovf) ? s : 0;  // half-lanes to drop
        const int t = sh >> 1;
        const bool odd = (sh & 1) != 0;
        const bool lo_ok = 2 * gl + sh < 2 * G;
        const bool hi_ok = 2 * gl + sh + 1 < 2 * G;
        const uint32_t keep = (lo_ok ? 0x0000ffffu : 0u) | (hi_ok ? 0xffff0000u : 0u);
        // an odd number of half-lanes moves rows k + 16 to k (code + 16) and
        // the next lane's rows k to k + 16 (code - 16)
        const uint32_t rebase = odd ? 16u - (16u << 16) : 0u;
        auto slide = [&](uint32_t& r) {
            uint32_t x = __shfl_down_sync(FULL, r, t, G);
            const uint32_t y = __shfl_down_sync(FULL, r, t + 1, G);
            if (odd) x = __byte_perm(x, y, 0x5432);
            if (sh > 0) r = ((x + rebase) & keep) | (DEAD2 & ~keep);
        };
#pragma unroll
        for (int h = 0; h < 16; ++h) {
            slide(H2[h]);
            slide(H1[h]);
            slide(E[h]);
            slide(F[h]);
        }
        auto slide_plane = [&](uint32_t& p) {
            uint32_t x = __shfl_down_sync(FULL, p, t, G);
            const uint32_t y = __shfl_down_sync(FULL, p, t + 1, G);
            if (odd) x = __funnelshift_r(x, y, 16);
            if (sh > 0) p = x;
        };
        slide_plane(u.a0[0]);
        slide_plane(u.a1[0]);
        slide_plane(u.b0[0]);
        slide_plane(u.b1[0]);
        if (sh > 0) {
            u.base += 16 * sh;
            if (!(lo_ok && hi_ok)) {
                // rows new to the window: codes from memory (b' as of d-1)
                load_a_planes(ka, u, gl);
                load_b_planes(ka, u, gl, u.d - 1);
            }
        }
        if (ovf) {
            u.active = false;
            u.done = true;
            u.overflow = true;
        }
    }
    // the next three steps read b' stream indices q .. q+2
    const int q = u.d - u.base - 1;
    const bool refill = u.active && (q < u.q0 || q + 2 >= u.q0 + PA<G>::PREFETCH);
    if (__any_sync(FULL, refill)) {
        if (refill) {
            u.q0 = q;
            u.bpre = b_codes16_of(ka, u, q + 16 * gl);
        }
    }
}

// One anti-diagonal of every unit of the warp: H2 = H on d-2, H1 = H on
// d-1, O receives H on d; E and F on d-1 are replaced by d.
template <int G>
__device__ __forceinline__ void a16_step(const KernelArgs& ka, int go, int ge, S16<1>& u, int gl,
                                         int unit, const uint32_t (&H2)[16],
                                         const uint32_t (&H1)[16], uint32_t (&O)[16],
                                         uint32_t (&E)[16], uint32_t (&F)[16]) {
    constexpr int W = PA<G>::W;
    const int rlo = max(u.lo, u.d - u.n);
    const int rhi = min(u.hi + 1, u.m);
    const bool run = u.active && rlo <= rhi;
    // b' shift register: every row takes the code its lower neighbour row
    // held on d-1; window row 0 takes stream index d - base - 1
    const int qq = u.d - u.base - 1 - u.q0;
    const uint32_t pre = __shfl_sync(FULL, u.bpre, unit * G + ((qq >> 4) & (G - 1)));
    const uint32_t front = pre >> (uint32_t(qq & 15) * 2u);
    uint32_t c0 = __shfl_up_sync(FULL, u.b0[0], 1, G);
    uint32_t c1 = __shfl_up_sync(FULL, u.b1[0], 1, G);
    c0 = gl == 0 ? (front << 31) : c0;
    c1 = gl == 0 ? ((front >> 1) << 31) : c1;
    u.b0[0] = __funnelshift_l(c0, u.b0[0], 1);
    u.b1[0] = __funnelshift_l(c1, u.b1[0], 1);
    const uint32_t eq = ~((u.a0[0] ^ u.b0[0]) | (u.a1[0] ^ u.b1[0]));  // bit r: row r matches
    const uint32_t eqB = eq >> 8;  // rows 8.. and 24.. for registers 8..15
    // register 0's row below: (lane g-1's row 31, own row 15) of H on d-1,
    // H on d-2 and F on d-1; the lower lane's row 31 has code 0 where row 0
    // expects code 32 from a predecessor: +32 on the low half
    uint32_t xu = __shfl_up_sync(FULL, H1[15], 1, G);
    uint32_t xd = __shfl_up_sync(FULL, H2[15], 1, G);
    uint32_t xf = __shfl_up_sync(FULL, F[15], 1, G);
    xu = gl == 0 ? DEAD2 : xu;
    xd = gl == 0 ? DEAD2 : xd;
    xf = gl == 0 ? DEAD2 : xf;
    const uint32_t one = uint32_t(ka.one);
    const uint32_t U0 = __byte_perm(xu, H1[15], 0x5432) * one + 32u;
    const uint32_t D0 = __byte_perm(xd, H2[15], 0x5432) * one + 32u;
    const uint32_t F0 = __byte_perm(xf, F[15], 0x5432) * one + 32u;
    // per-step offsets in key units, both halves at once
    const int gE = (ge + u.T1 - u.T) * KS;       // E along its row
    const int gH = (go + ge + u.T1 - u.T) * KS;  // a gap opened from H
    const uint32_t GE = uint32_t(gE) * 0x10001u;
    const uint32_t GH = uint32_t(gH) * 0x10001u;
    const uint32_t GEu = uint32_t(gE - 1) * 0x10001u;  // from the row below: code - 1
    const uint32_t GHu = uint32_t(gH - 1) * 0x10001u;
    const uint32_t SM = uint32_t((ka.sc.mismatch + u.T2 - u.T) * KS - 1) * 0x10001u;
    const int dsw = (ka.sc.match - ka.sc.mismatch) * KS;
    // rows of this lane inside [rlo, rhi]: bits [k0, k1) of rb
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
        const uint32_t t = dg * one + SM;
        const uint32_t Mh = (h < 8 ? eq : eqB) & (0x10001u << (h & 7));
        const uint32_t t2 = Mh * uint32_t(dsw >> (h & 7)) + t;
        const uint32_t v = __vimax3_u16x2(t2, e, f);
        // row h's range bit -> bit 15, row h+16's -> bit 31
        const uint32_t x = v & (rb * ka.pw16[h]);
        const uint32_t mk = sign_mask16(x);  // 0xffff per live half
        O[h] = (v & mk) | (DEAD2 & ~mk);
        E[h] = (e & mk) | (DEAD2 & ~mk);
        F[h] = (f & mk) | (DEAD2 & ~mk);
        L |= mk & (0x10001u << h);
    }
#pragma unroll
    for (int h = 0; h < 16; h += 2) lk1 = __vimax3_u16x2(lk1, O[h], O[h + 1]);
    // the unit's largest key and its first / last live rows
    const uint32_t lkey = max(lk1 & 0xffffu, lk1 >> 16);
    const uint32_t fkey = lkey >= LIVE ? (((lkey - LIVE) >> LOG2KS) << PA<G>::LOG2W) |
                                             uint32_t(W - 32 - gl * 32) + (lkey & 31u)
                                       : 0u;
    const int fr = __ffs(L) - 1, lr = 31 - __clz(L);
    const uint32_t flw = L ? (uint32_t(W - (gl * 32 + fr)) | (uint32_t(gl * 32 + lr + 1) << 16)) : 0u;
    const uint32_t wkey = unit_max_u32<G>(fkey);
    const uint32_t fl = unit_max_u16x2<G>(flw);
    u.c32 += run ? uint32_t(rhi - rlo + 1) : 0u;
    // the anti-diagonal's outcome, without branches: it advances when it
    // had a range and a live cell, else the extension ends here
    const bool adv = run && fl != 0u;
    const int umax = int(wkey >> PA<G>::LOG2W);
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
__global__ void __launch_bounds__(128, 3)
    k_affine16(KernelArgs ka, int go, int ge, int level, int n_levels) {
    const int lane = threadIdx.x & 31;
    const int gl = lane % G, unit = lane / G;
    const uint32_t* q = ka.queues + size_t(level) * ka.qcap;
    uint32_t P0[16], P1[16], P2[16], E[16], F[16];
#pragma unroll
    for (int h = 0; h < 16; ++h) P0[h] = P1[h] = P2[h] = E[h] = F[h] = DEAD2;
    S16<1> u;
    u.active = false;
    u.done = false;
    u.overflow = false;
    u.item = 0;
    u.m = u.n = 0;
    u.base = u.lo = u.hi = 0;
    u.d = 1;
    u.T = u.T1 = u.T2 = u.best = u.bi = u.bj = 0;
    u.X = 0;
    u.cells = 0ull;
    u.cells0 = 0ull;
    u.migrated = false;
    u.apos = u.bpos = 0;
    u.dir = 1;
    u.q0 = 0;
    u.bpre = 0u;
    u.a0[0] = u.a1[0] = u.b0[0] = u.b1[0] = 0u;
    u.c32 = 0u;
    bool exhausted = false;
    for (;;) {
        u.cells += u.c32;
        u.c32 = 0u;
        if (__any_sync(FULL, u.done || (!u.active && !exhausted))) {
            if (u.done) {
                a16_finish(ka, u, level, gl, n_levels);
                u.done = false;
            }
            const bool need = !u.active && !exhausted;  // the same in all lanes of a unit
            uint32_t id = 0xffffffffu;
            const uint32_t want = __ballot_sync(FULL, need && gl == 0);
            if (want) {
                const int leader = __ffs(want) - 1;
                // levels run one after another, so a level's queue (its
                // binned items, then those that outgrew the level below) is
                // complete
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
                if (id != 0xffffffffu) a16_init<G>(ka, u, id, gl, P0, P1, E, F);
                else exhausted = true;
            }
        }
        if (!__any_sync(FULL, u.active)) break;
        a16_prepare<G>(ka, u, gl, P0, P1, E, F);
        a16_step<G>(ka, go, ge, u, gl, unit, P0, P1, P2, E, F);
        a16_step<G>(ka, go, ge, u, gl, unit, P1, P2, P0, E, F);
        a16_step<G>(ka, go, ge, u, gl, unit, P2, P0, P1, E, F);
        // roles are back to P0 = d-2, P1 = d-1
    }
}

}  // namespace

// affine level -> G of its packed form (one 32-row lane; level 0, 64 rows,
// has none)
#define LOGAN_AFFINE16_LEVELS(X) X(1, 4) X(2, 8) X(3, 16)

bool affine16_level(int level) {
    switch (level) {
#define CASE(L, G) case L: return true;
        LOGAN_AFFINE16_LEVELS(CASE)
#undef CASE
        default: return false;
    }
}

cudaError_t launch_affine16_level(int level, const KernelArgs& ka, int go, int ge, int n_levels,
                                  int grid, cudaStream_t s) {
    switch (level) {
#define CASE(L, G) \
    case L: k_affine16<G><<<grid, 128, 0, s>>>(ka, go, ge, level, n_levels); break;
        LOGAN_AFFINE16_LEVELS(CASE)
#undef CASE
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

int affine16_blocks_per_sm(int level) {
    int n = 0;
    cudaError_t e = cudaErrorInvalidValue;
    switch (level) {
#define CASE(L, G) \
    case L: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_affine16<G>, 128, 0); break;
        LOGAN_AFFINE16_LEVELS(CASE)
#undef CASE
        default: break;
    }
    return e == cudaSuccess ? n : 0;
}

}  // namespace logan
