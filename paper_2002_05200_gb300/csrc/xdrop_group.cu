// X-drop extension with G-lane units, 32/G extensions per warp, band held
// in registers (window levels 0..5).
//
// Method (paper Sec. III-A recurrence and X-drop rule; Algorithm 1 sweep;
// Algorithm 2 cell update; Sec. IV-A parallel max reduction):
//   anti-diagonal d holds cells (i, d-i).  Lane g of a unit owns rows
//   i = base + g*C + k (k < C) of a window [base, base + W), W = G*C, that
//   slides up in whole lanes.  The three rolling anti-diagonals (d-2, d-1,
//   d) are three register arrays that swap roles every step (the loop is
//   unrolled three times), so no value moves in memory:
//     up   = S(i-1, j)   on d-1: own register k-1, or lane g-1's C-1 (shuffle)
//     left = S(i, j-1)   on d-1: own register k
//     diag = S(i-1, j-1) on d-2: own register k-1, or lane g-1's C-1 (shuffle)
//
// Scores are held relative to the pruning threshold of their anti-diagonal,
// u = S - T_d with T_d = best_{<d} - X, so a cell is live iff u >= 0 and -inf
// is NEGU.  Moving a value from d-1 or d-2 to d adds T_{d-1} - T_d or
// T_{d-2} - T_d; both are folded into the per-step gap and match/mismatch
// constants, so re-basing costs nothing per cell.  (The one-warp forms,
// G = 32 with C < 32, hold anti-diagonal d relative to T_{d-1} instead and
// prune against T_d - T_{d-1}: the same values shifted by a constant, with
// the same cost per cell, but a step's additions and maxima no longer wait
// for the previous step's reductions -- what a lone long extension waits
// on.)  Every live cell's
// key = u*W + (W-1-row) is reduced by one max per unit: the largest key holds
// the anti-diagonal's best score and, for equal scores, the smallest row --
// the best cell's tie-break without a second search.  Live rows are one warp
// ballot; the first/last set lanes give the trimmed band (Algorithm 1's trims
// from both ends).
//
// Several extensions share a warp so that the per-anti-diagonal bookkeeping
// is paid once per warp.  Window slides, result writes and item refills run
// once per three steps at the loop top (the window keeps three rows of slack
// above the band), so the unrolled steps hold only the hot path.  A band that
// outgrows the window writes its last two anti-diagonals and scalars to a
// band-state record and is handed to the next, wider level, which resumes
// from the record (unit_init); only when the record pool is full does that
// level recompute the extension from the start.  Items with X > kGroupMaxX
// never start here (binning sends them to the multi-warp levels): the keys
// need (X + max score) * W < 2^31.
#include "internal.h"

namespace logan {

namespace {

constexpr uint32_t FULL = 0xffffffffu;
constexpr int NEGU = -(1 << 20);  // -inf of the relative scores

// 2-bit codes of a lane's C rows: 32 bits up to 16 rows, 64 bits above
template <int C>
struct CodeWord {
    using T = uint32_t;
};
template <>
struct CodeWord<32> {
    using T = unsigned long long;
};

template <int G, int C>
struct Group {
    using Code = typename CodeWord<C>::T;
    static constexpr int U = 32 / G;  // units per warp
    static constexpr int W = G * C;   // window rows (a power of two)
    static constexpr int LOG2W =
        W == 32 ? 5 : W == 64 ? 6 : W == 128 ? 7 : W == 256 ? 8 : W == 512 ? 9 : 10;
    static constexpr Code MASK2C = (C >= 16) ? ~Code(0) : ((Code(1) << (2 * C)) - 1u);
    static constexpr uint32_t ALLC = (C >= 32) ? 0xffffffffu : ((1u << C) - 1u);
    static constexpr int PREFETCH = 16 * G;  // b' codes held by a unit
    // one extension per warp (G = 32) with C < 32: each anti-diagonal is
    // stored relative to the threshold of the one before it (see group_step)
    static constexpr bool LAT = G == 32 && C < 32;
    static_assert((1 << LOG2W) == W, "window must be a power of two");
};

// Per-unit state, replicated in every lane of the unit.
template <int C>
struct UState {
    int base, lo, hi, d;
    int best, T, T1, T2;  // T = T_d for the coming step, T1 = T_{d-1}, T2 = T_{d-2}
    int R1, R2;           // one-warp forms: the thresholds the d-1 / d-2 values are relative to
    int bi, bj;
    int m, n, X;
    unsigned long long cells;
    unsigned long long cells0;  // cells computed before this level (resumed items)
    uint32_t c32;               // cells of the current loop iteration, folded into cells at its top
    int64_t apos, bpos;
    int dir;
    int q0;          // first b' stream index held in the unit's prefetch words
    uint32_t bpre;   // this lane's 16 prefetched b' codes: q0 + 16*g ...
    uint32_t item;
    bool active;     // extension in progress
    bool done;       // finished, result not written yet
    bool overflow;   // finished because the band left the window
    bool migrated;   // the overflowing band was saved for the next level
    typename CodeWord<C>::T aw, bw;  // a' / b' codes of the lane's rows, row k at bits 2k
};

template <int C>
__device__ __forceinline__ uint32_t a_code(const KernelArgs& ka, const UState<C>& u, int64_t q) {
    return stream_code(ka.wa, u.apos, u.dir, uint32_t(u.m), q);
}
template <int C>
__device__ __forceinline__ uint32_t b_code(const KernelArgs& ka, const UState<C>& u, int64_t q) {
    return stream_code(ka.wb, u.bpos, u.dir, uint32_t(u.n), q);
}

// b' stream codes q..q+15 in stream order (0 for indices outside [0, n)).
template <int C>
__device__ __forceinline__ uint32_t b_codes16(const KernelArgs& ka, const UState<C>& u, int q) {
    return stream_codes16(ka.wb, u.bpos, u.dir, u.n, q);
}

template <int G>
__device__ __forceinline__ int unit_max(int v) {
    if constexpr (G == 32) {
        return __reduce_max_sync(FULL, v);
    } else {
#pragma unroll
        for (int o = G / 2; o >= 1; o >>= 1) v = max(v, __shfl_xor_sync(FULL, v, o, G));
        return v;
    }
}

template <int G, int C>
__device__ __forceinline__ void unit_init(const KernelArgs& ka, UState<C>& u, uint32_t id, int gl,
                                          int (&Q2)[C], int (&Q1)[C]) {
    using Code = typename Group<G, C>::Code;
    const Item it = ka.items[id];
    u.item = id;
    u.apos = it.a_pos;
    u.bpos = it.b_pos;
    u.dir = (it.flags & ITEM_LEFT) ? -1 : 1;
    u.m = int(it.m);
    u.n = int(it.n);
    u.X = it.X;
    u.bw = 0u;
    u.aw = 0u;
    const int32_t slot = ka.mig_slot[id];
    const int32_t* rec = slot >= 0 ? mig_record(ka, slot) : nullptr;
    if (rec && rec[MIG_KIND] == MIG_RELATIVE) {
        // resume a band saved by a narrower level
        const int rows = rec[MIG_ROWS];
        u.d = rec[MIG_D];
        u.base = rec[MIG_BASE];
        u.lo = rec[MIG_LO];
        u.hi = rec[MIG_HI];
        u.best = rec[MIG_BEST];
        u.T = rec[MIG_T];
        u.T1 = rec[MIG_T1];
        u.T2 = rec[MIG_T2];
        u.R1 = u.T1;  // a record holds d-1 relative to T_{d-1}, d-2 relative to T_{d-2}
        u.R2 = u.T2;
        u.bi = rec[MIG_BI];
        u.bj = rec[MIG_BJ];
        u.cells = (unsigned long long)uint32_t(rec[MIG_CELLS_LO]) |
                  ((unsigned long long)uint32_t(rec[MIG_CELLS_HI]) << 32);
        u.cells0 = u.cells;
        const int i0 = u.base + gl * C;
#pragma unroll
        for (int k = 0; k < C; ++k) {
            const int r = gl * C + k;
            Q1[k] = r < rows ? rec[kMigHeader + r] : NEGU;
            Q2[k] = r < rows ? rec[kMigHeader + rows + r] : NEGU;
            u.aw |= Code(a_code(ka, u, int64_t(i0) + k - 1)) << (2 * k);
            // b' codes as of anti-diagonal d-1: index (d-1) - i - 1
            u.bw |= Code(b_code(ka, u, int64_t(u.d) - 2 - (i0 + k))) << (2 * k);
        }
        u.q0 = -(1 << 30);  // forces a prefetch refill at the loop top
        u.bpre = 0u;
    } else {
        u.base = 0;
        u.lo = 0;
        u.hi = 0;
        u.d = 1;
        u.best = 0;
        u.T = -it.X;
        u.T1 = -it.X;
        u.T2 = -it.X;
        u.R1 = -it.X;
        u.R2 = -it.X;
        u.bi = 0;
        u.bj = 0;
        u.cells = 0ull;
        u.cells0 = 0ull;
        u.q0 = 0;
        u.bpre = b_codes16(ka, u, 16 * gl);
#pragma unroll
        for (int k = 0; k < C; ++k) {
            Q2[k] = NEGU;
            Q1[k] = NEGU;
            u.aw |= Code(a_code(ka, u, int64_t(gl) * C + k - 1)) << (2 * k);
        }
        if (gl == 0) Q1[0] = it.X;  // S(0,0) = 0, relative to T_0 = -X
    }
    const bool too_big = it.X > kGroupMaxX;  // only reachable in the plain form
    u.active = !too_big;
    u.done = too_big;
    u.overflow = too_big;
    u.migrated = false;
}

// Result or escalation of a finished unit (its leader lane writes).
template <int C>
__device__ __forceinline__ void unit_finish(const KernelArgs& ka, const UState<C>& u, int level,
                                            int gl, bool twin) {
    if (gl != 0) return;
    if (u.overflow) {
        if (u.migrated) atomicAdd(&ka.counters->cells[level], u.cells - u.cells0);
        const int nq = escalate_queue(ka, level, twin);
        const unsigned int t = atomicAdd(&ka.counters->tail[nq], 1u);
        ka.queues[size_t(nq) * ka.qcap + t] = u.item;
    } else {
        ExtRes r;
        r.best = u.best;
        r.bi = u.bi;
        r.bj = u.bj;
        r.status = 0;
        r.cells = u.cells;
        ka.ext[u.item] = r;
        atomicAdd(&ka.counters->cells[level], u.cells - u.cells0);
    }
}

// Loop top: slide windows so that the next three steps fit, and keep the b'
// prefetch covering them.  Q2 = d-2, Q1 = d-1.
template <int G, int C>
__device__ __forceinline__ void unit_prepare(const KernelArgs& ka, UState<C>& u, int level, int gl,
                                             int unit, int (&Q2)[C], int (&Q1)[C]) {
    using Gr = Group<G, C>;
    const int rlo = max(u.lo, u.d - u.n);
    const int top = min(u.hi + 3, u.m);  // highest row the next three steps can reach
    const bool need = u.active && top >= u.base + Gr::W;
    if (__any_sync(FULL, need)) {
        const int s = need ? (rlo - 1 - u.base) / C : 0;
        const bool ovf = need && (s <= 0 || top >= u.base + s * C + Gr::W);
        const int sh = (need && !ovf) ? s : 0;
#pragma unroll
        for (int k = 0; k < C; ++k) {
            Q2[k] = __shfl_down_sync(FULL, Q2[k], sh, G);
            Q1[k] = __shfl_down_sync(FULL, Q1[k], sh, G);
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
                Q2[k] = NEGU;
                Q1[k] = NEGU;
                u.aw |= typename Gr::Code(a_code(ka, u, int64_t(i0) + k - 1)) << (2 * k);
                // b' codes as of anti-diagonal d-1: index (d-1) - i - 1
                u.bw |= typename Gr::Code(b_code(ka, u, int64_t(u.d) - 2 - (i0 + k))) << (2 * k);
            }
        }
        if (__any_sync(FULL, ovf)) {
            // save the band for the next level (arrays are unshifted: sh = 0)
            int32_t slot = -1;
            if (ovf && gl == 0) slot = mig_alloc(ka, level);
            slot = __shfl_sync(FULL, slot, unit * G);
            if (ovf && slot >= 0) {
                int32_t* rec = mig_record(ka, slot);
                // (records hold d-1 relative to T_{d-1} and d-2 relative to
                // T_{d-2}; the one-warp forms re-base their values)
#pragma unroll
                for (int k = 0; k < C; ++k) {
                    if constexpr (Gr::LAT) {
                        rec[kMigHeader + gl * C + k] = Q1[k] >= 0 ? Q1[k] + (u.R1 - u.T1) : NEGU;
                        rec[kMigHeader + Gr::W + gl * C + k] =
                            Q2[k] >= 0 ? Q2[k] + (u.R2 - u.T2) : NEGU;
                    } else {
                        rec[kMigHeader + gl * C + k] = Q1[k];
                        rec[kMigHeader + Gr::W + gl * C + k] = Q2[k];
                    }
                }
                if (gl == 0) {
                    rec[MIG_KIND] = MIG_RELATIVE;
                    rec[MIG_ROWS] = Gr::W;
                    rec[MIG_D] = u.d;
                    rec[MIG_BASE] = u.base;
                    rec[MIG_LO] = u.lo;
                    rec[MIG_HI] = u.hi;
                    rec[MIG_BEST] = u.best;
                    rec[MIG_T] = u.T;
                    rec[MIG_T1] = u.T1;
                    rec[MIG_T2] = u.T2;
                    rec[MIG_BI] = u.bi;
                    rec[MIG_BJ] = u.bj;
                    rec[MIG_CELLS_LO] = int32_t(uint32_t(u.cells));
                    rec[MIG_CELLS_HI] = int32_t(uint32_t(u.cells >> 32));
                    rec[MIG_LEVEL] = level;
                    ka.mig_slot[u.item] = slot;
                }
            }
            if (ovf) {
                u.active = false;
                u.done = true;
                u.overflow = true;
                u.migrated = slot >= 0;
            }
        }
    }
    // the next three steps read b' stream indices q .. q+2
    const int q = u.d - u.base - 1;
    const bool refill = u.active && (q < u.q0 || q + 2 >= u.q0 + Gr::PREFETCH);
    if (__any_sync(FULL, refill)) {
        if (refill) {
            u.q0 = q;
            u.bpre = b_codes16(ka, u, q + 16 * gl);
        }
    }
}

// One anti-diagonal step of every unit of the warp.  Q2 = d-2, Q1 = d-1 on
// entry (relative to T2, T1); O receives d (relative to T).  Inactive units
// compute garbage without effects.
template <int G, int C>
__device__ __forceinline__ void group_step(const KernelArgs& ka, UState<C>& u, int gl, int unit,
                                           int (&Q2)[C], int (&Q1)[C], int (&O)[C]) {
    using Gr = Group<G, C>;
    const int rlo = max(u.lo, u.d - u.n);
    const int rhi = min(u.hi + 1, u.m);
    const bool run = u.active && rlo <= rhi;
    // b' shift register: lane 0 takes stream index d - base - 1
    const int qq = u.d - u.base - 1 - u.q0;
    const uint32_t pre = __shfl_sync(FULL, u.bpre, unit * G + ((qq >> 4) & (G - 1)));
    const uint32_t front = (pre >> (uint32_t(qq & 15) * 2u)) & 3u;
    uint32_t carry = uint32_t(__shfl_up_sync(FULL, u.bw, 1, G) >> (2 * (C - 1))) & 3u;
    carry = gl == 0 ? front : carry;
    u.bw = ((u.bw << 2) | typename Gr::Code(carry)) & Gr::MASK2C;
    int upc = __shfl_up_sync(FULL, Q1[C - 1], 1, G);
    int dgc = __shfl_up_sync(FULL, Q2[C - 1], 1, G);
    upc = gl == 0 ? NEGU : upc;
    dgc = gl == 0 ? NEGU : dgc;
    const typename Gr::Code x = u.aw ^ u.bw;
    const typename Gr::Code eq = ~(x | (x >> 1));  // bit 2k set iff row k's bases match
    const uint32_t eq_lo = uint32_t(eq);
    const uint32_t eq_hi = uint32_t(uint64_t(eq) >> 32);  // rows 16..31 (C = 32 only)
    // per-step constants: re-basing of d-1 and d-2 values onto T_d; in the
    // one-warp forms onto T_{d-1} instead (d-1 and d-2 are held relative to
    // R1 = T_{d-2} and R2 = T_{d-3}), so that nothing before the prune waits
    // for the previous anti-diagonal's reductions -- the cells' additions and
    // maxima overlap them -- and a cell is live iff its value >= T_d - T_{d-1}
    const int o1 = Gr::LAT ? ka.sc.gap + u.R1 - u.T1 : ka.sc.gap + u.T1 - u.T;
    const int o2 = Gr::LAT ? u.R2 - u.T1 : u.T2 - u.T;
    const int dT = Gr::LAT ? u.T - u.T1 : 0;
    const int sMM = ka.sc.mismatch + o2;
    const int dsub = ka.sc.mismatch - ka.sc.match;  // added back once per match (as -1 * dsub)
    // rows of this lane inside [rlo, rhi]: bits [k0, k1) of rb
    const int i0 = u.base + gl * C;
    const int k0 = __viaddmin_s32_relu(rlo, -i0, C);     // clamp(rlo - i0, 0, C)
    const int k1 = __viaddmin_s32_relu(rhi, 1 - i0, C);  // clamp(rhi + 1 - i0, 0, C)
    const uint32_t rb = __funnelshift_lc(~0u, 0u, k1) & ~__funnelshift_lc(~0u, 0u, k0);
    // Per row: v = max(up + o1, left + o1, diag + sub); the additions run as
    // multiply-adds (FMA pipe), the 3-way max is one DPX instruction, and
    // g = (d-1 value) + o1 of row k serves as "left" of row k and "up" of
    // row k+1.  Up to 16 rows per lane the substitution score is chosen on
    // the FMA pipe too: the row's match flag, shifted to the sign bit by a
    // multiply, gives y = -1 (match) or 0 as the high word of a product with
    // 1, and sub = mismatch - y * (mismatch - match).
    const int one = ka.one;
    const int wscale = one * Gr::W;  // a run-time W keeps the key a multiply-add
    int gp = upc * one + o1;
    // the dead-row bits and the lane's largest key are collected in NCH
    // independent chains over consecutive row blocks (short dependency chains
    // matter when a long extension runs alone on its SM)
    constexpr int NCH = C >= 16 ? 4 : C >= 2 ? 2 : 1, RB = C / NCH;
    int lk[NCH];
    // dead-row bits, collected by shifting in each row's sign (dead rows hold
    // NEGU < 0): after the loop bit RB-1-(k % RB) of chain k / RB is set iff
    // row k is dead
    uint32_t dc[NCH];
#pragma unroll
    for (int c = 0; c < NCH; ++c) {
        lk[c] = NEGU * Gr::W;
        dc[c] = 0u;
    }
#pragma unroll
    for (int k = 0; k < C; k += 2) {
        int key[2] = {NEGU * Gr::W, NEGU * Gr::W};
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int kk = k + h;
            if (kk >= C) break;  // C = 1
            const int g = Q1[kk] * one + o1;
            const int dg = kk ? Q2[kk - 1] : dgc;
            int t;
            if (C <= 16) {
                const uint32_t mw = eq_lo * ka.pw[kk];
                const int y = __mulhi(int(mw), one);  // -1 on a match, else 0
                t = y * dsub + (dg * one + sMM);
            } else {
                // the 32-row lanes are short of registers: a bit test and select
                const bool match = ((kk < 16 ? eq_lo : eq_hi) & (1u << (2 * (kk & 15)))) != 0u;
                t = dg * one + (match ? sMM - dsub : sMM);
            }
            int v = __vimax3_s32(gp, g, t);
            gp = g;
            const bool inr = (rb & (1u << kk)) != 0u;
            v = (inr & (v >= dT)) ? v : NEGU;
            O[kk] = v;
            key[h] = v * wscale + (C - 1 - kk);
            dc[kk / RB] = __funnelshift_l(uint32_t(v), dc[kk / RB], 1);
        }
        lk[k / RB] = __vimax3_s32(lk[k / RB], key[0], key[1]);
    }
    uint32_t dead = 0u;
    int lkey = lk[0];
#pragma unroll
    for (int c = 0; c < NCH; ++c) dead |= dc[c] << ((NCH - 1 - c) * RB);
#pragma unroll
    for (int c = 1; c < NCH; ++c) lkey = max(lkey, lk[c]);
    // live rows of this lane; bit C-1-k <-> row k
    const uint32_t bits = ~dead & Gr::ALLC;
    if constexpr (C >= 32) {  // (the 32-row lanes are short of registers)
        if (run) u.cells += (unsigned long long)(rhi - rlo + 1);
    } else {
        u.c32 += run ? uint32_t(rhi - rlo + 1) : 0u;
    }
    // the unit's first and last live window rows (W / -1 when none) and its
    // largest key
    int rfirst, rlast;
    const int wkey = unit_max<G>(lkey + (G - 1 - gl) * C);
    if constexpr (G == 32) {
        // whole-warp unit: two more warp reductions
        rfirst = __reduce_min_sync(FULL, bits ? gl * C + (__clz(bits) - (32 - C)) : Gr::W);
        rlast = __reduce_max_sync(FULL, bits ? gl * C + (C - __ffs(bits)) : -1);
    } else {
        // first / last lane with a live row (ballot), then the row inside it
        const uint32_t vote = __ballot_sync(FULL, bits != 0u);
        const uint32_t uvv = (vote >> (unit * G)) & ((1u << G) - 1u);
        const int fl = uvv ? __ffs(uvv) - 1 : 0, ll = uvv ? 31 - __clz(uvv) : 0;
        const uint32_t fb = __shfl_sync(FULL, bits, unit * G + fl);
        const uint32_t lb = __shfl_sync(FULL, bits, unit * G + ll);
        rfirst = uvv ? fl * C + (__clz(fb) - (32 - C)) : Gr::W;
        rlast = uvv ? ll * C + (C - __ffs(lb)) : -1;
    }
    // the anti-diagonal's outcome: it advances when it had a range and a
    // live cell, else the extension ends here.  The best: largest key =
    // highest relative score, smallest row on ties
    if constexpr (C >= 32) {
        // (branches: the 32-row lanes are short of registers)
        if (run && rlast >= 0) {
            const int umax = wkey >> Gr::LOG2W;
            if (umax > u.X) {  // S > best  <=>  S - T_d > X
                const int r = Gr::W - 1 - (wkey & (Gr::W - 1));
                u.best = u.T + umax;
                u.bi = u.base + r;
                u.bj = u.d - u.bi;
            }
            u.T2 = u.T1;
            u.T1 = u.T;
            u.T = u.best - u.X;
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
    const int umax = wkey >> Gr::LOG2W;
    // S > best  <=>  S - T_d > X (one-warp forms: S - T_{d-1} > best - T_{d-1})
    const int ref = Gr::LAT ? u.T1 : u.T;
    const bool imp = adv && umax > (Gr::LAT ? u.best - u.T1 : u.X);
    const int r = Gr::W - 1 - (wkey & (Gr::W - 1));
    const int best = imp ? ref + umax : u.best;
    u.bi = imp ? u.base + r : u.bi;
    u.bj = imp ? u.d - (u.base + r) : u.bj;
    u.best = best;
    const int T = u.T, T1 = u.T1;
    if constexpr (Gr::LAT) {
        // unconditional shifts: a step that does not advance ends the
        // extension, after which they are never read, and the next step's
        // offsets do not wait for the range reductions
        u.R2 = u.R1;
        u.R1 = T1;
        u.T2 = T1;
        u.T1 = T;
        u.T = best - u.X;
    } else {
        u.T2 = adv ? T1 : u.T2;
        u.T1 = adv ? T : T1;
        u.T = adv ? best - u.X : T;
    }
    u.lo = adv ? u.base + rfirst : u.lo;
    u.hi = adv ? u.base + rlast : u.hi;
    u.done = u.done || (u.active && !adv);
    u.active = u.active && adv;
    u.d += 1;
}

template <int G, int C>
__global__ void __launch_bounds__(128, (C == 32) ? 3 : (C == 16) ? 4 : (C == 8) ? 5 : 7)
    k_group(KernelArgs ka, int level, int queue, int phase) {
    using Gr = Group<G, C>;
    const int lane = threadIdx.x & 31;
    const int gl = lane % G, unit = lane / G;
    const bool plain = phase == PHASE_PLAIN;
    const bool twin = queue != level;  // the level's latency form
    const uint32_t* q = ka.queues + size_t(queue) * ka.qcap;
    // plain form: one fixed item per unit, in input order
    const uint32_t plain_id =
        (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * Gr::U + unit;
    bool fresh = true;
    int P0[C], P1[C], P2[C];
#pragma unroll
    for (int k = 0; k < C; ++k) {
        P0[k] = NEGU;
        P1[k] = NEGU;
        P2[k] = NEGU;
    }
    UState<C> u;
    u.active = false;
    u.done = false;
    u.overflow = false;
    u.item = 0;
    u.m = u.n = 0;
    u.base = u.lo = u.hi = 0;
    u.d = 1;
    u.T = u.T1 = u.T2 = u.best = u.bi = u.bj = 0;
    u.R1 = u.R2 = 0;
    u.X = 0;
    u.cells = 0ull;
    u.cells0 = 0ull;
    u.migrated = false;
    u.c32 = 0u;
    u.apos = u.bpos = 0;
    u.dir = 1;
    u.q0 = 0;
    u.bpre = u.aw = u.bw = 0u;
    bool exhausted = false;
    bool first_wave = true;  // the warp's first pop takes static slots
    for (;;) {
        if constexpr (C < 32) {
            u.cells += u.c32;
            u.c32 = 0u;
        }
        if (__any_sync(FULL, u.done || (!u.active && !exhausted))) {
            if (u.done) {
                unit_finish(ka, u, level, gl, twin);
                u.done = false;
            }
            const bool need = !u.active && !exhausted;  // the same in all lanes of a unit
            uint32_t id = 0xffffffffu;
            if (plain) {
                if (need && fresh && plain_id < ka.n_items &&
                    !(ka.items[plain_id].flags & ITEM_SKIP))
                    id = plain_id;
                if (need) fresh = false;
            } else {
                // one pop per warp for all of its idle units, so that a batch
                // with fewer items than unit slots fills whole warps (a warp
                // costs the same whether its units are busy or idle)
                const uint32_t want = __ballot_sync(FULL, need && gl == 0);
                if (want) {
                    unsigned int limit = 0u;
                    const unsigned int slot = pop_unit_slot<G>(ka.counters, queue, phase, want,
                                                               lane, unit, first_wave, limit);
                    if (need && slot < limit) id = q[slot];
                }
            }
            if (need) {
                if (id != 0xffffffffu) unit_init<G, C>(ka, u, id, gl, P0, P1);
                else exhausted = true;
            }
        }
        if (!__any_sync(FULL, u.active)) break;
        unit_prepare<G, C>(ka, u, level, gl, unit, P0, P1);
        group_step<G, C>(ka, u, gl, unit, P0, P1, P2);
        group_step<G, C>(ka, u, gl, unit, P1, P2, P0);
        group_step<G, C>(ka, u, gl, unit, P2, P0, P1);
        // roles are back to P0 = d-2, P1 = d-1
    }
}

}  // namespace

// level -> (G, C)
#define LOGAN_GROUP_LEVELS(X) \
    X(0, 8, 4) X(1, 8, 8) X(2, 8, 16) X(3, 16, 16) X(4, 32, 16) X(5, 32, 32)
// level -> (32, window / 32): the one-warp forms
#define LOGAN_TWIN_LEVELS(X) X(0, 32, 1) X(1, 32, 2) X(2, 32, 4) X(3, 32, 8)

cudaError_t launch_warp_level_persistent(int level, const KernelArgs& ka, int grid, int phase,
                                         cudaStream_t s) {
    switch (level) {
#define CASE(L, G, C) case L: k_group<G, C><<<grid, 128, 0, s>>>(ka, level, level, phase); break;
        LOGAN_GROUP_LEVELS(CASE)
#undef CASE
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_twin_persistent(int level, const KernelArgs& ka, int grid, int phase,
                                   cudaStream_t s) {
    switch (level) {
#define CASE(L, G, C)                                                                           \
    case L:                                                                                     \
        static_assert(G * C == level_window(L), "a one-warp form keeps its level's window");  \
        k_group<G, C><<<grid, 128, 0, s>>>(ka, level, twin_queue(level), phase);               \
        break;
        LOGAN_TWIN_LEVELS(CASE)
#undef CASE
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_warp_level_plain(int level, const KernelArgs& ka, cudaStream_t s) {
    int units_per_block = 0;
    switch (level) {
#define CASE(L, G, C) case L: units_per_block = 4 * (32 / G); break;
        LOGAN_GROUP_LEVELS(CASE)
#undef CASE
        default: return cudaErrorInvalidValue;
    }
    const unsigned int grid = (ka.n_items + units_per_block - 1) / units_per_block;
    if (grid == 0) return cudaSuccess;
    switch (level) {
#define CASE(L, G, C) \
    case L: k_group<G, C><<<grid, 128, 0, s>>>(ka, level, level, PHASE_PLAIN); break;
        LOGAN_GROUP_LEVELS(CASE)
#undef CASE
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

int warp_level_blocks_per_sm(int level) {
    int n = 0;
    cudaError_t e = cudaErrorInvalidValue;
    switch (level) {
#define CASE(L, G, C) \
    case L: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_group<G, C>, 128, 0); break;
        LOGAN_GROUP_LEVELS(CASE)
#undef CASE
        default: break;
    }
    return e == cudaSuccess ? n : 0;
}

int twin_blocks_per_sm(int level) {
    int n = 0;
    cudaError_t e = cudaErrorInvalidValue;
    switch (level) {
#define CASE(L, G, C) \
    case L: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_group<G, C>, 128, 0); break;
        LOGAN_TWIN_LEVELS(CASE)
#undef CASE
        default: break;
    }
    return e == cudaSuccess ? n : 0;
}

}  // namespace logan
