// X-drop extension with G-lane units and the band packed two rows to a
// 32-bit register (16-bit SIMD), for window levels whose score range
// provably fits 16 bits.
//
// Method: the paper's recurrence and X-drop rule (Sec. III-A), the
// anti-diagonal sweep of Algorithm 1 with the cell update of Algorithm 2,
// and the per-anti-diagonal maximum of Sec. IV-A -- the same computation as
// the 32-bit G-lane kernel (xdrop_group.cu), with the same results.
//
// Layout.  A unit is G lanes of V "virtual lanes" of 32 rows each: virtual
// lane l = g*V + v (v < V) of lane g owns window rows l*32 + k, k < 32, and
// its register h (h < 16) holds rows h (low half) and h + 16 (high half).
// So the "up" and "diag" predecessors of register h are register h - 1 of
// the same virtual lane (both halves move together); register 0 needs the
// top row of the virtual lane below: a byte permute of two registers of the
// same lane for v > 0, plus one shuffle from the lane below for v = 0.  Two
// virtual lanes per lane (V = 2) halve the units' shared per-anti-diagonal
// work per row (reductions, bookkeeping) at the price of registers.
//
// Values.  The cell in row k of lane g's 32 rows on anti-diagonal e holds
//     sigma = 32768 + 128*u + (31 - k),   u = S - T_e,  T_e = best_{<e} - X,
// when it is live (u >= 0, i.e. sigma >= 32768, bit 15 set), and DEAD =
// 16384 otherwise.  The low bits are the row's code within its lane, so one
// unsigned 16-bit maximum over a lane gives the lane's best score and, for
// equal scores, its smallest row; the unit's reduction then widens the key
// to 32 bits with the lane, (u << log2 W) | (W - 1 - row), so one maximum
// gives the anti-diagonal's best and its smallest row (the tie-break of the
// 32-bit kernel's keyed max).  Every candidate is re-based onto the cell's
// own code: "up" and "diag" come from row k - 1 (code + 1) and get -1, "left"
// from the same row; row 0's predecessors are the lower lane's row 31 (code
// 0), which first get +32.  The host enables this kernel only when
//     128*(Xmax + 2*max(match,0) + |gap| + 2) + 31 <= 32767   and
//     128*(|mismatch| + |gap| + 2*max(match,0) + 2) <= 16383,
// Xmax the largest X that can reach the level.  Then every half-word stays
// inside [0, 65536) through every addition, so the additions are plain
// 32-bit multiply-adds of both halves at once (FMA pipe, no carry or borrow
// between halves), a dead value never climbs to 32768 within the two steps
// it is read, and the only per-half operations are one 3-input 16-bit DPX
// maximum and the bit tests of the prune (ALU pipe).
//
// Range and prune: a cell outside the anti-diagonal's range [rlo, rhi] or
// with sigma < 32768 is stored as DEAD (the range bit of the row is moved to
// the half's bit 15 by a multiply, ANDed with the value, and a byte permute
// with sign replication turns bit 15 of each half into a half-word mask).
//
// Everything else -- the b' shift register fed by a per-unit prefetch,
// window slides at the loop top (here by half a virtual lane, 16 rows), band-state
// records for the next level (32-bit relative scores, the same records the
// 32-bit levels write and read), persistent queue pops -- follows the
// 32-bit kernel.  Codes are kept as two bit planes per lane (bit r = row r),
// so a row's match flag is one bit of ~((a0 ^ b0) | (a1 ^ b1)).
#include "packed16.cuh"

namespace logan {

namespace {

template <int G, int V>
__device__ __forceinline__ void unit_init16(const KernelArgs& ka, S16<V>& u, uint32_t id, int gl,
                                            uint32_t (&Q2)[16 * V], uint32_t (&Q1)[16 * V]) {
    const Item it = ka.items[id];
    u.item = id;
    u.apos = it.a_pos;
    u.bpos = it.b_pos;
    u.dir = (it.flags & ITEM_LEFT) ? -1 : 1;
    u.m = int(it.m);
    u.n = int(it.n);
    u.X = it.X;
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
        u.bi = rec[MIG_BI];
        u.bj = rec[MIG_BJ];
        u.cells = (unsigned long long)uint32_t(rec[MIG_CELLS_LO]) |
                  ((unsigned long long)uint32_t(rec[MIG_CELLS_HI]) << 32);
        u.cells0 = u.cells;
#pragma unroll
        for (int v = 0; v < V; ++v) {
#pragma unroll
            for (int h = 0; h < 16; ++h) {
                uint32_t q1 = 0u, q2 = 0u;
#pragma unroll
                for (int half = 0; half < 2; ++half) {
                    const int r = (gl * V + v) * 32 + h + 16 * half;
                    const int v1 = r < rows ? rec[kMigHeader + r] : NEGU;
                    const int v2 = r < rows ? rec[kMigHeader + rows + r] : NEGU;
                    q1 |= (v1 >= 0 ? live_key(v1, h + 16 * half) : 0x4000u) << (16 * half);
                    q2 |= (v2 >= 0 ? live_key(v2, h + 16 * half) : 0x4000u) << (16 * half);
                }
                Q1[v * 16 + h] = q1;
                Q2[v * 16 + h] = q2;
            }
        }
        load_a_planes(ka, u, gl);
        load_b_planes(ka, u, gl, u.d - 1);  // the shift register holds anti-diagonal d-1
        u.q0 = -(1 << 30);                  // forces a prefetch refill at the loop top
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
        u.bi = 0;
        u.bj = 0;
        u.cells = 0ull;
        u.cells0 = 0ull;
        u.q0 = 0;
        u.bpre = b_codes16_of(ka, u, 16 * gl);
#pragma unroll
        for (int h = 0; h < 16 * V; ++h) {
            Q2[h] = DEAD2;
            Q1[h] = DEAD2;
        }
        // S(0,0) = 0 relative to T_0 = -X, window row 0
        if (gl == 0) Q1[0] = (DEAD2 & 0xffff0000u) | live_key(it.X, 0);
        load_a_planes(ka, u, gl);
#pragma unroll
        for (int v = 0; v < V; ++v) u.b0[v] = u.b1[v] = 0u;
    }
    const bool too_big = it.X > kGroupMaxX;  // never binned here; kept for safety
    u.active = !too_big;
    u.done = too_big;
    u.overflow = too_big;
    u.migrated = false;
}

// Result or escalation of a finished unit (its leader lane writes).
template <int V>
__device__ __forceinline__ void unit_finish16(const KernelArgs& ka, const S16<V>& u, int level,
                                              int gl) {
    if (gl != 0) return;
    if (u.overflow) {
        if (u.migrated) atomicAdd(&ka.counters->cells[level], u.cells - u.cells0);
        const int nq = escalate_queue(ka, level, false);
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

// Loop top: slide windows (by half virtual lanes of 16 rows) so that the
// next three steps fit, save overflowing bands for the next level, and keep
// the b' prefetch covering the next three steps.  Q2 = d-2, Q1 = d-1.
template <int G, int V>
__device__ __forceinline__ void unit_prepare16(const KernelArgs& ka, S16<V>& u, int level, int gl,
                                               int unit, uint32_t (&Q2)[16 * V],
                                               uint32_t (&Q1)[16 * V]) {
    constexpr int W = P16<G, V>::W;
    constexpr int HL = 2 * V;  // half virtual lanes (16 rows) per lane
    const int rlo = max(u.lo, u.d - u.n);
    const int top = min(u.hi + 3, u.m);  // highest row the next three steps can reach
    const bool need = u.active && top >= u.base + W;
    if (__any_sync(FULL, need)) {
        // keep row rlo - 1 (a predecessor of the lowest cell) in the window
        const int s = need ? (rlo - 1 - u.base) / 16 : 0;
        const bool ovf = need && (s <= 0 || top >= u.base + s * 16 + W);
        const int sh = (need && !ovf) ? s : 0;  // half virtual lanes to drop
        // Half j (= 2v + half) of this lane takes half j + sh of the old
        // window.  Candidate c (c < 2V) is virtual lane c % V of lane
        // gl + t + c / V; virtual lane v takes candidate v + r2 whole, or,
        // for an odd shift, that candidate's high half as its low half and
        // the next candidate's low half as its high half.
        const int t = sh / HL;
        const int r2 = (sh % HL) >> 1;
        const bool odd = (sh & 1) != 0;
        // an odd shift moves rows k + 16 to k (code + 16) and the next virtual
        // lane's rows k to k + 16 (code - 16); whole virtual lanes keep codes
        const uint32_t rebase = odd ? 16u - (16u << 16) : 0u;
        // halves of this lane that receive a row of the old window
        uint32_t keep[V];
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const int j = gl * HL + 2 * v + sh;
            keep[v] = (j < HL * G ? 0x0000ffffu : 0u) | (j + 1 < HL * G ? 0xffff0000u : 0u);
        }
        const bool all_ok = gl * HL + HL - 1 + sh < HL * G;
#pragma unroll
        for (int h = 0; h < 16; ++h) {
            uint32_t c2[2 * V], c1[2 * V];
#pragma unroll
            for (int c = 0; c < 2 * V; ++c) {
                c2[c] = __shfl_down_sync(FULL, Q2[(c % V) * 16 + h], t + c / V, G);
                c1[c] = __shfl_down_sync(FULL, Q1[(c % V) * 16 + h], t + c / V, G);
            }
#pragma unroll
            for (int v = 0; v < V; ++v) {
                uint32_t x2 = c2[v], y2 = c2[v + 1], x1 = c1[v], y1 = c1[v + 1];
                if constexpr (V == 2) {
                    if (r2) {
                        x2 = c2[v + 1];
                        y2 = c2[v + 2];
                        x1 = c1[v + 1];
                        y1 = c1[v + 2];
                    }
                }
                if (odd) {
                    x2 = __byte_perm(x2, y2, 0x5432);
                    x1 = __byte_perm(x1, y1, 0x5432);
                }
                if (sh > 0) {
                    Q2[v * 16 + h] = ((x2 + rebase) & keep[v]) | (DEAD2 & ~keep[v]);
                    Q1[v * 16 + h] = ((x1 + rebase) & keep[v]) | (DEAD2 & ~keep[v]);
                }
            }
        }
        {
            uint32_t ca0[2 * V], ca1[2 * V], cb0[2 * V], cb1[2 * V];
#pragma unroll
            for (int c = 0; c < 2 * V; ++c) {
                ca0[c] = __shfl_down_sync(FULL, u.a0[c % V], t + c / V, G);
                ca1[c] = __shfl_down_sync(FULL, u.a1[c % V], t + c / V, G);
                cb0[c] = __shfl_down_sync(FULL, u.b0[c % V], t + c / V, G);
                cb1[c] = __shfl_down_sync(FULL, u.b1[c % V], t + c / V, G);
            }
#pragma unroll
            for (int v = 0; v < V; ++v) {
                uint32_t xa0 = ca0[v], ya0 = ca0[v + 1], xa1 = ca1[v], ya1 = ca1[v + 1];
                uint32_t xb0 = cb0[v], yb0 = cb0[v + 1], xb1 = cb1[v], yb1 = cb1[v + 1];
                if constexpr (V == 2) {
                    if (r2) {
                        xa0 = ca0[v + 1];
                        ya0 = ca0[v + 2];
                        xa1 = ca1[v + 1];
                        ya1 = ca1[v + 2];
                        xb0 = cb0[v + 1];
                        yb0 = cb0[v + 2];
                        xb1 = cb1[v + 1];
                        yb1 = cb1[v + 2];
                    }
                }
                if (odd) {
                    xa0 = __funnelshift_r(xa0, ya0, 16);
                    xa1 = __funnelshift_r(xa1, ya1, 16);
                    xb0 = __funnelshift_r(xb0, yb0, 16);
                    xb1 = __funnelshift_r(xb1, yb1, 16);
                }
                if (sh > 0) {
                    u.a0[v] = xa0;
                    u.a1[v] = xa1;
                    u.b0[v] = xb0;
                    u.b1[v] = xb1;
                }
            }
            if (sh > 0) {
                u.base += 16 * sh;
                if (!all_ok) {
                    // rows new to the window: codes from memory (b' as of d-1)
                    load_a_planes(ka, u, gl);
                    load_b_planes(ka, u, gl, u.d - 1);
                }
            }
        }
        if (__any_sync(FULL, ovf)) {
            // save the band (window rows [base, base + W) of d-1 and d-2, as
            // 32-bit relative scores) for the next level
            int32_t slot = -1;
            if (ovf && gl == 0) slot = mig_alloc(ka, level);
            slot = __shfl_sync(FULL, slot, unit * G);
            if (ovf && slot >= 0) {
                int32_t* rec = mig_record(ka, slot);
#pragma unroll
                for (int v = 0; v < V; ++v) {
#pragma unroll
                    for (int h = 0; h < 16; ++h) {
#pragma unroll
                        for (int half = 0; half < 2; ++half) {
                            const int r = (gl * V + v) * 32 + h + 16 * half;
                            const uint32_t s1 = (Q1[v * 16 + h] >> (16 * half)) & 0xffffu;
                            const uint32_t s2 = (Q2[v * 16 + h] >> (16 * half)) & 0xffffu;
                            rec[kMigHeader + r] = s1 >= LIVE ? int((s1 - LIVE) >> LOG2KS) : NEGU;
                            rec[kMigHeader + W + r] = s2 >= LIVE ? int((s2 - LIVE) >> LOG2KS) : NEGU;
                        }
                    }
                }
                if (gl == 0) {
                    rec[MIG_KIND] = MIG_RELATIVE;
                    rec[MIG_ROWS] = W;
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
    const bool refill = u.active && (q < u.q0 || q + 2 >= u.q0 + P16<G, V>::PREFETCH);
    if (__any_sync(FULL, refill)) {
        if (refill) {
            u.q0 = q;
            u.bpre = b_codes16_of(ka, u, q + 16 * gl);
        }
    }
}

// One anti-diagonal step of every unit of the warp.  Q2 = d-2, Q1 = d-1 on
// entry; O receives d.  Inactive units compute garbage without effects.
template <int G, int V>
__device__ __forceinline__ void step16(const KernelArgs& ka, S16<V>& u, int gl, int unit,
                                       uint32_t (&Q2)[16 * V], uint32_t (&Q1)[16 * V],
                                       uint32_t (&O)[16 * V]) {
    using P = P16<G, V>;
    constexpr int W = P::W;
    const int rlo = max(u.lo, u.d - u.n);
    const int rhi = min(u.hi + 1, u.m);
    const bool run = u.active && rlo <= rhi;
    // b' shift register: every row takes the code its lower neighbour row
    // held on d-1; window row 0 takes stream index d - base - 1
    const int qq = u.d - u.base - 1 - u.q0;
    const uint32_t pre = __shfl_sync(FULL, u.bpre, unit * G + ((qq >> 4) & (G - 1)));
    const uint32_t front = pre >> (uint32_t(qq & 15) * 2u);
    uint32_t c0 = __shfl_up_sync(FULL, u.b0[V - 1], 1, G);
    uint32_t c1 = __shfl_up_sync(FULL, u.b1[V - 1], 1, G);
    c0 = gl == 0 ? (front << 31) : c0;
    c1 = gl == 0 ? ((front >> 1) << 31) : c1;
#pragma unroll
    for (int v = V - 1; v >= 1; --v) {  // row 0 of virtual lane v takes row 31 of v - 1
        u.b0[v] = __funnelshift_l(u.b0[v - 1], u.b0[v], 1);
        u.b1[v] = __funnelshift_l(u.b1[v - 1], u.b1[v], 1);
    }
    u.b0[0] = __funnelshift_l(c0, u.b0[0], 1);
    u.b1[0] = __funnelshift_l(c1, u.b1[0], 1);
    // register 0's up / diag of virtual lane 0: (lane g-1's top row, own row
    // 15); of virtual lane v > 0: (row 31 of virtual lane v-1, own row 15)
    uint32_t xu = __shfl_up_sync(FULL, Q1[(V - 1) * 16 + 15], 1, G);
    uint32_t xd = __shfl_up_sync(FULL, Q2[(V - 1) * 16 + 15], 1, G);
    xu = gl == 0 ? DEAD2 : xu;
    xd = gl == 0 ? DEAD2 : xd;
    // per-step offsets in key units (the re-basing of d-1 and d-2 onto T_d),
    // both halves at once: v = o1W + max(up - 1, left, diag + SM + sub)
    const int one = ka.one;
    const int o1W = (ka.sc.gap + u.T1 - u.T) * KS;
    const uint32_t O1 = uint32_t(o1W) * 0x10001u;
    const int sm = (ka.sc.mismatch + u.T2 - u.T) * KS - 1 - o1W;
    const uint32_t SM = uint32_t(sm) * 0x10001u;
    const uint32_t M1 = 0x10001u * one;  // "- M1" = minus one in both halves (IMAD)
    const int dsw = (ka.sc.match - ka.sc.mismatch) * KS;
    uint32_t fkey = 0u;
    uint32_t L[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
        // row r matches iff both code bits agree: bit r of eq
        const uint32_t eq = ~((u.a0[v] ^ u.b0[v]) | (u.a1[v] ^ u.b1[v]));
        const uint32_t eqB = eq >> 8;  // rows 8.. and 24.. for registers 8..15
        // (the row below has code 0 where row 0 expects code 32 from a
        // predecessor: +32 on the low half)
        const uint32_t bu = v ? Q1[(v - 1) * 16 + 15] : xu;
        const uint32_t bd = v ? Q2[(v - 1) * 16 + 15] : xd;
        const uint32_t U0 = __byte_perm(bu, Q1[v * 16 + 15], 0x5432) * uint32_t(one) + 32u;
        const uint32_t D0 = __byte_perm(bd, Q2[v * 16 + 15], 0x5432) * uint32_t(one) + 32u;
        // rows of this virtual lane inside [rlo, rhi]: bits [k0, k1) of rb
        const int i0 = u.base + (gl * V + v) * 32;
        const int k0 = __viaddmin_s32_relu(rlo, -i0, 32);
        const int k1 = __viaddmin_s32_relu(rhi, 1 - i0, 32);
        const uint32_t rb = __funnelshift_lc(~0u, 0u, k1) & ~__funnelshift_lc(~0u, 0u, k0);
        uint32_t Lv = 0u;
        uint32_t lk1 = 0u;
#pragma unroll
        for (int h = 0; h < 16; ++h) {
            const int g = v * 16 + h;
            const uint32_t sU = h ? Q1[g - 1] : U0;
            const uint32_t sD = h ? Q2[g - 1] : D0;
            const uint32_t sUm = sU * uint32_t(one) - M1;
            const uint32_t t = sD * uint32_t(one) + SM;
            const uint32_t Mh = (h < 8 ? eq : eqB) & (0x10001u << (h & 7));
            const uint32_t t2 = Mh * uint32_t(dsw >> (h & 7)) + t;
            const uint32_t u3 = __vimax3_u16x2(sUm, Q1[g], t2);
            const uint32_t val = u3 * uint32_t(one) + O1;
            // row h's range bit -> bit 15, row h+16's -> bit 31
            const uint32_t x = val & (rb * ka.pw16[h]);
            const uint32_t mk = sign_mask16(x);  // 0xffff per live half
            const uint32_t p = (val & mk) | (DEAD2 & ~mk);
            Lv |= mk & (0x10001u << h);
            O[g] = p;
            if (h & 1) lk1 = __vimax3_u16x2(lk1, O[g - 1], p);
        }
        L[v] = Lv;
        // the virtual lane's largest key, widened with its position: (u,
        // code in the virtual lane) -> (u << log2 W) | (W - 1 - row)
        const uint32_t lkey = max(lk1 & 0xffffu, lk1 >> 16);
        const uint32_t fk = lkey >= LIVE ? (((lkey - LIVE) >> LOG2KS) << P::LOG2W) |
                                               uint32_t(W - 32 - (gl * V + v) * 32) + (lkey & 31u)
                                         : 0u;
        fkey = max(fkey, fk);
    }
    // the lane's first / last live rows, then the unit's
    int fr, lr;
    bool any;
    if constexpr (V == 1) {
        fr = __ffs(L[0]) - 1;
        lr = 31 - __clz(L[0]);
        any = L[0] != 0u;
    } else {
        const unsigned long long LL = (unsigned long long)L[0] | ((unsigned long long)L[1] << 32);
        fr = __ffsll(LL) - 1;
        lr = 63 - __clzll(LL);
        any = LL != 0ull;
    }
    const uint32_t flw =
        any ? (uint32_t(W - (gl * P::C + fr)) | (uint32_t(gl * P::C + lr + 1) << 16)) : 0u;
    const uint32_t wkey = unit_max_u32<G>(fkey);
    const uint32_t fl = unit_max_u16x2<G>(flw);
    u.c32 += run ? uint32_t(rhi - rlo + 1) : 0u;
    // the anti-diagonal's outcome, without branches: it advances when it
    // had a range and a live cell, else the extension ends here
    const bool adv = run && fl != 0u;
    const int umax = int(wkey >> P::LOG2W);
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

template <int G, int V>
__global__ void __launch_bounds__(128, V == 1 ? 4 : 3)
    k_group16(KernelArgs ka, int level, int queue, int phase) {
    const int lane = threadIdx.x & 31;
    const int gl = lane % G, unit = lane / G;
    const uint32_t* q = ka.queues + size_t(queue) * ka.qcap;
    uint32_t P0[16 * V], P1[16 * V], P2[16 * V];
#pragma unroll
    for (int h = 0; h < 16 * V; ++h) {
        P0[h] = DEAD2;
        P1[h] = DEAD2;
        P2[h] = DEAD2;
    }
    S16<V> u;
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
#pragma unroll
    for (int v = 0; v < V; ++v) u.a0[v] = u.a1[v] = u.b0[v] = u.b1[v] = 0u;
    u.c32 = 0u;
    bool exhausted = false;
    bool first_wave = true;  // the warp's first pop takes static slots
    for (;;) {
        u.cells += u.c32;
        u.c32 = 0u;
        if (__any_sync(FULL, u.done || (!u.active && !exhausted))) {
            if (u.done) {
                unit_finish16(ka, u, level, gl);
                u.done = false;
            }
            const bool need = !u.active && !exhausted;  // the same in all lanes of a unit
            uint32_t id = 0xffffffffu;
            // one pop per warp for all of its idle units
            const uint32_t want = __ballot_sync(FULL, need && gl == 0);
            if (want) {
                unsigned int limit = 0u;
                const unsigned int slot =
                    pop_unit_slot<G>(ka.counters, queue, phase, want, lane, unit, first_wave, limit);
                if (need && slot < limit) id = q[slot];
            }
            if (need) {
                if (id != 0xffffffffu) unit_init16<G, V>(ka, u, id, gl, P0, P1);
                else exhausted = true;
            }
        }
        if (!__any_sync(FULL, u.active)) break;
        unit_prepare16<G, V>(ka, u, level, gl, unit, P0, P1);
        step16<G, V>(ka, u, gl, unit, P0, P1, P2);
        step16<G, V>(ka, u, gl, unit, P1, P2, P0);
        step16<G, V>(ka, u, gl, unit, P2, P0, P1);
    }
}

}  // namespace

// level -> (G, V) of its packed form: G lanes of V virtual lanes of 32 rows
#define LOGAN_PACKED_LEVELS(X) X(2, 4, 1) X(3, 8, 1) X(4, 16, 1) X(5, 16, 2) X(6, 32, 2)

bool packed_level(int level) {
    switch (level) {
#define CASE(L, G, V) case L: return true;
        LOGAN_PACKED_LEVELS(CASE)
#undef CASE
        default: return false;
    }
}

cudaError_t launch_packed_level_persistent(int level, const KernelArgs& ka, int grid, int phase,
                                           cudaStream_t s) {
    switch (level) {
#define CASE(L, G, V)                                                                      \
    case L:                                                                                \
        static_assert(P16<G, V>::W == level_window(L), "a packed form keeps its level's window"); \
        k_group16<G, V><<<grid, 128, 0, s>>>(ka, level, level, phase);                    \
        break;
        LOGAN_PACKED_LEVELS(CASE)
#undef CASE
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

int packed_level_blocks_per_sm(int level) {
    int n = 0;
    cudaError_t e = cudaErrorInvalidValue;
    switch (level) {
#define CASE(L, G, V) \
    case L: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_group16<G, V>, 128, 0); break;
        LOGAN_PACKED_LEVELS(CASE)
#undef CASE
        default: break;
    }
    return e == cudaSuccess ? n : 0;
}

}  // namespace logan
