// Shared pieces of the packed 16-bit kernels (xdrop_group16.cu: linear
// gaps; xdrop_affine16.cu: affine gaps): the key encoding, the per-unit
// state, the code bit planes and the reductions.  Two band rows share one
// 32-bit register as 16-bit keys 32768 + 128*u + (31 - k) (u the score
// minus the anti-diagonal's pruning threshold, k the row within its
// 32-row lane) when live, DEAD = 16384 otherwise.
#pragma once

#include "internal.h"

namespace logan {

namespace {

constexpr uint32_t FULL = 0xffffffffu;
constexpr uint32_t LIVE = 0x8000u;
constexpr uint32_t DEAD2 = 0x40004000u;  // DEAD in both halves
constexpr int NEGU = -(1 << 20);         // -inf of the 32-bit relative records

template <int G, int V>
struct P16 {
    static constexpr int C = 32 * V;  // rows per lane (16 registers per virtual lane)
    static constexpr int W = G * C;
    static constexpr int LOG2W = W == 32    ? 5
                                 : W == 64  ? 6
                                 : W == 128 ? 7
                                 : W == 256 ? 8
                                 : W == 512 ? 9
                                 : W == 1024 ? 10
                                             : 11;
    static constexpr int PREFETCH = 16 * G;
    static_assert((1 << LOG2W) == W, "window must be a power of two");
    static_assert(V == 1 || V == 2, "one or two virtual lanes per lane");
};
// score scale of a key: the substitution step multiplies a match flag at bit
// h' < 8 by (match - mismatch) * 128 >> h', which is exact
constexpr int KS = 128;
constexpr int LOG2KS = 7;

template <int V>
struct S16 {
    int base, lo, hi, d;
    int best, T, T1, T2;
    int bi, bj;
    int m, n, X;
    unsigned long long cells, cells0;
    uint32_t c32;  // cells of the current loop iteration, folded into cells at its top
    int64_t apos, bpos;
    int dir;
    int q0;
    uint32_t bpre;
    uint32_t item;
    bool active, done, overflow, migrated;
    uint32_t a0[V], a1[V], b0[V], b1[V];  // code bit planes of each virtual lane's 32 rows
};

// 16 two-bit codes (code t at bits 2t) -> their low and high bit planes
// (bit t of each).
__device__ __forceinline__ void planes16(uint32_t c, uint32_t& p0, uint32_t& p1) {
    uint32_t x = c & 0x55555555u, y = (c >> 1) & 0x55555555u;
    x = (x | (x >> 1)) & 0x33333333u;
    y = (y | (y >> 1)) & 0x33333333u;
    x = (x | (x >> 2)) & 0x0f0f0f0fu;
    y = (y | (y >> 2)) & 0x0f0f0f0fu;
    x = (x | (x >> 4)) & 0x00ff00ffu;
    y = (y | (y >> 4)) & 0x00ff00ffu;
    p0 = (x | (x >> 8)) & 0xffffu;
    p1 = (y | (y >> 8)) & 0xffffu;
}

// stream codes q..q+15 (code q in the low bits), 0 for indices below 0 and
// outside [0, len) when the whole group is
__device__ __forceinline__ uint32_t codes16z(const uint32_t* __restrict__ w, int64_t pos, int dir,
                                             int len, int q) {
    if (q >= 0) return stream_codes16(w, pos, dir, len, q);
    if (q <= -16) return 0u;
    return stream_codes16(w, pos, dir, len, 0) << (2u * uint32_t(-q));
}

// a' codes of virtual lane l's 32 rows (row r needs a' index base + l*32 + r - 1)
template <int V>
__device__ __forceinline__ void load_a_planes(const KernelArgs& ka, S16<V>& u, int gl) {
#pragma unroll
    for (int v = 0; v < V; ++v) {
        const int q = u.base + (gl * V + v) * 32 - 1;
        uint32_t p0, p1, h0, h1;
        planes16(codes16z(ka.wa, u.apos, u.dir, u.m, q), p0, p1);
        planes16(codes16z(ka.wa, u.apos, u.dir, u.m, q + 16), h0, h1);
        u.a0[v] = p0 | (h0 << 16);
        u.a1[v] = p1 | (h1 << 16);
    }
}

// b' codes of the lane's rows as of anti-diagonal e: row r of virtual lane
// l needs b' index e - (base + l*32 + r) - 1, decreasing with r
template <int V>
__device__ __forceinline__ void load_b_planes(const KernelArgs& ka, S16<V>& u, int gl, int e) {
#pragma unroll
    for (int v = 0; v < V; ++v) {
        const int top = e - (u.base + (gl * V + v) * 32) - 1;  // index of row 0
        uint32_t p0, p1, h0, h1;
        // rows 0..15: indices top-15 .. top (row 15 .. row 0)
        planes16(rev16(codes16z(ka.wb, u.bpos, u.dir, u.n, top - 15)), p0, p1);
        planes16(rev16(codes16z(ka.wb, u.bpos, u.dir, u.n, top - 31)), h0, h1);
        u.b0[v] = p0 | (h0 << 16);
        u.b1[v] = p1 | (h1 << 16);
    }
}

// 0xffff in each 16-bit half whose bit 15 is set, else 0: a byte permute in
// its sign-replicating form (a selector nibble with its top bit set copies
// the sign of the selected byte; the __byte_perm intrinsic uses only the
// low three bits of each nibble, so this is written in PTX)
__device__ __forceinline__ uint32_t sign_mask16(uint32_t x) {
    uint32_t r;
    asm("prmt.b32 %0, %1, 0, 0xBB99;" : "=r"(r) : "r"(x));
    return r;
}

template <int G>
__device__ __forceinline__ uint32_t unit_max_u32(uint32_t v) {
#pragma unroll
    for (int o = G / 2; o >= 1; o >>= 1) v = max(v, __shfl_xor_sync(FULL, v, o, G));
    return v;
}

template <int G>
__device__ __forceinline__ uint32_t unit_max_u16x2(uint32_t v) {
#pragma unroll
    for (int o = G / 2; o >= 1; o >>= 1) v = __vimax3_u16x2(v, __shfl_xor_sync(FULL, v, o, G), 0u);
    return v;
}

// b' stream codes q..q+15 (code q in the low bits; 0 when q is outside [0, n))
template <int V>
__device__ __forceinline__ uint32_t b_codes16_of(const KernelArgs& ka, const S16<V>& u, int q) {
    return stream_codes16(ka.wb, u.bpos, u.dir, u.n, q);
}

// live key of row k of a lane with relative score u (u >= 0)
__device__ __forceinline__ uint32_t live_key(int u, int k) {
    return LIVE + uint32_t(u) * uint32_t(KS) + uint32_t(31 - k);
}

}  // namespace

}  // namespace logan
