// Internal device-side definitions shared by the library's kernels.
//
// Data layout in HBM (all inside the caller's workspace, 256-byte aligned
// chunks; see api.cu for the carve-up):
//   * 2-bit sequence words: base k of a pool in word k/16, bits 2(k%16)..+1,
//     codes A0 C1 G2 T3.  Caller-packed pools are read in place; ASCII pools
//     are packed once into the workspace at the same base positions.
//   * Item[2*n_pairs]: one extension per pair side (2p = left, 2p+1 = right).
//     An extension reads stream index q of a' and b' at pool position
//     pos + dir*q, so the left extension reads both sequences backwards
//     without a reversed copy (the paper reverses one sequence in memory
//     for coalescing, Sec. IV-B; here the few bases a step needs come from
//     L1-resident words, so direction is just an index sign).
//   * ExtRes[2*n_pairs]: best score, its cell and the computed-cell count of
//     each extension.
//   * per-level work queues of item ids + counters.
//   * fallback ring slots for bands wider than every register window.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace logan {

// -infinity of the recurrence.  Every live score lies in
// [-X, max|score| * (m+n)] subset of (-2^29, 2^29) (host and device
// validation), so NEG + any score parameter stays below any threshold
// best - X >= -2^29 and no sum involving NEG overflows int32.
constexpr int32_t NEG = -(1 << 30);

constexpr int32_t kMaxParam = 1000;
constexpr int32_t kMaxX = 1 << 29;
constexpr int64_t kScoreRange = int64_t(1) << 29;

// item flags
constexpr uint32_t ITEM_LEFT = 1u;   // reads both sequences backwards
constexpr uint32_t ITEM_SKIP = 2u;   // invalid pair or empty extension: not run

struct Item {
    int64_t a_pos;   // pool position of a'[0]
    int64_t b_pos;   // pool position of b'[0]
    uint32_t m, n;   // lengths of a' and b'
    int32_t X;
    uint32_t flags;
};
static_assert(sizeof(Item) == 32, "Item layout");

struct ExtRes {
    int32_t best, bi, bj, status;
    unsigned long long cells;
};
static_assert(sizeof(ExtRes) == 24, "ExtRes layout");

struct PairInfo {
    int32_t seed_score;
    int32_t status;
};

struct Scoring {
    int32_t match, mismatch, gap;
};

// Window levels: level k runs a unit of level_threads(k) threads holding
// level_cells(k) rows each (window = threads * cells).  Levels
// 0..kWarpLevels-1 are G-lane units (32/G extensions per warp): (G, C) =
// (8,4) (8,8) (8,16) (16,16) (32,16) (32,32); level 6 is a 4-warp unit
// with 16 rows per thread (2048 rows), level 7 a 16-warp unit with 8 rows
// per thread (4096 rows).  After the last level comes the global-memory
// ring fallback (index kNumLevels).
constexpr int kNumLevels = 8;
constexpr int kWarpLevels = 6;
// largest X the G-lane levels take (their score keys need
// (X + max score) * window < 2^31); larger X starts at level kWarpLevels
constexpr int32_t kGroupMaxX = (1 << 20) - 4096;
__host__ __device__ constexpr int level_cells(int k) {
    return k == 0 ? 4 : k == 1 ? 8 : k <= 4 ? 16 : k == 5 ? 32 : k == 6 ? 16 : 8;
}
__host__ __device__ constexpr int level_threads(int k) {
    return k <= 2 ? 8 : k == 3 ? 16 : k <= 5 ? 32 : k == 6 ? 128 : 512;
}
__host__ __device__ constexpr int level_window(int k) { return level_cells(k) * level_threads(k); }

// Latency forms.  Levels 0..kTwinLevels-1 put several extensions in a warp,
// which keeps the lanes busy but makes every anti-diagonal step of one
// extension cost a whole warp's instructions.  A long item (the one a
// batch waits for) or an item of a batch too small to fill the GPU runs
// instead in its level's latency form: the same window, one warp of 32
// lanes x window/32 rows, so a step is about half the instructions and its
// reductions are single warp reductions.  (A 4-warp block form of the
// 512-row level, one barrier per step, measured 2x slower per step than
// its one-warp kernel, so levels 4 and up have none.)
constexpr int kTwinLevels = 4;
__host__ __device__ constexpr int twin_cells(int k) { return level_window(k) / 32; }

// Work queues: queue k (k <= kNumLevels) holds the items that level k runs,
// first those binned to it (longest first), then those escalated from k-1;
// queue twin_queue(k) the same for level k's one-warp form.
constexpr int kQueues = kNumLevels + 1 + kTwinLevels;
__host__ __device__ constexpr int twin_queue(int level) { return kNumLevels + 1 + level; }
struct Counters {
    unsigned int tail[kQueues];
    unsigned int head[kQueues];
    unsigned int started[kQueues];             // items that began in this queue (binning)
    unsigned int pad;
    unsigned long long cells[kNumLevels + 1];  // cells computed by each level (both forms)
    unsigned int mig_used[kNumLevels];         // migration records written per level
    unsigned int head2[kQueues];               // pop cursor of the escalated entries
};

// Which entries of a level's queue a launch processes: the binned (initial)
// entries [0, started) in phase 1, the escalated ones [started, tail) in
// phase 2; the plain form takes item i directly.
constexpr int PHASE_INITIAL = 0;
constexpr int PHASE_ESCALATED = 1;
constexpr int PHASE_PLAIN = 2;
constexpr int PHASE_WHOLE = 3;  // every entry [0, tail): levels that run one after another

// Queue slot of each idle unit of a warp (the units whose leader lane is set
// in `want`; `unit` is this lane's unit of G lanes).  A warp's first call in
// a launch takes static slots -- unit u of the launch's warp w gets entry
// w * (32 / G) + u of the phase's range -- so the first entries (the
// longest: binning orders a queue longest first) go to the warps in launch
// order, and with them to the SMs and their schedulers in turn (a block's
// warps sit on one SM's four schedulers, consecutive blocks on different
// SMs), instead of following the order in which warps reach an atomic;
// consecutive entries share a warp, so its units start on items of similar
// length.  Later calls pop dynamically after the static entries.  Every
// unit must be idle at the first call (true at kernel start).  Returns the
// slot; one at or past `limit` means the range is used up.
template <int G>
__device__ __forceinline__ unsigned int pop_unit_slot(Counters* c, int q, int phase, uint32_t want,
                                                      int lane, int unit, bool& first_wave,
                                                      unsigned int& limit) {
    constexpr unsigned int U = 32 / G;
    const unsigned int nwarps = gridDim.x * (blockDim.x >> 5);
    const unsigned int gw = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const unsigned int lo = phase == PHASE_ESCALATED ? c->started[q] : 0u;
    limit = phase == PHASE_INITIAL ? c->started[q] : c->tail[q];
    if (first_wave) {
        first_wave = false;
        return lo + gw * U + unsigned(unit);
    }
    const int leader = __ffs(want) - 1;
    unsigned int first = 0u;
    if (lane == leader)
        first = atomicAdd(phase == PHASE_ESCALATED ? &c->head2[q] : &c->head[q],
                          unsigned(__popc(want)));
    first = __shfl_sync(0xffffffffu, first, leader);
    return lo + U * nwarps + first + unsigned(__popc(want & ((1u << (unit * G)) - 1u)));
}

// Next slot of queue `q` for this phase, or ~0u when the range is used up.
__device__ __forceinline__ unsigned int pop_slot(Counters* c, int q, int phase) {
    if (phase == PHASE_INITIAL) {
        const unsigned int s = atomicAdd(&c->head[q], 1u);
        return s < c->started[q] ? s : ~0u;
    }
    const unsigned int s = c->started[q] + atomicAdd(&c->head2[q], 1u);
    return s < c->tail[q] ? s : ~0u;
}

// Band-state migration.  A unit whose band outgrows its window writes its
// last two anti-diagonals (rows [base, base + rows)) and its scalars to a
// record in HBM; the level it escalates to resumes from there instead of
// recomputing the extension.  Record = kMigHeader int32 header + d-1 rows +
// d-2 rows.  RELATIVE records hold scores minus the threshold of their
// anti-diagonal (T1 for d-1, T2 for d-2; -inf = any negative value),
// ABSOLUTE records hold scores (-inf = NEG).
constexpr int kMigHeader = 16;
enum MigField {
    MIG_KIND = 0, MIG_ROWS, MIG_D, MIG_BASE, MIG_LO, MIG_HI, MIG_BEST, MIG_T, MIG_T1, MIG_T2,
    MIG_BI, MIG_BJ, MIG_CELLS_LO, MIG_CELLS_HI, MIG_LEVEL
};
constexpr int MIG_RELATIVE = 1;
constexpr int MIG_ABSOLUTE = 2;
__host__ __device__ constexpr int mig_stride(int level) { return kMigHeader + 2 * level_window(level); }

// One 2-bit code of a pool (p must lie inside the pool).
__device__ __forceinline__ uint32_t code_at(const uint32_t* __restrict__ w, int64_t p) {
    return (__ldg(w + (p >> 4)) >> (uint32_t(p & 15) * 2u)) & 3u;
}

// Code of stream index q of an extension operand; indices outside [0, len)
// return 0 without touching memory (such cells are out of range anyway).
__device__ __forceinline__ uint32_t stream_code(const uint32_t* __restrict__ w, int64_t pos,
                                                int dir, uint32_t len, int64_t q) {
    if (q < 0 || q >= int64_t(len)) return 0u;
    return code_at(w, pos + (dir > 0 ? q : -q));
}

// 16 consecutive codes of pool positions s..s+15 (s >= 0; the pool keeps one
// spare word after its last base), code of s in the low bits.
__device__ __forceinline__ uint32_t load16(const uint32_t* __restrict__ w, int64_t s) {
    const int64_t wi = s >> 4;
    return __funnelshift_r(__ldg(w + wi), __ldg(w + wi + 1), uint32_t(s & 15) * 2u);
}

// reverses the order of the sixteen 2-bit codes of a word
__device__ __forceinline__ uint32_t rev16(uint32_t x) {
    x = __brev(x);
    return ((x >> 1) & 0x55555555u) | ((x & 0x55555555u) << 1);
}

// stream codes q..q+15 of an operand read from pool position pos in
// direction dir (code q in the low bits); 0 for indices outside [0, len)
__device__ __forceinline__ uint32_t stream_codes16(const uint32_t* __restrict__ w, int64_t pos,
                                                   int dir, int len, int q) {
    if (q < 0 || q >= len) return 0u;
    if (dir > 0) return load16(w, pos + q);
    const int64_t p = pos - q;  // position of code q; codes q+t sit at p-t
    int64_t s = p - 15;
    uint32_t sh = 0u;
    if (s < 0) {
        sh = uint32_t(-s) * 2u;
        s = 0;
    }
    return rev16(load16(w, s)) >> sh;
}

}  // namespace logan
