// Host-side declarations shared by the library's translation units.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "logan_dev.cuh"

namespace logan {

// Everything an extension kernel needs, passed by value to every launch.
struct KernelArgs {
    const uint32_t* wa;      // 2-bit words of pool A
    const uint32_t* wb;      // 2-bit words of pool B
    const Item* items;
    ExtRes* ext;
    uint32_t* queues;        // (kNumLevels + 1) queues of qcap item ids
    Counters* counters;
    int32_t* ring;           // fallback ring slots: n_ring_slots * 3 * ring_cap ints
    uint32_t qcap;           // = number of items
    uint32_t n_items;
    uint32_t ring_cap;       // power of two
    uint32_t n_ring_slots;
    uint32_t max_level;      // last register level before the ring
    Scoring sc;
    // always 1; read at run time so that "x * one + y" stays a multiply-add
    // (FMA pipe) instead of an integer add on the busier ALU pipe
    int32_t one;
    // pw[k] = 2^(31 - 2k): multiplying a 2-bit-per-row flag word by it moves
    // row k's flag to the sign bit (a multiply-add, FMA pipe)
    uint32_t pw[16];
    // pw16[h] = 2^(15 - h): moves bits h and h + 16 of a row mask to bits 15
    // and 31 (the halves' top bits) as a multiply-add
    uint32_t pw16[16];
    // level an item goes to when its band outgrows level k (kNumLevels = ring)
    int8_t next_level[kNumLevels];
    // migration records written by level k (nullptr or cap 0: restart instead)
    int32_t* mig_pool[kNumLevels];
    uint32_t mig_cap[kNumLevels];
    int32_t* mig_slot;  // per item: (level << 24) | record, or -1
};

__device__ __forceinline__ int32_t* mig_record(const KernelArgs& ka, int32_t slot) {
    const int lv = slot >> 24;
    return ka.mig_pool[lv] + size_t(slot & 0xffffff) * size_t(mig_stride(lv));
}

// A record slot of `level`, or -1 when its pool is full (the item restarts).
__device__ __forceinline__ int32_t mig_alloc(const KernelArgs& ka, int level) {
    if (ka.mig_pool[level] == nullptr || ka.mig_cap[level] == 0) return -1;
    const unsigned int idx = atomicAdd(&ka.counters->mig_used[level], 1u);
    return idx < ka.mig_cap[level] ? int32_t((unsigned(level) << 24) | idx) : -1;
}

__device__ __forceinline__ int escalate(const KernelArgs& ka, int level) {
    const int nl = ka.next_level[level];
    return nl <= int(ka.max_level) ? nl : kNumLevels;
}

// queue an item outgrowing `level` goes to: a one-warp form's items stay in
// one-warp forms while the next level has one
__device__ __forceinline__ int escalate_queue(const KernelArgs& ka, int level, bool twin) {
    const int nl = escalate(ka, level);
    return (twin && nl < kTwinLevels) ? twin_queue(nl) : nl;
}

// extension kernels (xdrop_group.cu / xdrop_cta.cu / xdrop_ring.cu)
cudaError_t launch_warp_level_persistent(int level, const KernelArgs& ka, int grid, int phase,
                                         cudaStream_t s);
cudaError_t launch_warp_level_plain(int level, const KernelArgs& ka, cudaStream_t s);
int warp_level_blocks_per_sm(int level);
// packed 16-bit form of a register level (xdrop_group16.cu): same queues,
// results and band-state records as the level's 32-bit kernel
bool packed_level(int level);
cudaError_t launch_packed_level_persistent(int level, const KernelArgs& ka, int grid, int phase,
                                           cudaStream_t s);
int packed_level_blocks_per_sm(int level);
// level k's one-warp form (k < kTwinLevels), persistent over twin_queue(k)
cudaError_t launch_twin_persistent(int level, const KernelArgs& ka, int grid, int phase,
                                   cudaStream_t s);
int twin_blocks_per_sm(int level);
cudaError_t launch_cta_level(int level, const KernelArgs& ka, int grid, int phase, cudaStream_t s);
int cta_level_blocks_per_sm(int level);
cudaError_t launch_ring(const KernelArgs& ka, int grid, cudaStream_t s);
// affine-gap window levels (xdrop_affine.cu): level l pops queue l
int affine_levels();
int affine_blocks_per_sm(int level);
cudaError_t launch_affine_level(int level, const KernelArgs& ka, int gap_open, int gap_extend,
                                int grid, cudaStream_t s);
// their packed 16-bit forms (xdrop_affine16.cu), for the levels that have one
bool affine16_level(int level);
cudaError_t launch_affine16_level(int level, const KernelArgs& ka, int gap_open, int gap_extend,
                                  int n_levels, int grid, cudaStream_t s);
int affine16_blocks_per_sm(int level);
// bands that outgrow the affine windows, and X too large for their keys:
// every entry of queue q continues in the device-memory ring kernel
// (xdrop_matrix.cu) at the workspace ring's width
cudaError_t launch_affine_ring(const KernelArgs& ka, int q, int go, int ge, int grid,
                               cudaStream_t s);

// pre/post-processing kernels (prep.cu)
struct PoolDev {
    const void* bases;
    const uint64_t* offsets;
    const uint32_t* lengths;
    uint32_t count;
    uint32_t packed2bit;
    uint64_t pool_bases;
    const uint32_t* words;   // 2-bit words used by the kernels
    uint8_t* bad;            // per-sequence invalid flag
};

cudaError_t launch_pack(const PoolDev& p, uint32_t* words_out, cudaStream_t s);
cudaError_t launch_validate(const PoolDev& p, cudaStream_t s);
cudaError_t launch_split(const PoolDev& A, const PoolDev& B, const void* seeds, uint32_t n_pairs,
                         Scoring sc, int32_t X, const int32_t* Xs, Item* items, PairInfo* info,
                         ExtRes* ext, int32_t* mig_slot, cudaStream_t s);
constexpr int kBuckets = 128;
// X class -> starting window level (the autotune table), plus the highest
// register level in use and an optional X-class filter (-1 = all classes).
struct LevelTable {
    int8_t lv[8];
    int max_level;
    // items with m + n >= long_min that start below level kTwinLevels go to
    // that level's one-warp form (0xffffffff: none)
    uint32_t long_min;
};
cudaError_t launch_bin(const Item* items, uint32_t n_items, LevelTable table, int force_level, uint32_t* hist, uint32_t* queues, uint32_t qcap,
                       Counters* counters, cudaStream_t s);
cudaError_t launch_reset_counters(Counters* c, uint32_t first_level_items, int first_level,
                                  cudaStream_t s);
cudaError_t launch_combine(const void* seeds, const PairInfo* info, const ExtRes* ext,
                           uint32_t n_pairs, void* out, cudaStream_t s);

// X classes used by the autotune table: X <= 15, <= 35, <= 75, <= 150, <= 300,
// <= 700, <= 2000, larger.
constexpr int kXClasses = 8;
__host__ __device__ inline int x_class(int32_t X) {
    return X <= 15 ? 0 : X <= 35 ? 1 : X <= 75 ? 2 : X <= 150 ? 3 : X <= 300 ? 4
         : X <= 700 ? 5 : X <= 2000 ? 6 : 7;
}

}  // namespace logan
