// What the alignment-path and overlap calls (traceback.cu, overlap.cu) need
// from the context and from a finished logan_extend_batch, defined in api.cu.
#pragma once

#include "internal.h"

#include "../../include/logan.h"

namespace logan {

struct TracebackTiming {
    logan_traceback_stats_t last{};
    bool valid = false;  // a timed call completed
};

// the context's record; never null for a valid context
TracebackTiming* ctx_traceback_timing(logan_ctx_t* c);

// The context's pool for the scratch of the overlap and alignment-path
// calls: freed scratch stays mapped until the context is destroyed, so
// repeated calls do not map gigabytes again.  Null if it cannot be created
// (the callers then use the device's default pool).
cudaMemPool_t ctx_scratch_pool(logan_ctx_t* c);

// the matrix call's record of the windows that ran packed (read back with
// LOGAN_OPT_MATRIX_PACKED)
void ctx_set_matrix_packed(logan_ctx_t* c, uint32_t levels);

// Device views into the workspace of a finished logan_extend_batch call
// with the same pools and pair count: the 2-bit words of both pools, the
// split items (two per pair, left first), every item's result (best cell,
// cells) and every pair's status.
struct ExtensionViews {
    const uint32_t* wa = nullptr;
    const uint32_t* wb = nullptr;
    const Item* items = nullptr;
    const ExtRes* ext = nullptr;
    const PairInfo* info = nullptr;
    uint32_t launches = 0;  // kernels that call launched
};
void extension_views(const logan_ctx_t* c, const logan_seqs_t* A, const logan_seqs_t* B,
                     uint32_t n_pairs, const void* ws, ExtensionViews* v);

}  // namespace logan
