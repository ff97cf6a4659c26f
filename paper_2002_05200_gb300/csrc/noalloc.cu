// logan_extend_batch_noalloc: the persistent batch extension for callers
// that cannot allocate device memory.
//
// Who needs it: a caller whose device memory is already owned by another
// allocator (a framework's caching pool that reserved most of the GPU), a
// latency-critical loop that must not call cudaMalloc/cudaFree (both can
// synchronise the whole device and stall unrelated streams), or a plugin
// host whose hot path forbids allocation.  Such a caller still passes the
// sequences, seeds and result buffer; the scratch memory the pipeline needs
// (item tables, work queues, counters, the fallback window) comes from one
// file-scope device array instead of a caller workspace.
//
// The array is sized once, at library load, on every GPU that loads the
// library, and stays allocated until the process exits.  In host code its
// name is only a host-side stand-in for the device object: its device
// address is looked up with cudaGetSymbolAddress once per device (with that
// device current) and that address is what the pipeline receives.
#include <mutex>

#include <cuda_runtime.h>

#include "../../include/logan.h"

// Scratch shared by every no-alloc call on a device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[LOGAN_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;

std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on `device` (looked up on the first
// call for that device, with that device made current).
int scratch_address(int device, void** out) {
    if (device < 0 || device >= kMaxDevices) return LOGAN_EINVAL;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[device]) {
        int prev = -1;
        if (cudaGetDevice(&prev) != cudaSuccess) return LOGAN_ECUDA;
        if (prev != device && cudaSetDevice(device) != cudaSuccess) return LOGAN_ECUDA;
        void* ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (prev != device) cudaSetDevice(prev);
        if (e != cudaSuccess || !ptr) return LOGAN_ECUDA;
        g_scratch_addr[device] = ptr;
    }
    *out = g_scratch_addr[device];
    return LOGAN_OK;
}

}  // namespace

extern "C" int logan_extend_batch_noalloc(logan_ctx_t* ctx, const logan_seqs_t* seqsA,
                                          const logan_seqs_t* seqsB, const logan_seed_t* seeds,
                                          uint32_t n_pairs, int32_t match, int32_t mismatch,
                                          int32_t gap, int32_t X, const int32_t* X_per_pair,
                                          logan_result_t* out, void* stream) {
    if (!ctx) return LOGAN_EINVAL;
    int64_t device = -1, ring = 0, graphs = 0, mig = 0, conc = 0;
    if (logan_get_option(ctx, LOGAN_OPT_DEVICE, &device) != LOGAN_OK ||
        logan_get_option(ctx, LOGAN_OPT_RING_CAP, &ring) != LOGAN_OK ||
        logan_get_option(ctx, LOGAN_OPT_GRAPHS, &graphs) != LOGAN_OK ||
        logan_get_option(ctx, LOGAN_OPT_MIGRATION_MB, &mig) != LOGAN_OK ||
        logan_get_option(ctx, LOGAN_OPT_CONCURRENT, &conc) != LOGAN_OK)
        return LOGAN_EINVAL;
    void* scratch = nullptr;
    int rc = scratch_address(int(device), &scratch);
    if (rc != LOGAN_OK) return rc;
    // this form always uses the smaller fallback window, keeps no band-state
    // records (a band that outgrows its window restarts at the next level),
    // runs all levels on the caller's stream and never builds a CUDA graph
    // (instantiating one allocates); the caller's settings are restored
    // afterwards
    rc = logan_set_option(ctx, LOGAN_OPT_RING_CAP, LOGAN_NOALLOC_RING_LOG2);
    if (rc == LOGAN_OK) rc = logan_set_option(ctx, LOGAN_OPT_GRAPHS, 0);
    if (rc == LOGAN_OK) rc = logan_set_option(ctx, LOGAN_OPT_MIGRATION_MB, 0);
    // runs every level on the caller's stream (no auxiliary streams to create)
    if (rc == LOGAN_OK) rc = logan_set_option(ctx, LOGAN_OPT_CONCURRENT, 0);
    size_t need = 0;
    if (rc == LOGAN_OK) rc = logan_workspace_size(ctx, seqsA, seqsB, n_pairs, &need);
    if (rc == LOGAN_OK && need > size_t(LOGAN_NOALLOC_SCRATCH_BYTES)) rc = LOGAN_ENOMEM;
    if (rc == LOGAN_OK)
        rc = logan_extend_batch(ctx, seqsA, seqsB, seeds, n_pairs, match, mismatch, gap, X,
                                X_per_pair, scratch, size_t(LOGAN_NOALLOC_SCRATCH_BYTES), out,
                                stream);
    logan_set_option(ctx, LOGAN_OPT_RING_CAP, ring);
    logan_set_option(ctx, LOGAN_OPT_GRAPHS, graphs);
    logan_set_option(ctx, LOGAN_OPT_MIGRATION_MB, mig);
    logan_set_option(ctx, LOGAN_OPT_CONCURRENT, conc);
    return rc;
}
