// Integer-instruction throughput microbenchmark (the ALU roofline's measured
// denominator; the paper's roofline, Sec. VII, counts warp instructions).
// Each thread runs 8 independent dependency chains so that issue, not
// latency, bounds the rate.  The chain values are folded into one store so
// the compiler cannot drop them.
#include <cuda_runtime.h>

#include "../../include/logan.h"

namespace {

template <int OP>
__global__ void __launch_bounds__(256) k_intpeak(int iters, int seed, int* out) {
    int a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = seed + threadIdx.x * 8 + k;
    const int b = seed * 3 + 1, c = seed - 7;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 16; ++r) {
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                if (OP == 0) a[k] = a[k] + b;
                else if (OP == 1) a[k] = max(a[k], c + k) ^ r;  // max + xor: 2 instr
                else a[k] = __viaddmax_s32(a[k], b, c);
            }
        }
    }
    int acc = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) acc ^= a[k];
    if (acc == 0x7fffffff) out[blockIdx.x] = acc;
}

}  // namespace

extern "C" int logan_intpeak(int device, int op, int iters, double* instr_per_s, float* ms) {
    if (!instr_per_s || !ms || op < 0 || op > 2 || iters <= 0) return LOGAN_EINVAL;
    if (cudaSetDevice(device) != cudaSuccess) return LOGAN_ECUDA;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
        return LOGAN_ECUDA;
    const int grid = sms * 8;  // 8 x 256 threads = 2048 per SM
    int* out = nullptr;
    if (cudaMalloc(&out, sizeof(int) * grid) != cudaSuccess) return LOGAN_ECUDA;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    auto launch = [&](int n) {
        if (op == 0) k_intpeak<0><<<grid, 256>>>(n, 1, out);
        else if (op == 1) k_intpeak<1><<<grid, 256>>>(n, 1, out);
        else k_intpeak<2><<<grid, 256>>>(n, 1, out);
    };
    launch(iters / 8 + 1);  // warm-up
    cudaEventRecord(e0);
    launch(iters);
    cudaEventRecord(e1);
    cudaError_t e = cudaEventSynchronize(e1);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (e != cudaSuccess || t <= 0.f) return LOGAN_ECUDA;
    const double per_iter = (op == 1) ? 2.0 : 1.0;  // instructions per chain step
    const double instr = double(grid) * 256.0 * iters * 16.0 * 8.0 * per_iter;
    *instr_per_s = instr / (double(t) * 1e-3);
    *ms = t;
    return LOGAN_OK;
}
