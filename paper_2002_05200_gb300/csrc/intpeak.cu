// Instruction-throughput microbenchmark (the ALU roofline's measured
// denominator; the paper's roofline, Sec. VII, counts warp instructions).
// Each thread runs 8 independent dependency chains of one operation so that
// issue, not latency, bounds the rate.  The chains are folded into one
// conditional store so the compiler cannot drop them.
//
// ops (one instruction per chain step unless noted); every step reads a
// neighbouring chain's previous value, so the chains cannot be folded:
//   0 int add         1 int max         2 int add+max (DPX)
//   3 int16x2 3-in max 4 int16x2 add+max 5 fp32 max
//   6 fp16x2 max      7 fp16x2 add      8 int multiply-add
//   9 fp32 add        10 fp32 fma       11 3-input logic
//   12 bit test + select (2)            13 byte permute
//   14 fp32 compare + select (2)
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "../../include/logan.h"

namespace {

template <int OP>
__global__ void __launch_bounds__(256) k_intpeak(int iters, int seed, int* out) {
    int a[8];
    float f[8];
    __half2 h[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        a[k] = seed + int(threadIdx.x) * 8 + k;
        f[k] = float(a[k]);
        h[k] = __halves2half2(__int2half_rn(a[k] & 7), __int2half_rn(k & 3));
    }
    const int b = seed * 3 + 1, c = seed - 7;
    const unsigned int ub = unsigned(b) * 0x00010001u, uc = unsigned(c) & 0xffffu;
    const float fb = float(b);
    const __half2 hb = __halves2half2(__int2half_rn(b & 7), __int2half_rn(c & 7));
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 16; ++r) {
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int n1 = (k + 1) & 7, n2 = (k + 2) & 7;
                if (OP == 0) a[k] = a[k] + a[n1];
                else if (OP == 1) a[k] = max(a[k], a[n1]);
                else if (OP == 2) a[k] = __viaddmax_s32(a[k], b, a[n1]);
                else if (OP == 3) a[k] = int(__vimax3_s16x2(unsigned(a[k]), unsigned(a[n1]), unsigned(a[n2])));
                else if (OP == 4) a[k] = int(__viaddmax_s16x2(unsigned(a[k]), ub, unsigned(a[n1])));
                else if (OP == 5) f[k] = fmaxf(f[k], f[n1]);
                else if (OP == 6) h[k] = __hmax2(h[k], h[n1]);
                else if (OP == 7) h[k] = __hadd2(h[k], h[n1]);
                else if (OP == 8) a[k] = a[k] * a[n1] + b;
                else if (OP == 9) f[k] = f[k] + f[n1];
                else if (OP == 10) f[k] = fmaf(f[k], fb, f[n1]);
                else if (OP == 11) a[k] = a[k] ^ a[n1] ^ (a[n2] & b);
                else if (OP == 12) a[k] = (a[n1] & 4) ? a[k] : c;
                else if (OP == 13) a[k] = int(__byte_perm(unsigned(a[k]), unsigned(a[n1]), 0x5432u));
                else f[k] = f[n1] >= 0.f ? f[k] : -1e30f;
            }
        }
    }
    int acc = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k)
        acc ^= a[k] ^ __float_as_int(f[k]) ^ int(__half_as_short(__low2half(h[k])));
    if (acc == 0x7fffffff) out[blockIdx.x] = acc;
}

template <int OP>
void launch(int grid, int n, int* out) {
    k_intpeak<OP><<<grid, 256>>>(n, 1, out);
}

}  // namespace

extern "C" int logan_intpeak(int device, int op, int iters, double* instr_per_s, float* ms) {
    if (!instr_per_s || !ms || op < 0 || op > 14 || iters <= 0) return LOGAN_EINVAL;
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
    void (*fns[15])(int, int, int*) = {launch<0>,  launch<1>,  launch<2>,  launch<3>,  launch<4>,
                                       launch<5>,  launch<6>,  launch<7>,  launch<8>,  launch<9>,
                                       launch<10>, launch<11>, launch<12>, launch<13>, launch<14>};
    fns[op](grid, iters / 8 + 1, out);  // warm-up
    cudaEventRecord(e0);
    fns[op](grid, iters, out);
    cudaEventRecord(e1);
    cudaError_t e = cudaEventSynchronize(e1);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (e != cudaSuccess || t <= 0.f) return LOGAN_ECUDA;
    // chain steps executed (ops 12 and 14 take two instructions per step)
    const double per_step = (op == 12 || op == 14) ? 2.0 : 1.0;
    const double instr = double(grid) * 256.0 * iters * 16.0 * 8.0 * per_step;
    *instr_per_s = instr / (double(t) * 1e-3);
    *ms = t;
    return LOGAN_OK;
}
