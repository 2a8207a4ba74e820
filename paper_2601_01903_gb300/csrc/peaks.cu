// Throughput microbenchmark of the arithmetic pipes the FSI kernels lean on:
// float64 add, float64 fused multiply-add and 32-bit / 64-bit integer add.
// The float64 rate is the ALU roofline of the float64 arithmetic
// (TT_FSI_ARITH_F64); the integer rates bound the exact arithmetic.  Each
// thread runs kChains independent dependency chains (enough to cover the
// pipe latency), so the kernel is bound by issue on the measured pipe only.
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "tt_fsi.h"

namespace ttfsi {
namespace {

constexpr int kChains = 8;

template <int KIND>
__global__ void __launch_bounds__(256) peak_kernel(int iters, double seed, double *out) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    if constexpr (KIND == 0 || KIND == 1) {
        double x[kChains];
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = seed + tid * 1e-9 + c;
        const double a = 1.0 - 1e-12 * seed, b = 1e-9 * seed;
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int u = 0; u < 16; ++u)
#pragma unroll
                for (int c = 0; c < kChains; ++c) {
                    if constexpr (KIND == 0)
                        x[c] = __dadd_rn(x[c], b);
                    else
                        x[c] = __fma_rn(x[c], a, b);
                }
        }
        double s = 0.0;
#pragma unroll
        for (int c = 0; c < kChains; ++c) s += x[c];
        if (s == 12345.678) out[tid] = s;  // never true for these inputs; keeps the chains live
    } else {
        // integer adds: x_c <- x_c + x_(c+1 mod 8) from the previous round's
        // values, a linear recurrence the compiler cannot fold into fewer adds
        using U = typename std::conditional<KIND == 2, unsigned, unsigned long long>::type;
        U x[kChains];
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = (U)tid * (U)7 + (U)c + (U)seed;
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                U y[kChains];
#pragma unroll
                for (int c = 0; c < kChains; ++c) y[c] = x[c] + x[(c + 1) % kChains];
#pragma unroll
                for (int c = 0; c < kChains; ++c) x[c] = y[c];
            }
        }
        U s = 0;
#pragma unroll
        for (int c = 0; c < kChains; ++c) s ^= x[c];
        if (s == (U)0x9e3779b9u) out[tid] = (double)s;
    }
}

}  // namespace
}  // namespace ttfsi

extern "C" tt_fsi_status tt_fsi_peak_launch(int kind, int blocks, int iters, double *out_dev,
                                            int64_t *ops_per_launch, struct CUstream_st *stream) {
    using namespace ttfsi;
    if (kind < 0 || kind > 3 || blocks < 1 || iters < 1 || !out_dev || !ops_per_launch)
        return TT_FSI_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const double seed = 1.25;
    switch (kind) {
        case 0: ttfsi::peak_kernel<0><<<blocks, 256, 0, st>>>(iters, seed, out_dev); break;
        case 1: ttfsi::peak_kernel<1><<<blocks, 256, 0, st>>>(iters, seed, out_dev); break;
        case 2: ttfsi::peak_kernel<2><<<blocks, 256, 0, st>>>(iters, seed, out_dev); break;
        default: ttfsi::peak_kernel<3><<<blocks, 256, 0, st>>>(iters, seed, out_dev); break;
    }
    *ops_per_launch = (int64_t)blocks * 256 * (int64_t)iters * 16 * kChains;
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? TT_FSI_OK : TT_FSI_ERR_CUDA;
}
