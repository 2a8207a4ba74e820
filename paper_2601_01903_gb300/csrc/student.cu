// Amortised FSI explainer ("student"): a GELU MLP that maps an instance x to
// its FSI scores, trained on (x, exact FSI of v_x) pairs, run through the
// tcgen05 BF16 GEMM of gemm_tcgen05.cuh.  This file holds the GEMM launcher
// and its C ABI entry point.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "gemm_tcgen05.cuh"
#include "tt_fsi.h"

namespace {

tt_fsi_status st_status(cudaError_t e) {
    if (e == cudaSuccess) return TT_FSI_OK;
    return e == cudaErrorMemoryAllocation ? TT_FSI_ERR_NO_MEMORY : TT_FSI_ERR_CUDA;
}

bool g_gemm_attr_set[64] = {false};

tt_fsi_status gemm_launch(const ttfsi_gemm::GemmArgs &a, cudaStream_t st) {
    using namespace ttfsi_gemm;
    if (a.M <= 0 || a.N <= 0 || a.K <= 0) return TT_FSI_OK;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return TT_FSI_ERR_CUDA;
    if (dev >= 0 && dev < 64 && !g_gemm_attr_set[dev]) {
        cudaError_t e = cudaFuncSetAttribute(gemm_bf16_tcgen05, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
        if (e != cudaSuccess) return st_status(e);
        g_gemm_attr_set[dev] = true;
    }
    dim3 grid((unsigned)((a.N + BN - 1) / BN), (unsigned)((a.M + BM - 1) / BM));
    gemm_bf16_tcgen05<<<grid, THREADS, SMEM_BYTES, st>>>(a);
    return st_status(cudaGetLastError());
}

}  // namespace

extern "C" tt_fsi_status tt_fsi_gemm_bf16(const void *A, int lda, const void *B, int ldb, int M, int N, int K,
                                          const float *bias, int act, const float *dgelu_z, int ldz, float *Cf,
                                          int ldcf, void *Cb, int ldcb, void *Ct, int ldct, int *err_dev,
                                          struct CUstream_st *stream) {
    if (M < 0 || N < 0 || K < 0 || !A || !B || !err_dev) return TT_FSI_ERR_INVALID_ARG;
    if ((lda % 8) || (ldb % 8) || lda < K || ldb < K) return TT_FSI_ERR_INVALID_ARG;  // 16-byte rows
    if ((((uintptr_t)A) | ((uintptr_t)B)) & 15) return TT_FSI_ERR_INVALID_ARG;
    if (act != 0 && act != 1) return TT_FSI_ERR_INVALID_ARG;
    ttfsi_gemm::GemmArgs a{};
    a.A = static_cast<const __nv_bfloat16 *>(A);
    a.B = static_cast<const __nv_bfloat16 *>(B);
    a.lda = lda;
    a.ldb = ldb;
    a.M = M;
    a.N = N;
    a.K = K;
    a.bias = bias;
    a.act = act;
    a.dgelu_z = dgelu_z;
    a.ldz = ldz;
    a.Cf = Cf;
    a.ldcf = ldcf;
    a.Cb = static_cast<__nv_bfloat16 *>(Cb);
    a.ldcb = ldcb;
    a.Ct = static_cast<__nv_bfloat16 *>(Ct);
    a.ldct = ldct;
    a.err = err_dev;
    return gemm_launch(a, reinterpret_cast<cudaStream_t>(stream));
}
