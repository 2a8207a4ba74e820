// Masked-model value function on the tcgen05 tensor cores (label path).
//
// v_x(S) = f(z), z_i = x_i for i in S and baseline_i otherwise, f the GELU
// MLP d -> 128 -> 128 -> 1 (Section 2.1's value function of a model with
// absent features set to a baseline).  One CTA (4 warps) takes 128
// coalitions at a time:
//   layer 1 (CUDA cores): thread k owns hidden unit k and forms its 128
//     pre-activations -- for the 128 consecutive coalitions of a dense tile
//     by walking the 7 low bits in Gray-code order (one add per coalition),
//     for a list of coalitions by a d-term dot product each -- then GELU,
//     rounded to BF16 into shared memory in the 128-byte-swizzled K-major
//     layout the tensor cores read;
//   layer 2 (tensor cores): eight tcgen05.mma (M = 128 coalitions, N = 128
//     units, K = 16 each) of the BF16 activations against W2 (rounded to BF16
//     once per CTA and kept in shared memory), FP32 accumulators in tensor
//     memory, completion signalled on an mbarrier (bounded wait);
//   layer 3 (epilogue): thread r reads accumulator row r with tcgen05.ld and
//     forms b3 + sum_n W3[n] GELU(acc[n] + b2[n]) in FP32.
// The BF16 rounding of the layer-2 operands is this path's precision (the
// float64 kernel in masked_game.cu is the parity path).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

// only the tcgen05 helpers (the GEMM kernel itself lives in student.cu)
#define TTFSI_GEMM_HELPERS_ONLY
#include "gemm_tcgen05.cuh"
#include "tt_fsi.h"

namespace ttfsi_mgtc {

using ttfsi_gemm::mbar_init;
using ttfsi_gemm::mbar_wait;
using ttfsi_gemm::mma_bf16;
using ttfsi_gemm::mma_commit;
using ttfsi_gemm::smem_desc;
using ttfsi_gemm::smem_u32;

constexpr int ROWS = 128;                  // coalitions per tile (MMA M)
constexpr int H = 128;                     // hidden width (MMA N and K)
constexpr int THREADS = 128;
constexpr int KB_BYTES = ROWS * 128;       // one 64-wide K block of 128 rows: 16 KB
constexpr int OPERAND_BYTES = 2 * KB_BYTES;  // K = 128: two blocks
constexpr int SMEM_BYTES = 2 * OPERAND_BYTES + 1024;
constexpr int kErrTimeout = 1;

struct Args {
    const float *W1, *b1, *W2, *b2, *W3;
    float b3;
    const double *x, *base;
    int d;
    long long B;
    const unsigned *coal;  // list mode when non-null: rows are (instance r / K, coal[r])
    int K;
    float *out;
    long long n_tiles, n_rows;
    int *err;
};

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }

// Byte offset of element (row r, column k) of a 128 x 128 BF16 operand in
// two 128-byte-swizzled K blocks.
__device__ __forceinline__ uint32_t operand_offset(int r, int k) {
    return (uint32_t)((k >> 6) * KB_BYTES + r * 128 + ((((k & 63) >> 3) ^ (r & 7)) << 4) + (k & 7) * 2);
}

__global__ void __launch_bounds__(THREADS) masked_game_tc_kernel(Args a) {
    extern __shared__ __align__(1024) unsigned char sm_raw[];
    const uint32_t raw = smem_u32(sm_raw);
    const uint32_t pad = ((raw + 1023) & ~1023u) - raw;
    unsigned char *wB = sm_raw + pad;            // W2 as the B operand [n][k]
    unsigned char *aA = wB + OPERAND_BYTES;      // activations as the A operand [row][k]
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base_sh;
    __shared__ int s_fail;
    __shared__ float zrow[ROWS][33];             // list mode: each row's input vector
    __shared__ float sb2[H], sw3[H];
    __shared__ float sdelta[7][THREADS];         // dense mode: w1[k][q] (x_q - baseline_q)

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    sb2[tid] = a.b2[tid];
    sw3[tid] = a.W3[tid];
    // W2 -> BF16 B operand (once per CTA)
    for (int i = tid; i < H * H; i += THREADS) {
        const int n = i / H, k = i - n * H;
        *reinterpret_cast<__nv_bfloat16 *>(wB + operand_offset(n, k)) = __float2bfloat16_rn(a.W2[i]);
    }
    if (tid == 0) {
        mbar_init(smem_u32(&mbar), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_fail = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                     "r"(H));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base_sh;
    const uint32_t idesc = ttfsi_gemm::instr_desc_bf16(ROWS, H);
    const uint32_t a_base = smem_u32(aA), b_base = smem_u32(wB);

    // this thread's hidden unit k = tid: its row of W1 and its bias
    const int k = tid;
    float w1[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) w1[i] = (i < a.d) ? a.W1[k * a.d + i] : 0.f;
    const float bias1 = a.b1[k];
    const long long tiles_per_inst = a.coal ? 0 : (1ll << (a.d - 7));
    uint32_t parity = 0;

    for (long long t = blockIdx.x; t < a.n_tiles; t += gridDim.x) {
        // ---- layer 1 into the A operand ----
        if (!a.coal) {
            const long long inst = t / tiles_per_inst;
            const unsigned c0 = (unsigned)((t - inst * tiles_per_inst) << 7);
            const double *x = a.x + inst * a.d;
            float pre = bias1;
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                if (i >= a.d) break;
                const float xi = (float)x[i], bi = (float)a.base[i];
                if (i < 7) sdelta[i][k] = w1[i] * (xi - bi);
                pre += w1[i] * ((((c0 >> i) & 1u) != 0u) ? xi : bi);
            }
            // Gray-code walk over the 7 low bits: row g = r ^ (r >> 1)
            unsigned g = 0;
            for (int r = 0; r < ROWS; ++r) {
                if (r > 0) {
                    const int q = __ffs(r) - 1;  // the bit that flips between g(r-1) and g(r)
                    pre += ((g >> q) & 1u) ? -sdelta[q][k] : sdelta[q][k];
                    g ^= 1u << q;
                }
                *reinterpret_cast<__nv_bfloat16 *>(aA + operand_offset((int)g, k)) = __float2bfloat16_rn(gelu(pre));
            }
        } else {
            // each thread builds one row's input vector
            {
                const long long row = t * ROWS + tid;
                if (row < a.n_rows) {
                    const long long inst = row / a.K;
                    const unsigned m = a.coal[row];
                    const double *x = a.x + inst * a.d;
                    for (int i = 0; i < a.d; ++i) zrow[tid][i] = (float)(((m >> i) & 1u) ? x[i] : a.base[i]);
                } else {
                    for (int i = 0; i < a.d; ++i) zrow[tid][i] = 0.f;
                }
            }
            __syncthreads();
            for (int r = 0; r < ROWS; ++r) {
                float pre = bias1;
#pragma unroll
                for (int i = 0; i < 32; ++i)
                    if (i < a.d) pre += w1[i] * zrow[r][i];
                *reinterpret_cast<__nv_bfloat16 *>(aA + operand_offset(r, k)) = __float2bfloat16_rn(gelu(pre));
            }
        }
        // ---- layer 2 on the tensor cores ----
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int kb = 0; kb < 2; ++kb)
#pragma unroll
                for (int k16 = 0; k16 < 4; ++k16) {
                    const uint64_t da = smem_desc(a_base + kb * KB_BYTES + k16 * 32);
                    const uint64_t db = smem_desc(b_base + kb * KB_BYTES + k16 * 32);
                    mma_bf16(tmem, da, db, idesc, (kb > 0 || k16 > 0) ? 1u : 0u);
                }
            mma_commit(smem_u32(&mbar));
        }
        const bool ok = mbar_wait(smem_u32(&mbar), parity);
        parity ^= 1u;
        if (__syncthreads_or(ok ? 0 : 1)) {
            if (tid == 0) s_fail = 1;
            break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // ---- layer 3 in the epilogue: thread = accumulator row ----
        float v = a.b3;
#pragma unroll 1
        for (int c0 = 0; c0 < H; c0 += 16) {
            uint32_t r[16];
            const uint32_t taddr = tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                "[%16];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                  "=r"(r[15])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int j = 0; j < 16; ++j) v += sw3[c0 + j] * gelu(__uint_as_float(r[j]) + sb2[c0 + j]);
        }
        const long long row = t * ROWS + 32 * warp + lane;
        if (row < a.n_rows) a.out[row] = v;
        // the accumulators and the A operand are rewritten by the next tile
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
    }
    if (s_fail && tid == 0) atomicOr(a.err, kErrTimeout);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(H));
}

}  // namespace ttfsi_mgtc

extern "C" tt_fsi_status tt_fsi_masked_game_tc(const tt_fsi_mlp *model, const double *x_dev,
                                              const double *baseline_dev, int64_t B, const unsigned *coal_dev,
                                              int K, float *out_dev, int *err_dev, struct CUstream_st *stream) {
    using namespace ttfsi_mgtc;
    if (!model || B < 0) return TT_FSI_ERR_INVALID_ARG;
    if (B == 0) return TT_FSI_OK;
    if (!x_dev || !baseline_dev || !out_dev || !err_dev) return TT_FSI_ERR_INVALID_ARG;
    if (!model->W1f || !model->b1f || !model->W2f || !model->b2f || !model->W3f) return TT_FSI_ERR_INVALID_ARG;
    if (model->h1 != H || model->h2 != H) return TT_FSI_ERR_UNSUPPORTED;
    if (coal_dev) {
        if (K < 1 || model->d < 1 || model->d > 32) return TT_FSI_ERR_INVALID_ARG;
    } else if (model->d < 7 || model->d > 30) {
        return TT_FSI_ERR_UNSUPPORTED;  // a dense tile is 128 coalitions of one instance
    }
    Args a{};
    a.W1 = model->W1f;
    a.b1 = model->b1f;
    a.W2 = model->W2f;
    a.b2 = model->b2f;
    a.W3 = model->W3f;
    a.b3 = (float)model->b3;
    a.x = x_dev;
    a.base = baseline_dev;
    a.d = model->d;
    a.B = B;
    a.coal = coal_dev;
    a.K = coal_dev ? K : 0;
    a.out = out_dev;
    a.n_rows = coal_dev ? B * (long long)K : (B << model->d);
    a.n_tiles = (a.n_rows + ROWS - 1) / ROWS;
    a.err = err_dev;
    int dev = 0, sms = 0, occ = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(masked_game_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, masked_game_tc_kernel, THREADS, SMEM_BYTES);
    if (e != cudaSuccess) return TT_FSI_ERR_CUDA;
    const long long grid = std::min<long long>(a.n_tiles, (long long)std::max(1, occ) * sms);
    masked_game_tc_kernel<<<(unsigned)grid, THREADS, SMEM_BYTES, reinterpret_cast<cudaStream_t>(stream)>>>(a);
    return cudaGetLastError() == cudaSuccess ? TT_FSI_OK : TT_FSI_ERR_CUDA;
}
