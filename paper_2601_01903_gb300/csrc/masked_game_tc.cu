// Masked-model value function on the tcgen05 tensor cores (label path).
//
// v_x(S) = f(z), z_i = x_i for i in S and baseline_i otherwise, f the GELU
// MLP d -> 128 -> 128 -> 1 (Section 2.1's value function of a model with
// absent features set to a baseline).  One CTA (8 warps) takes 128
// coalitions at a time:
//   layer 1 (CUDA cores): for the consecutive coalitions of a dense tile a
//     thread owns two hidden units and 32 coalitions, walking their 5 low
//     bits in Gray-code order (one add per coalition and unit, every flip a
//     compile-time constant); for a list of coalitions threads k and k + 128
//     own unit k, 64 rows each, by a d-term dot product per row -- then GELU,
//     rounded to BF16 into shared memory in the 128-byte-swizzled K-major
//     layout the tensor cores read;
//   layer 2 (tensor cores): eight tcgen05.mma (M = 128 coalitions, N = 128
//     units, K = 16 each) of the BF16 activations against W2 (rounded to BF16
//     once per CTA and kept in shared memory), FP32 accumulators in tensor
//     memory, completion signalled on an mbarrier (bounded wait);
//   layer 3 (epilogue): warps w and w + 4 read accumulator rows 32w..32w+31
//     (their TMEM lane quarter), columns 0-63 and 64-127, with tcgen05.ld and
//     form b3 + sum_n W3[n] GELU(acc[n] + b2[n]) in FP32.
// The interventional value function of Section 4.1 (the mean of f over
// background rows standing in for the absent features) repeats the three
// layers per background row on the same tile and averages in FP32; one row
// is the baseline value function.  The BF16 rounding of the layer-2 operands
// is this path's precision (the float64 kernel in masked_game.cu is the
// parity path).
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
constexpr int THREADS = 256;  // 8 warps
constexpr int KB_BYTES = ROWS * 128;       // one 64-wide K block of 128 rows: 16 KB
constexpr int OPERAND_BYTES = 2 * KB_BYTES;  // K = 128: two blocks
constexpr int SMEM_BYTES = 2 * OPERAND_BYTES + 1024;
constexpr int kErrTimeout = 1;

struct Args {
    const float *W1, *b1, *W2, *b2, *W3;
    float b3;
    const double *x, *base;  // base: n_bg background rows [n_bg, d] (one row: the baseline)
    int n_bg;
    int d;
    long long B;
    const unsigned *coal;  // list mode when non-null: rows are (instance r / K, coal[r])
    int K;
    float *out;
    long long n_tiles, n_rows;
    int *err;
};

// GELU(z) = z Phi(z) with the normal tail by Abramowitz & Stegun, Handbook
// of Mathematical Functions, formula 7.1.26 (Hastings' approximation of
// erfc(x) = P(t) exp(-x^2), t = 1 / (1 + p x), x >= 0; absolute error of
// erf below 1.5e-7, far below the BF16 rounding this path applies next):
// Phi(z) = 1 - q for z >= 0 and q for z < 0, q = erfc(|z| / sqrt 2) / 2.
// The reciprocal and the exponential run on the special-function unit.
__device__ __forceinline__ float gelu(float z) {
    const float x = fabsf(z) * 0.70710678118654752f;
    float t;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(t) : "f"(fmaf(0.3275911f, x, 1.0f)));
    float p = fmaf(1.061405429f, t, -1.453152027f);
    p = fmaf(p, t, 1.421413741f);
    p = fmaf(p, t, -0.284496736f);
    p = fmaf(p, t, 0.254829592f);
    const float q = 0.5f * p * t * __expf(-x * x);
    return z * (z >= 0.f ? 1.0f - q : q);
}

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
    __shared__ float zrow[ROWS][33];             // list mode: each row's input vector
    __shared__ float sb2[H], sw3[H];
    __shared__ float sdelta[5][H];               // dense mode: w1[k][q] (x_q - baseline_q)
    __shared__ float spart[ROWS];                // epilogue: the second half's partial sums

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid < H) {
        sb2[tid] = a.b2[tid];
        sw3[tid] = a.W3[tid];
    }
    // W2 -> BF16 B operand (once per CTA)
    for (int i = tid; i < H * H; i += THREADS) {
        const int n = i / H, k = i - n * H;
        *reinterpret_cast<__nv_bfloat16 *>(wB + operand_offset(n, k)) = __float2bfloat16_rn(a.W2[i]);
    }
    if (tid == 0) {
        mbar_init(smem_u32(&mbar), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
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

    // list mode: this thread's hidden unit k and half of the tile's rows
    const int k = tid & (H - 1), half = tid >> 7;
    float w1[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) w1[i] = (i < a.d) ? a.W1[k * a.d + i] : 0.f;
    const float bias1 = a.b1[k];
    const long long tiles_per_inst = a.coal ? 0 : (1ll << (a.d - 7));
    uint32_t parity = 0;

    bool failed = false;
    for (long long t = blockIdx.x; t < a.n_tiles && !failed; t += gridDim.x) {
      // one pass per background row; each adds its partial layer-3 sums
      float vsum = 0.f;
      for (int bgi = 0; bgi < a.n_bg; ++bgi) {
        const double *base = a.base + (long long)bgi * a.d;
        // ---- layer 1 into the A operand ----
        if (!a.coal) {
            // thread (unit pair kp, quarter qr of the rows): units 2kp, 2kp + 1,
            // rows 32 qr .. 32 qr + 31, walked in Gray-code order over their 5
            // low bits
            const long long inst = t / tiles_per_inst;
            const unsigned c0 = (unsigned)((t - inst * tiles_per_inst) << 7);
            const double *x = a.x + inst * a.d;
            const int kp = tid & 63, qr = tid >> 6, k0 = 2 * kp;
            const unsigned cb = c0 | ((unsigned)qr << 5);
            float p0 = a.b1[k0], p1 = a.b1[k0 + 1];
            for (int i = 0; i < a.d; ++i) {
                const float xi = (float)x[i], bi = (float)base[i];
                const float wa = __ldg(a.W1 + k0 * a.d + i), wb = __ldg(a.W1 + (k0 + 1) * a.d + i);
                if (i < 5 && qr == 0) {
                    sdelta[i][k0] = wa * (xi - bi);
                    sdelta[i][k0 + 1] = wb * (xi - bi);
                }
                const float zi = ((cb >> i) & 1u) ? xi : bi;
                p0 = fmaf(wa, zi, p0);
                p1 = fmaf(wb, zi, p1);
            }
            __syncthreads();  // sdelta of this tile
            float da[5], db[5];
#pragma unroll
            for (int q = 0; q < 5; ++q) {
                da[q] = sdelta[q][k0];
                db[q] = sdelta[q][k0 + 1];
            }
            const int row0 = qr << 5;
#pragma unroll
            for (int r = 0; r < 32; ++r) {
                if (r > 0) {
                    // the bit that flips between gray(r - 1) and gray(r), and its old value
                    const int q = (r & 1) ? 0 : (r & 2) ? 1 : (r & 4) ? 2 : (r & 8) ? 3 : 4;
                    const bool was_set = (((r - 1) ^ ((r - 1) >> 1)) >> q) & 1;
                    p0 += was_set ? -da[q] : da[q];
                    p1 += was_set ? -db[q] : db[q];
                }
                const int row = row0 + (r ^ (r >> 1));
                *reinterpret_cast<__nv_bfloat162 *>(aA + operand_offset(row, k0)) =
                    __floats2bfloat162_rn(gelu(p0), gelu(p1));
            }
        } else {
            // the first 128 threads build one row's input vector each
            if (tid < ROWS) {
                const long long row = t * ROWS + tid;
                if (row < a.n_rows) {
                    const long long inst = row / a.K;
                    const unsigned m = a.coal[row];
                    const double *x = a.x + inst * a.d;
                    for (int i = 0; i < a.d; ++i) zrow[tid][i] = (float)(((m >> i) & 1u) ? x[i] : base[i]);
                } else {
                    for (int i = 0; i < a.d; ++i) zrow[tid][i] = 0.f;
                }
            }
            __syncthreads();
            for (int r = half * (ROWS / 2); r < (half + 1) * (ROWS / 2); ++r) {
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
        // one lane per warp polls; the others wait at the warp barrier
        bool ok = true;
        if ((tid & 31) == 0) ok = mbar_wait(smem_u32(&mbar), parity);
        __syncwarp();
        parity ^= 1u;
        if (__syncthreads_or(ok ? 0 : 1)) {
            failed = true;
            break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // ---- layer 3 in the epilogue: warps w, w + 4 share accumulator rows ----
        const int quarter = warp & 3, col0 = (warp >> 2) * (H / 2);
        float v = 0.f;
#pragma unroll 1
        for (int c0 = col0; c0 < col0 + H / 2; c0 += 16) {
            uint32_t r[16];
            const uint32_t taddr = tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)c0;
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
        vsum += v;
        // the accumulators and the A operand are rewritten by the next pass
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      }
      if (failed) break;
      const int quarter = warp & 3;
      if (warp >= 4) spart[32 * quarter + lane] = vsum;
      __syncthreads();
      const long long row = t * ROWS + 32 * quarter + lane;
      if (warp < 4 && row < a.n_rows) a.out[row] = a.b3 + (vsum + spart[32 * quarter + lane]) / (float)a.n_bg;
      __syncthreads();
    }
    if (failed && tid == 0) atomicOr(a.err, kErrTimeout);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(H));
}

}  // namespace ttfsi_mgtc

extern "C" tt_fsi_status tt_fsi_masked_game_tc_interventional(const tt_fsi_mlp *model, const double *x_dev,
                                                             const double *background_dev, int n_background,
                                                             int64_t B, const unsigned *coal_dev, int K,
                                                             float *out_dev, int *err_dev, struct CUstream_st *stream);

extern "C" tt_fsi_status tt_fsi_masked_game_tc(const tt_fsi_mlp *model, const double *x_dev,
                                              const double *baseline_dev, int64_t B, const unsigned *coal_dev,
                                              int K, float *out_dev, int *err_dev, struct CUstream_st *stream) {
    // a baseline is the interventional value function with one background row
    return tt_fsi_masked_game_tc_interventional(model, x_dev, baseline_dev, 1, B, coal_dev, K, out_dev, err_dev,
                                                stream);
}

extern "C" tt_fsi_status tt_fsi_masked_game_tc_interventional(const tt_fsi_mlp *model, const double *x_dev,
                                                             const double *background_dev, int n_background,
                                                             int64_t B, const unsigned *coal_dev, int K,
                                                             float *out_dev, int *err_dev, struct CUstream_st *stream) {
    using namespace ttfsi_mgtc;
    const double *baseline_dev = background_dev;
    if (!model || B < 0 || n_background < 1) return TT_FSI_ERR_INVALID_ARG;
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
    a.n_bg = n_background;
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
    // two CTAs per SM fit (shared memory and registers); a persistent grid of
    // at least that many keeps one CTA's CUDA-core layers beside the other's
    // tensor-core wait
    const long long grid = std::min<long long>(a.n_tiles, (long long)std::max(2, occ) * sms);
    masked_game_tc_kernel<<<(unsigned)grid, THREADS, SMEM_BYTES, reinterpret_cast<cudaStream_t>(stream)>>>(a);
    return cudaGetLastError() == cudaSuccess ? TT_FSI_OK : TT_FSI_ERR_CUDA;
}
