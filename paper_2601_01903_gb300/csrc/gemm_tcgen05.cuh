// BF16 x BF16 -> FP32 GEMM on the 5th-generation tensor cores of sm_103a
// (tcgen05.mma, accumulators in tensor memory), with fused epilogues, in
// two forms: operands fed by the Tensor Memory Accelerator (the default,
// below) or by cp.async (used where an operand has no tensor map).
//
//   C[M, N] = A[M, K] . B[N, K]^T      (both operands K-major, row-major in HBM)
//
// One CTA (4 warps) computes a 128 x BN tile (of one K slice when K is
// split over the grid's third dimension).  Operand tiles of 128 x 64
// bf16 are staged in shared memory in the 128-byte swizzled K-major layout
// (row r at r * 128 bytes, its 16-byte chunk c at chunk c ^ (r & 7)), two
// stages deep: cp.async fills stage s + 1 while the tensor cores read stage
// s.  One thread issues four 128 x BN x 16 MMAs per stage and commits them to
// an mbarrier; every wait on an mbarrier is bounded and, when it runs out,
// records an error, drains and returns.  The epilogue reads the accumulator
// rows back with tcgen05.ld (warp w owns TMEM lanes 32w..32w+31 = tile rows
// 32w..32w+31), stages them through shared memory so that every global
// store is coalesced, and applies bias, GELU or a GELU-derivative factor,
// writing FP32 and/or BF16 outputs, optionally also transposed.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace ttfsi_gemm {

constexpr int BM = 128;
constexpr int BN = 128;
constexpr int BK = 64;
constexpr int THREADS = 128;
constexpr int STAGES = 2;
constexpr int TILE_BYTES = BM * BK * 2;  // 16 KB per operand tile
constexpr int SMEM_BYTES = STAGES * 2 * TILE_BYTES + 1024;
constexpr long long WAIT_LIMIT = 20000000;  // mbarrier polls before giving up

enum : int { kErrGemmTimeout = 1 };

struct GemmArgs {
    const __nv_bfloat16 *A;
    const __nv_bfloat16 *B;
    int lda, ldb;
    int M, N, K;
    const float *bias;         // [N] or null
    int act;                   // 0: none, 1: GELU
    const float *dgelu_z;      // [M, N] pre-activations: multiply by gelu'(z), or null
    int ldz;
    float *Cf;                 // FP32 result (before the activation), or null
    int ldcf;
    __nv_bfloat16 *Cb;         // BF16 result (after the activation), or null
    int ldcb;
    __nv_bfloat16 *Ct;         // BF16 result transposed ([N, M]), or null
    int ldct;
    int *err;
    // split K: CTA z of the grid's third dimension takes K blocks
    // [z kbc, (z + 1) kbc) and writes its raw FP32 partial product to
    // Cf + z cf_zstride (only Cf; the caller adds the slices); kbc = 0: all of K
    int kbc;
    long long cf_zstride;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor: 128-byte swizzle, K-major, 8-row groups
// 1024 bytes apart (stride byte offset), descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFF) >> 4);
    d |= (uint64_t)1 << 16;              // leading byte offset (unused by swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;    // stride byte offset
    d |= (uint64_t)1 << 46;              // version
    d |= (uint64_t)2 << 61;              // 128-byte swizzle
    return d;
}

// Instruction descriptor of kind::f16: FP32 accumulate, BF16 A and B, both
// K-major, M = 128, N = BN.
__host__ __device__ constexpr uint32_t instr_desc_bf16(int m, int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}

// Bounded wait for phase `parity` of the mbarrier; false if the limit ran out.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    for (long long i = 0; i < WAIT_LIMIT; ++i) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, bool valid) {
    const int n = valid ? 16 : 0;  // 0 source bytes: the 16 destination bytes are zero-filled
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(n) : "memory");
}

// The normal distribution function Phi(z) and density phi(z) for GELU and
// its derivative.  The tail q = erfc(|z| / sqrt 2) / 2 follows Abramowitz &
// Stegun, Handbook of Mathematical Functions, formula 7.1.26 (Hastings'
// approximation erfc(x) = P(t) exp(-x^2), t = 1 / (1 + p x); absolute error
// of erf below 1.5e-7, under the BF16 rounding of the activations); the
// reciprocal and the exponential run on the special-function unit.
__device__ __forceinline__ void normal_cdf_pdf(float z, float &cdf, float &pdf) {
    const float x = fabsf(z) * 0.70710678118654752f;
    float t;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(t) : "f"(fmaf(0.3275911f, x, 1.0f)));
    float p = fmaf(1.061405429f, t, -1.453152027f);
    p = fmaf(p, t, 1.421413741f);
    p = fmaf(p, t, -0.284496736f);
    p = fmaf(p, t, 0.254829592f);
    const float e = __expf(-x * x);  // exp(-z^2 / 2)
    const float q = 0.5f * p * t * e;
    cdf = z >= 0.f ? 1.0f - q : q;
    pdf = 0.39894228040143268f * e;
}

__device__ __forceinline__ float gelu_f(float z) {
    float cdf, pdf;
    normal_cdf_pdf(z, cdf, pdf);
    return z * cdf;
}

__device__ __forceinline__ float gelu_grad_f(float z) {
    // d/dz [z Phi(z)] = Phi(z) + z phi(z)
    float cdf, pdf;
    normal_cdf_pdf(z, cdf, pdf);
    return cdf + z * pdf;
}

// Fills one 128 x 64 operand tile (rows r0.., columns k0..) into the swizzled
// layout; rows >= rows_valid or columns >= K are zero.
__device__ __forceinline__ void load_tile(uint32_t tile, const __nv_bfloat16 *G, int ld, int r0, int rows_valid,
                                          int k0, int K) {
    for (int i = threadIdx.x; i < BM * 8; i += THREADS) {
        const int r = i >> 3, c = i & 7;
        const int gr = r0 + r, gk = k0 + c * 8;
        const bool ok = (gr < rows_valid) && (gk < K);
        const __nv_bfloat16 *src = ok ? G + (long long)gr * ld + gk : G;
        cp_async16(tile + r * 128 + ((c ^ (r & 7)) << 4), src, ok);
    }
}

#ifndef TTFSI_GEMM_HELPERS_ONLY
// Epilogue of one 128 x BN tile from its TMEM accumulators (see the header).
// `stage_all` is idle shared memory, 32 x 33 floats per warp; `slot` picks
// the warp's block, the warp reads TMEM lane quarter `quarter` (tile rows
// 32 quarter ..) over accumulator columns [cb, ce).
__device__ __forceinline__ void gemm_epilogue(const GemmArgs &a, float *Cf, uint32_t tmem, float *stage_all, int m0,
                                              int n0, int slot, int quarter, int cb, int ce, int lane) {
        float *stage = stage_all + slot * (32 * 33);
        // Epilogue, 32 columns at a time.  Warp w owns accumulator rows
        // 32w..32w+31 (its TMEM lane quarter); tcgen05.ld gives each lane one
        // row, so the values go through a per-warp 32 x 33 staging block in
        // the (now idle) operand tiles and leave with lanes over columns
        // (row-major outputs) or over rows (the transposed output), i.e. as
        // coalesced stores.
        const int rbase = m0 + 32 * quarter;
        for (int c0 = cb; c0 < ce; c0 += 32) {
            uint32_t r[32];
            const uint32_t taddr = tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                "[%16];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                  "=r"(r[15])
                : "r"(taddr));
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                "[%16];"
                : "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]),
                  "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
                  "=r"(r[30]), "=r"(r[31])
                : "r"(taddr + 16u));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int j = 0; j < 32; ++j) stage[lane * 33 + j] = __uint_as_float(r[j]);
            __syncwarp();
            // row pass: lane = column; the pre-activations of the GELU factor
            // are loaded 8 rows at a time ahead of their use, so the loads overlap
            const int col = n0 + c0 + lane;
            const bool col_ok = col < a.N;
            const float bias = (a.bias && col_ok) ? a.bias[col] : 0.f;
#pragma unroll 1
            for (int i0 = 0; i0 < 32; i0 += 8) {
                float zin[8];
                if (a.dgelu_z) {
#pragma unroll
                    for (int i = 0; i < 8; ++i)
                        zin[i] = (col_ok && rbase + i0 + i < a.M) ? a.dgelu_z[(long long)(rbase + i0 + i) * a.ldz + col]
                                                                  : 0.f;
                }
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int row = rbase + i0 + i;
                    if (row < a.M && col_ok) {
                        float z = stage[(i0 + i) * 33 + lane] + bias;
                        if (a.dgelu_z) z *= gelu_grad_f(zin[i]);
                        if (Cf) Cf[(long long)row * a.ldcf + col] = z;
                        const float y = (a.act == 1) ? gelu_f(z) : z;
                        if (a.Cb) a.Cb[(long long)row * a.ldcb + col] = __float2bfloat16_rn(y);
                        stage[(i0 + i) * 33 + lane] = y;
                    }
                }
            }
            if (a.Ct) {
                __syncwarp();
                // column pass: lane = row
                const int row = rbase + lane;
                if (row < a.M)
                    for (int j = 0; j < 32; ++j) {
                        const int colj = n0 + c0 + j;
                        if (colj < a.N) a.Ct[(long long)colj * a.ldct + row] = __float2bfloat16_rn(stage[lane * 33 + j]);
                    }
            }
            __syncwarp();
        }
}

__global__ void __launch_bounds__(THREADS) gemm_bf16_tcgen05(GemmArgs a) {
    extern __shared__ __align__(1024) unsigned char gsm_raw[];
    // 1024-byte alignment of the operand tiles (the swizzle is address based)
    const uint32_t raw = smem_u32(gsm_raw);
    const uint32_t base = (raw + 1023) & ~1023u;
    __shared__ __align__(8) uint64_t mbar[STAGES];
    __shared__ uint32_t tmem_base_sh;
    __shared__ int s_fail;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int nk_all = (a.K + BK - 1) / BK;
    const int kb0 = a.kbc > 0 ? (int)blockIdx.z * a.kbc : 0;
    const int nk = a.kbc > 0 ? min(a.kbc, nk_all - kb0) : nk_all;  // K blocks of this CTA
    float *const Cf = a.Cf ? a.Cf + (long long)blockIdx.z * a.cf_zstride : nullptr;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) mbar_init(smem_u32(&mbar[s]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_fail = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                     "r"(BN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base_sh;
    const uint32_t idesc = instr_desc_bf16(BM, BN);

    auto tileA = [&](int s) { return base + (uint32_t)(s * 2) * TILE_BYTES; };
    auto tileB = [&](int s) { return base + (uint32_t)(s * 2 + 1) * TILE_BYTES; };

    uint32_t phase_bits = 0, issued_bits = 0;  // bit s: parity to wait for / MMAs pending on stage s
    bool fail = false;

    // prologue: stage 0
    load_tile(tileA(0), a.A, a.lda, m0, a.M, kb0 * BK, a.K);
    load_tile(tileB(0), a.B, a.ldb, n0, a.N, kb0 * BK, a.K);
    asm volatile("cp.async.commit_group;" ::: "memory");

    for (int kb = 0; kb < nk && !fail; ++kb) {
        const int s = kb & 1, sn = s ^ 1;
        // prefetch the next stage once the MMAs that last read it are done
        if (kb + 1 < nk) {
            if ((issued_bits >> sn) & 1u) {
                if (!mbar_wait(smem_u32(&mbar[sn]), (phase_bits >> sn) & 1u)) fail = true;
                phase_bits ^= 1u << sn;
                issued_bits &= ~(1u << sn);
            }
            if (!fail) {
                load_tile(tileA(sn), a.A, a.lda, m0, a.M, (kb0 + kb + 1) * BK, a.K);
                load_tile(tileB(sn), a.B, a.ldb, n0, a.N, (kb0 + kb + 1) * BK, a.K);
            }
            asm volatile("cp.async.commit_group;" ::: "memory");
            asm volatile("cp.async.wait_group 1;" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
        }
        // the current stage's bytes are in shared memory; make them visible to
        // the tensor cores (async proxy)
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        fail = __syncthreads_or(fail ? 1 : 0) != 0;  // one decision for the whole CTA
        if (fail) break;
        if (threadIdx.x == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int kmax = min(BK, a.K - (kb0 + kb) * BK);
            for (int k16 = 0; k16 * 16 < kmax; ++k16) {
                const uint64_t da = smem_desc(tileA(s) + k16 * 32);
                const uint64_t db = smem_desc(tileB(s) + k16 * 32);
                mma_bf16(tmem, da, db, idesc, (kb > 0 || k16 > 0) ? 1u : 0u);
            }
            mma_commit(smem_u32(&mbar[s]));
        }
        issued_bits |= 1u << s;
    }
    // wait for the last MMAs
    for (int s = 0; s < STAGES; ++s)
        if ((issued_bits >> s) & 1u) {
            if (!mbar_wait(smem_u32(&mbar[s]), (phase_bits >> s) & 1u)) fail = true;
            phase_bits ^= 1u << s;
        }
    if (fail) atomicOr(&s_fail, 1);
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

    if (!s_fail) {
        gemm_epilogue(a, Cf, tmem, reinterpret_cast<float *>(gsm_raw + (base - raw)), m0, n0, warp, warp, 0, BN, lane);
    } else if (threadIdx.x == 0) {
        atomicOr(a.err, kErrGemmTimeout);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BN));
}

// ----------------------------------------------------------------------------
// The same product with the operands fed by the Tensor Memory Accelerator:
// one thread (warp 0) issues 2D tiled bulk-tensor loads of the 128 x 64
// operand tiles, 128-byte swizzled by the copy engine into the layout the
// MMA descriptors describe, into TMA_STAGES stages; each stage has a "full"
// mbarrier (the loads' transaction bytes) and an "empty" one (the MMAs that
// read it, via tcgen05.commit).  One thread (warp 1) waits on "full" and
// issues the MMAs; all 8 warps then run the epilogue once a final commit
// signals that the accumulator is complete (two warps per TMEM lane
// quarter, one per half of the columns).  Rows, columns and K beyond the
// operands are zero-filled by the loads.  Every wait is bounded; a wait that
// runs out records kErrGemmTimeout and the CTA skips its epilogue.
// ----------------------------------------------------------------------------
constexpr int TMA_STAGES = 2;     // 66.5 KB: three CTAs per SM
constexpr int TMA_THREADS = 256;  // 8 warps for the epilogue
constexpr int TMA_SMEM_BYTES = TMA_STAGES * 2 * TILE_BYTES + 1024;

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const void *tmap, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(dst), "l"(tmap), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__global__ void __launch_bounds__(TMA_THREADS) gemm_bf16_tcgen05_tma(const __grid_constant__ GemmArgs a,
                                                                 const __grid_constant__ CUtensorMap tmA,
                                                                 const __grid_constant__ CUtensorMap tmB) {
    extern __shared__ __align__(1024) unsigned char gsm_raw[];
    const uint32_t raw = smem_u32(gsm_raw);
    const uint32_t base = (raw + 1023) & ~1023u;
    __shared__ __align__(8) uint64_t full[TMA_STAGES], empty[TMA_STAGES], done;
    __shared__ uint32_t tmem_base_sh;
    __shared__ int s_fail;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int nk_all = (a.K + BK - 1) / BK;
    const int kb0 = a.kbc > 0 ? (int)blockIdx.z * a.kbc : 0;
    const int nk = a.kbc > 0 ? min(a.kbc, nk_all - kb0) : nk_all;
    float *const Cf = a.Cf ? a.Cf + (long long)blockIdx.z * a.cf_zstride : nullptr;

    if (threadIdx.x == 0) {
        for (int s = 0; s < TMA_STAGES; ++s) {
            mbar_init(smem_u32(&full[s]), 1);
            mbar_init(smem_u32(&empty[s]), 1);
        }
        mbar_init(smem_u32(&done), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_fail = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                     "r"(BN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base_sh;

    auto tileA = [&](int s) { return base + (uint32_t)(s * 2) * TILE_BYTES; };
    auto tileB = [&](int s) { return base + (uint32_t)(s * 2 + 1) * TILE_BYTES; };

    // Warp 0 lane 0 produces, warp 1 lane 0 issues the MMAs; the other lanes
    // of those two warps park at __syncwarp, so no spinning lane of the same
    // warp competes with the one that does the work.
    if (warp == 0) {
        if (lane == 0) {
        // producer
        for (int kb = 0; kb < nk; ++kb) {
            const int s = kb % TMA_STAGES;
            const uint32_t use = (uint32_t)(kb / TMA_STAGES);
            if (use > 0 && !mbar_wait(smem_u32(&empty[s]), (use - 1) & 1u)) {
                atomicOr(&s_fail, 1);
                break;
            }
            if (*(volatile int *)&s_fail) break;
            mbar_expect_tx(smem_u32(&full[s]), 2u * TILE_BYTES);
            const int k0 = (kb0 + kb) * BK;
            tma_load_2d(tileA(s), &tmA, k0, m0, smem_u32(&full[s]));
            tma_load_2d(tileB(s), &tmB, k0, n0, smem_u32(&full[s]));
        }
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {
        // MMA issuer
        const uint32_t idesc = instr_desc_bf16(BM, BN);
        bool ok = true;
        for (int kb = 0; kb < nk; ++kb) {
            const int s = kb % TMA_STAGES;
            if (!mbar_wait(smem_u32(&full[s]), (uint32_t)(kb / TMA_STAGES) & 1u)) {
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int k16 = 0; k16 < BK / 16; ++k16) {
                const uint64_t da = smem_desc(tileA(s) + k16 * 32);
                const uint64_t db = smem_desc(tileB(s) + k16 * 32);
                mma_bf16(tmem, da, db, idesc, (kb > 0 || k16 > 0) ? 1u : 0u);
            }
            mma_commit(smem_u32(&empty[s]));
        }
        if (!ok) atomicOr(&s_fail, 1);
        mma_commit(smem_u32(&done));  // arrives once every MMA issued above has completed
        }
        __syncwarp();
    }
    // every warp: lane 0 waits for the accumulator (or the failure flag), the
    // other lanes wait at the warp barrier without issuing
    bool done_ok = true;
    if (lane == 0) done_ok = mbar_wait(smem_u32(&done), 0);
    __syncwarp();
    if (lane == 0 && !done_ok) atomicOr(&s_fail, 1);
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!s_fail) {
        // the stage buffers are idle: every load was consumed by an MMA that has completed
        // 8 warps: warps w and w + 4 share TMEM lane quarter w & 3 and take
        // the accumulator columns [0, BN/2) and [BN/2, BN)
        gemm_epilogue(a, Cf, tmem, reinterpret_cast<float *>(gsm_raw + (base - raw)), m0, n0, warp, warp & 3,
                      (warp >> 2) * (BN / 2), (warp >> 2) * (BN / 2) + BN / 2, lane);
    } else if (threadIdx.x == 0) {
        atomicOr(a.err, kErrGemmTimeout);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BN));
}
#endif  // TTFSI_GEMM_HELPERS_ONLY

}  // namespace ttfsi_gemm
