// Amortised FSI explainer ("student"): a GELU MLP that maps an instance x to
// its FSI scores, trained on (x, exact FSI of v_x) pairs, run through the
// tcgen05 BF16 GEMM of gemm_tcgen05.cuh.  This file holds the GEMM launcher
// and its C ABI entry point.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cudaTypedefs.h>

#include <algorithm>

#include "gemm_tcgen05.cuh"
#include "tt_fsi.h"

namespace {

tt_fsi_status st_status(cudaError_t e) {
    if (e == cudaSuccess) return TT_FSI_OK;
    return e == cudaErrorMemoryAllocation ? TT_FSI_ERR_NO_MEMORY : TT_FSI_ERR_CUDA;
}

bool g_gemm_attr_set[64] = {false};

// The driver's tensor-map encoder, looked up through the runtime (so the
// library does not link the driver library itself); null if unavailable.
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool looked = false;
    if (!looked) {
        looked = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// Tensor map of a row-major BF16 operand [rows, K] with row pitch ld
// elements: 128 x 64 boxes, 128-byte swizzle, zero fill outside the matrix.
bool operand_tensor_map(CUtensorMap *map, const __nv_bfloat16 *ptr, int rows, int K, int ld) {
    PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();
    if (!encode) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * sizeof(__nv_bfloat16)};
    const cuuint32_t box[2] = {(cuuint32_t)ttfsi_gemm::BK, (cuuint32_t)ttfsi_gemm::BM};
    const cuuint32_t estr[2] = {1, 1};
    return encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16 *>(ptr), dims, strides, box,
                  estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Launches the TMA-fed kernel, or the cp.async kernel where an operand has
// no valid tensor map (the two compute the same products).
tt_fsi_status gemm_launch(const ttfsi_gemm::GemmArgs &a, cudaStream_t st) {
    using namespace ttfsi_gemm;
    if (a.M <= 0 || a.N <= 0 || a.K <= 0) return TT_FSI_OK;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return TT_FSI_ERR_CUDA;
    if (dev >= 0 && dev < 64 && !g_gemm_attr_set[dev]) {
        cudaError_t e = cudaFuncSetAttribute(gemm_bf16_tcgen05, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(gemm_bf16_tcgen05_tma, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     TMA_SMEM_BYTES);
        if (e != cudaSuccess) return st_status(e);
        g_gemm_attr_set[dev] = true;
    }
    const int nk = (a.K + BK - 1) / BK;
    const int kslices = a.kbc > 0 ? (nk + a.kbc - 1) / a.kbc : 1;
    dim3 grid((unsigned)((a.N + BN - 1) / BN), (unsigned)((a.M + BM - 1) / BM), (unsigned)kslices);
    CUtensorMap tmA, tmB;
    if (operand_tensor_map(&tmA, a.A, a.M, a.K, a.lda) && operand_tensor_map(&tmB, a.B, a.N, a.K, a.ldb))
        gemm_bf16_tcgen05_tma<<<grid, TMA_THREADS, TMA_SMEM_BYTES, st>>>(a, tmA, tmB);
    else
        gemm_bf16_tcgen05<<<grid, THREADS, SMEM_BYTES, st>>>(a);
    return st_status(cudaGetLastError());
}

// Sum of the K-slice partial products in slice order, plus an optional bias
// per column: C[r, c] = sum_z P_z[r, c] (+ bias[c]).
__global__ void ksum_kernel(const float *part, long long zstride, int slices, int M, int N, int ld, const float *bias,
                            float *C) {
    const long long n = (long long)M * N;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long r = i / N, c = i - r * N;
        float s = 0.f;
        for (int z = 0; z < slices; ++z) s += part[z * zstride + r * ld + c];
        C[r * ld + c] = bias ? s + bias[c] : s;
    }
}

// K blocks per slice for a plain (Cf-only) product: split K when the output
// tiles alone cannot fill the GPU, keeping at least 4 K blocks per slice.
int split_kbc(int M, int N, int K) {
    const int tiles = ((M + ttfsi_gemm::BM - 1) / ttfsi_gemm::BM) * ((N + ttfsi_gemm::BN - 1) / ttfsi_gemm::BN);
    const int nk = (K + ttfsi_gemm::BK - 1) / ttfsi_gemm::BK;
    if (tiles >= 128 || nk < 8) return 0;
    int slices = std::min((2 * 152 + tiles - 1) / tiles, nk / 4);
    if (slices < 2) return 0;
    return (nk + slices - 1) / slices;
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

// ============================================================================
// Student network d -> H -> H -> n_out (GELU), BF16 operands on the tensor
// cores, FP32 master weights and Adam state, output projected onto the
// efficiency constraint.
// ============================================================================
#include <cmath>
#include <new>
#include <vector>

namespace ttfsi_student {

using bf16 = __nv_bfloat16;
constexpr int kErrTimeout = 1;

// FP32 [rows, cols] (row-major) -> BF16 copy Wb [rows_pad, cols] (rows >= rows
// zero; optional) and transposed BF16 copy Wt [cols, ldt] with Wt[c][r] =
// W[r][c] for r < rows_pad (zero for r >= rows; optional), through 32 x 32
// shared-memory tiles so that the reads and both writes are coalesced.
// Block 32 x 8 threads, grid (ceil(cols / 32), ceil(rows_pad / 32)).
__device__ __forceinline__ void to_bf16_tile(const float *W, int rows, int cols, int rows_pad, bf16 *Wb, bf16 *Wt,
                                             int ldt, int c0, int r0) {
    __shared__ float tile[32][33];
    const int tx = threadIdx.x, ty = threadIdx.y;
    for (int i = ty; i < 32; i += 8) {
        const int r = r0 + i, c = c0 + tx;
        const float w = (r < rows && c < cols) ? W[(long long)r * cols + c] : 0.0f;
        tile[i][tx] = w;
        if (Wb && r < rows_pad && c < cols) Wb[(long long)r * cols + c] = __float2bfloat16_rn(w);
    }
    if (!Wt) return;
    __syncthreads();
    for (int i = ty; i < 32; i += 8) {
        const int c = c0 + i, r = r0 + tx;
        if (c < cols && r < rows_pad) Wt[(long long)c * ldt + r] = __float2bfloat16_rn(tile[tx][i]);
    }
}

__global__ void to_bf16_tiled_kernel(const float *W, int rows, int cols, int rows_pad, bf16 *Wb, bf16 *Wt, int ldt) {
    to_bf16_tile(W, rows, cols, rows_pad, Wb, Wt, ldt, blockIdx.x * 32, blockIdx.y * 32);
}

// Several casts in one launch: block b takes tile b - first[j] of cast j
// (the casts' tiles are numbered one after another, column tiles fastest).
struct CastJob {
    const float *W;
    bf16 *Wb, *Wt;
    int rows, cols, rows_pad, ldt, tiles_x, first;
};
struct CastJobs {
    CastJob j[3];
    int n;
};
__global__ void to_bf16_multi_kernel(CastJobs jobs) {
    int k = 0;
    while (k + 1 < jobs.n && (int)blockIdx.x >= jobs.j[k + 1].first) ++k;
    const CastJob &c = jobs.j[k];
    const int t = (int)blockIdx.x - c.first;
    to_bf16_tile(c.W, c.rows, c.cols, c.rows_pad, c.Wb, c.Wt, c.ldt, (t % c.tiles_x) * 32, (t / c.tiles_x) * 32);
}

// Projection onto sum_{S != empty} phi(S) = target, phi(empty) = v_empty, then
// (if labels are given) the squared-error loss and its gradient with respect
// to the raw outputs: dL/dY = P (2 (phi_p - phi) / (B n_out)), P = I - 11^T/(n_out-1)
// on the non-empty coordinates, 0 on the empty one.  One warp per instance.
__global__ void project_loss_kernel(const float *Y, int B, int n_out, const float *target, float v_empty, float *phi,
                                    const float *labels, float *loss_rows, float *dYf, bf16 *dYb, int ld_dyb, bf16 *dYt,
                                    int ld_dyt) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= B) return;
    const float *y = Y + (long long)warp * n_out;
    float s = 0.f;
    for (int k = 1 + lane; k < n_out; k += 32) s += y[k];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    const float shift = (target[warp] - s) / (float)(n_out - 1);
    float loss = 0.f, gsum = 0.f;
    const float scale = 2.0f / ((float)B * (float)n_out);
    for (int k = lane; k < n_out; k += 32) {
        const float p = (k == 0) ? v_empty : y[k] + shift;
        if (phi) phi[(long long)warp * n_out + k] = p;
        if (labels) {
            const float e = p - labels[(long long)warp * n_out + k];
            loss += e * e;
            if (k > 0) gsum += scale * e;
        }
    }
    if (!labels) return;
    for (int o = 16; o > 0; o >>= 1) {
        loss += __shfl_xor_sync(0xffffffffu, loss, o);
        gsum += __shfl_xor_sync(0xffffffffu, gsum, o);
    }
    if (lane == 0) loss_rows[warp] = loss;
    const float gmean = gsum / (float)(n_out - 1);
    for (int k = lane; k < ld_dyb; k += 32) {
        float g = 0.f;
        if (k > 0 && k < n_out) {
            const float p = y[k] + shift;
            g = scale * (p - labels[(long long)warp * n_out + k]) - gmean;
        }
        if (k < n_out) dYf[(long long)warp * n_out + k] = g;
        const bf16 gb = __float2bfloat16_rn(g);
        dYb[(long long)warp * ld_dyb + k] = gb;
        if (dYt && k < n_out) dYt[(long long)k * ld_dyt + warp] = gb;
    }
}

// Column sums of an FP32 [M, N] matrix in a fixed order, one launch.  Block
// (32 columns, a slab of 256 rows), 32 x 8 threads; thread (x, y) sums rows
// 32y..32y+31 of the slab, the 8 partials are added in order and written to
// part[slab][N].  The last block to finish a column block (an arrival
// counter per column block, reset by that block for the next call) adds the
// slab partials of its 32 columns in slab order.  No block waits for
// another.
__global__ void colsum_kernel(const float *X, int M, int N, float *part, int *arrivals, float *out) {
    __shared__ float red[8][33];
    __shared__ int s_last;
    const int c = blockIdx.x * 32 + threadIdx.x;
    const int r0 = blockIdx.y * 256 + threadIdx.y * 32;
    float s = 0.f;
    if (c < N) {
        const int r1 = min(r0 + 32, M);
        for (int r = r0; r < r1; ++r) s += X[(long long)r * N + c];
    }
    red[threadIdx.y][threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.y == 0) {
        if (c < N) {
            float t = 0.f;
            for (int k = 0; k < 8; ++k) t += red[k][threadIdx.x];
            part[(long long)blockIdx.y * N + c] = t;
        }
        __threadfence();
    }
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0)
        s_last = atomicAdd(arrivals + blockIdx.x, 1) == (int)gridDim.y - 1;
    __syncthreads();
    if (!s_last) return;
    if (threadIdx.y == 0) {
        __threadfence();
        if (c < N) {
            float t = 0.f;
            for (int k = 0; k < (int)gridDim.y; ++k) t += __ldcg(part + (long long)k * N + c);
            out[c] = t;
        }
        if (threadIdx.x == 0) arrivals[blockIdx.x] = 0;
    }
}

// Sum of the per-instance losses, one block, fixed order.
__global__ void sum_kernel(const float *x, int n, float scale, float *out) {
    __shared__ float red[256];
    float s = 0.f;
    for (int i = threadIdx.x; i < n; i += 256) s += x[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0] * scale;
}

// Adam (Kingma & Ba): m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
// p -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps), over a flat buffer.
__global__ void adam_kernel(float *p, float *m, float *v, const float *g, long long n, float lr, float b1, float b2,
                            float eps, float c1, float c2) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// Surrogate residual of each instance on its sampled coalitions:
// g(T) = sum over scores S subset of T of phi(S);
// r = sqrt(mean_k (g(T_k) - v(T_k))^2).  One warp per instance.
__global__ void residual_kernel(const float *phi, int B, int n_out, const unsigned *masks, const unsigned *coal,
                                const float *vcoal, int K, float *resid) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= B) return;
    float acc = 0.f;
    for (int k = lane; k < K; k += 32) {
        const unsigned T = coal[(long long)warp * K + k];
        float g = 0.f;
        for (int q = 0; q < n_out; ++q)
            if ((masks[q] & T) == masks[q]) g += phi[(long long)warp * n_out + q];
        const float e = g - vcoal[(long long)warp * K + k];
        acc += e * e;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) resid[warp] = sqrtf(acc / (float)K);
}

int grid_for(long long n) {
    long long g = (n + 255) / 256;
    if (g > 4096) g = 4096;
    return (int)(g < 1 ? 1 : g);
}

}  // namespace ttfsi_student

struct tt_fsi_student_s {
    int d = 0, H = 0, n_out = 0, n_pad = 0, max_batch = 0, ldB = 0;
    long long n_params = 0;
    long long off_W1 = 0, off_b1 = 0, off_W2 = 0, off_b2 = 0, off_W3 = 0, off_b3 = 0;
    float *params = nullptr, *m = nullptr, *v = nullptr, *grads = nullptr;
    __nv_bfloat16 *W1b = nullptr, *W2b = nullptr, *W2bT = nullptr, *W3b = nullptr, *W3bT = nullptr;
    __nv_bfloat16 *Xb = nullptr, *XbT = nullptr, *A1 = nullptr, *A1T = nullptr, *A2 = nullptr, *A2T = nullptr;
    __nv_bfloat16 *dYb = nullptr, *dYt = nullptr, *dH2 = nullptr, *dH2T = nullptr, *dH1T = nullptr;
    float *Z1 = nullptr, *Z2 = nullptr, *Y = nullptr, *dYf = nullptr, *dH2f = nullptr, *dH1f = nullptr;
    float *loss_rows = nullptr;
    float *colpart = nullptr;  // column-sum partials [ceil(max_batch / 256)][max(H, n_out)]
    int *colarrive = nullptr;  // column-sum arrival counters [ceil(max(H, n_out) / 32)], zero between calls
    float *gpart = nullptr;    // K-slice partial products of the weight gradients
    int *err = nullptr;
    float lr = 1e-3f, beta1 = 0.9f, beta2 = 0.999f, eps = 1e-8f;
    long long step = 0;
    std::vector<void *> allocs;
};

namespace {

using ttfsi_student::bf16;

template <typename T>
cudaError_t st_alloc(tt_fsi_student_s *s, T **p, size_t count) {
    cudaError_t e = cudaMalloc((void **)p, count * sizeof(T) + 16);
    if (e == cudaSuccess) {
        s->allocs.push_back(*p);
        e = cudaMemset(*p, 0, count * sizeof(T) + 16);
    }
    return e;
}

tt_fsi_status gemm(const bf16 *A, int lda, const bf16 *B, int ldb, int M, int N, int K, const float *bias, int act,
                   const float *dz, int ldz, float *Cf, int ldcf, bf16 *Cb, int ldcb, bf16 *Ct, int ldct, int *err,
                   cudaStream_t st, float *gpart = nullptr) {
    ttfsi_gemm::GemmArgs a{};
    a.A = A;
    a.B = B;
    a.lda = lda;
    a.ldb = ldb;
    a.M = M;
    a.N = N;
    a.K = K;
    a.bias = bias;
    a.act = act;
    a.dgelu_z = dz;
    a.ldz = ldz;
    a.Cf = Cf;
    a.ldcf = ldcf;
    a.Cb = Cb;
    a.ldcb = ldcb;
    a.Ct = Ct;
    a.ldct = ldct;
    a.err = err;
    // plain products with a long K (the weight gradients) are split over K
    // into the student's partial buffer and summed in slice order
    const int kbc = (!act && !dz && !Cb && !Ct && Cf && gpart) ? split_kbc(M, N, K) : 0;
    if (kbc > 0) {
        const int nk = (K + ttfsi_gemm::BK - 1) / ttfsi_gemm::BK, slices = (nk + kbc - 1) / kbc;
        a.kbc = kbc;
        a.bias = nullptr;  // added once, in the slice sum
        a.Cf = gpart;
        a.cf_zstride = (long long)M * ldcf;
        tt_fsi_status r = gemm_launch(a, st);
        if (r != TT_FSI_OK) return r;
        const long long n = (long long)M * N;
        ksum_kernel<<<(unsigned)std::min<long long>((n + 255) / 256, 4096), 256, 0, st>>>(gpart, a.cf_zstride, slices, M,
                                                                                          N, ldcf, bias, Cf);
        return st_status(cudaGetLastError());
    }
    return gemm_launch(a, st);
}

void to_bf16(const float *W, int rows, int cols, int rows_pad, bf16 *Wb, bf16 *Wt, int ldt, cudaStream_t st) {
    const dim3 grid((unsigned)((cols + 31) / 32), (unsigned)((rows_pad + 31) / 32));
    ttfsi_student::to_bf16_tiled_kernel<<<grid, dim3(32, 8), 0, st>>>(W, rows, cols, rows_pad, Wb, Wt, ldt);
}

// Bias gradient: column sums of an FP32 [M, N] matrix (fixed order).
void colsum(tt_fsi_student_s *s, const float *X, int M, int N, float *out, cudaStream_t st) {
    const int slabs = (M + 255) / 256;
    ttfsi_student::colsum_kernel<<<dim3((unsigned)((N + 31) / 32), (unsigned)slabs), dim3(32, 8), 0, st>>>(
        X, M, N, s->colpart, s->colarrive, out);
}

// BF16 copies of the three weight matrices (and the transposes the backward
// pass reads), one launch.
tt_fsi_status refresh_bf16(tt_fsi_student_s *s, cudaStream_t st) {
    using ttfsi_student::CastJob;
    ttfsi_student::CastJobs jobs{};
    auto add = [&](const float *W, int rows, int cols, int rows_pad, bf16 *Wb, bf16 *Wt, int ldt) {
        CastJob &c = jobs.j[jobs.n];
        c.W = W;
        c.Wb = Wb;
        c.Wt = Wt;
        c.rows = rows;
        c.cols = cols;
        c.rows_pad = rows_pad;
        c.ldt = ldt;
        c.tiles_x = (cols + 31) / 32;
        c.first = jobs.n ? jobs.j[jobs.n - 1].first + jobs.j[jobs.n - 1].tiles_x * ((jobs.j[jobs.n - 1].rows_pad + 31) / 32)
                         : 0;
        ++jobs.n;
    };
    add(s->params + s->off_W1, s->H, s->d, s->H, s->W1b, nullptr, 0);
    add(s->params + s->off_W2, s->H, s->H, s->H, s->W2b, s->W2bT, s->H);
    add(s->params + s->off_W3, s->n_out, s->H, s->n_pad, s->W3b, s->W3bT, s->n_pad);
    const CastJob &last = jobs.j[jobs.n - 1];
    const unsigned blocks = (unsigned)(last.first + last.tiles_x * ((last.rows_pad + 31) / 32));
    ttfsi_student::to_bf16_multi_kernel<<<blocks, dim3(32, 8), 0, st>>>(jobs);
    return st_status(cudaGetLastError());
}

// Forward pass into s->Y (raw outputs); `train` also keeps what the backward
// pass needs (transposed activations).
tt_fsi_status forward(tt_fsi_student_s *s, const float *x, int B, bool train, cudaStream_t st) {
    using namespace ttfsi_student;
    to_bf16(x, B, s->d, B, s->Xb, train ? s->XbT : nullptr, s->ldB, st);
    tt_fsi_status r = st_status(cudaGetLastError());
    if (r != TT_FSI_OK) return r;
    const float *P = s->params;
    // the FP32 pre-activations Z1, Z2 and the transposed activations are
    // read only by the backward pass
    r = gemm(s->Xb, s->d, s->W1b, s->d, B, s->H, s->d, P + s->off_b1, 1, nullptr, 0, train ? s->Z1 : nullptr, s->H,
             s->A1, s->H, train ? s->A1T : nullptr, s->ldB, s->err, st);
    if (r != TT_FSI_OK) return r;
    r = gemm(s->A1, s->H, s->W2b, s->H, B, s->H, s->H, P + s->off_b2, 1, nullptr, 0, train ? s->Z2 : nullptr, s->H,
             s->A2, s->H, train ? s->A2T : nullptr, s->ldB, s->err, st);
    if (r != TT_FSI_OK) return r;
    return gemm(s->A2, s->H, s->W3b, s->H, B, s->n_out, s->H, P + s->off_b3, 0, nullptr, 0, s->Y, s->n_out, nullptr, 0,
                nullptr, 0, s->err, st, s->gpart);
}

// Gradients of the mean squared error of the projected outputs into s->grads.
tt_fsi_status backward(tt_fsi_student_s *s, const float *labels, const float *target, float v_empty, int B,
                       float *loss_dev, cudaStream_t st) {
    using namespace ttfsi_student;
    const int warps_per_block = 8;
    project_loss_kernel<<<(B + warps_per_block - 1) / warps_per_block, 32 * warps_per_block, 0, st>>>(
        s->Y, B, s->n_out, target, v_empty, nullptr, labels, s->loss_rows, s->dYf, s->dYb, s->n_pad, nullptr, 0);
    // dY^T (rows n_out..n_pad of dYt stay zero)
    to_bf16(s->dYf, B, s->n_out, B, nullptr, s->dYt, s->ldB, st);
    tt_fsi_status r = st_status(cudaGetLastError());
    if (r != TT_FSI_OK) return r;
    if (loss_dev) sum_kernel<<<1, 256, 0, st>>>(s->loss_rows, B, 1.0f / ((float)B * s->n_out), loss_dev);
    float *G = s->grads;
    // layer 3
    r = gemm(s->dYt, s->ldB, s->A2T, s->ldB, s->n_out, s->H, B, nullptr, 0, nullptr, 0, G + s->off_W3, s->H, nullptr, 0,
             nullptr, 0, s->err, st, s->gpart);
    if (r != TT_FSI_OK) return r;
    colsum(s, s->dYf, B, s->n_out, G + s->off_b3, st);
    r = gemm(s->dYb, s->n_pad, s->W3bT, s->n_pad, B, s->H, s->n_pad, nullptr, 0, s->Z2, s->H, s->dH2f, s->H, s->dH2,
             s->H, s->dH2T, s->ldB, s->err, st);
    if (r != TT_FSI_OK) return r;
    // layer 2
    colsum(s, s->dH2f, B, s->H, G + s->off_b2, st);
    r = gemm(s->dH2T, s->ldB, s->A1T, s->ldB, s->H, s->H, B, nullptr, 0, nullptr, 0, G + s->off_W2, s->H, nullptr, 0,
             nullptr, 0, s->err, st, s->gpart);
    if (r != TT_FSI_OK) return r;
    r = gemm(s->dH2, s->H, s->W2bT, s->H, B, s->H, s->H, nullptr, 0, s->Z1, s->H, s->dH1f, s->H, nullptr, 0, s->dH1T,
             s->ldB, s->err, st);
    if (r != TT_FSI_OK) return r;
    // layer 1
    colsum(s, s->dH1f, B, s->H, G + s->off_b1, st);
    r = gemm(s->dH1T, s->ldB, s->XbT, s->ldB, s->H, s->d, B, nullptr, 0, nullptr, 0, G + s->off_W1, s->d, nullptr, 0,
             nullptr, 0, s->err, st, s->gpart);
    if (r != TT_FSI_OK) return r;
    return st_status(cudaGetLastError());
}

void student_free(tt_fsi_student_s *s) {
    for (void *p : s->allocs) cudaFree(p);
    s->allocs.clear();
}

}  // namespace

extern "C" {

tt_fsi_status tt_fsi_student_create(int d, int hidden, int n_out, int max_batch, const float *params_host,
                                    tt_fsi_student *out) {
    if (!out || !params_host || d < 1 || hidden < 8 || n_out < 2 || max_batch < 1) return TT_FSI_ERR_INVALID_ARG;
    if ((d % 8) || (hidden % 8)) return TT_FSI_ERR_UNSUPPORTED;  // 16-byte rows of the BF16 operands
    *out = nullptr;
    tt_fsi_student_s *s = new (std::nothrow) tt_fsi_student_s();
    if (!s) return TT_FSI_ERR_NO_MEMORY;
    s->d = d;
    s->H = hidden;
    s->n_out = n_out;
    s->n_pad = (n_out + 15) / 16 * 16;
    s->max_batch = max_batch;
    s->ldB = (max_batch + 7) / 8 * 8;
    long long o = 0;
    s->off_W1 = o;
    o += (long long)hidden * d;
    s->off_b1 = o;
    o += hidden;
    s->off_W2 = o;
    o += (long long)hidden * hidden;
    s->off_b2 = o;
    o += hidden;
    s->off_W3 = o;
    o += (long long)n_out * hidden;
    s->off_b3 = o;
    o += n_out;
    s->n_params = o;
    const size_t Bm = (size_t)s->ldB, H = (size_t)hidden;
    cudaError_t e = cudaSuccess;
    auto A = [&](auto **p, size_t n) {
        if (e == cudaSuccess) e = st_alloc(s, p, n);
    };
    A(&s->params, (size_t)o);
    A(&s->m, (size_t)o);
    A(&s->v, (size_t)o);
    A(&s->grads, (size_t)o);
    A(&s->W1b, H * d);
    A(&s->W2b, H * H);
    A(&s->W2bT, H * H);
    A(&s->W3b, (size_t)s->n_pad * H);
    A(&s->W3bT, H * s->n_pad);
    A(&s->Xb, Bm * d);
    A(&s->XbT, (size_t)d * Bm);
    A(&s->A1, Bm * H);
    A(&s->A1T, H * Bm);
    A(&s->A2, Bm * H);
    A(&s->A2T, H * Bm);
    A(&s->Z1, Bm * H);
    A(&s->Z2, Bm * H);
    A(&s->Y, Bm * n_out);
    A(&s->dYf, Bm * n_out);
    A(&s->dYb, Bm * s->n_pad);
    A(&s->dYt, (size_t)s->n_pad * Bm);
    A(&s->dH2f, Bm * H);
    A(&s->dH2, Bm * H);
    A(&s->dH2T, H * Bm);
    A(&s->dH1f, Bm * H);
    A(&s->dH1T, H * Bm);
    A(&s->loss_rows, Bm);
    A(&s->colpart, ((Bm + 255) / 256) * (size_t)std::max(hidden, n_out));
    A(&s->colarrive, ((size_t)std::max(hidden, n_out) + 31) / 32);
    {
        // the largest split product: the weight gradients W3 [n_out, H], W2 [H, H], W1 [H, d] with
        // K = max_batch
        size_t need = 0;
        // (and the forward output layer [max_batch, n_out] with K = H)
        const int shapes[4][3] = {{n_out, hidden, max_batch}, {hidden, hidden, max_batch}, {hidden, d, max_batch},
                                  {max_batch, n_out, hidden}};
        for (auto &sh : shapes) {
            const int kbc = split_kbc(sh[0], sh[1], sh[2]);
            if (!kbc) continue;
            const int nk = (sh[2] + ttfsi_gemm::BK - 1) / ttfsi_gemm::BK;
            need = std::max(need, (size_t)((nk + kbc - 1) / kbc) * sh[0] * sh[1]);
        }
        if (need) A(&s->gpart, need);
    }
    A(&s->err, 1);
    if (e == cudaSuccess) e = cudaMemcpy(s->params, params_host, (size_t)o * sizeof(float), cudaMemcpyHostToDevice);
    tt_fsi_status r = st_status(e);
    if (r == TT_FSI_OK) r = refresh_bf16(s, nullptr);
    if (r == TT_FSI_OK) r = st_status(cudaDeviceSynchronize());
    if (r != TT_FSI_OK) {
        student_free(s);
        delete s;
        return r;
    }
    *out = s;
    return TT_FSI_OK;
}

void tt_fsi_student_destroy(tt_fsi_student s) {
    if (!s) return;
    cudaDeviceSynchronize();
    student_free(s);
    delete s;
}

int64_t tt_fsi_student_num_params(tt_fsi_student s) { return s ? s->n_params : -1; }

tt_fsi_status tt_fsi_student_set_adam(tt_fsi_student s, float lr, float beta1, float beta2, float eps) {
    if (!s || !(lr >= 0.f) || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) || !(eps > 0.f))
        return TT_FSI_ERR_INVALID_ARG;
    s->lr = lr;
    s->beta1 = beta1;
    s->beta2 = beta2;
    s->eps = eps;
    return TT_FSI_OK;
}

tt_fsi_status tt_fsi_student_gradients(tt_fsi_student s, const float *x_dev, const float *labels_dev,
                                       const float *target_dev, float v_empty, int B, float *loss_dev,
                                       struct CUstream_st *stream) {
    if (!s || !x_dev || !labels_dev || !target_dev || B < 1 || B > s->max_batch) return TT_FSI_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    tt_fsi_status r = forward(s, x_dev, B, true, st);
    if (r == TT_FSI_OK) r = backward(s, labels_dev, target_dev, v_empty, B, loss_dev, st);
    return r;
}

tt_fsi_status tt_fsi_student_train_step(tt_fsi_student s, const float *x_dev, const float *labels_dev,
                                        const float *target_dev, float v_empty, int B, float *loss_dev,
                                        struct CUstream_st *stream) {
    tt_fsi_status r = tt_fsi_student_gradients(s, x_dev, labels_dev, target_dev, v_empty, B, loss_dev, stream);
    if (r != TT_FSI_OK) return r;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    s->step += 1;
    const float c1 = 1.0f - (float)std::pow((double)s->beta1, (double)s->step);
    const float c2 = 1.0f - (float)std::pow((double)s->beta2, (double)s->step);
    ttfsi_student::adam_kernel<<<ttfsi_student::grid_for(s->n_params), 256, 0, st>>>(
        s->params, s->m, s->v, s->grads, s->n_params, s->lr, s->beta1, s->beta2, s->eps, c1, c2);
    r = st_status(cudaGetLastError());
    if (r == TT_FSI_OK) r = refresh_bf16(s, st);
    return r;
}

tt_fsi_status tt_fsi_student_predict(tt_fsi_student s, const float *x_dev, const float *target_dev, float v_empty,
                                     int B, float *phi_dev, struct CUstream_st *stream) {
    if (!s || !x_dev || !target_dev || !phi_dev || B < 1 || B > s->max_batch) return TT_FSI_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    tt_fsi_status r = forward(s, x_dev, B, false, st);
    if (r != TT_FSI_OK) return r;
    ttfsi_student::project_loss_kernel<<<(B + 7) / 8, 256, 0, st>>>(s->Y, B, s->n_out, target_dev, v_empty, phi_dev,
                                                                  nullptr, nullptr, nullptr, nullptr, 0, nullptr, 0);
    return st_status(cudaGetLastError());
}

tt_fsi_status tt_fsi_student_get_state(tt_fsi_student s, float *params_host, float *adam_m_host, float *adam_v_host,
                                       int64_t *step) {
    if (!s) return TT_FSI_ERR_INVALID_ARG;
    const size_t bytes = (size_t)s->n_params * sizeof(float);
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess && params_host) e = cudaMemcpy(params_host, s->params, bytes, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && adam_m_host) e = cudaMemcpy(adam_m_host, s->m, bytes, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && adam_v_host) e = cudaMemcpy(adam_v_host, s->v, bytes, cudaMemcpyDeviceToHost);
    if (step) *step = s->step;
    return st_status(e);
}

tt_fsi_status tt_fsi_student_set_state(tt_fsi_student s, const float *params_host, const float *adam_m_host,
                                       const float *adam_v_host, int64_t step) {
    if (!s || step < 0) return TT_FSI_ERR_INVALID_ARG;
    const size_t bytes = (size_t)s->n_params * sizeof(float);
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess && params_host) e = cudaMemcpy(s->params, params_host, bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && adam_m_host) e = cudaMemcpy(s->m, adam_m_host, bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && adam_v_host) e = cudaMemcpy(s->v, adam_v_host, bytes, cudaMemcpyHostToDevice);
    s->step = step;
    tt_fsi_status r = st_status(e);
    if (r == TT_FSI_OK) r = refresh_bf16(s, nullptr);
    if (r == TT_FSI_OK) r = st_status(cudaDeviceSynchronize());
    return r;
}

tt_fsi_status tt_fsi_student_get_grads(tt_fsi_student s, float *grads_host) {
    if (!s || !grads_host) return TT_FSI_ERR_INVALID_ARG;
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess)
        e = cudaMemcpy(grads_host, s->grads, (size_t)s->n_params * sizeof(float), cudaMemcpyDeviceToHost);
    return st_status(e);
}

tt_fsi_status tt_fsi_student_check(tt_fsi_student s, struct CUstream_st *stream) {
    if (!s) return TT_FSI_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, s->err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->err, 0, sizeof(int), st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return st_status(e);
    return h ? TT_FSI_ERR_TIMEOUT : TT_FSI_OK;
}

tt_fsi_status tt_fsi_surrogate_residual(const float *phi_dev, int B, int n_out, const unsigned *score_masks_dev,
                                        const unsigned *coal_dev, const float *vcoal_dev, int K, float *resid_dev,
                                        struct CUstream_st *stream) {
    if (B < 0 || n_out < 1 || K < 1) return TT_FSI_ERR_INVALID_ARG;
    if (B == 0) return TT_FSI_OK;
    if (!phi_dev || !score_masks_dev || !coal_dev || !vcoal_dev || !resid_dev) return TT_FSI_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    ttfsi_student::residual_kernel<<<(B + 7) / 8, 256, 0, st>>>(phi_dev, B, n_out, score_masks_dev, coal_dev, vcoal_dev,
                                                              K, resid_dev);
    return st_status(cudaGetLastError());
}

}  // extern "C"
