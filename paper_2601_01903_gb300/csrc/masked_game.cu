// Masked-model value function on GB300: v_x(S) = f(z), z_i = x_i for i in S
// and baseline_i otherwise, f a GELU MLP d -> h1 -> h2 -> 1 (the value
// function of Section 2.1, "the model's prediction when only the features in
// S are present", with absent features replaced by a baseline).
//
// One CTA evaluates 2^G coalitions of one instance that share their high
// bits.  Layer 1 is built as a subset sum: W1 z + b1 = (W1 z_high + b1) +
// sum_{i in S_low} W1[:, i] (x_i - baseline_i), so the 2^G pre-activations of
// a CTA cost one d-term dot product per hidden unit plus one add per
// coalition (doubling over the G low bits).  Layer 2 is a [2^G, h1] x
// [h1, h2] product from shared memory, layer 3 a dot product reduced across
// the two threads that share a coalition.  The float64 instantiation is the
// parity path; the float32 one generates training labels faster.  The
// interventional value function of Section 4.1 (the mean of f over
// background rows standing in for the absent features) runs as one launch
// per background row, each adding f / K to v in ascending row order.
#include <cuda_runtime.h>

#include <cstdint>

#include "tt_fsi.h"

namespace ttfsi_mg {

constexpr int G = 6;                 // coalitions per CTA = 64
constexpr int NC = 1 << G;
constexpr int THREADS = 128;         // two threads per coalition in layer 2
constexpr int MAX_H = 256;

template <typename T>
__device__ __forceinline__ T gelu(T z);
template <>
__device__ __forceinline__ double gelu<double>(double z) {
    return 0.5 * z * (1.0 + erf(z * 0.70710678118654752440));
}
template <>
__device__ __forceinline__ float gelu<float>(float z) {
    return 0.5f * z * (1.0f + erff(z * 0.70710678118654752440f));
}

struct Args {
    const double *W1, *b1, *W2, *b2, *W3;
    double b3;
    const double *x, *base;
    void *v;
    int d, h1, h2;
    long long game0;
    const float *W1f, *b1f, *W2f, *b2f, *W3f;
    double scale;    // v = scale * f (1 for the baseline value function, 1/K per background row)
    int accumulate;  // add to v instead of overwriting it
};

// Weights in the arithmetic of the instantiation (float64 or float32 copies).
template <typename T>
struct W;
template <>
struct W<double> {
    static __device__ __forceinline__ const double *w2(const Args &a) { return a.W2; }
    static __device__ __forceinline__ double b2(const Args &a, int j) { return a.b2[j]; }
    static __device__ __forceinline__ double w3(const Args &a, int j) { return a.W3[j]; }
};
template <>
struct W<float> {
    static __device__ __forceinline__ const float *w2(const Args &a) { return a.W2f; }
    static __device__ __forceinline__ float b2(const Args &a, int j) { return a.b2f[j]; }
    static __device__ __forceinline__ float w3(const Args &a, int j) { return a.W3f[j]; }
};

template <typename T>
__global__ void __launch_bounds__(THREADS) masked_game_kernel(Args a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *pre = reinterpret_cast<T *>(smem_raw);       // [NC][h1 + 1]
    __shared__ T part[THREADS];
    const int tid = threadIdx.x;
    const int ld = a.h1 + 1;
    const long long game = a.game0 + blockIdx.y;
    const long long S_high = (long long)blockIdx.x << G;
    const double *x = a.x + game * a.d;
    const int g = a.d < G ? a.d : G;

    // layer-1 pre-activations by subset sums over the low bits
    for (int j = tid; j < a.h1; j += THREADS) {
        double acc = a.b1[j];
        for (int i = 0; i < a.d; ++i) {
            const bool on = (i >= g) && ((S_high >> i) & 1);
            acc += a.W1[(long long)j * a.d + i] * (on ? x[i] : a.base[i]);
        }
        pre[j] = (T)acc;
        for (int k = 0; k < g; ++k) {
            const T delta = (T)(a.W1[(long long)j * a.d + k] * (x[k] - a.base[k]));
            for (int c = 0; c < (1 << k); ++c) pre[(c | (1 << k)) * ld + j] = pre[c * ld + j] + delta;
        }
    }
    __syncthreads();
    const int nc = 1 << g;
    for (int idx = tid; idx < nc * a.h1; idx += THREADS) {
        const int c = idx / a.h1, j = idx - c * a.h1;
        pre[c * ld + j] = gelu<T>(pre[c * ld + j]);
    }
    __syncthreads();

    // layer 2 (+ GELU) and layer 3: thread pair (c, half) covers coalition c
    const int c = tid % NC, half = tid / NC;
    T acc3 = 0;
    if (c < nc) {
        const T *row = pre + c * ld;
        for (int j = half; j < a.h2; j += 2) {
            const T *w = W<T>::w2(a) + (long long)j * a.h1;
            T acc = W<T>::b2(a, j);
            for (int i = 0; i < a.h1; ++i) acc += __ldg(w + i) * row[i];
            acc3 += W<T>::w3(a, j) * gelu<T>(acc);
        }
    }
    part[tid] = acc3;
    __syncthreads();
    if (tid < NC && tid < nc) {
        const T val = part[tid] + part[tid + NC] + (T)a.b3;
        T *out = reinterpret_cast<T *>(a.v) + (game << a.d) + S_high + tid;
        if (a.accumulate)
            *out += (T)a.scale * val;
        else
            *out = (a.scale == 1.0) ? val : (T)a.scale * val;
    }
}

}  // namespace ttfsi_mg

namespace ttfsi_mg {
tt_fsi_status masked_game_launch(const tt_fsi_mlp *model, const double *x_dev, const double *baseline_dev, int64_t B,
                                 void *v_dev, int out_f32, double scale, int accumulate, struct CUstream_st *stream);
}  // namespace ttfsi_mg

extern "C" tt_fsi_status tt_fsi_masked_game(const tt_fsi_mlp *model, const double *x_dev,
                                           const double *baseline_dev, int64_t B, void *v_dev,
                                           int out_f32, struct CUstream_st *stream) {
    return ttfsi_mg::masked_game_launch(model, x_dev, baseline_dev, B, v_dev, out_f32, 1.0, 0, stream);
}

extern "C" tt_fsi_status tt_fsi_masked_game_interventional(const tt_fsi_mlp *model, const double *x_dev,
                                                          const double *background_dev, int n_background, int64_t B,
                                                          void *v_dev, int out_f32, struct CUstream_st *stream) {
    if (!model || n_background < 1 || !background_dev) return TT_FSI_ERR_INVALID_ARG;
    const double scale = 1.0 / (double)n_background;
    for (int k = 0; k < n_background; ++k) {
        const tt_fsi_status s = ttfsi_mg::masked_game_launch(model, x_dev, background_dev + (size_t)k * model->d, B,
                                                             v_dev, out_f32, scale, k > 0, stream);
        if (s != TT_FSI_OK) return s;
    }
    return TT_FSI_OK;
}

tt_fsi_status ttfsi_mg::masked_game_launch(const tt_fsi_mlp *model, const double *x_dev, const double *baseline_dev,
                                           int64_t B, void *v_dev, int out_f32, double scale, int accumulate,
                                           struct CUstream_st *stream) {
    using namespace ttfsi_mg;
    if (!model || B < 0) return TT_FSI_ERR_INVALID_ARG;
    if (B == 0) return TT_FSI_OK;
    if (!x_dev || !baseline_dev || !v_dev || !model->W1 || !model->b1 || !model->W2 || !model->b2 ||
        !model->W3)
        return TT_FSI_ERR_INVALID_ARG;
    if (model->d < 1 || model->d > 30 || model->h1 < 1 || model->h2 < 1 || model->h1 > MAX_H ||
        model->h2 > MAX_H)
        return TT_FSI_ERR_INVALID_ARG;
    if (out_f32 && (!model->W2f || !model->b2f || !model->W3f)) return TT_FSI_ERR_INVALID_ARG;
    Args a{model->W1, model->b1, model->W2, model->b2, model->W3, model->b3,
           x_dev, baseline_dev, v_dev, model->d, model->h1, model->h2, 0,
           model->W1f, model->b1f, model->W2f, model->b2f, model->W3f, scale, accumulate};
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int g = model->d < G ? model->d : G;
    const size_t elem = out_f32 ? sizeof(float) : sizeof(double);
    const size_t smem = (size_t)(1 << g) * (model->h1 + 1) * elem;
    cudaError_t e;
    if (out_f32)
        e = cudaFuncSetAttribute(masked_game_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    else
        e = cudaFuncSetAttribute(masked_game_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return TT_FSI_ERR_CUDA;
    const unsigned groups = 1u << (model->d - g);
    for (int64_t g0 = 0; g0 < B; g0 += 65535) {
        const unsigned nb = (unsigned)((B - g0) < 65535 ? (B - g0) : 65535);
        a.game0 = g0;
        dim3 grid(groups, nb);
        if (out_f32)
            masked_game_kernel<float><<<grid, THREADS, smem, st>>>(a);
        else
            masked_game_kernel<double><<<grid, THREADS, smem, st>>>(a);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? TT_FSI_ERR_NO_MEMORY : TT_FSI_ERR_CUDA;
    }
    return TT_FSI_OK;
}

// ----------------------------------------------------------------------------
// Value function at sampled coalitions (FP32): one warp per (instance,
// coalition); layer-1 and layer-2 units are spread over the lanes, layer 3 is
// a warp reduction.  Used by the student's residual spot check.
// ----------------------------------------------------------------------------
namespace ttfsi_mg {

constexpr int SW = 8;  // warps per block

__global__ void __launch_bounds__(32 * SW) masked_game_sampled_kernel(Args a, const unsigned *coal, int K, long long total,
                                                                      float *out) {
    extern __shared__ __align__(16) unsigned char smem_s[];
    float *h1 = reinterpret_cast<float *>(smem_s) + (threadIdx.x >> 5) * (a.h1 + 64);
    const int lane = threadIdx.x & 31;
    for (long long w = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; w < total;
         w += ((long long)gridDim.x * blockDim.x) >> 5) {
        const long long b = w / K;
        const unsigned T = coal[w];
        const double *x = a.x + b * a.d;
        // the instance's features and the baseline, converted once per coalition
        float *zf = h1 + a.h1;
        for (int i = lane; i < a.d; i += 32) {
            zf[i] = (float)x[i];
            zf[32 + i] = (float)a.base[i];
        }
        __syncwarp();
        for (int j = lane; j < a.h1; j += 32) {
            float acc = a.b1f[j];
            for (int i = 0; i < a.d; ++i) acc += a.W1f[(long long)j * a.d + i] * zf[((T >> i) & 1u) ? i : 32 + i];
            h1[j] = gelu<float>(acc);
        }
        __syncwarp();
        float acc3 = 0.f;
        for (int j = lane; j < a.h2; j += 32) {
            float acc = a.b2f[j];
            const float *w = a.W2f + (long long)j * a.h1;
            for (int i = 0; i < a.h1; ++i) acc += __ldg(w + i) * h1[i];
            acc3 += a.W3f[j] * gelu<float>(acc);
        }
        for (int o = 16; o > 0; o >>= 1) acc3 += __shfl_xor_sync(0xffffffffu, acc3, o);
        if (lane == 0) out[w] = acc3 + (float)a.b3;
        __syncwarp();
    }
}

}  // namespace ttfsi_mg

extern "C" tt_fsi_status tt_fsi_masked_game_sampled(const tt_fsi_mlp *model, const double *x_dev,
                                                   const double *baseline_dev, int64_t B, const unsigned *coal_dev,
                                                   int K, float *out_dev, struct CUstream_st *stream) {
    using namespace ttfsi_mg;
    if (!model || B < 0 || K < 1) return TT_FSI_ERR_INVALID_ARG;
    if (B == 0) return TT_FSI_OK;
    if (!x_dev || !baseline_dev || !coal_dev || !out_dev || !model->W1 || !model->b1 || !model->W2 ||
        !model->b2 || !model->W3)
        return TT_FSI_ERR_INVALID_ARG;
    if (model->d < 1 || model->d > 32 || model->h1 < 1 || model->h2 < 1 || model->h1 > MAX_H || model->h2 > MAX_H)
        return TT_FSI_ERR_INVALID_ARG;
    if (!model->W1f || !model->b1f || !model->W2f || !model->b2f || !model->W3f) return TT_FSI_ERR_INVALID_ARG;
    Args a{model->W1, model->b1, model->W2, model->b2, model->W3, model->b3,
           x_dev, baseline_dev, nullptr, model->d, model->h1, model->h2, 0,
           model->W1f, model->b1f, model->W2f, model->b2f, model->W3f, 1.0, 0};
    const long long total = B * (long long)K;
    long long blocks = (total + SW - 1) / SW;
    if (blocks > 65535LL * 16) blocks = 65535LL * 16;
    const size_t smem = (size_t)SW * (model->h1 + 64) * sizeof(float);
    masked_game_sampled_kernel<<<(unsigned)blocks, 32 * SW, smem, reinterpret_cast<cudaStream_t>(stream)>>>(
        a, coal_dev, K, total, out_dev);
    return cudaGetLastError() == cudaSuccess ? TT_FSI_OK : TT_FSI_ERR_CUDA;
}
