// FSI operator kernels for GB300 (sm_103a) and the C ABI of include/tt_fsi.h.
//
// Two kernels per call:
//  1. fsi_tile_kernel: one CTA per tile (game, high pattern U_H) of 2^b
//     coalitions.  Loads the tile, (exact path) rounds it once to a per-tile
//     fixed-point grid, applies the Moebius transform on the b low bits
//     (Section 3.2: the operator is a Kronecker product of [[1,0],[-1,1]], one
//     butterfly level per bit), then the ranked superset sums of the
//     correction (Section 3.3: per output prefix sigma the counter pair
//     (|S|, |T|), here as (sigma, j = |T \ S|)), level by level through two
//     shared-memory buffers.  Writes the n_ch channels Y(U_H, S_L, j).
//  2. fsi_combine_kernel: one CTA per (score S, game).  Reduces the channels
//     of S's low part over all tiles with the combined weights omega_s(p, q)
//     (see fsi_plan.cpp for the derivation) and writes phi(S).
// On the exact path every sum is wrap-around int64 / int128 arithmetic, so
// results are independent of summation order; the weights are exact
// rationals over one denominator per |S|.
#include <cuda_runtime.h>

#include <cstdio>
#include <algorithm>
#include <array>
#include <cstring>
#include <new>
#include <vector>

#include "fast_layout.h"
#include "fast_tile.cuh"
#include "fsi_plan.h"
#include "tile_common.cuh"
#include "tt_fsi.h"

namespace ttfsi {


struct TileArgs {
    const void *v;
    void *Y;
    int *tile_exp;
    int *err;
    const int32_t *trans;
    int d, b, h, n_ch, buf_elems, prec_bits, mob_only;
    int n_states[kMaxLevels];
    int lvl_off[kMaxLevels];
    long long game0;  // first game of this launch
};

struct CombineArgs {
    const void *Y;
    const int *tile_exp;
    const int32_t *tasks;
    const long long *wnum;
    const long long *wden;
    const double *winv;  // 1 / wden[s]
    const double *wf64;
    const float *wf32;
    void *phi;
    int b, h, n_ch, shift_cap, mob_only;
    long long n_out;
    long long game0;
};

// PRE: the precontracted sweep (input v, the Moebius step of bit k fused
// into level k); a template flag so that the plain sweep keeps its loop.
template <typename Acc, bool PRE = false>
__global__ void __launch_bounds__(kTileThreads) fsi_tile_kernel(TileArgs a) {
    using In = typename TileTraits<Acc>::In;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Acc *bufA = reinterpret_cast<Acc *>(smem_raw);
    Acc *bufB = bufA + a.buf_elems;
    __shared__ int s_emax;

    const int tid = threadIdx.x;
    const int n = 1 << a.b;
    const long long game = a.game0 + blockIdx.y;
    const long long tile = blockIdx.x;
    const In *src = reinterpret_cast<const In *>(a.v) + (game << a.d) + (tile << a.b);

    constexpr int VPT = (1 << kMaxTileBits) / kTileThreads;
    int E = 0;
    if constexpr (TileTraits<Acc>::exact) {
        In vals[VPT];
        int emax = 0;
#pragma unroll
        for (int r = 0; r < VPT; ++r) {
            int e = tid + r * kTileThreads;
            vals[r] = (e < n) ? __ldg(src + e) : 0ull;
            emax = max(emax, (int)((vals[r] >> 52) & 0x7ff));
        }
        for (int o = 16; o > 0; o >>= 1) emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, o));
        if (tid == 0) s_emax = 0;
        __syncthreads();
        if ((tid & 31) == 0) atomicMax(&s_emax, emax);
        __syncthreads();
        E = s_emax;
        const bool bad = (E == 0x7ff);
        if (bad && tid == 0) atomicOr(a.err, kErrNonFinite);
        if (E == 0) E = 1;
#pragma unroll
        for (int r = 0; r < VPT; ++r) {
            int e = tid + r * kTileThreads;
            if (e < n) bufA[e] = bad ? 0ll : to_fixed(vals[r], E, a.prec_bits);
        }
    } else {
        for (int e = tid; e < n; e += kTileThreads) bufA[e] = (Acc)__ldg(src + e);
    }
    __syncthreads();

    // Moebius transform on the b tile bits: x[T u {k}] -= x[T] for T without k
    // (skipped by the precontracted sweep, which applies it level by level).
    for (int k = 0; k < (PRE ? 0 : a.b); ++k) {
        const int lo_mask = (1 << k) - 1;
        for (int i = tid; i < (n >> 1); i += kTileThreads) {
            int e0 = ((i >> k) << (k + 1)) | (i & lo_mask);
            bufA[e0 | (1 << k)] -= bufA[e0];
        }
        __syncthreads();
    }

    Acc *out = bufA;
    if (!a.mob_only) {
        // Ranked superset sums, one bit per level.  Level k holds
        // X_k[tau][state] (tau = pattern of bits k..b-1, state = (sigma, j));
        // an output state takes its tau_k = 0 source and its tau_k = 1 source.
        Acc *in = bufA, *nxt = bufB;
        for (int k = 0; k < a.b; ++k) {
            const int nk = a.n_states[k], nk1 = a.n_states[k + 1];
            const int half = n >> (k + 1);
            const int total = nk1 * half;
            const int2 *tr = reinterpret_cast<const int2 *>(a.trans) + a.lvl_off[k];
            for (int idx = tid; idx < total; idx += kTileThreads) {
                int t2 = idx / nk1;
                int st = idx - t2 * nk1;
                int2 s = __ldg(tr + st);
                Acc val = 0;
                if (s.x >= 0) val += in[(2 * t2) * nk + s.x];
                if (s.y >= 0) {
                    val += in[(2 * t2 + 1) * nk + s.y];
                    // B_corr = A_trunc o Moebius (Section 3.5): the tau_k = 1 input
                    // of a core is x[tau_k = 1] - x[tau_k = 0]
                    if constexpr (PRE) val -= in[(2 * t2) * nk + s.y];
                }
                nxt[idx] = val;
            }
            __syncthreads();
            Acc *t = in;
            in = nxt;
            nxt = t;
        }
        out = in;
    }

    Acc *dst = reinterpret_cast<Acc *>(a.Y) + ((game << a.h) + tile) * (long long)a.n_ch;
    for (int c = tid; c < a.n_ch; c += kTileThreads) dst[c] = out[c];
    if constexpr (TileTraits<Acc>::exact) {
        if (tid == 0) a.tile_exp[(game << a.h) + tile] = a.prec_bits + 1022 - E;
    }
}

// ----------------------------------------------------------------------------
// Combine of the fast path: phi(S) = sum over tiles of G(S_L, s, |U_H n S_H|),
// one warp per score, lanes over tiles.  Exact path: tile partial scores are
// aligned to a common exponent by exact left shifts and summed in
// wrap-around int128; the sum, scaled to a double with integer instructions,
// is multiplied once by the reciprocal of the weight denominator.
// ----------------------------------------------------------------------------
constexpr int kCombineFastWarps = 8;

struct CombineFastArgs {
    const void *G;
    const int *tile_exp;
    const int32_t *tasks;
    const long long *wden;
    const double *winv;  // 1 / wden[s]
    void *phi;
    int h, n_g, shift_cap;
    long long n_out;
    long long game0;
};

__device__ __forceinline__ __int128 shfl_down_i128(__int128 v, int o) {
    unsigned long long lo = (unsigned long long)v, hi = (unsigned long long)((unsigned __int128)v >> 64);
    lo = __shfl_down_sync(0xffffffffu, lo, o);
    hi = __shfl_down_sync(0xffffffffu, hi, o);
    return (__int128)(((unsigned __int128)hi << 64) | lo);
}

// x 2^-F rounded to the nearest double (ties to even) with integer
// instructions only (float64 is slow on this part): the leading one of |x|
// gives the exponent, the next 52 bits the mantissa, the rest the rounding.
// Returns false when the result is not a normal double (the caller then
// takes the float64 route); the magnitude is taken in unsigned arithmetic,
// so x = -2^127 is converted too.
__device__ __forceinline__ bool i128_scaled_to_double(__int128 x, int F, double &out) {
    if (x == 0) {
        out = 0.0;
        return true;
    }
    const unsigned long long sign = x < 0 ? (1ull << 63) : 0ull;
    const unsigned __int128 u = x < 0 ? (unsigned __int128)0 - (unsigned __int128)x : (unsigned __int128)x;
    const unsigned long long hi = (unsigned long long)(u >> 64), lo = (unsigned long long)u;
    const int lz = hi ? __clzll((long long)hi) : 64 + __clzll((long long)lo);  // 0 .. 127
    unsigned long long top, rest;  // |x| << lz: bits 127..64 and 63..0
    if (lz >= 64) {
        top = lo << (lz - 64);
        rest = 0;
    } else if (lz == 0) {
        top = hi;
        rest = lo;
    } else {
        top = (hi << lz) | (lo >> (64 - lz));
        rest = lo << lz;
    }
    unsigned long long mant = top >> 11;  // 53 bits, leading one at bit 52
    const unsigned long long low11 = top & 0x7ff;
    mant += (low11 > 0x400 || (low11 == 0x400 && (rest != 0 || (mant & 1)))) ? 1 : 0;
    int e = 127 - lz - F;
    if (mant >> 53) {
        mant >>= 1;
        ++e;
    }
    if (e < -1022 || e > 1023) return false;
    out = __longlong_as_double((long long)(sign | ((unsigned long long)(e + 1023) << 52) | (mant & 0xFFFFFFFFFFFFFull)));
    return true;
}

// Scores [task_begin, task_end) of one game; warp w takes task_begin + w,
// + kCombineFastWarps, ...  Partial scores are read past L1 (ld.global.cg):
// in the persistent batch kernel other CTAs wrote them during this launch.
template <typename Acc>
__device__ __forceinline__ void combine_fast_body(const CombineFastArgs &a, const long long game,
                                                  const long long task_begin, const long long task_end) {
    using GT = typename GTraits<Acc>::G;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ntile = 1 << a.h;
    const GT *Gg = reinterpret_cast<const GT *>(a.G) + (game << a.h) * (long long)a.n_g;
    if constexpr (TileTraits<Acc>::exact) {
        __shared__ int s_fmin, s_fmax;
        const int *texp = a.tile_exp + (game << a.h);
        int fmin = 0x7fffffff, fmax = -0x7fffffff;
        for (int u = threadIdx.x; u < ntile; u += blockDim.x) {
            const int f = __ldcg(texp + u);
            fmin = min(fmin, f);
            fmax = max(fmax, f);
        }
        if (threadIdx.x == 0) {
            s_fmin = 0x7fffffff;
            s_fmax = -0x7fffffff;
        }
        __syncthreads();
        atomicMin(&s_fmin, fmin);
        atomicMax(&s_fmax, fmax);
        __syncthreads();
        const int Fc = min(s_fmax, s_fmin + a.shift_cap);
        // When the game's tile exponents span at most shift_cap (all but games
        // of extreme dynamic range), Fc = fmax and every alignment is a left
        // shift by 0 .. shift_cap < 64: two 64-bit shifts, no rounding.
        const bool left_only = s_fmax - s_fmin <= a.shift_cap;
        constexpr int U = 8;  // independent loads in flight per lane
        for (long long task = task_begin + warp; task < task_end; task += kCombineFastWarps) {
            const unsigned SH = (unsigned)a.tasks[task * 4 + 1];
            const int s = a.tasks[task * 4 + 2] & 0xff;
            const GT *Gs = Gg + (long long)a.tasks[task * 4 + 3] * ntile;
            __int128 acc = 0;
            for (int u0 = lane; u0 < ntile; u0 += 32 * U) {
                longlong2 raw[U];
                int f[U];
#pragma unroll
                for (int k = 0; k < U; ++k) {
                    const int u = u0 + 32 * k;
                    if (u < ntile) {
                        raw[k] = __ldcg(reinterpret_cast<const longlong2 *>(
                            Gs + (long long)__popc((unsigned)u & SH) * ntile + u));
                        f[k] = __ldcg(texp + u);
                    } else {
                        raw[k] = make_longlong2(0, 0);
                        f[k] = Fc;
                    }
                }
                if (left_only) {
#pragma unroll
                    for (int k = 0; k < U; ++k) {
                        const int delta = Fc - f[k];  // 0 .. shift_cap (0 for the padding slots)
                        const unsigned long long lo = (unsigned long long)raw[k].x;
                        const unsigned long long hi =
                            ((unsigned long long)raw[k].y << delta) | ((lo >> 1) >> (63 - delta));
                        acc += (__int128)(((unsigned __int128)hi << 64) | (lo << delta));
                    }
                } else {
#pragma unroll
                    for (int k = 0; k < U; ++k) {
                        __int128 g = (__int128)(((unsigned __int128)(unsigned long long)raw[k].y << 64) |
                                                (unsigned long long)raw[k].x);
                        const int delta = Fc - f[k];
                        if (delta >= 0)
                            g = (__int128)((unsigned __int128)g << delta);
                        else
                            g = (-delta >= 127) ? (__int128)0 : ((g + ((__int128)1 << (-delta - 1))) >> (-delta));
                        acc += g;
                    }
                }
            }
            for (int o = 16; o > 0; o >>= 1) acc += shfl_down_i128(acc, o);
            if (lane == 0) {
                // phi = acc 2^-Fc / D_s.  Float64 is slow on this part: acc 2^-Fc
                // is rounded to a double with integer instructions and the
                // quotient is a product with 1 / D_s (rounded once on the host),
                // one float64 instruction per score; ldexp where acc 2^-Fc is
                // not a normal double.
                double x, out;
                if (i128_scaled_to_double(acc, Fc, x))
                    out = x * __ldg(a.winv + s);
                else
                    out = ldexp(i128_to_double(acc) * __ldg(a.winv + s), -Fc);
                reinterpret_cast<double *>(a.phi)[game * a.n_out + task] = out;
            }
        }
    } else {
        constexpr int U = 8;
        for (long long task = task_begin + warp; task < task_end; task += kCombineFastWarps) {
            const unsigned SH = (unsigned)a.tasks[task * 4 + 1];
            const GT *Gs = Gg + (long long)a.tasks[task * 4 + 3] * ntile;
            Acc acc = 0;
            for (int u0 = lane; u0 < ntile; u0 += 32 * U) {
                Acc part[U];
#pragma unroll
                for (int k = 0; k < U; ++k) {
                    const int u = u0 + 32 * k;
                    part[k] = (u < ntile) ? __ldcg(Gs + (long long)__popc((unsigned)u & SH) * ntile + u) : (Acc)0;
                }
#pragma unroll
                for (int k = 0; k < U; ++k) acc += part[k];
            }
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
            if (lane == 0) reinterpret_cast<Acc *>(a.phi)[game * a.n_out + task] = acc;
        }
    }
}

template <typename Acc>
__global__ void __launch_bounds__(32 * kCombineFastWarps) fsi_combine_fast_kernel(CombineFastArgs a) {
    // as the tile launch's programmatic dependent: wait for its results
    // (returns at once otherwise); combine_fast_body reads them past L1
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const long long t0 = (long long)blockIdx.x * kCombineFastWarps;
    const long long t1 = (t0 + kCombineFastWarps < a.n_out) ? t0 + kCombineFastWarps : a.n_out;
    combine_fast_body<Acc>(a, a.game0 + blockIdx.y, t0, t1);
}

// ----------------------------------------------------------------------------
// Combine of the split schedule for games of at most 2^12 tiles (exact
// arithmetic): kC4Lanes lanes per score, each summing every kC4Lanes-th tile
// (so the lanes of a score read consecutive partial scores), 32 / kC4Lanes
// scores per warp.  Compared with one warp per score, each lane sums
// 2^h / kC4Lanes terms in registers and the cross-lane reduction is three
// shuffle steps, not five; the first batch of partial-score loads is issued
// before the game's exponent range is known, so the exponent pass overlaps
// it; the tiles' alignment shifts are computed once per CTA into shared
// memory and skipped when all tiles of the game share one exponent.  Partial
// scores come from the previous (tile) launch, so loads may go through L1.
// Games whose tile exponents span more than shift_cap take the one-warp-per-
// score routine (its rounding right shifts).
// ----------------------------------------------------------------------------
constexpr int kC4Warps = 8;
constexpr int kC4Lanes = 8;                                // lanes per score
constexpr int kC4Scores = kC4Warps * (32 / kC4Lanes);     // scores per CTA
constexpr int kC4MaxTiles = 4096;                          // h <= 12: per-tile shifts in shared memory

__device__ __forceinline__ __int128 shfl_xor_i128(__int128 v, int o) {
    unsigned long long lo = (unsigned long long)v, hi = (unsigned long long)((unsigned __int128)v >> 64);
    lo = __shfl_xor_sync(0xffffffffu, lo, o);
    hi = __shfl_xor_sync(0xffffffffu, hi, o);
    return (__int128)(((unsigned __int128)hi << 64) | lo);
}

template <typename Acc>
__global__ void __launch_bounds__(32 * kC4Warps, 3) fsi_combine_split_kernel(CombineFastArgs a) {
    static_assert(TileTraits<Acc>::exact, "exact arithmetic only");
    using GT = typename GTraits<Acc>::G;
    constexpr int U = 8;  // partial-score loads in flight per lane
    // launched as the tile grid's programmatic dependent: wait until that
    // grid has finished and its partial scores and exponents are visible
    // (returns at once otherwise); they are read past L1 (ld.global.cg)
    asm volatile("griddepcontrol.wait;" ::: "memory");
    __shared__ unsigned char s_shift[kC4MaxTiles];
    __shared__ int s_f[kC4MaxTiles];  // the game's tile exponents
    __shared__ int s_fmin, s_fmax;
    const long long game = a.game0 + blockIdx.y;
    const int ntile = 1 << a.h;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, q = lane % kC4Lanes;
    const long long t_begin = (long long)blockIdx.x * kC4Scores;
    const long long t_end = t_begin + kC4Scores < a.n_out ? t_begin + kC4Scores : a.n_out;
    const long long task = t_begin + warp * (32 / kC4Lanes) + lane / kC4Lanes;
    const bool active = task < t_end;
    // lanes past the last score stay for the shuffles but sum nothing
    const long long tk = active ? task : t_begin;
    const unsigned SH = (unsigned)__ldg(a.tasks + tk * 4 + 1);
    const int s = __ldg(a.tasks + tk * 4 + 2) & 0xff;
    const GT *row = reinterpret_cast<const GT *>(a.G) + (game << a.h) * (long long)a.n_g +
                    (long long)__ldg(a.tasks + tk * 4 + 3) * ntile;
    const int u_first = active ? q : ntile;
    auto load_batch = [&](int u0, longlong2 (&raw)[U]) {
#pragma unroll
        for (int k = 0; k < U; ++k) {
            const int u = u0 + kC4Lanes * k;
            raw[k] = u < ntile ? __ldcg(reinterpret_cast<const longlong2 *>(
                                     row + (long long)__popc((unsigned)u & SH) * ntile + u))
                               : make_longlong2(0, 0);
        }
    };
    longlong2 raw[U];
    load_batch(u_first, raw);  // in flight during the exponent pass

    const int *texp = a.tile_exp + (game << a.h);
    int fmin = 0x7fffffff, fmax = -0x7fffffff;
    for (int u = threadIdx.x; u < ntile; u += blockDim.x) {
        const int f = __ldcg(texp + u);
        s_f[u] = f;  // kept for the shift table (no second trip to L2)
        fmin = min(fmin, f);
        fmax = max(fmax, f);
    }
    for (int o = 16; o > 0; o >>= 1) {
        fmin = min(fmin, __shfl_xor_sync(0xffffffffu, fmin, o));
        fmax = max(fmax, __shfl_xor_sync(0xffffffffu, fmax, o));
    }
    if (threadIdx.x == 0) {
        s_fmin = 0x7fffffff;
        s_fmax = -0x7fffffff;
    }
    __syncthreads();
    if (lane == 0) {
        atomicMin(&s_fmin, fmin);
        atomicMax(&s_fmax, fmax);
    }
    __syncthreads();
    const int gmin = s_fmin, gmax = s_fmax;
    if (gmax - gmin > a.shift_cap) {
        // rounding right shifts needed: the one-warp-per-score routine
        combine_fast_body<Acc>(a, game, t_begin, t_end);
        return;
    }
    // every alignment is a left shift by Fc - f in [0, shift_cap], Fc = gmax
    const bool shifts = gmax != gmin;
    if (shifts)
        for (int u = threadIdx.x; u < ntile; u += blockDim.x) s_shift[u] = (unsigned char)(gmax - s_f[u]);
    __syncthreads();
    __int128 acc = 0;
    for (int u0 = u_first;;) {
#pragma unroll
        for (int k = 0; k < U; ++k) {
            const unsigned long long lo = (unsigned long long)raw[k].x;
            unsigned long long hi = (unsigned long long)raw[k].y, l2 = lo;
            if (shifts) {
                const int u = u0 + kC4Lanes * k;
                const int delta = u < ntile ? s_shift[u] : 0;
                hi = (hi << delta) | ((lo >> 1) >> (63 - delta));
                l2 = lo << delta;
            }
            acc += (__int128)(((unsigned __int128)hi << 64) | l2);
        }
        u0 += kC4Lanes * U;
        if (u0 >= ntile) break;
        load_batch(u0, raw);
    }
#pragma unroll
    for (int o = 1; o < kC4Lanes; o <<= 1) acc += shfl_xor_i128(acc, o);
    if (active && q == 0) {
        // phi = acc 2^-Fc / D_s (see combine_fast_body)
        double x, out;
        if (i128_scaled_to_double(acc, gmax, x))
            out = x * __ldg(a.winv + s);
        else
            out = ldexp(i128_to_double(acc) * __ldg(a.winv + s), -gmax);
        reinterpret_cast<double *>(a.phi)[game * a.n_out + task] = out;
    }
}

// ----------------------------------------------------------------------------
// Fused apply of a fast-path plan: one persistent launch runs the tiles and
// the combine of all B games.  Work items come from a device counter in the
// order T(0), T(1), S(0), T(2), S(1), ..., T(B-1), S(B-2), S(B-1), where T(g)
// are the tiles of game g (tiles_per_item at a time) and S(g) its score
// chunks, so the combine of a game runs beside the tiles of later games.  A
// score chunk waits until every tile of its game is done; those tiles were
// handed out earlier to running CTAs that never wait, so the wait ends, and
// it is bounded all the same (spin_limit polls, then kErrTimeout is latched
// and every later wait gives up at once).  A CTA that takes a tile item asks
// L2 to prefetch the input of the item one grid width ahead, which hides most
// of the HBM latency of the next tile's load.
// ----------------------------------------------------------------------------
struct ApplyArgs {
    FastArgs fa;
    CombineFastArgs ca;
    int B, n_tiles, tpi, spi, nt, ns;  // games, tiles per game, tiles / scores per item, items per game
    long long n_items;
    int *counters;                     // [0] queue head, [1 + g] finished tiles of game g
    long long spin_limit;
    int inject_missing;                // test hook: every wait expects one tile more than exists
};

struct ApplyItem {
    int tile, game, first, count;
};

__device__ __forceinline__ ApplyItem apply_item(const ApplyArgs &a, long long k) {
    ApplyItem it;
    int r;
    if (k < a.nt) {
        it.tile = 1;
        it.game = 0;
        r = (int)k;
    } else {
        const long long per = a.nt + a.ns, kk = k - a.nt, blk = kk / per;
        const int rr = (int)(kk - blk * per);
        if (blk < a.B - 1) {
            it.tile = rr < a.nt;
            it.game = it.tile ? (int)blk + 1 : (int)blk;
            r = it.tile ? rr : rr - a.nt;
        } else {
            it.tile = 0;
            it.game = a.B - 1;
            r = (int)(kk - (long long)(a.B - 1) * per);
        }
    }
    if (it.tile) {
        it.first = r * a.tpi;
        it.count = min(a.tpi, a.n_tiles - it.first);
    } else {
        it.first = r * a.spi;
        it.count = (int)min((long long)a.spi, a.ca.n_out - it.first);
    }
    return it;
}

template <typename Acc, int L>
__global__ void __launch_bounds__(kTileThreads, 2) fsi_apply_fast_kernel(ApplyArgs a) {
    using In = typename TileTraits<Acc>::In;
    __shared__ long long s_item;
    __shared__ int s_ok;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(a.counters, 1);
        __syncthreads();
        const long long item = s_item;
        __syncthreads();
        if (item >= a.n_items) break;
        const ApplyItem it = apply_item(a, item);
        if (it.tile) {
            const long long ahead = item + gridDim.x;
            if (ahead < a.n_items) {
                const ApplyItem pf = apply_item(a, ahead);
                if (pf.tile) {
                    const char *base = reinterpret_cast<const char *>(
                        reinterpret_cast<const In *>(a.fa.v) + ((long long)pf.game << a.fa.d) +
                        ((long long)pf.first << fast::kBits));
                    const long long bytes = (long long)pf.count * (a.fa.load_mask + 1) * (long long)sizeof(In);
                    for (long long o = threadIdx.x * 128ll; o < bytes; o += kTileThreads * 128ll)
                        asm volatile("prefetch.global.L2 [%0];" ::"l"(base + o));
                }
            }
            for (int t = it.first; t < it.first + it.count; ++t) {
                tile_fast_body<Acc, L>(a.fa, it.game, t);
                __syncthreads();
            }
            __threadfence();
            __syncthreads();
            if (threadIdx.x == 0) atomicAdd(a.counters + 1 + it.game, it.count);
        } else {
            if (threadIdx.x == 0) {
                int ok = 1;
                long long polls = 0;
                while (atomicAdd(a.counters + 1 + it.game, 0) < a.n_tiles + a.inject_missing) {
                    if ((atomicAdd(a.fa.err, 0) & kErrTimeout) || ++polls > a.spin_limit) {
                        atomicOr(a.fa.err, kErrTimeout);
                        ok = 0;
                        break;
                    }
                    __nanosleep(200);
                }
                __threadfence();
                s_ok = ok;
            }
            __syncthreads();
            if (s_ok) combine_fast_body<Acc>(a.ca, it.game, it.first, it.first + it.count);
            __syncthreads();
        }
    }
}

// ----------------------------------------------------------------------------
// combine
// ----------------------------------------------------------------------------

constexpr int kCombineThreads = 128;

template <typename Acc>
__global__ void __launch_bounds__(kCombineThreads) fsi_combine_kernel(CombineArgs a) {
    const long long game = a.game0 + blockIdx.y;
    const long long task = blockIdx.x;
    const int tid = threadIdx.x;
    const int ch_base = a.tasks[task * 4 + 0];
    const unsigned SH = (unsigned)a.tasks[task * 4 + 1];
    const int code = a.tasks[task * 4 + 2];
    const int s = code & 0xff, sL = (code >> 8) & 0xff, sH = (code >> 16) & 0xff;
    const int ntile = 1 << a.h;
    const int J = a.mob_only ? 1 : (a.b - sL + 1);
    const int P1 = a.h + 1, Q1 = a.b + 1;
    const Acc *Yg = reinterpret_cast<const Acc *>(a.Y) + (game << a.h) * (long long)a.n_ch;

    if constexpr (TileTraits<Acc>::exact) {
        __shared__ int s_fmin, s_fmax;
        __shared__ __int128 red[kCombineThreads];
        const int *texp = a.tile_exp + (game << a.h);
        int fmin = 0x7fffffff, fmax = -0x7fffffff;
        for (int u = tid; u < ntile; u += kCombineThreads) {
            int f = texp[u];
            fmin = min(fmin, f);
            fmax = max(fmax, f);
        }
        if (tid == 0) {
            s_fmin = 0x7fffffff;
            s_fmax = -0x7fffffff;
        }
        __syncthreads();
        atomicMin(&s_fmin, fmin);
        atomicMax(&s_fmax, fmax);
        __syncthreads();
        const int Fc = min(s_fmax, s_fmin + a.shift_cap);
        const long long den = a.wden[s];
        const long long *wrow = a.wnum + (long long)s * P1 * Q1;
        __int128 acc = 0;
        for (int u = tid; u < ntile; u += kCombineThreads) {
            const int i = __popc((unsigned)u & SH);
            const int m = __popc((unsigned)u & ~SH);
            const int p = sH + m;
            const long long *y = Yg + (long long)u * a.n_ch + ch_base;
            const long long *w = wrow + (long long)p * Q1 + sL;
            __int128 inner = 0;
            for (int j = 0; j < J; ++j) {
                long long c = w[j] + ((m == 0 && j == 0) ? den : 0ll);
                inner += (__int128)y[j] * (__int128)c;
            }
            const int delta = Fc - texp[u];
            if (delta >= 0) {
                inner = (__int128)((unsigned __int128)inner << delta);
            } else {
                const int r = -delta;
                inner = (r >= 127) ? (__int128)0 : ((inner + ((__int128)1 << (r - 1))) >> r);
            }
            if ((sH - i) & 1) inner = -inner;
            acc += inner;
        }
        red[tid] = acc;
        __syncthreads();
        for (int o = kCombineThreads / 2; o > 0; o >>= 1) {
            if (tid < o) red[tid] += red[tid + o];
            __syncthreads();
        }
        if (tid == 0) {
            // as in the fast combine: acc 2^-Fc rounded with integer
            // instructions, then one product with 1 / D_s
            double x, out;
            if (i128_scaled_to_double(red[0], Fc, x))
                out = x * a.winv[s];
            else
                out = ldexp(i128_to_double(red[0]) * a.winv[s], -Fc);
            reinterpret_cast<double *>(a.phi)[game * a.n_out + task] = out;
        }
    } else {
        __shared__ Acc red[kCombineThreads];
        const bool f32 = sizeof(Acc) == 4;
        Acc acc = 0;
        for (int u = tid; u < ntile; u += kCombineThreads) {
            const int i = __popc((unsigned)u & SH);
            const int m = __popc((unsigned)u & ~SH);
            const int p = sH + m;
            const Acc *y = Yg + (long long)u * a.n_ch + ch_base;
            const long long wo = ((long long)s * P1 + p) * Q1 + sL;
            Acc inner = 0;
            for (int j = 0; j < J; ++j) {
                Acc c = f32 ? (Acc)a.wf32[wo + j] : (Acc)a.wf64[wo + j];
                if (m == 0 && j == 0) c += (Acc)1;
                inner += y[j] * c;
            }
            acc += ((sH - i) & 1) ? -inner : inner;
        }
        red[tid] = acc;
        __syncthreads();
        for (int o = kCombineThreads / 2; o > 0; o >>= 1) {
            if (tid < o) red[tid] += red[tid + o];
            __syncthreads();
        }
        if (tid == 0) reinterpret_cast<Acc *>(a.phi)[game * a.n_out + task] = red[0];
    }
}

// ----------------------------------------------------------------------------
// host side
// ----------------------------------------------------------------------------
namespace {

thread_local cudaError_t g_last_cuda_error = cudaSuccess;

tt_fsi_status cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return TT_FSI_OK;
    g_last_cuda_error = e;
    if (e == cudaErrorMemoryAllocation) return TT_FSI_ERR_NO_MEMORY;
    return TT_FSI_ERR_CUDA;
}

// Raises a kernel's dynamic shared-memory cap to the device's opt-in maximum.
// The cap is per kernel, not per plan, so it must never be lowered by a plan
// that needs less than another plan created earlier.
template <typename K>
cudaError_t allow_max_smem(K *kernel) {
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - 1024);
    return e;
}

// Every device-side table of a plan, so that plan creation and the
// allocation-free entry point place the same set.
struct TableRef {
    void **dev;
    const void *host;
    size_t bytes;
};

constexpr int kPlanTables = 9;

std::array<TableRef, kPlanTables> plan_tables(Plan &p) {
    return {{
        {(void **)&p.d_trans, p.trans.data(), p.trans.size() * sizeof(int32_t)},
        {(void **)&p.d_tasks, p.tasks.data(), p.tasks.size() * sizeof(int32_t)},
        {(void **)&p.d_wnum, p.wnum.data(), p.wnum.size() * sizeof(long long)},
        {(void **)&p.d_wden, p.wden.data(), p.wden.size() * sizeof(long long)},
        {(void **)&p.d_wf64, p.wf64.data(), p.wf64.size() * sizeof(double)},
        {(void **)&p.d_wf32, p.wf32.data(), p.wf32.size() * sizeof(float)},
        {(void **)&p.d_gtab, p.gtab.data(), p.gtab.size() * sizeof(int32_t)},
        {(void **)&p.d_wstage, p.wstage.data(), p.wstage.size()},
        {(void **)&p.d_winv, p.winv.data(), p.winv.size() * sizeof(double)},
    }};
}

// Bytes of per-tile output one game needs: partial scores on the fast path
// (int128 on the exact path), channels otherwise.
size_t tile_out_bytes_per_game(const Plan &p) {
    const size_t ntile = (size_t)1 << p.h;
    if (p.fast12) {
        const size_t g = p.arith == TT_FSI_ARITH_EXACT ? 16 : (p.arith == TT_FSI_ARITH_F64 ? 8 : 4);
        return ntile * (size_t)p.n_g * g;
    }
    const size_t e = (p.arith == TT_FSI_ARITH_F32) ? 4 : 8;
    return ntile * (size_t)p.n_ch * e;
}

void free_plan_device(Plan *p) {
    cudaFree(p->d_trans);
    cudaFree(p->d_tasks);
    cudaFree(p->d_wnum);
    cudaFree(p->d_wden);
    cudaFree(p->d_wf64);
    cudaFree(p->d_wf32);
    cudaFree(p->d_Y);
    cudaFree(p->d_exp);
    cudaFree(p->d_err);
    cudaFree(p->d_gtab);
    cudaFree(p->d_wstage);
    cudaFree(p->d_winv);
    cudaFree(p->d_counters);
}

// Kernel arguments of a fast-path plan that do not depend on the call.
FastArgs fast_args(const Plan &p) {
    FastArgs fa{};
    fa.gtab = p.d_gtab;
    fa.n_g = p.n_g;
    fa.d = p.d;
    fa.h = p.h;
    fa.ell = p.ell_eff;
    fa.prec_bits = p.prec_bits;
    fa.load_mask = (1 << p.load_bits) - 1;
    fa.g_split31 = p.g_split31 ? 1 : 0;
    fa.wstage = p.d_wstage;
    fa.wstage_block = p.wstage_block;
    return fa;
}

// Kernel arguments of the fast combine that do not depend on the call.
CombineFastArgs combine_fast_args(const Plan &p) {
    CombineFastArgs cf{};
    cf.G = p.d_Y;
    cf.tile_exp = p.d_exp;
    cf.tasks = p.d_tasks;
    cf.wden = p.d_wden;
    cf.winv = p.d_winv;
    cf.h = p.h;
    cf.n_g = p.n_g;
    cf.shift_cap = p.shift_cap;
    cf.n_out = p.n_out;
    return cf;
}

// Raises the shared-memory cap of every order's fast tile and fused kernels.
template <typename Acc>
cudaError_t allow_max_smem_fast() {
    cudaError_t e = allow_max_smem(fsi_tile_fast_kernel<Acc, 1>);
    if (e == cudaSuccess) e = allow_max_smem(fsi_tile_fast_kernel<Acc, 2>);
    if (e == cudaSuccess) e = allow_max_smem(fsi_tile_fast_kernel<Acc, 3>);
    if (e == cudaSuccess) e = allow_max_smem(fsi_tile_fast_kernel<Acc, 4>);
    if (e == cudaSuccess) e = allow_max_smem(fsi_apply_fast_kernel<Acc, 1>);
    if (e == cudaSuccess) e = allow_max_smem(fsi_apply_fast_kernel<Acc, 2>);
    if (e == cudaSuccess) e = allow_max_smem(fsi_apply_fast_kernel<Acc, 3>);
    if (e == cudaSuccess) e = allow_max_smem(fsi_apply_fast_kernel<Acc, 4>);
    return e;
}

// Persistent grid of the fused kernel: SMs x resident CTAs per SM.
template <typename Acc>
cudaError_t fused_grid(const Plan &p, int *grid) {
    int dev = 0, sms = 0, occ = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    switch (p.ell_eff) {
        case 1: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fsi_apply_fast_kernel<Acc, 1>, kTileThreads, p.smem_fast); break;
        case 2: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fsi_apply_fast_kernel<Acc, 2>, kTileThreads, p.smem_fast); break;
        case 3: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fsi_apply_fast_kernel<Acc, 3>, kTileThreads, p.smem_fast); break;
        default: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fsi_apply_fast_kernel<Acc, 4>, kTileThreads, p.smem_fast); break;
    }
    *grid = std::max(1, occ) * sms;
    return e;
}

// Launches a combine kernel as the programmatic dependent of the tile
// launch just before it on `st`: its CTAs may be placed while the tile grid
// drains, and each waits in the kernel (griddepcontrol.wait) for the tile
// grid's results before reading them.
template <typename Args>
cudaError_t launch_dependent(void (*kernel)(Args), dim3 grid, dim3 block, cudaStream_t st, const Args &args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args);
}

template <typename Acc>
tt_fsi_status launch_apply(const Plan &p, const void *v, int64_t B, void *phi, cudaStream_t st,
                           cudaEvent_t ev0 = nullptr, cudaEvent_t ev1 = nullptr,
                           cudaEvent_t ev2 = nullptr) {
    // every table a kernel of this plan will read must be in place
    const bool exact = TileTraits<Acc>::exact;
    if (!p.d_tasks || !p.d_Y || !p.d_err || (p.fast12 && !p.d_gtab) || (p.fast12 && (p.wstage_block <= 0 || !p.d_wstage)) ||
        (!p.mob_only && !p.fast12 && !p.d_trans) ||
        (exact && (!p.d_wnum || !p.d_wden || !p.d_winv || !p.d_exp)) ||
        (!exact && sizeof(Acc) == 8 && !p.d_wf64) || (!exact && sizeof(Acc) == 4 && !p.d_wf32))
        return TT_FSI_ERR_INVALID_ARG;
    TileArgs ta{};
    ta.v = v;
    ta.Y = p.d_Y;
    ta.tile_exp = p.d_exp;
    ta.err = p.d_err;
    ta.trans = p.d_trans;
    ta.d = p.d;
    ta.b = p.b;
    ta.h = p.h;
    ta.n_ch = p.n_ch;
    ta.buf_elems = p.buf_elems;
    ta.prec_bits = p.prec_bits;
    ta.mob_only = p.mob_only ? 1 : 0;
    for (int k = 0; k < kMaxLevels; ++k) {
        ta.n_states[k] = p.n_states[k];
        ta.lvl_off[k] = p.lvl_off[k];
    }
    CombineArgs ca{};
    ca.Y = p.d_Y;
    ca.tile_exp = p.d_exp;
    ca.tasks = p.d_tasks;
    ca.wnum = p.d_wnum;
    ca.wden = p.d_wden;
    ca.winv = p.d_winv;
    ca.wf64 = p.d_wf64;
    ca.wf32 = p.d_wf32;
    ca.phi = phi;
    ca.b = p.b;
    ca.h = p.h;
    ca.n_ch = p.n_ch;
    ca.shift_cap = p.shift_cap;
    ca.mob_only = ta.mob_only;
    ca.n_out = p.n_out;
    if (p.fast12 && p.fused) {
        if (!p.d_counters || p.apply_grid < 1) return TT_FSI_ERR_INVALID_ARG;
        ApplyArgs aa{};
        aa.fa = fast_args(p);
        aa.fa.v = v;
        aa.fa.G = p.d_Y;
        aa.fa.tile_exp = p.d_exp;
        aa.fa.err = p.d_err;
        aa.ca = combine_fast_args(p);
        aa.ca.phi = phi;
        aa.B = (int)B;
        aa.n_tiles = 1 << p.h;
        aa.tpi = p.tiles_per_item;
        aa.spi = p.scores_per_item;
        aa.nt = (aa.n_tiles + aa.tpi - 1) / aa.tpi;
        aa.ns = (int)((p.n_out + aa.spi - 1) / aa.spi);
        aa.n_items = (long long)B * (aa.nt + aa.ns);
        aa.counters = p.d_counters;
        aa.spin_limit = p.spin_limit;
        aa.inject_missing = p.inject_missing ? 1 : 0;
        const unsigned grid = (unsigned)std::min<long long>(aa.n_items, p.apply_grid);
        if (ev0) cudaEventRecord(ev0, st);
        cudaError_t e = cudaMemsetAsync(p.d_counters, 0, (size_t)(B + 1) * sizeof(int), st);
        if (e != cudaSuccess) return cuda_status(e);
        switch (p.ell_eff) {
            case 1: fsi_apply_fast_kernel<Acc, 1><<<grid, kTileThreads, p.smem_fast, st>>>(aa); break;
            case 2: fsi_apply_fast_kernel<Acc, 2><<<grid, kTileThreads, p.smem_fast, st>>>(aa); break;
            case 3: fsi_apply_fast_kernel<Acc, 3><<<grid, kTileThreads, p.smem_fast, st>>>(aa); break;
            default: fsi_apply_fast_kernel<Acc, 4><<<grid, kTileThreads, p.smem_fast, st>>>(aa); break;
        }
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_status(e);
        if (ev1) cudaEventRecord(ev1, st);
        if (ev2) cudaEventRecord(ev2, st);
        return TT_FSI_OK;
    }
    const int64_t chunk = 65535;
    for (int64_t g0 = 0; g0 < B; g0 += chunk) {
        const int nb = (int)((B - g0 < chunk) ? (B - g0) : chunk);
        ta.game0 = g0;
        ca.game0 = g0;
        dim3 g1((unsigned)(1u << p.h), (unsigned)nb);
        if (ev0 && g0 == 0) cudaEventRecord(ev0, st);
        if (p.fast12) {
            FastArgs fa = fast_args(p);
            fa.v = v;
            fa.G = p.d_Y;
            fa.tile_exp = p.d_exp;
            fa.err = p.d_err;
            fa.game0 = g0;
            // no L2 prefetch: with three resident CTAs per SM on the exact
            // path the other CTAs hide each tile's load, and the prefetch
            // instructions cost more than they save (distances of 0.66 to 3
            // waves measured 1 to 3 % slower than none)
            fa.prefetch_ahead = 0;
            switch (p.ell_eff) {
                case 1: fsi_tile_fast_kernel<Acc, 1><<<g1, kTileThreads, p.smem_fast, st>>>(fa); break;
                case 2: fsi_tile_fast_kernel<Acc, 2><<<g1, kTileThreads, p.smem_fast, st>>>(fa); break;
                case 3: fsi_tile_fast_kernel<Acc, 3><<<g1, kTileThreads, p.smem_fast, st>>>(fa); break;
                default: fsi_tile_fast_kernel<Acc, 4><<<g1, kTileThreads, p.smem_fast, st>>>(fa); break;
            }
        } else {
            if (p.precontract)
                fsi_tile_kernel<Acc, true><<<g1, kTileThreads, p.smem_tile, st>>>(ta);
            else
                fsi_tile_kernel<Acc><<<g1, kTileThreads, p.smem_tile, st>>>(ta);
        }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_status(e);
        if (ev1 && g0 + chunk >= B) cudaEventRecord(ev1, st);
        if (p.fast12) {
            CombineFastArgs cf{};
            cf.G = p.d_Y;
            cf.tile_exp = p.d_exp;
            cf.tasks = p.d_tasks;
            cf.wden = p.d_wden;
            cf.winv = p.d_winv;
            cf.phi = phi;
            cf.h = p.h;
            cf.n_g = p.n_g;
            cf.shift_cap = p.shift_cap;
            cf.n_out = p.n_out;
            cf.game0 = g0;
            // exact arithmetic: any summation order gives the same integers, so
            // the lane-split combine can replace the fused schedule's routine;
            // the float paths keep that routine's order (bitwise equal to the
            // fused schedule)
            if constexpr (TileTraits<Acc>::exact) {
                if (p.h <= 12) {
                    dim3 g2((unsigned)((p.n_out + kC4Scores - 1) / kC4Scores), (unsigned)nb);
                    cudaError_t le = launch_dependent(fsi_combine_split_kernel<Acc>, g2, dim3(32 * kC4Warps), st, cf);
                    if (le != cudaSuccess) return cuda_status(le);
                } else {
                    dim3 g2((unsigned)((p.n_out + kCombineFastWarps - 1) / kCombineFastWarps), (unsigned)nb);
                    cudaError_t le = launch_dependent(fsi_combine_fast_kernel<Acc>, g2, dim3(32 * kCombineFastWarps), st, cf);
                    if (le != cudaSuccess) return cuda_status(le);
                }
            } else {
                dim3 g2((unsigned)((p.n_out + kCombineFastWarps - 1) / kCombineFastWarps), (unsigned)nb);
                cudaError_t le = launch_dependent(fsi_combine_fast_kernel<Acc>, g2, dim3(32 * kCombineFastWarps), st, cf);
                if (le != cudaSuccess) return cuda_status(le);
            }
        } else {
            dim3 g2((unsigned)p.n_out, (unsigned)nb);
            fsi_combine_kernel<Acc><<<g2, kCombineThreads, 0, st>>>(ca);
        }
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_status(e);
    }
    if (ev2) cudaEventRecord(ev2, st);
    return TT_FSI_OK;
}

}  // namespace
}  // namespace ttfsi

using namespace ttfsi;

struct tt_fsi_plan_s {
    Plan p;
    // tracing: events recorded around each kernel while profiling is on
    bool profiling = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::array<cudaEvent_t, 3>> ev_rec;
    // staging for tt_fsi_apply_host: device buffers, the copy stream that
    // fills them chunk by chunk, and the games per chunk (0: automatic)
    void *d_v_stage = nullptr;
    void *d_phi_stage = nullptr;
    cudaStream_t s_copy = nullptr;
    cudaEvent_t ev_copy = nullptr;
    int64_t host_chunk = 0;
    // tt_fsi_apply_host on page-locked input: the tile kernel reads the host
    // buffer in place (one pass over the host link) instead of a staged copy
    bool host_zero_copy = true;
};

namespace {
cudaEvent_t pool_event(tt_fsi_plan_s *h) {
    if (!h->ev_pool.empty()) {
        cudaEvent_t e = h->ev_pool.back();
        h->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}
}  // namespace

extern "C" {

int64_t tt_fsi_num_scores(int d, int ell) { return ttfsi::num_scores(d, ell); }

tt_fsi_status tt_fsi_score_masks(int d, int ell, uint64_t *masks_host) {
    if (!masks_host || ttfsi::num_scores(d, ell) < 0) return TT_FSI_ERR_INVALID_ARG;
    ttfsi::score_masks(d, ell, masks_host);
    return TT_FSI_OK;
}

tt_fsi_status tt_fsi_plan_create(int d, int ell, tt_fsi_arith arith, int64_t max_batch,
                                 tt_fsi_plan *out) {
    return tt_fsi_plan_create_index(d, ell, TT_FSI_INDEX_FSI, arith, max_batch, out);
}

tt_fsi_status tt_fsi_plan_create_index(int d, int ell, tt_fsi_index index, tt_fsi_arith arith,
                                       int64_t max_batch, tt_fsi_plan *out) {
    return tt_fsi_plan_create_ex(d, ell, index, arith, max_batch, 0u, out);
}

tt_fsi_status tt_fsi_plan_create_ex(int d, int ell, tt_fsi_index index, tt_fsi_arith arith, int64_t max_batch,
                                    unsigned flags, tt_fsi_plan *out) {
    if (!out || (flags & ~(unsigned)(TT_FSI_PLAN_SITE_SWEEP | TT_FSI_PLAN_PRECONTRACT))) return TT_FSI_ERR_INVALID_ARG;
    *out = nullptr;
    tt_fsi_plan_s *h = new (std::nothrow) tt_fsi_plan_s();
    if (!h) return TT_FSI_ERR_NO_MEMORY;
    Plan &p = h->p;
    tt_fsi_status st = plan_build_host(p, d, ell, arith, max_batch, index, (flags & TT_FSI_PLAN_SITE_SWEEP) != 0,
                                       (flags & TT_FSI_PLAN_PRECONTRACT) != 0);
    if (st != TT_FSI_OK) {
        delete h;
        return st;
    }
    const size_t elem = (arith == TT_FSI_ARITH_F32) ? 4 : 8;
    const size_t ntile = (size_t)1 << p.h;
    p.scratch_bytes = (size_t)max_batch * tile_out_bytes_per_game(p);
    if (arith == TT_FSI_ARITH_EXACT) p.scratch_bytes += (size_t)max_batch * ntile * sizeof(int);
    do {
        for (const TableRef &t : plan_tables(p)) {
            *t.dev = nullptr;
            if (!t.bytes) continue;
            cudaError_t e = cudaMalloc(t.dev, t.bytes);
            if (e == cudaSuccess) e = cudaMemcpy(*t.dev, t.host, t.bytes, cudaMemcpyHostToDevice);
            if (e != cudaSuccess) {
                st = cuda_status(e);
                break;
            }
        }
        if (st != TT_FSI_OK) break;
        cudaError_t e = cudaMalloc(&p.d_Y, (size_t)max_batch * tile_out_bytes_per_game(p));
        if (e != cudaSuccess) {
            st = cuda_status(e);
            break;
        }
        e = cudaMalloc((void **)&p.d_exp, (size_t)max_batch * ntile * sizeof(int));
        if (e != cudaSuccess) {
            st = cuda_status(e);
            break;
        }
        e = cudaMalloc((void **)&p.d_err, sizeof(int));
        if (e == cudaSuccess) e = cudaMemset(p.d_err, 0, sizeof(int));
        if (e != cudaSuccess) {
            st = cuda_status(e);
            break;
        }
        const int smem = (int)p.smem_tile;
        if (arith == TT_FSI_ARITH_EXACT) {
            e = allow_max_smem(fsi_tile_kernel<long long>);
            if (e == cudaSuccess) e = allow_max_smem(fsi_tile_kernel<long long, true>);
        } else if (arith == TT_FSI_ARITH_F64) {
            e = allow_max_smem(fsi_tile_kernel<double>);
            if (e == cudaSuccess) e = allow_max_smem(fsi_tile_kernel<double, true>);
        } else {
            e = allow_max_smem(fsi_tile_kernel<float>);
            if (e == cudaSuccess) e = allow_max_smem(fsi_tile_kernel<float, true>);
        }
        if (e != cudaSuccess) {
            st = cuda_status(e);
            break;
        }
        if (p.fast12) {
            if (arith == TT_FSI_ARITH_EXACT)
                e = allow_max_smem_fast<long long>();
            else if (arith == TT_FSI_ARITH_F64)
                e = allow_max_smem_fast<double>();
            else
                e = allow_max_smem_fast<float>();
            if (e == cudaSuccess) {
                if (arith == TT_FSI_ARITH_EXACT)
                    e = fused_grid<long long>(p, &p.apply_grid);
                else if (arith == TT_FSI_ARITH_F64)
                    e = fused_grid<double>(p, &p.apply_grid);
                else
                    e = fused_grid<float>(p, &p.apply_grid);
            }
            if (e == cudaSuccess) e = cudaMalloc((void **)&p.d_counters, (size_t)(max_batch + 1) * sizeof(int));
            if (e != cudaSuccess) {
                st = cuda_status(e);
                break;
            }
        }
        st = TT_FSI_OK;
    } while (0);
    if (st != TT_FSI_OK) {
        free_plan_device(&p);
        delete h;
        return st;
    }
    *out = h;
    return TT_FSI_OK;
}

void tt_fsi_plan_destroy(tt_fsi_plan plan) {
    if (!plan) return;
    cudaDeviceSynchronize();
    free_plan_device(&plan->p);
    cudaFree(plan->d_v_stage);
    cudaFree(plan->d_phi_stage);
    if (plan->ev_copy) cudaEventDestroy(plan->ev_copy);
    if (plan->s_copy) cudaStreamDestroy(plan->s_copy);
    for (auto &r : plan->ev_rec)
        for (cudaEvent_t ev : r) cudaEventDestroy(ev);
    for (cudaEvent_t ev : plan->ev_pool) cudaEventDestroy(ev);
    delete plan;
}

size_t tt_fsi_plan_scratch_bytes(tt_fsi_plan plan) { return plan ? plan->p.scratch_bytes : 0; }

int tt_fsi_plan_tile_bits(tt_fsi_plan plan) { return plan ? plan->p.b : -1; }

tt_fsi_status tt_fsi_apply(tt_fsi_plan plan, const void *v_dev, int64_t B, void *phi_dev,
                           struct CUstream_st *stream) {
    if (!plan || B < 0) return TT_FSI_ERR_INVALID_ARG;
    if (B == 0) return TT_FSI_OK;
    if (!v_dev || !phi_dev || B > plan->p.max_batch) return TT_FSI_ERR_INVALID_ARG;
    const Plan &p = plan->p;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaEvent_t e0 = nullptr, e1 = nullptr, e2 = nullptr;
    if (plan->profiling) {
        e0 = pool_event(plan);
        e1 = pool_event(plan);
        e2 = pool_event(plan);
        if (!e0 || !e1 || !e2) return TT_FSI_ERR_CUDA;
        plan->ev_rec.push_back({e0, e1, e2});
    }
    switch (p.arith) {
        case TT_FSI_ARITH_EXACT: return launch_apply<long long>(p, v_dev, B, phi_dev, st, e0, e1, e2);
        case TT_FSI_ARITH_F64: return launch_apply<double>(p, v_dev, B, phi_dev, st, e0, e1, e2);
        case TT_FSI_ARITH_F32: return launch_apply<float>(p, v_dev, B, phi_dev, st, e0, e1, e2);
    }
    return TT_FSI_ERR_INVALID_ARG;
}

tt_fsi_status tt_fsi_apply_host(tt_fsi_plan plan, const void *v_host, int64_t B, void *phi_host,
                                struct CUstream_st *stream) {
    if (!plan || B < 0) return TT_FSI_ERR_INVALID_ARG;
    if (B == 0) return TT_FSI_OK;
    if (!v_host || !phi_host || B > plan->p.max_batch) return TT_FSI_ERR_INVALID_ARG;
    const Plan &p = plan->p;
    const size_t elem = (p.arith == TT_FSI_ARITH_F32) ? 4 : 8;
    const size_t vbytes = ((size_t)1 << p.d) * elem, obytes = (size_t)p.n_out * elem;
    // Page-locked input: the tile kernel streams it from host memory itself.
    // It reads every input value exactly once, so the host link carries the
    // same bytes as a copy would, in one pass and without a staging buffer.
    const void *v_mapped = nullptr;
    if (plan->host_zero_copy) {
        cudaPointerAttributes at{};
        if (cudaPointerGetAttributes(&at, v_host) == cudaSuccess && at.type == cudaMemoryTypeHost &&
            at.devicePointer != nullptr)
            v_mapped = at.devicePointer;
        else
            cudaGetLastError();  // pageable memory: not an error, take the staged copies
    }
    if (!plan->d_v_stage) {
        cudaError_t e = cudaMalloc(&plan->d_v_stage, vbytes * (size_t)p.max_batch);
        if (e == cudaSuccess) e = cudaMalloc(&plan->d_phi_stage, obytes * (size_t)p.max_batch);
        if (e != cudaSuccess) {
            cudaFree(plan->d_v_stage);
            cudaFree(plan->d_phi_stage);
            plan->d_v_stage = plan->d_phi_stage = nullptr;
            return cuda_status(e);
        }
    }
    if (!plan->s_copy) {
        cudaError_t e = cudaStreamCreateWithFlags(&plan->s_copy, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&plan->ev_copy, cudaEventDisableTiming);
        if (e != cudaSuccess) {
            if (plan->s_copy) cudaStreamDestroy(plan->s_copy);
            plan->s_copy = nullptr;
            return cuda_status(e);
        }
    }
    cudaStream_t st0 = reinterpret_cast<cudaStream_t>(stream);
    if (v_mapped) {
        tt_fsi_status s = tt_fsi_apply(plan, v_mapped, B, plan->d_phi_stage, stream);
        if (s != TT_FSI_OK) return s;
        cudaError_t e = cudaMemcpyAsync(phi_host, plan->d_phi_stage, obytes * (size_t)B, cudaMemcpyDeviceToHost, st0);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st0);
        return cuda_status(e);
    }
    // Games per chunk: explicit, or chunks of at least 16 MiB and at most 16
    // chunks.  The copy stream moves chunk k + 1 while `stream` computes
    // chunk k, so only the last chunk's compute is added to the transfer.
    // (d = 20, 16 games: 8 MiB chunks 2.29e10 coalitions/s, 16 MiB 2.34e10.)
    int64_t chunk = plan->host_chunk;
    if (chunk <= 0) {
        const int64_t min_games = (int64_t)(((size_t)16 << 20) + vbytes - 1) / (int64_t)vbytes;
        chunk = std::max(min_games, (B + 15) / 16);
    }
    chunk = std::min(std::max<int64_t>(chunk, 1), B);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    // the staging buffer may still be read by earlier work on `stream`
    cudaError_t e = cudaEventRecord(plan->ev_copy, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(plan->s_copy, plan->ev_copy, 0);
    if (e != cudaSuccess) return cuda_status(e);
    const char *src = static_cast<const char *>(v_host);
    char *stage = static_cast<char *>(plan->d_v_stage);
    char *phi_stage = static_cast<char *>(plan->d_phi_stage);
    for (int64_t g0 = 0; g0 < B; g0 += chunk) {
        const int64_t nb = std::min(chunk, B - g0);
        e = cudaMemcpyAsync(stage + (size_t)g0 * vbytes, src + (size_t)g0 * vbytes, (size_t)nb * vbytes,
                            cudaMemcpyHostToDevice, plan->s_copy);
        // a wait takes the event's most recent record, so one event serves all chunks
        if (e == cudaSuccess) e = cudaEventRecord(plan->ev_copy, plan->s_copy);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, plan->ev_copy, 0);
        if (e != cudaSuccess) return cuda_status(e);
        tt_fsi_status s = tt_fsi_apply(plan, stage + (size_t)g0 * vbytes, nb, phi_stage + (size_t)g0 * obytes, stream);
        if (s != TT_FSI_OK) return s;
    }
    e = cudaMemcpyAsync(phi_host, plan->d_phi_stage, obytes * (size_t)B, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return cuda_status(e);
}

tt_fsi_status tt_fsi_plan_set_host_zero_copy(tt_fsi_plan plan, int enable) {
    if (!plan) return TT_FSI_ERR_INVALID_ARG;
    plan->host_zero_copy = enable != 0;
    return TT_FSI_OK;
}

tt_fsi_status tt_fsi_plan_set_host_chunk(tt_fsi_plan plan, int64_t games) {
    if (!plan || games < 0) return TT_FSI_ERR_INVALID_ARG;
    plan->host_chunk = games;
    return TT_FSI_OK;
}

tt_fsi_status tt_fsi_plan_profile(tt_fsi_plan plan, int enable) {
    if (!plan) return TT_FSI_ERR_INVALID_ARG;
    plan->profiling = enable != 0;
    return TT_FSI_OK;
}

tt_fsi_status tt_fsi_plan_profile_read(tt_fsi_plan plan, double *ms_tile, double *ms_combine,
                                       int64_t *n_calls) {
    if (!plan) return TT_FSI_ERR_INVALID_ARG;
    double t1 = 0.0, t2 = 0.0;
    tt_fsi_status st = TT_FSI_OK;
    for (auto &r : plan->ev_rec) {
        float a = 0.f, b = 0.f;
        cudaError_t e = cudaEventSynchronize(r[2]);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&a, r[0], r[1]);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&b, r[1], r[2]);
        if (e != cudaSuccess) st = cuda_status(e);
        t1 += a;
        t2 += b;
        for (cudaEvent_t ev : r) plan->ev_pool.push_back(ev);
    }
    if (n_calls) *n_calls = (int64_t)plan->ev_rec.size();
    plan->ev_rec.clear();
    if (ms_tile) *ms_tile = t1;
    if (ms_combine) *ms_combine = t2;
    return st;
}

tt_fsi_status tt_fsi_plan_check(tt_fsi_plan plan, struct CUstream_st *stream) {
    if (!plan) return TT_FSI_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int h_err = 0;
    cudaError_t e = cudaMemcpyAsync(&h_err, plan->p.d_err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaMemsetAsync(plan->p.d_err, 0, sizeof(int), st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_status(e);
    if (h_err & kErrTimeout) return TT_FSI_ERR_TIMEOUT;
    if (h_err & kErrNonFinite) return TT_FSI_ERR_NONFINITE;
    return TT_FSI_OK;
}

tt_fsi_status tt_fsi_plan_set_schedule(tt_fsi_plan plan, int fused, int tiles_per_item, int scores_per_item) {
    if (!plan || tiles_per_item < 1 || scores_per_item < 1) return TT_FSI_ERR_INVALID_ARG;
    plan->p.fused = fused != 0;
    plan->p.tiles_per_item = tiles_per_item;
    plan->p.scores_per_item = scores_per_item;
    return TT_FSI_OK;
}

tt_fsi_status tt_fsi_plan_set_wait_limit(tt_fsi_plan plan, long long polls, int inject_missing) {
    if (!plan || polls < 0) return TT_FSI_ERR_INVALID_ARG;
    plan->p.spin_limit = polls;
    plan->p.inject_missing = inject_missing != 0;
    return TT_FSI_OK;
}

const char *tt_fsi_last_cuda_error(void) { return cudaGetErrorString(ttfsi::g_last_cuda_error); }

const char *tt_fsi_status_string(tt_fsi_status s) {
    switch (s) {
        case TT_FSI_OK: return "ok";
        case TT_FSI_ERR_INVALID_ARG: return "invalid argument";
        case TT_FSI_ERR_UNSUPPORTED: return "unsupported";
        case TT_FSI_ERR_NO_MEMORY: return "out of memory";
        case TT_FSI_ERR_CUDA: return "CUDA error";
        case TT_FSI_ERR_TIMEOUT: return "device wait timed out";
        case TT_FSI_ERR_NONFINITE: return "non-finite input";
        case TT_FSI_ERR_CHECK_FAILED: return "self-check failed";
    }
    return "unknown status";
}

}  // extern "C"

// ----------------------------------------------------------------------------
// Allocation-free FSI (exact arithmetic) for callers that cannot allocate
// device memory.  The scratch and the plan tables live in one file-scope
// device array; nothing is allocated per call.  The array's device address is
// taken once per device with cudaGetSymbolAddress (in host code the symbol
// name only stands in for the array, it is not a device address).
// ----------------------------------------------------------------------------
#include <map>
#include <mutex>

namespace ttfsi {
namespace {

constexpr size_t kNoAllocBytes = (size_t)64 << 20;  // 64 MiB on every device that loads the library
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kNoAllocMaxDevices = 64;
std::mutex g_na_mutex;
unsigned char *g_na_base[kNoAllocMaxDevices] = {nullptr};
std::map<std::pair<int, int>, Plan> g_na_plans;  // host tables per (d, l)

// Writes NaN over every score when the tile kernel flagged a non-finite input.
__global__ void noalloc_poison_kernel(const int *fault, double *phi, long long count) {
    if (*fault == 0) return;
    const double nan = __longlong_as_double(0x7ff8000000000000ll);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x)
        phi[i] = nan;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace
}  // namespace ttfsi

extern "C" tt_fsi_status tt_fsi_apply_noalloc(int d, int ell, const double *v_dev, int64_t B,
                                              double *phi_dev, struct CUstream_st *stream) {
    using namespace ttfsi;
    if (B < 0) return TT_FSI_ERR_INVALID_ARG;
    if (num_scores(d, ell) < 0) return TT_FSI_ERR_INVALID_ARG;
    if (B == 0) return TT_FSI_OK;
    if (!v_dev || !phi_dev) return TT_FSI_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(g_na_mutex);

    // host tables for (d, l), built once
    auto key = std::make_pair(d, ell);
    auto it = g_na_plans.find(key);
    if (it == g_na_plans.end()) {
        Plan hp;
        tt_fsi_status s = plan_build_host(hp, d, ell, TT_FSI_ARITH_EXACT, 1);
        if (s != TT_FSI_OK) return s;
        it = g_na_plans.emplace(key, std::move(hp)).first;
    }
    Plan &p = it->second;  // cached host tables; device pointers are set below, under the lock

    // carve the static array: fault word, tables, tile exponents, channels
    const size_t ntile = (size_t)1 << p.h;
    size_t off = 256;
    std::array<TableRef, kPlanTables> tabs = plan_tables(p);
    size_t tab_off[kPlanTables];
    for (size_t i = 0; i < tabs.size(); ++i) {
        tab_off[i] = off;
        off = align256(off + tabs[i].bytes);
    }
    const size_t o_exp = off;
    off = align256(off + (size_t)B * ntile * sizeof(int));
    const size_t o_Y = off;
    off = align256(off + (size_t)B * tile_out_bytes_per_game(p));
    const size_t o_cnt = off;
    off = align256(off + (size_t)(B + 1) * sizeof(int));
    if (off > kNoAllocBytes) return TT_FSI_ERR_UNSUPPORTED;  // beyond the 64 MiB array

    // once per device: the array's device address (with that device current)
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return TT_FSI_ERR_CUDA;
    if (dev < 0 || dev >= kNoAllocMaxDevices) return TT_FSI_ERR_UNSUPPORTED;
    if (!g_na_base[dev]) {
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return TT_FSI_ERR_CUDA;
        if (allow_max_smem(fsi_tile_kernel<long long>) != cudaSuccess ||
            allow_max_smem_fast<long long>() != cudaSuccess)
            return TT_FSI_ERR_CUDA;
        g_na_base[dev] = static_cast<unsigned char *>(ptr);
    }
    if (p.fast12 && p.apply_grid == 0 && fused_grid<long long>(p, &p.apply_grid) != cudaSuccess)
        return TT_FSI_ERR_CUDA;
    unsigned char *base = g_na_base[dev];
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);

    // every call: clear the fault word, upload the tables, then run
    cudaError_t e = cudaMemsetAsync(base, 0, sizeof(int), st);
    for (size_t i = 0; i < tabs.size() && e == cudaSuccess; ++i) {
        *tabs[i].dev = tabs[i].bytes ? (void *)(base + tab_off[i]) : nullptr;
        if (tabs[i].bytes)
            e = cudaMemcpyAsync(base + tab_off[i], tabs[i].host, tabs[i].bytes, cudaMemcpyHostToDevice, st);
    }
    if (e != cudaSuccess) return cuda_status(e);
    p.d_err = reinterpret_cast<int *>(base);
    p.d_exp = reinterpret_cast<int *>(base + o_exp);
    p.d_Y = base + o_Y;
    p.d_counters = reinterpret_cast<int *>(base + o_cnt);
    tt_fsi_status s = launch_apply<long long>(p, v_dev, B, phi_dev, st);
    if (s != TT_FSI_OK) return s;
    noalloc_poison_kernel<<<64, 256, 0, st>>>(p.d_err, phi_dev, (long long)B * p.n_out);
    return cuda_status(cudaGetLastError());
}

// ============================================================================
// Batches of uneven games (different d and l) in one persistent launch.
//
// Work items: first the tiles of every game (largest games first, a few
// consecutive tiles per item), then the score chunks of every game.  One CTA
// per SM pulls items from a device counter.  A score chunk of game g needs
// every tile of g: its CTA waits on g's finished-tile counter with a bounded
// number of polls; every tile it waits for was handed out earlier to a CTA
// that is running and never waits itself, so the wait ends unless something
// is broken -- then the kernel records TT_FSI_ERR_TIMEOUT and the remaining
// waits give up at once.
// ============================================================================
#include <memory>

namespace ttfsi {
namespace {

struct BatchGameDev {
    long long v_off, phi_off, g_off, exp_off;  // element offsets into v, phi, partial scores, exponents
    int plan, n_tiles;
};

struct BatchItem {
    int game, first, count;  // tiles [first, first + count) or scores [first, first + count)
};

struct BatchArgs {
    const void *v;
    void *phi;
    void *G;
    int *tile_exp;
    int *err;
    const FastArgs *fplans;
    const CombineFastArgs *cplans;
    const BatchGameDev *games;
    const BatchItem *items;
    int n_tile_items, n_items;
    int *head;
    int *done;
    long long spin_limit;
    int inject_missing;  // test hook: every wait expects one tile more than exists
};

template <typename Acc>
__global__ void __launch_bounds__(kTileThreads, 2) fsi_batch_kernel(BatchArgs a) {
    using GT = typename GTraits<Acc>::G;
    using In = typename TileTraits<Acc>::In;
    using Out = typename std::conditional<sizeof(Acc) == 4, float, double>::type;
    __shared__ int s_item, s_ok;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(a.head, 1);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= a.n_items) break;
        const BatchItem it = a.items[item];
        const BatchGameDev g = a.games[it.game];
        if (item < a.n_tile_items) {
            FastArgs fa = a.fplans[g.plan];
            fa.v = reinterpret_cast<const In *>(a.v) + g.v_off;
            fa.G = reinterpret_cast<GT *>(a.G) + g.g_off;
            fa.tile_exp = a.tile_exp + g.exp_off;
            fa.err = a.err;
            for (int t = it.first; t < it.first + it.count; ++t) {
                tile_fast_dispatch<Acc>(fa, 0, t);
                __syncthreads();
            }
            __threadfence();
            __syncthreads();
            if (threadIdx.x == 0) atomicAdd(a.done + it.game, it.count);
        } else {
            if (threadIdx.x == 0) {
                const int need = g.n_tiles + (a.inject_missing ? 1 : 0);
                int ok = 1;
                long long polls = 0;
                while (atomicAdd(a.done + it.game, 0) < need) {
                    if ((atomicAdd(a.err, 0) & kErrTimeout) || ++polls > a.spin_limit) {
                        atomicOr(a.err, kErrTimeout);
                        ok = 0;
                        break;
                    }
                    __nanosleep(200);
                }
                __threadfence();
                s_ok = ok;
            }
            __syncthreads();
            if (s_ok) {
                CombineFastArgs ca = a.cplans[g.plan];
                ca.G = reinterpret_cast<GT *>(a.G) + g.g_off;
                ca.tile_exp = a.tile_exp + g.exp_off;
                ca.phi = reinterpret_cast<Out *>(a.phi) + g.phi_off;
                combine_fast_body<Acc>(ca, 0, it.first, it.first + it.count);
            }
            __syncthreads();
        }
    }
}

}  // namespace
}  // namespace ttfsi

struct tt_fsi_batch_s {
    tt_fsi_arith arith = TT_FSI_ARITH_EXACT;
    std::vector<tt_fsi_game> games;
    std::vector<tt_fsi_plan> plans;                // one per distinct (d, l)
    std::vector<int> plan_of_game;
    std::vector<ttfsi::BatchGameDev> hgames;
    std::vector<int> fast_games, slow_games;
    int tiles_per_item = 1, scores_per_item = 64;
    int n_tile_items = 0, n_items = 0;
    ttfsi::FastArgs *d_fplans = nullptr;
    ttfsi::CombineFastArgs *d_cplans = nullptr;
    ttfsi::BatchGameDev *d_games = nullptr;
    ttfsi::BatchItem *d_items = nullptr;
    int *d_counters = nullptr;  // [0] queue head, [1 + g] finished tiles of game g
    int *d_err = nullptr;
    void *d_G = nullptr;
    int *d_exp = nullptr;
    size_t smem = 0;
    int grid = 0;
    long long spin_limit = 4000000;
    int inject_missing = 0;
    cudaGraphExec_t graph = nullptr;
    cudaGraph_t graph_def = nullptr;
    const void *graph_v = nullptr;
    void *graph_phi = nullptr;
};

namespace ttfsi {
namespace {

size_t in_elem(tt_fsi_arith a) { return a == TT_FSI_ARITH_F32 ? 4 : 8; }
size_t g_elem(tt_fsi_arith a) { return a == TT_FSI_ARITH_EXACT ? 16 : (a == TT_FSI_ARITH_F64 ? 8 : 4); }

// Builds the work list for the current item sizes and uploads it.
tt_fsi_status batch_build_items(tt_fsi_batch_s *b) {
    std::vector<int> order = b->fast_games;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        return b->hgames[x].n_tiles > b->hgames[y].n_tiles;
    });
    std::vector<BatchItem> items;
    for (int g : order)
        for (int t = 0; t < b->hgames[g].n_tiles; t += b->tiles_per_item)
            items.push_back({g, t, std::min(b->tiles_per_item, b->hgames[g].n_tiles - t)});
    b->n_tile_items = (int)items.size();
    for (int g : order) {
        const int64_t n_out = b->plans[b->plan_of_game[g]]->p.n_out;
        for (int64_t t = 0; t < n_out; t += b->scores_per_item)
            items.push_back({g, (int)t, (int)std::min<int64_t>(b->scores_per_item, n_out - t)});
    }
    b->n_items = (int)items.size();
    cudaFree(b->d_items);
    b->d_items = nullptr;
    if (items.empty()) return TT_FSI_OK;
    cudaError_t e = cudaMalloc((void **)&b->d_items, items.size() * sizeof(BatchItem));
    if (e == cudaSuccess)
        e = cudaMemcpy(b->d_items, items.data(), items.size() * sizeof(BatchItem), cudaMemcpyHostToDevice);
    return cuda_status(e);
}

void batch_free(tt_fsi_batch_s *b) {
    if (b->graph) cudaGraphExecDestroy(b->graph);
    if (b->graph_def) cudaGraphDestroy(b->graph_def);
    cudaFree(b->d_fplans);
    cudaFree(b->d_cplans);
    cudaFree(b->d_games);
    cudaFree(b->d_items);
    cudaFree(b->d_counters);
    cudaFree(b->d_err);
    cudaFree(b->d_G);
    cudaFree(b->d_exp);
    for (tt_fsi_plan p : b->plans) tt_fsi_plan_destroy(p);
}

template <typename Acc>
tt_fsi_status batch_launch(tt_fsi_batch_s *b, const void *v, void *phi, cudaStream_t st) {
    if (b->n_items > 0) {
        const size_t nc = 1 + b->games.size();
        cudaError_t e = cudaMemsetAsync(b->d_counters, 0, nc * sizeof(int), st);
        if (e != cudaSuccess) return cuda_status(e);
        BatchArgs a{};
        a.v = v;
        a.phi = phi;
        a.G = b->d_G;
        a.tile_exp = b->d_exp;
        a.err = b->d_err;
        a.fplans = b->d_fplans;
        a.cplans = b->d_cplans;
        a.games = b->d_games;
        a.items = b->d_items;
        a.n_tile_items = b->n_tile_items;
        a.n_items = b->n_items;
        a.head = b->d_counters;
        a.done = b->d_counters + 1;
        a.spin_limit = b->spin_limit;
        a.inject_missing = b->inject_missing;
        fsi_batch_kernel<Acc><<<b->grid, kTileThreads, b->smem, st>>>(a);
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_status(e);
    }
    // games outside the fast path (l > 3 or l >= d): one plan call each
    const size_t ie = in_elem(b->arith);
    for (int g : b->slow_games) {
        const tt_fsi_game &gm = b->games[g];
        tt_fsi_status s = tt_fsi_apply(b->plans[b->plan_of_game[g]], (const char *)v + gm.v_offset * ie, 1,
                                       (char *)phi + gm.phi_offset * ie, reinterpret_cast<CUstream_st *>(st));
        if (s != TT_FSI_OK) return s;
    }
    return TT_FSI_OK;
}

}  // namespace
}  // namespace ttfsi

extern "C" {

tt_fsi_status tt_fsi_batch_create(const tt_fsi_game *games_host, int64_t n_games, tt_fsi_arith arith,
                                  tt_fsi_batch *out) {
    return tt_fsi_batch_create_index(games_host, n_games, arith, TT_FSI_INDEX_FSI, out);
}

tt_fsi_status tt_fsi_batch_create_index(const tt_fsi_game *games_host, int64_t n_games, tt_fsi_arith arith,
                                        tt_fsi_index index, tt_fsi_batch *out) {
    using namespace ttfsi;
    if (!out || n_games < 0 || (n_games > 0 && !games_host)) return TT_FSI_ERR_INVALID_ARG;
    if (arith != TT_FSI_ARITH_EXACT && arith != TT_FSI_ARITH_F64 && arith != TT_FSI_ARITH_F32)
        return TT_FSI_ERR_INVALID_ARG;
    *out = nullptr;
    std::unique_ptr<tt_fsi_batch_s> b(new (std::nothrow) tt_fsi_batch_s());
    if (!b) return TT_FSI_ERR_NO_MEMORY;
    b->arith = arith;
    b->games.assign(games_host, games_host + n_games);
    std::map<std::pair<int, int>, int> plan_idx;
    tt_fsi_status st = TT_FSI_OK;
    for (int64_t g = 0; g < n_games && st == TT_FSI_OK; ++g) {
        const tt_fsi_game &gm = b->games[g];
        if (gm.d < 1 || gm.d > 30 || gm.ell < 1 || gm.v_offset < 0 || gm.phi_offset < 0) {
            st = TT_FSI_ERR_INVALID_ARG;
            break;
        }
        auto key = std::make_pair(gm.d, gm.ell);
        auto it = plan_idx.find(key);
        if (it == plan_idx.end()) {
            tt_fsi_plan p = nullptr;
            st = tt_fsi_plan_create_index(gm.d, gm.ell, index, arith, 1, &p);
            if (st != TT_FSI_OK) break;
            it = plan_idx.emplace(key, (int)b->plans.size()).first;
            b->plans.push_back(p);
        }
        b->plan_of_game.push_back(it->second);
    }
    if (st != TT_FSI_OK) {
        batch_free(b.get());
        return st;
    }
    // per-game offsets of the partial scores and exponents
    long long goff = 0, eoff = 0;
    b->hgames.resize(n_games);
    for (int64_t g = 0; g < n_games; ++g) {
        const Plan &p = b->plans[b->plan_of_game[g]]->p;
        BatchGameDev &hg = b->hgames[g];
        hg.v_off = b->games[g].v_offset;
        hg.phi_off = b->games[g].phi_offset;
        hg.plan = b->plan_of_game[g];
        hg.n_tiles = 1 << p.h;
        hg.g_off = goff;
        hg.exp_off = eoff;
        if (p.fast12) {
            b->fast_games.push_back((int)g);
            goff += (long long)hg.n_tiles * p.n_g;
            eoff += hg.n_tiles;
            b->smem = std::max(b->smem, p.smem_fast);
        } else {
            b->slow_games.push_back((int)g);
        }
    }
    // device copies of each plan's kernel arguments
    std::vector<FastArgs> fpl(b->plans.size());
    std::vector<CombineFastArgs> cpl(b->plans.size());
    for (size_t i = 0; i < b->plans.size(); ++i) {
        const Plan &p = b->plans[i]->p;
        FastArgs &fa = fpl[i];
        fa = fast_args(p);
        CombineFastArgs &ca = cpl[i];
        ca = CombineFastArgs{};
        ca.tasks = p.d_tasks;
        ca.wden = p.d_wden;
        ca.winv = p.d_winv;
        ca.h = p.h;
        ca.n_g = p.n_g;
        ca.shift_cap = p.shift_cap;
        ca.n_out = p.n_out;
    }
    cudaError_t e = cudaSuccess;
    auto up = [&](void **dst, const void *src, size_t bytes) {
        if (e != cudaSuccess || bytes == 0) return;
        e = cudaMalloc(dst, bytes);
        if (e == cudaSuccess) e = cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice);
    };
    up((void **)&b->d_fplans, fpl.data(), fpl.size() * sizeof(FastArgs));
    up((void **)&b->d_cplans, cpl.data(), cpl.size() * sizeof(CombineFastArgs));
    up((void **)&b->d_games, b->hgames.data(), b->hgames.size() * sizeof(BatchGameDev));
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->d_counters, (1 + (size_t)n_games) * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->d_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(b->d_err, 0, sizeof(int));
    if (e == cudaSuccess && goff > 0) e = cudaMalloc(&b->d_G, (size_t)goff * g_elem(arith));
    if (e == cudaSuccess && eoff > 0) e = cudaMalloc((void **)&b->d_exp, (size_t)eoff * sizeof(int));
    if (e == cudaSuccess && !b->fast_games.empty()) {
        int occ = 0, dev = 0, sms = 0;
        if (arith == TT_FSI_ARITH_EXACT) {
            e = allow_max_smem(fsi_batch_kernel<long long>);
            if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fsi_batch_kernel<long long>, kTileThreads, b->smem);
        } else if (arith == TT_FSI_ARITH_F64) {
            e = allow_max_smem(fsi_batch_kernel<double>);
            if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fsi_batch_kernel<double>, kTileThreads, b->smem);
        } else {
            e = allow_max_smem(fsi_batch_kernel<float>);
            if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fsi_batch_kernel<float>, kTileThreads, b->smem);
        }
        if (e == cudaSuccess) e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        b->grid = std::max(1, occ) * sms;  // every CTA resident at once: waits can always be served
        if (occ < 1) e = cudaErrorInvalidConfiguration;
    }
    st = cuda_status(e);
    if (st == TT_FSI_OK) st = batch_build_items(b.get());
    if (st != TT_FSI_OK) {
        batch_free(b.get());
        return st;
    }
    *out = b.release();
    return TT_FSI_OK;
}

void tt_fsi_batch_destroy(tt_fsi_batch batch) {
    if (!batch) return;
    cudaDeviceSynchronize();
    ttfsi::batch_free(batch);
    delete batch;
}

tt_fsi_status tt_fsi_batch_apply(tt_fsi_batch b, const void *v_dev, void *phi_dev, struct CUstream_st *stream) {
    using namespace ttfsi;
    if (!b) return TT_FSI_ERR_INVALID_ARG;
    if (b->games.empty()) return TT_FSI_OK;
    if (!v_dev || !phi_dev) return TT_FSI_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    switch (b->arith) {
        case TT_FSI_ARITH_EXACT: return batch_launch<long long>(b, v_dev, phi_dev, st);
        case TT_FSI_ARITH_F64: return batch_launch<double>(b, v_dev, phi_dev, st);
        case TT_FSI_ARITH_F32: return batch_launch<float>(b, v_dev, phi_dev, st);
    }
    return TT_FSI_ERR_INVALID_ARG;
}

tt_fsi_status tt_fsi_batch_apply_per_game(tt_fsi_batch b, const void *v_dev, void *phi_dev,
                                          struct CUstream_st *stream) {
    using namespace ttfsi;
    if (!b) return TT_FSI_ERR_INVALID_ARG;
    if (b->games.empty()) return TT_FSI_OK;
    if (!v_dev || !phi_dev) return TT_FSI_ERR_INVALID_ARG;
    const size_t ie = in_elem(b->arith);
    for (size_t g = 0; g < b->games.size(); ++g) {
        const tt_fsi_game &gm = b->games[g];
        tt_fsi_status s = tt_fsi_apply(b->plans[b->plan_of_game[g]], (const char *)v_dev + gm.v_offset * ie, 1,
                                       (char *)phi_dev + gm.phi_offset * ie, stream);
        if (s != TT_FSI_OK) return s;
    }
    return TT_FSI_OK;
}

tt_fsi_status tt_fsi_batch_apply_graph(tt_fsi_batch b, const void *v_dev, void *phi_dev,
                                       struct CUstream_st *stream) {
    using namespace ttfsi;
    if (!b) return TT_FSI_ERR_INVALID_ARG;
    if (b->games.empty()) return TT_FSI_OK;
    if (!v_dev || !phi_dev) return TT_FSI_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (!b->graph || b->graph_v != v_dev || b->graph_phi != phi_dev) {
        if (b->graph) cudaGraphExecDestroy(b->graph);
        if (b->graph_def) cudaGraphDestroy(b->graph_def);
        b->graph = nullptr;
        b->graph_def = nullptr;
        cudaStream_t cap = nullptr;
        cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
        if (e != cudaSuccess) return cuda_status(e);
        e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        tt_fsi_status s = TT_FSI_OK;
        if (e == cudaSuccess) s = tt_fsi_batch_apply_per_game(b, v_dev, phi_dev, reinterpret_cast<CUstream_st *>(cap));
        cudaGraph_t gdef = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(cap, &gdef);
        cudaStreamDestroy(cap);
        if (e != cudaSuccess || e2 != cudaSuccess || s != TT_FSI_OK) {
            if (gdef) cudaGraphDestroy(gdef);
            return s != TT_FSI_OK ? s : cuda_status(e != cudaSuccess ? e : e2);
        }
        e = cudaGraphInstantiate(&b->graph, gdef, 0);
        if (e != cudaSuccess) {
            cudaGraphDestroy(gdef);
            b->graph = nullptr;
            return cuda_status(e);
        }
        b->graph_def = gdef;
        b->graph_v = v_dev;
        b->graph_phi = phi_dev;
    }
    return cuda_status(cudaGraphLaunch(b->graph, st));
}

tt_fsi_status tt_fsi_batch_autotune(tt_fsi_batch b, const void *v_dev, void *phi_dev, struct CUstream_st *stream,
                                    int *tiles_per_item, int *scores_per_item) {
    using namespace ttfsi;
    if (!b || !v_dev || !phi_dev) return TT_FSI_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int tpi[] = {1, 2, 4, 8};
    const int spi[] = {16, 64, 256};
    float best = 1e30f;
    int bt = b->tiles_per_item, bs = b->scores_per_item;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return TT_FSI_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return TT_FSI_ERR_CUDA;
    }
    tt_fsi_status s = TT_FSI_OK;
    for (int t : tpi) {
        for (int c : spi) {
            b->tiles_per_item = t;
            b->scores_per_item = c;
            if ((s = batch_build_items(b)) != TT_FSI_OK) break;
            if ((s = tt_fsi_batch_apply(b, v_dev, phi_dev, stream)) != TT_FSI_OK) break;  // warm-up
            cudaEventRecord(e0, st);
            for (int r = 0; r < 3 && s == TT_FSI_OK; ++r) s = tt_fsi_batch_apply(b, v_dev, phi_dev, stream);
            cudaEventRecord(e1, st);
            if (s != TT_FSI_OK || cudaEventSynchronize(e1) != cudaSuccess) {
                if (s == TT_FSI_OK) s = TT_FSI_ERR_CUDA;
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best) {
                best = ms;
                bt = t;
                bs = c;
            }
        }
        if (s != TT_FSI_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->tiles_per_item = bt;
    b->scores_per_item = bs;
    tt_fsi_status s2 = batch_build_items(b);
    if (s == TT_FSI_OK) s = s2;
    if (tiles_per_item) *tiles_per_item = bt;
    if (scores_per_item) *scores_per_item = bs;
    return s;
}

tt_fsi_status tt_fsi_batch_set_schedule(tt_fsi_batch b, int tiles_per_item, int scores_per_item) {
    if (!b || tiles_per_item < 1 || scores_per_item < 1) return TT_FSI_ERR_INVALID_ARG;
    b->tiles_per_item = tiles_per_item;
    b->scores_per_item = scores_per_item;
    return ttfsi::batch_build_items(b);
}

tt_fsi_status tt_fsi_batch_set_wait_limit(tt_fsi_batch b, long long polls, int inject_missing_tile) {
    if (!b || polls < 1) return TT_FSI_ERR_INVALID_ARG;
    b->spin_limit = polls;
    b->inject_missing = inject_missing_tile ? 1 : 0;
    return TT_FSI_OK;
}

tt_fsi_status tt_fsi_batch_check(tt_fsi_batch b, struct CUstream_st *stream) {
    using namespace ttfsi;
    if (!b) return TT_FSI_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int h_err = 0;
    cudaError_t e = cudaMemcpyAsync(&h_err, b->d_err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_err, 0, sizeof(int), st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_status(e);
    for (tt_fsi_plan p : b->plans) {
        tt_fsi_status s = tt_fsi_plan_check(p, stream);
        if (s != TT_FSI_OK) h_err |= (s == TT_FSI_ERR_NONFINITE) ? kErrNonFinite : 0;
    }
    if (h_err & kErrTimeout) return TT_FSI_ERR_TIMEOUT;
    if (h_err & kErrNonFinite) return TT_FSI_ERR_NONFINITE;
    return TT_FSI_OK;
}

}  // extern "C"
