// The fast tile path (12-bit tiles, orders l <= 4): per-tile Moebius,
// ranked superset sums and partial scores, and its tile kernel.  Kept in
// one file so that the measured traffic of this kernel can be tied to its
// exact source.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "fast_layout.h"
#include "fsi_plan.h"
#include "tile_common.cuh"

namespace ttfsi {

// ----------------------------------------------------------------------------
// Fast tile kernel for b = 12, l <= 4.
//
// Moebius: the 16 values a thread holds always differ in 4 tile bits; three
// register phases (bits 8-11, 4-7, 0-3) with two shared-memory transposes.
// Shared layout of the tile: element e at e ^ ((e >> 8) & 15), which keeps
// every half-warp on 16 distinct 8-byte bank pairs in all three phases.
//
// Ranked superset sums (the (|S|, |T|) counters of Section 3.3) in three
// 4-bit groups, ranked by the absolute count u = |T n processed bits| (the
// layout and its closed-form offsets are in fast_layout.h).  With u fixed,
// every input of a group step has exactly one rank, so each step is a plain
// superset sum over 4 bits in registers:
//   block 1 (group A, registers): Z_A(sigma_A, t) from the Moebius values;
//   block 2 (group B): item (sigma_A, u) x 16 lanes tau_C gathers the 16
//     values Z_A(sigma_A, u - |tau_B|; tau_B) and writes Z_AB(sigma_A u
//     sigma_B, u) for every sigma_B the order allows;
//   block 3 (group C): item (sigma_8, u') per thread gathers Z_AB(sigma_8,
//     u' - |tau_C|; tau_C) and writes the channels Z(sigma_8 u sigma_C, u').
// Each output state is written by exactly one thread.  States are processed
// in rounds rd = |sigma_A| (a state's round never changes), on the exact
// path the rounds with 4 or 6 patterns sigma_A in two chunks, so only one
// chunk's level-4 and level-8 states are held in shared memory at a time
// (62 KB per CTA at l = 3 with the channels: three CTAs per SM).  The kernel is instantiated
// per order l, which makes every offset and every pruning decision a
// compile-time constant; the chunks of a round share one copy of the block
// 2 and 3 code (the kernel's instruction footprint matters as much as its
// instruction count: larger unrolled variants lost to instruction fetch).
//
// Weighting: the tile, whose high pattern U_H has u_H = |U_H| set bits, forms
// one partial score per (S_L, s, i) -- i the size of U_H n S_H that a score
// S = S_L u S_H of size s would see --
//   G = (-1)^(r-i) sum_j [omega_s(u_H + r - i, |S_L| + j) + [i = u_H][j = 0]] Y(S_L, j),
// r = s - |S_L|, so that phi(S) = sum over tiles of G(S_L, s, |U_H n S_H|).
// On the exact path G is an exact int128 (weights as integer numerators).
// ----------------------------------------------------------------------------
struct FastArgs {
    const void *v;
    void *G;
    int *tile_exp;
    int *err;
    const int32_t *gtab;
    int n_g;
    int d, h, ell, prec_bits, load_mask;
    int g_split31;        // exact weighting by 32 x 32-bit products (see the plan)
    int prefetch_ahead;   // tile launch: prefetch the tile this many CTAs ahead into L2 (0: off)
    long long game0;
    const void *wstage;   // weight rows per u_H (built by every fast plan)
    int wstage_block;     // bytes per u_H, a multiple of 16
};

template <typename Acc>
struct GTraits {
    using G = Acc;
};
// Chunked rounds (fast_layout.h) on the exact path, which then fits three
// CTAs per SM; the float paths keep whole rounds (fewer barriers: float32
// fits four CTAs per SM either way, float64 is bound by its float64 pipe).
template <typename Acc>
constexpr int kChunked = TileTraits<Acc>::exact ? 1 : 0;
// The tile launch (fsi_tile_fast_kernel) runs round 2 in three chunks
// (fast_layout.h, mode 2): one pass of block 2 per chunk.  The persistent
// kernels, which carry the combine as well, keep mode 1 (two chunks), which
// measured faster for them.  Mode 2 needs no more shared memory than mode 1,
// so the plan sizes every launch by mode 1.
template <typename Acc>
constexpr int kTileChunkMode = TileTraits<Acc>::exact ? 2 : 0;
template <>
struct GTraits<long long> {
    using G = __int128;
};

__device__ __forceinline__ double i128_to_double(__int128 x) {
    const bool neg = x < 0;
    unsigned __int128 u = neg ? (unsigned __int128)(-x) : (unsigned __int128)x;
    unsigned long long hi = (unsigned long long)(u >> 64), lo = (unsigned long long)u;
    double r = (double)hi * 18446744073709551616.0 + (double)lo;
    return neg ? -r : r;
}

// Full 128-bit product of two signed 64-bit integers.
__device__ __forceinline__ __int128 mul_wide(long long a, long long b) {
    const unsigned long long lo = (unsigned long long)a * (unsigned long long)b;
    const long long hi = __mul64hi(a, b);
    return (__int128)(((unsigned __int128)(unsigned long long)hi << 64) | lo);
}

__device__ __forceinline__ int tile_phys(int e) { return e ^ ((e >> 8) & 15); }

// L2 eviction priorities: the input is read once and streams through L2
// (evict first), the partial scores are read again by the combine launch
// (evict last), so that they stay in L2 while the input passes.
__device__ __forceinline__ unsigned long long l2_policy_evict_first() {
    unsigned long long p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ unsigned long long l2_policy_evict_last() {
    unsigned long long p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ unsigned long long ld_stream_u64(const unsigned long long *ptr, unsigned long long pol) {
    unsigned long long v;
    asm volatile("ld.global.nc.L2::cache_hint.u64 %0, [%1], %2;" : "=l"(v) : "l"(ptr), "l"(pol));
    return v;
}
__device__ __forceinline__ void st_keep_i128(__int128 *ptr, __int128 v, unsigned long long pol) {
    const unsigned long long lo = (unsigned long long)v, hi = (unsigned long long)((unsigned __int128)v >> 64);
    asm volatile("st.global.L2::cache_hint.v2.u64 [%0], {%1, %2}, %3;" ::"l"(ptr), "l"(lo), "l"(hi), "l"(pol)
                 : "memory");
}

// Moebius transform over 4 bits, two bits at a time: for the four entries
// x0..x3 that differ in bits q, q+1 (x3 has both) the result is x0,
// x1 - x0, x2 - x0 and x3 - x1 - (x2 - x0), i.e. three additions of at most
// three operands (one 64-bit add instruction pair each) instead of four.
template <typename Acc>
__device__ __forceinline__ void mobius16(Acc (&x)[16]) {
#pragma unroll
    for (int q = 0; q < 4; q += 2)
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            if ((r >> q) & 3) continue;
            const int r1 = r | (1 << q), r2 = r | (2 << q), r3 = r | (3 << q);
            const Acc y2 = x[r2] - x[r];
            x[r3] = x[r3] - x[r1] - y2;
            x[r1] = x[r1] - x[r];
            x[r2] = y2;
        }
}

// Superset sums over 4 bits, correct wherever |sigma_r| <= O, two bits at a
// time.  Bit by bit, an entry is still needed after the level of bit q only
// if it has at most O set bits among bits 0..q; for the four entries that
// differ in bits q, q+1, with c set bits of r below q:
//   c <= O - 1: x0 + x1 + x2 + x3, x1 + x3, x2 + x3 (all three needed);
//   c == O:     x0 + x1 + x2 + x3 and x2 + x3 (x1's sum is never read);
//   c >  O:     nothing.
template <int O, typename Acc>
__device__ __forceinline__ void zeta16(Acc (&x)[16]) {
#pragma unroll
    for (int q = 0; q < 4; q += 2)
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            if ((r >> q) & 3) continue;
            const int c = fast::pc4(r & ((1 << q) - 1));
            if (c > O) continue;
            const int r1 = r | (1 << q), r2 = r | (2 << q), r3 = r | (3 << q);
            const Acc t2 = x[r2] + x[r3];
            x[r] = x[r] + x[r1] + t2;
            if (c <= O - 1) x[r1] = x[r1] + x[r3];
            x[r2] = t2;
        }
}

// Block 1 of chunk C of round RD: the level-4 states (sigma_A, t),
// |sigma_A| = RD, rank of sigma_A in the chunk, of this thread's position
// (tau_B, tau_C) from its 16 Moebius values.
template <int L, int RD, int C, int CM, typename Acc>
__device__ __forceinline__ void fast_block1(const Acc (&x)[16], Acc *regB, int pos) {
    constexpr int CA = fast::chunk_a(RD, CM), A0 = C * CA;
#pragma unroll
    for (int sg = 0; sg < 16; ++sg) {
        if (fast::pc4(sg) != RD) continue;
        const int ra = fast::rank4(sg);
        if (ra < A0 || ra >= A0 + CA) continue;
        const int base = (ra - A0) * (5 - RD) - RD;
#pragma unroll
        for (int t = RD; t <= 4; ++t) {
            Acc acc = 0;
#pragma unroll
            for (int tau = 0; tau < 16; ++tau)
                if ((tau & sg) == sg && fast::pc4(tau) == t) acc += x[tau];
            regB[(base + t) * 256 + pos] = acc;
        }
    }
}

// Block 2 item (rank sigma_A = rA within the chunk, u = RD + uu) of round
// RD on lane tau_C: gathers the 16 level-4 states Z_A(sigma_A, u - |tau_B|;
// tau_B), zero where that rank is outside [RD, 4], and writes the level-8
// states (sigma_A u sigma_B, u) to regA[tau_C * NST + state].  UU >= 0
// fixes uu at compile time, so the zero inputs and the states that cannot
// exist fold away; UU = -1 takes uu at run time.
template <int L, int RD, int UU, int CM, typename Acc>
__device__ __forceinline__ void fast_block2_item(const Acc *regB, Acc *regA, int rA, int uu_rt, int t3) {
    constexpr int O = L - RD;
    constexpr int S8 = fast::s8(L, RD);
    constexpr int NST = fast::nst(L, CM);
    const int uu = UU >= 0 ? UU : uu_rt;
    // input tau_B: level-4 state (sigma_A, t = u - |tau_B|), t in [RD, 4]
    const Acc *src = regB + (rA * (5 - RD) + uu) * 256 + t3;
    Acc x[16];
#pragma unroll
    for (int tau = 0; tau < 16; ++tau) {
        const int pc = fast::pc4(tau);
        Acc val = 0;
        if (uu >= pc && uu - pc <= 4 - RD) val = src[16 * tau - 256 * pc];
        x[tau] = val;
    }
    zeta16<O>(x);
    Acc *dst = regA + t3 * NST + rA * S8 + uu;
#pragma unroll
    for (int sb = 0; sb < 16; ++sb) {
        const int kB = fast::pc4(sb);
        if (kB > O) continue;
        // state (sigma_A u sigma_B, u): off8 + rank * (9 - RD - kB) + (u - RD - kB)
        if (uu >= kB) dst[fast::off8(RD, kB) + fast::rank4(sb) * (9 - RD - kB) - kB] = x[sb];
    }
}

// Block 2 of one chunk of round RD: items (rank sigma_A in the chunk, u),
// u in [RD, 8], 16 lanes over tau_C, in the order (k, rank sigma_A) with
// uu = k / 2 for even k and 8 - RD - k / 2 for odd k: the items with uu in
// {0, 1, 7 - RD, 8 - RD} (at most 5 of their 16 inputs nonzero) come first,
// and the two half-warps of a warp take the same uu whenever the number of
// sigma_A is even (for one sigma_A they pair uu with 8 - RD - uu).  On the
// float paths those items run bodies compiled for their uu (the zero terms
// fold away, which the float64 pipe needs); the exact path runs one body
// for every uu (bodies compiled per uu cost it more in instruction fetch
// than they save).
template <int L, int RD, int CM, typename Acc>
__device__ __forceinline__ void fast_block2(const Acc *regB, Acc *regA, int tid) {
    constexpr int NU = 9 - RD;
    constexpr int NA = fast::chunk_a(RD, CM);
    constexpr int NIT = NA * NU;
    const int t3 = tid & 15;
    for (int it = tid >> 4; it < NIT; it += kTileThreads / 16) {
        const int k = it / NA, rA = it - k * NA;
        const int uu = (k & 1) ? NU - 1 - (k >> 1) : (k >> 1);
        if constexpr (TileTraits<Acc>::exact) {
            fast_block2_item<L, RD, -1, CM>(regB, regA, rA, uu, t3);
        } else {
            if (uu == 0)
                fast_block2_item<L, RD, 0, CM>(regB, regA, rA, uu, t3);
            else if (uu == 1)
                fast_block2_item<L, RD, 1, CM>(regB, regA, rA, uu, t3);
            else if (uu == NU - 2)
                fast_block2_item<L, RD, NU - 2, CM>(regB, regA, rA, uu, t3);
            else if (uu == NU - 1)
                fast_block2_item<L, RD, NU - 1, CM>(regB, regA, rA, uu, t3);
            else
                fast_block2_item<L, RD, -1, CM>(regB, regA, rA, uu, t3);
        }
    }
}

// Block 3 item of round RD, group kB = |sigma_B|: (rank sigma_A, rank
// sigma_B, u'), u' in [RD + KB, 12]; writes the channels of sigma_8 u sigma_C.
template <int L, int RD, int KB, int CM, typename Acc>
__device__ __forceinline__ void fast_block3_item(int local, const Acc *regA, Acc *regY, int pair0) {
    constexpr int K8 = RD + KB;
    constexpr int O = L - K8;
    constexpr int NU = 13 - K8;
    constexpr int NB = fast::c4(KB);
    constexpr int S8 = fast::s8(L, RD);
    constexpr int NST = fast::nst(L, CM);
    constexpr int OFF8 = fast::off8(RD, KB);
    constexpr int CG = fast::chan_group(L, RD, KB);
    constexpr int CH = fast::ch8(L, K8);
    const int pair = local / NU, uu = local - pair * NU;  // u' = K8 + uu
    const int rA = pair / NB, rB = pair - rA * NB;
    // input tau_C: level-8 state (sigma_8, u' - |tau_C|), u' - |tau_C| in [K8, 8]
    const Acc *src = regA + rA * S8 + OFF8 + rB * (9 - K8) + uu;
    Acc x[16];
#pragma unroll
    for (int tau = 0; tau < 16; ++tau) {
        const int pc = fast::pc4(tau);
        Acc val = 0;
        if (uu >= pc && uu - pc <= 8 - K8) val = src[tau * NST - pc];
        x[tau] = val;
    }
    zeta16<O>(x);
    Acc *dst = regY + CG + (pair0 + pair) * CH + uu;
#pragma unroll
    for (int sc = 0; sc < 16; ++sc) {
        const int kC = fast::pc4(sc);
        if (kC > O) continue;
        // channel (sigma_8 u sigma_C, j = u' - K8 - kC)
        if (uu >= kC) dst[fast::offC(K8, kC) + fast::rank4(sc) * (13 - K8 - kC) - kC] = x[sc];
    }
}

// Block 3 of chunk C of round RD: the groups kB = 0..L-RD one after
// another, each padded to whole warps so that a warp never mixes two
// pruning orders.  Item pairs are numbered within the chunk; their channels
// sit at the round's pair index (chunk C starts at pair C * CA * C(4, kB)).
template <int L, int RD, int CM, typename Acc>
__device__ __forceinline__ void fast_block3(const Acc *regA, Acc *regY, int tid, int C) {
    constexpr int M = L - RD;
    constexpr int CA = fast::chunk_a(RD, CM);
    constexpr int P0 = fast::pad32(fast::g3(RD, 0, CM));
    constexpr int P1 = M >= 1 ? fast::pad32(fast::g3(RD, 1, CM)) : 0;
    constexpr int P2 = M >= 2 ? fast::pad32(fast::g3(RD, 2, CM)) : 0;
    constexpr int P3 = M >= 3 ? fast::pad32(fast::g3(RD, 3, CM)) : 0;
    constexpr int P4 = M >= 4 ? fast::pad32(fast::g3(RD, 4, CM)) : 0;
    constexpr int TOTAL = P0 + P1 + P2 + P3 + P4;
    for (int it = tid; it < TOTAL; it += kTileThreads) {
        if (it < P0) {
            if (it < fast::g3(RD, 0, CM)) fast_block3_item<L, RD, 0, CM>(it, regA, regY, C * CA * fast::c4(0));
        } else if (it < P0 + P1) {
            if constexpr (M >= 1) {
                const int l = it - P0;
                if (l < fast::g3(RD, 1, CM)) fast_block3_item<L, RD, 1, CM>(l, regA, regY, C * CA * fast::c4(1));
            }
        } else if (it < P0 + P1 + P2) {
            if constexpr (M >= 2) {
                const int l = it - P0 - P1;
                if (l < fast::g3(RD, 2, CM)) fast_block3_item<L, RD, 2, CM>(l, regA, regY, C * CA * fast::c4(2));
            }
        } else if (it < P0 + P1 + P2 + P3) {
            if constexpr (M >= 3) {
                const int l = it - P0 - P1 - P2;
                if (l < fast::g3(RD, 3, CM)) fast_block3_item<L, RD, 3, CM>(l, regA, regY, C * CA * fast::c4(3));
            }
        } else {
            if constexpr (M >= 4) {
                const int l = it - P0 - P1 - P2 - P3;
                if (l < fast::g3(RD, 4, CM)) fast_block3_item<L, RD, 4, CM>(l, regA, regY, C * CA * fast::c4(4));
            }
        }
    }
}

// Block 1 of chunk C (run time) of round RD.
template <int L, int RD, int CM, typename Acc>
__device__ __forceinline__ void fast_block1_chunk(const Acc (&x)[16], Acc *regB, int pos, int C) {
    constexpr int NC = fast::n_chunks(RD, CM);
    static_assert(NC >= 1 && NC <= 3, "at most three chunks per round");
    if constexpr (NC == 1) {
        fast_block1<L, RD, 0, CM>(x, regB, pos);
    } else if constexpr (NC == 2) {
        if (C == 0)
            fast_block1<L, RD, 0, CM>(x, regB, pos);
        else
            fast_block1<L, RD, 1, CM>(x, regB, pos);
    } else {
        if (C == 0)
            fast_block1<L, RD, 0, CM>(x, regB, pos);
        else if (C == 1)
            fast_block1<L, RD, 1, CM>(x, regB, pos);
        else
            fast_block1<L, RD, 2, CM>(x, regB, pos);
    }
}

// Round RD, chunk by chunk (a run-time loop, so that the chunks share the
// code of blocks 2 and 3): blocks 2 and 3 of the chunk, then block 1 of the
// next chunk (of this round or the next), which only touches the level-4
// region that block 2 has finished reading.
template <int L, int RD, int CM, typename Acc>
__device__ __forceinline__ void fast_round(const Acc (&x)[16], Acc *regA, Acc *regB, Acc *regY, int tid,
                                           int pos) {
    constexpr int NC = fast::n_chunks(RD, CM);
#pragma unroll 1
    for (int c = 0; c < NC; ++c) {
        fast_block2<L, RD, CM>(regB, regA, tid);
        __syncthreads();
        fast_block3<L, RD, CM>(regA, regY, tid, c);
        if (c + 1 < NC)
            fast_block1_chunk<L, RD, CM>(x, regB, pos, c + 1);
        else if constexpr (RD < L)
            fast_block1<L, RD + 1, 0, CM>(x, regB, pos);
        __syncthreads();
    }
    if constexpr (RD < L) fast_round<L, RD + 1, CM>(x, regA, regB, regY, tid, pos);
}

// Weight rows in shared memory per tile, row (s, |S_L|, i) holding the
// weights omega_s(u_H + r - i, |S_L| + j) of j = 0 .. 12 - |S_L| with the
// identity term (1, or D_s on the exact path) at j = 0 when i = u_H and the
// sign (-1)^(r - i) folded in, r = s - |S_L|: int32 on the exact path when
// g_split31 holds (every weight plus the identity term fits), int64 on the
// exact path otherwise, the arithmetic's own type on the float paths.  The
// plan holds the rows of every u_H; a tile copies its u_H block with
// cp.async when it starts and waits for the copy only before the ranked
// sums, so the copy costs no latency.
template <typename Acc>
struct WTraits {
    using W = Acc;
};
template <>
struct WTraits<long long> {
    using W = int;
};

// One partial score from a staged row: sum over j < J = 13 - |S_L| of
// w[j] Y(S_L, j).  Exact path: two 32 x 32-bit multiply-add chains on the
// split channel y = yh 2^31 + yl.
template <typename Acc, int J>
__device__ __forceinline__ typename GTraits<Acc>::G fast_g_staged(const typename WTraits<Acc>::W *w, const Acc *y) {
    using GT = typename GTraits<Acc>::G;
    using WT = typename WTraits<Acc>::W;
    Acc yv[J];
    WT c[J];
#pragma unroll
    for (int j = 0; j < J; ++j) yv[j] = y[j];
#pragma unroll
    for (int j = 0; j < J; ++j) c[j] = w[j];
    if constexpr (TileTraits<Acc>::exact) {
        long long acc_h = 0, acc_l = 0;
#pragma unroll
        for (int j = 0; j < J; ++j) {
            acc_h += (long long)c[j] * (int)(yv[j] >> 31);
            acc_l += (long long)c[j] * (int)(yv[j] & 0x7fffffffll);
        }
        return (GT)(((unsigned __int128)(__int128)acc_h) << 31) + (GT)acc_l;
    } else {
        Acc acc = 0;
#pragma unroll
        for (int j = 0; j < J; ++j) acc += yv[j] * c[j];
        return acc;
    }
}

// Exact path with 64-bit weight rows (numerators beyond the split): full
// 64 x 64 -> 128-bit products.
template <int J>
__device__ __forceinline__ __int128 fast_g_staged64(const long long *w, const long long *y) {
    long long yv[J], c[J];
#pragma unroll
    for (int j = 0; j < J; ++j) yv[j] = y[j];
#pragma unroll
    for (int j = 0; j < J; ++j) c[j] = w[j];
    __int128 acc = 0;
#pragma unroll
    for (int j = 0; j < J; ++j) acc += mul_wide(yv[j], c[j]);
    return acc;
}

template <typename Acc, int L, int CM = kChunked<Acc>>
__device__ __forceinline__ void tile_fast_body(const FastArgs &a, const long long game, const long long tile) {
    using In = typename TileTraits<Acc>::In;
    using GT = typename GTraits<Acc>::G;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Acc *tileS = reinterpret_cast<Acc *>(smem_raw);  // the tile during the Moebius transform
    Acc *regB = tileS;                                // then one chunk's level-4 states
    Acc *regA = regB + fast::reg4_elems(L, CM);  // and one chunk's level-8 states
    Acc *regY = tileS + fast::regT_elems(L, CM);  // channels
    using WT = typename WTraits<Acc>::W;
    // this tile's weight rows: the first 16-byte boundary after the channels
    constexpr size_t kWOff =
        ((size_t)(fast::regT_elems(L, CM) + fast::n_chan(L)) * sizeof(Acc) + 15) & ~(size_t)15;
    WT *wst = reinterpret_cast<WT *>(smem_raw + kWOff);
    __shared__ int s_emax;

    const int tid = threadIdx.x;
    const In *src = reinterpret_cast<const In *>(a.v) + (game << a.d) + (tile << 12);
    const int uH = __popcll((unsigned long long)tile);
    {
        const char *wsrc = reinterpret_cast<const char *>(a.wstage) + (size_t)uH * a.wstage_block;
        const unsigned wdst = (unsigned)__cvta_generic_to_shared(wst);
        for (int o = tid * 16; o < a.wstage_block; o += kTileThreads * 16)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(wdst + o), "l"(wsrc + o) : "memory");
        asm volatile("cp.async.commit_group;" ::: "memory");
    }

    Acc x[16];
    int E = 0;
    // ---- load (element tid + 256 r), register bits 8-11 ----
    if constexpr (TileTraits<Acc>::exact) {
        In raw[16];
        int emax = 0;
        const unsigned long long pol_in = l2_policy_evict_first();
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            raw[r] = ld_stream_u64(src + ((tid + 256 * r) & a.load_mask), pol_in);
            emax = max(emax, (int)((raw[r] >> 52) & 0x7ff));
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
        if (bad) {
#pragma unroll
            for (int r = 0; r < 16; ++r) x[r] = 0;
        } else if (E >= a.prec_bits + 1) {  // every tile but one of tiny values
            const int C = 53 - a.prec_bits + E;
#pragma unroll
            for (int r = 0; r < 16; ++r) x[r] = to_fixed_big_tile(raw[r], C);
        } else {
#pragma unroll
            for (int r = 0; r < 16; ++r) x[r] = to_fixed(raw[r], E, a.prec_bits);
        }
    } else {
#pragma unroll
        for (int r = 0; r < 16; ++r) x[r] = (Acc)__ldg(src + ((tid + 256 * r) & a.load_mask));
    }
    mobius16(x);
#pragma unroll
    for (int r = 0; r < 16; ++r) tileS[tile_phys(tid + 256 * r)] = x[r];
    __syncthreads();
    // ---- bits 4-7: e = (tid & 15) | r << 4 | (tid >> 4) << 8 ----
    {
        const int e0 = (tid & 15) | ((tid >> 4) << 8);
#pragma unroll
        for (int r = 0; r < 16; ++r) x[r] = tileS[tile_phys(e0 | (r << 4))];
        mobius16(x);
#pragma unroll
        for (int r = 0; r < 16; ++r) tileS[tile_phys(e0 | (r << 4))] = x[r];
    }
    __syncthreads();
    // ---- bits 0-3: t3 = tid & 15 (tau_C, bits 8-11), t2 = tid >> 4 (tau_B, bits 4-7) ----
    const int t3 = tid & 15, t2 = tid >> 4;
    {
        const int e0 = (t2 << 4) | (t3 << 8);
#pragma unroll
        for (int r = 0; r < 16; ++r) x[r] = tileS[tile_phys(e0 | r)];
        mobius16(x);
    }
    // the level-4 and level-8 states overwrite the tile
    __syncthreads();
    // ---- ranked sums: block 1 of round 0, then the rounds ----
    const int pos = t3 + 16 * t2;
    fast_block1<L, 0, 0, CM>(x, regB, pos);
    // the weight rows are read only after this barrier
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
    fast_round<L, 0, CM>(x, regA, regB, regY, tid, pos);
    // ---- partial scores G(S_L, s, i) of this tile ----
    // partial scores of a game are stored entry-major, [n_g][2^h tiles], so
    // that the combine's lanes (consecutive tiles) read consecutive addresses
    const long long ntile = 1ll << a.h;
    GT *gdst = reinterpret_cast<GT *>(a.G) + (game << a.h) * (long long)a.n_g + tile;
    const unsigned long long pol_g = l2_policy_evict_last();
    {
        for (int g = tid; g < a.n_g; g += kTileThreads) {
            const int cb = __ldg(a.gtab + 2 * g), code = __ldg(a.gtab + 2 * g + 1);
            const int sL = code & 0xff, s = (code >> 8) & 0xff, i = code >> 16;
            const WT *w = wst + fast::wcombo(s, sL, i) * fast::kWRow;
            GT acc;
            if constexpr (TileTraits<Acc>::exact) {
                // 13 products for every entry: the row's weights past
                // 12 - |S_L| are zero, and the channels read there (the next
                // channel's, or past the last channel the alignment gap and
                // the weight rows, all inside the allocation) are integers,
                // so every entry runs the same code
                if (a.g_split31)
                    acc = fast_g_staged<Acc, 13>(w, regY + cb);
                else
                    acc = fast_g_staged64<13>(reinterpret_cast<const long long *>(wst) +
                                                  fast::wcombo(s, sL, i) * fast::kWRow,
                                              reinterpret_cast<const long long *>(regY) + cb);
            } else {
                // entries are sorted by |S_L|, so a warp almost always takes one case
                switch (sL) {
                    case 0: acc = fast_g_staged<Acc, 13>(w, regY + cb); break;
                    case 1: acc = fast_g_staged<Acc, 12>(w, regY + cb); break;
                    case 2: acc = fast_g_staged<Acc, 11>(w, regY + cb); break;
                    case 3: acc = fast_g_staged<Acc, 10>(w, regY + cb); break;
                    default: acc = fast_g_staged<Acc, 9>(w, regY + cb); break;
                }
            }
            if constexpr (TileTraits<Acc>::exact)
                st_keep_i128(gdst + g * ntile, acc, pol_g);
            else
                gdst[g * ntile] = acc;
        }
    }
    if constexpr (TileTraits<Acc>::exact) {
        if (tid == 0) a.tile_exp[(game << a.h) + tile] = a.prec_bits + 1022 - E;
    }
}

// One tile of a plan with order a.ell (1..4): the instantiation for that order.
template <typename Acc>
__device__ __forceinline__ void tile_fast_dispatch(const FastArgs &a, const long long game, const long long tile) {
    switch (a.ell) {
        case 1: tile_fast_body<Acc, 1>(a, game, tile); break;
        case 2: tile_fast_body<Acc, 2>(a, game, tile); break;
        case 3: tile_fast_body<Acc, 3>(a, game, tile); break;
        default: tile_fast_body<Acc, 4>(a, game, tile); break;
    }
}

// One CTA per (tile, game).  With prefetch_ahead > 0 each CTA asks L2 to
// prefetch the input of the tile prefetch_ahead CTAs later (CTAs start
// roughly in linear order); the split schedule launches it with 0 (see the
// launch).
// Resident CTAs per SM the tile kernel is compiled for: three on the
// chunked exact path at l <= 3 (62 KB of shared memory, at most 80
// registers), four for float32 at l <= 3, two otherwise.
template <typename Acc, int L>
constexpr int kTileMinBlocks = L > 3 ? 2 : TileTraits<Acc>::exact ? 3 : sizeof(Acc) == 4 ? 4 : 2;

template <typename Acc, int L>
__global__ void __launch_bounds__(kTileThreads, kTileMinBlocks<Acc, L>) fsi_tile_fast_kernel(FastArgs a) {
    using In = typename TileTraits<Acc>::In;
    // a combine launched as this grid's programmatic dependent may be placed
    // on the SMs from now on; it waits for this grid's results before reading
    asm volatile("griddepcontrol.launch_dependents;");
    if (a.prefetch_ahead > 0) {
        const long long lin = (long long)blockIdx.y * gridDim.x + blockIdx.x + a.prefetch_ahead;
        if (lin < (long long)gridDim.x * gridDim.y) {
            const long long gy = lin / gridDim.x, gx = lin - gy * gridDim.x;
            const char *base = reinterpret_cast<const char *>(reinterpret_cast<const In *>(a.v) +
                                                              ((a.game0 + gy) << a.d) + (gx << fast::kBits));
            const int bytes = (a.load_mask + 1) * (int)sizeof(In);
            for (int o = threadIdx.x * 128; o < bytes; o += kTileThreads * 128)
                asm volatile("prefetch.global.L2 [%0];" ::"l"(base + o));
        }
    }
    tile_fast_body<Acc, L, kTileChunkMode<Acc>>(a, a.game0 + blockIdx.y, blockIdx.x);
}

}  // namespace ttfsi
