// Host-side plan of the FSI operator: tile schedule, the transition tables of
// the ranked superset sums, the combined correction weights, and the
// per-score tasks of the combine kernel.  Everything here depends only on
// (d, l, arithmetic) and is built once per plan.
#pragma once

#include <cstdint>
#include <vector>

#include "tt_fsi.h"

namespace ttfsi {

// Largest tile the tile kernel handles (2^12 coalitions per CTA, 16 values
// per thread at 256 threads).
constexpr int kMaxTileBits = 12;
constexpr int kTileThreads = 256;
constexpr int kMaxLevels = kMaxTileBits + 1;

// Exact rational with 128-bit numerator and denominator (denominator > 0,
// reduced).  Used only on the host to build weight tables.
struct Rational {
    __int128 num = 0;
    __int128 den = 1;
};
Rational rat_make(__int128 num, __int128 den);
Rational rat_add(const Rational &a, const Rational &b);
Rational rat_mul(const Rational &a, const Rational &b);

// Correction weight w(s, t) of Eq. weight as an exact rational; zero for
// s = 0, s > l or t <= l (where C(t-1, l) vanishes).
Rational weight_rational(int ell, int s, int t);

// Weight W(s, t), t > s, of an interaction index on the Moebius coefficient
// of a superset T of S (|S| = s, |T| = t); the T = S term is always 1 and is
// applied separately.
Rational index_weight(tt_fsi_index index, int ell, int s, int t);

struct Plan {
    bool precontract = false;  // site-by-site sweep of B_corr on v (no Moebius pass)
    int d = 0, ell = 0, ell_eff = 0;
    tt_fsi_index index = TT_FSI_INDEX_FSI;
    tt_fsi_arith arith = TT_FSI_ARITH_EXACT;
    int64_t max_batch = 0;
    int b = 0, h = 0;         // tile bits, high bits (d = b + h, or d < b = 12 on the fast path)
    int load_bits = 0;        // bits of a tile present in v (min(d, b)); the rest are null players
    bool mob_only = false;    // FSI or STII with l >= d: scores are the Moebius coefficients
    int64_t n_out = 0;        // scores per game
    int n_ch = 0;             // channels per tile (states at the last level)
    int prec_bits = 0;        // fixed-point headroom P of the exact path
    bool g_split31 = false;   // fast exact path: weights small enough for 32 x 32-bit products
    int shift_cap = 0;        // largest exponent gap aligned exactly across tiles

    // ranked superset sums: states per level and (src for tau=0, src for tau=1)
    int n_states[kMaxLevels] = {0};
    int lvl_off[kMaxLevels] = {0};
    std::vector<int32_t> trans;   // 2 entries per (level, output state)
    int buf_elems = 0;            // elements of one ping-pong buffer

    // Fast tile path (b = 12, l <= 4): Moebius in registers, ranked sums in
    // three 4-bit groups by absolute rank, run in rounds r = |sigma n bits
    // 0..3|; every offset is a closed form (fast_layout.h), so the only table
    // is gtab.  Shared memory: regA (tile, then one round's level-8 states),
    // regB (one round's level-4 states), then the n_ch channels.
    bool fast12 = false;
    int fast_regA = 0, fast_regB = 0;       // shared-memory regions (elements)
    size_t smem_fast = 0;
    // Schedule of a fast-path apply: one fused persistent launch (tiles and
    // combine from one work queue; default) or a tile launch then a combine
    // launch.  Work-item sizes and the bound on the combine's wait.
    bool fused = false;
    int tiles_per_item = 1, scores_per_item = 64;
    int apply_grid = 0;                     // persistent CTAs (SMs x resident CTAs per SM)
    long long spin_limit = 4000000;
    bool inject_missing = false;            // test hook of the bounded wait
    int *d_counters = nullptr;              // [0] queue head, [1 + g] finished tiles of game g
    // Partial scores per tile on the fast path: one entry per (S_L, s, i)
    // (low set, |S|, |U_H n S_H|), gtab = {ch_base, s_L | s << 8 | i << 16}.
    // The combine tasks' 4th field is the entry of (S_L, s, i = 0).
    std::vector<int32_t> gtab;
    int n_g = 0;
    int32_t *d_gtab = nullptr;

    // combine tasks, one per score in output order:
    // [ch_base, high mask (bits b..d-1 shifted down), s | s_L << 8 | s_H << 16, 0]
    std::vector<int32_t> tasks;

    // weights omega_s(p, q), index (s * (h+1) + p) * (b+1) + q
    std::vector<long long> wnum;  // exact path: numerators over den[s]
    std::vector<long long> wden;  // exact path: one common denominator per s
    std::vector<double> wf64;     // float paths
    std::vector<float> wf32;

    // device memory
    int32_t *d_trans = nullptr;
    int32_t *d_tasks = nullptr;
    long long *d_wnum = nullptr;
    std::vector<double> winv;  // exact path: 1 / den[s], rounded once (the combine's scale)
    double *d_winv = nullptr;
    // fast path: weight rows per u_H = |U_H| ([h + 1][n_wcombo][kWRow], int32
    // on the exact split path, float / double otherwise), copied into shared
    // memory by each tile; empty when the exact path needs 64-bit weights
    std::vector<uint8_t> wstage;
    int wstage_block = 0;  // bytes per u_H
    void *d_wstage = nullptr;
    long long *d_wden = nullptr;
    double *d_wf64 = nullptr;
    float *d_wf32 = nullptr;
    void *d_Y = nullptr;          // [max_batch][2^h][n_ch] elements (8 B, 4 B for f32)
    int *d_exp = nullptr;         // [max_batch][2^h] tile exponents (exact path)
    int *d_err = nullptr;         // fault word
    size_t scratch_bytes = 0;
    size_t smem_tile = 0;         // dynamic shared memory of the tile kernel
};

// Builds every host table of the plan (no CUDA calls).  Returns a status.
tt_fsi_status plan_build_host(Plan &p, int d, int ell, tt_fsi_arith arith, int64_t max_batch,
                              tt_fsi_index index = TT_FSI_INDEX_FSI, bool site_sweep = false,
                              bool precontract = false);

// Scores and their order.
int64_t num_scores(int d, int ell);
void score_masks(int d, int ell, uint64_t *out);

}  // namespace ttfsi
