// Host-side plan construction for the FSI operator (see fsi_plan.h).
//
// Decomposition used by the kernels.  Split the d players into the b low
// "tile" bits and the h = d - b high bits; a tile is the 2^b coalitions that
// share one high pattern U_H.  Per tile the kernel forms the Moebius transform
// on the low bits, a_L, and the ranked superset sums
//   Y(U_H, S_L, j) = sum_{T_L superset of S_L, |T_L \ S_L| = j} a_L(U_H, T_L)
// for every low set S_L with |S_L| <= l (the two counters |S|, |T| of the
// correction operator of Section 3.3, kept per output prefix).  Expanding
// a(T) over the high bits and summing the correction of Eq. correction over
// the high supersets gives, for S = S_L u S_H,
//   phi(S) = sum_{U_H} (-1)^(|S_H| - |U_H n S_H|) sum_j
//              [omega_s(|S_H u U_H|, |S_L| + j) + [U_H subset S_H][j = 0]] Y(U_H, S_L, j)
// with s = |S| and
//   omega_s(p, q) = sum_{n=0}^{h-p} (-1)^n C(h-p, n) w(s, p + q + n),
// w the weight of Eq. weight.  The bracket's second term is the Moebius part
// a(S) of Eq. fsi_closed.  omega is exact rational; the exact path scales
// each omega_s by the common denominator of its entries.
#include "fsi_plan.h"
#include "fast_layout.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <tuple>

namespace ttfsi {

namespace {

__int128 iabs128(__int128 x) { return x < 0 ? -x : x; }

__int128 gcd128(__int128 a, __int128 b) {
    a = iabs128(a);
    b = iabs128(b);
    while (b != 0) {
        __int128 t = a % b;
        a = b;
        b = t;
    }
    return a;
}

// Binomial coefficients by Pascal's rule, exact for n <= 126.
struct Pascal {
    std::vector<std::vector<__int128>> c;
    explicit Pascal(int nmax) : c(nmax + 1) {
        for (int n = 0; n <= nmax; ++n) {
            c[n].assign(n + 1, 0);
            c[n][0] = c[n][n] = 1;
            for (int k = 1; k < n; ++k) c[n][k] = c[n - 1][k - 1] + c[n - 1][k];
        }
    }
    __int128 operator()(int n, int k) const {
        if (n < 0 || k < 0 || k > n) return 0;
        return c[n][k];
    }
};

const Pascal &pascal() {
    static Pascal p(126);
    return p;
}

int popc64(uint64_t x) { return __builtin_popcountll(x); }

}  // namespace

Rational rat_make(__int128 num, __int128 den) {
    Rational r;
    if (den < 0) {
        num = -num;
        den = -den;
    }
    __int128 g = gcd128(num, den);
    if (g == 0) g = 1;
    r.num = num / g;
    r.den = den / g;
    if (r.num == 0) r.den = 1;
    return r;
}

Rational rat_add(const Rational &a, const Rational &b) {
    __int128 g = gcd128(a.den, b.den);
    __int128 den = a.den / g * b.den;
    return rat_make(a.num * (b.den / g) + b.num * (a.den / g), den);
}

Rational rat_mul(const Rational &a, const Rational &b) {
    __int128 g1 = gcd128(a.num, b.den), g2 = gcd128(b.num, a.den);
    if (g1 == 0) g1 = 1;
    if (g2 == 0) g2 = 1;
    return rat_make((a.num / g1) * (b.num / g2), (a.den / g2) * (b.den / g1));
}

Rational weight_rational(int ell, int s, int t) {
    const Pascal &C = pascal();
    if (s <= 0 || s > ell || t < 1) return Rational{};
    __int128 top = C(t - 1, ell);
    if (top == 0) return Rational{};
    // s/(l+s) * C(l,s) * C(t-1,l) / C(t+l-1, l+s), sign (-1)^(l-s)
    Rational r = rat_make((__int128)s * C(ell, s), (__int128)(ell + s));
    r = rat_mul(r, rat_make(top, C(t + ell - 1, ell + s)));
    if ((ell - s) & 1) r.num = -r.num;
    return r;
}

// Bernoulli numbers B_0 .. B_n (B_1 = -1/2) from sum_{j<=m} C(m+1, j) B_j = 0.
const std::vector<Rational> &bernoulli_table() {
    static const std::vector<Rational> tab = [] {
        const Pascal &C = pascal();
        std::vector<Rational> B(1, rat_make(1, 1));
        for (int m = 1; m <= 30; ++m) {
            Rational acc;
            for (int j = 0; j < m; ++j) acc = rat_add(acc, rat_mul(rat_make(C(m + 1, j), 1), B[j]));
            B.push_back(rat_mul(acc, rat_make(-1, m + 1)));
        }
        return B;
    }();
    return tab;
}

Rational index_weight(tt_fsi_index index, int ell, int s, int t) {
    if (t <= s || s < 0) return Rational{};
    switch (index) {
        case TT_FSI_INDEX_KSII: {
            // Moebius form of the Bernoulli aggregation of SII: a superset T
            // of S reaches S through every T' with S <= T' <= T, |T'| <= l,
            // with B_{|T'|-s} / (t - |T'| + 1); the sums vanish for t <= l
            if (s == 0 || t <= ell) return Rational{};
            const Pascal &C = pascal();
            const std::vector<Rational> &B = bernoulli_table();
            Rational acc;
            for (int j = 0; j <= std::min(ell - s, (int)B.size() - 1); ++j) {
                if (B[j].num == 0) continue;
                acc = rat_add(acc, rat_mul(B[j], rat_make(C(t - s, j), (__int128)(t - s - j + 1))));
            }
            return acc;
        }
        case TT_FSI_INDEX_FSI: return weight_rational(ell, s, t);
        case TT_FSI_INDEX_SII: return rat_make(1, (__int128)(t - s + 1));
        case TT_FSI_INDEX_BII: return rat_make(1, (__int128)1 << (t - s));
        case TT_FSI_INDEX_STII: {
            if (s != ell) return Rational{};
            const Pascal &C = pascal();
            return rat_make(1, C(t, ell));
        }
    }
    return Rational{};
}

int64_t num_scores(int d, int ell) {
    if (d < 1 || d > 62 || ell < 1) return -1;
    const Pascal &C = pascal();
    int64_t n = 0;
    for (int k = 0; k <= std::min(ell, d); ++k) n += (int64_t)C(d, k);
    return n;
}

namespace {
void emit_grade(int d, int k, int first, uint64_t prefix, uint64_t *out, int64_t &pos) {
    if (k == 0) {
        out[pos++] = prefix;
        return;
    }
    for (int i = first; i <= d - k; ++i) emit_grade(d, k - 1, i + 1, prefix | (1ull << i), out, pos);
}
}  // namespace

void score_masks(int d, int ell, uint64_t *out) {
    int64_t pos = 0;
    for (int k = 0; k <= std::min(ell, d); ++k) emit_grade(d, k, 0, 0, out, pos);
}

tt_fsi_status plan_build_host(Plan &p, int d, int ell, tt_fsi_arith arith, int64_t max_batch,
                              tt_fsi_index index, bool site_sweep, bool precontract) {
    if (d < 1 || ell < 1 || max_batch < 1) return TT_FSI_ERR_INVALID_ARG;
    if (index != TT_FSI_INDEX_FSI && index != TT_FSI_INDEX_SII && index != TT_FSI_INDEX_BII &&
        index != TT_FSI_INDEX_STII && index != TT_FSI_INDEX_KSII)
        return TT_FSI_ERR_INVALID_ARG;
    if (arith != TT_FSI_ARITH_EXACT && arith != TT_FSI_ARITH_F64 && arith != TT_FSI_ARITH_F32)
        return TT_FSI_ERR_INVALID_ARG;
    if (d > 30) return TT_FSI_ERR_UNSUPPORTED;
    p.d = d;
    p.ell = ell;
    p.ell_eff = std::min(ell, d);
    p.index = index;
    p.arith = arith;
    p.max_batch = max_batch;
    // With l >= d, FSI, STII and k-SII leave every Moebius coefficient in place
    // (no superset has more than d >= l players); SII and BII still sum
    // over supersets.
    p.mob_only = ell >= d && (index == TT_FSI_INDEX_FSI || index == TT_FSI_INDEX_STII || index == TT_FSI_INDEX_KSII);
    p.n_out = num_scores(d, ell);
    const size_t elem = (arith == TT_FSI_ARITH_F32) ? 4 : 8;
    const size_t smem_budget = 224 * 1024;  // 227 KB opt-in per CTA, minus static

    // Tile width.  Orders l <= 4 (below d) take the fast path, whose tile is
    // always 12 bits: a game with d < 12 is processed as the 12-player game
    // with 12 - d null players appended (v_ext(S) = v(S n [d])); its
    // Moebius coefficients vanish on every T that contains a null player and
    // Eq. correction's weights depend only on |S| and |T|, so the scores of
    // the sets inside [d] are unchanged.  Otherwise: the largest b <=
    // min(d, 12) whose two ranked-sum buffers fit in shared memory.
    // (site_sweep, precontract: always the site-by-site kernels, as comparison
    // variants; precontract applies only where there are ranked sums)
    const bool want_fast = !site_sweep && !precontract && !p.mob_only && p.ell_eff <= 4;
    p.precontract = precontract && !p.mob_only;
    int b = want_fast ? kMaxTileBits : std::min(d, kMaxTileBits);
    for (;; --b) {
        if (want_fast) {
            p.buf_elems = 1 << b;
            break;
        }
        // state count after k processed bits: sum_{s <= min(k, l)} C(k, s)(k - s + 1)
        const Pascal &C = pascal();
        int64_t peak = (int64_t)1 << b;
        if (!p.mob_only) {
            for (int k = 0; k <= b; ++k) {
                int64_t nk = 0;
                for (int s = 0; s <= std::min(k, p.ell_eff); ++s) nk += (int64_t)C(k, s) * (k - s + 1);
                peak = std::max(peak, nk << (b - k));
            }
        }
        if ((size_t)peak * 2 * elem <= smem_budget || b == 1) {
            p.buf_elems = (int)peak;
            break;
        }
    }
    p.b = b;
    p.h = std::max(0, d - b);
    p.load_bits = std::min(d, b);
    p.smem_tile = (size_t)p.buf_elems * 2 * elem;

    // ---------------- ranked superset states and transitions --------------
    // State at level k: (sigma subset of bits 0..k-1 with |sigma| <= l,
    // j in [0, k - |sigma|]); ordered by (sigma, j).
    std::vector<std::pair<uint32_t, int>> cur{{0u, 0}};
    p.trans.clear();
    p.n_states[0] = 1;
    if (!p.mob_only) {
        for (int k = 0; k < b; ++k) {
            std::map<std::pair<uint32_t, int>, int> idx;
            for (size_t i = 0; i < cur.size(); ++i) idx[cur[i]] = (int)i;
            std::vector<std::pair<uint32_t, int>> nxt;
            for (auto &st : cur) {
                int s = popc64(st.first);
                for (int j = 0; j <= k + 1 - s; ++j) nxt.push_back({st.first, j});
                if (s + 1 <= p.ell_eff)
                    for (int j = 0; j <= k - s; ++j) nxt.push_back({st.first | (1u << k), j});
            }
            std::sort(nxt.begin(), nxt.end());
            nxt.erase(std::unique(nxt.begin(), nxt.end()), nxt.end());
            p.lvl_off[k] = (int)(p.trans.size() / 2);
            for (auto &st : nxt) {
                int src0 = -1, src1 = -1;
                if (st.first >> k & 1u) {
                    // sigma_k = 1 needs tau_k = 1; rank unchanged
                    uint32_t sig = st.first & ~(1u << k);
                    auto it = idx.find({sig, st.second});
                    if (it != idx.end()) src1 = it->second;
                } else {
                    // sigma_k = 0: tau_k = 0 keeps the rank, tau_k = 1 adds one
                    auto it0 = idx.find({st.first, st.second});
                    if (it0 != idx.end()) src0 = it0->second;
                    if (st.second >= 1) {
                        auto it1 = idx.find({st.first, st.second - 1});
                        if (it1 != idx.end()) src1 = it1->second;
                    }
                }
                p.trans.push_back(src0);
                p.trans.push_back(src1);
            }
            cur.swap(nxt);
            p.n_states[k + 1] = (int)cur.size();
        }
        p.lvl_off[b] = (int)(p.trans.size() / 2);
        p.n_ch = p.n_states[b];
    } else {
        p.n_ch = 1 << b;
    }

    // fast tile path: shared-memory regions of fast_layout.h
    if (want_fast) {
        if (fast::n_chan(p.ell_eff) != p.n_ch) return TT_FSI_ERR_UNSUPPORTED;  // layouts disagree
        // the fast launches are sized for chunk mode 1 (the persistent
        // kernels' layout); the tile launch runs mode 2, which must fit in that
        static_assert(fast::regT_elems(1, 2) <= fast::regT_elems(1, 1) && fast::regT_elems(2, 2) <= fast::regT_elems(2, 1) &&
                          fast::regT_elems(3, 2) <= fast::regT_elems(3, 1) && fast::regT_elems(4, 2) <= fast::regT_elems(4, 1),
                      "three round-2 chunks must not need more shared memory than two");
        const bool chunked = arith == TT_FSI_ARITH_EXACT;  // as the kernels' kChunked (mode 1)
        p.fast_regA = fast::reg8_elems(p.ell_eff, chunked);
        p.fast_regB = fast::reg4_elems(p.ell_eff, chunked);
        // tile / chunk states and channels, then the tile's weight rows
        // (int32 or int64 on the exact path, the arithmetic's own type
        // otherwise; int32 rows are sized below once the split is decided)
        const size_t wbytes = (arith == TT_FSI_ARITH_F32) ? 4 : 8;
        p.smem_fast = (size_t)(fast::regT_elems(p.ell_eff, chunked) + p.n_ch) * elem + 16 +
                      (size_t)fast::n_wcombo(p.ell_eff) * fast::kWRow * wbytes;
        p.fast12 = p.smem_fast <= smem_budget;
    }

    // channel base of each low set S_L: index of (S_L, j = 0)
    std::map<uint32_t, int> ch_base;
    if (p.fast12) {
        for (auto &st : cur)
            if (st.second == 0) ch_base[st.first] = fast::channel_base(p.ell_eff, (int)st.first);
    } else if (!p.mob_only) {
        for (size_t i = 0; i < cur.size(); ++i)
            if (cur[i].second == 0) ch_base[cur[i].first] = (int)i;
    }

    // ---------------- combine tasks in output order ----------------------
    std::vector<uint64_t> masks((size_t)p.n_out);
    score_masks(d, ell, masks.data());
    p.tasks.assign((size_t)p.n_out * 4, 0);
    const uint64_t low_mask = (b >= 64) ? ~0ull : ((1ull << b) - 1);
    for (int64_t i = 0; i < p.n_out; ++i) {
        uint64_t S = masks[i];
        uint32_t SL = (uint32_t)(S & low_mask);
        uint32_t SH = (uint32_t)(S >> b);
        int sL = popc64(SL), sH = popc64(SH);
        int base = p.mob_only ? (int)SL : ch_base.at(SL);
        p.tasks[i * 4 + 0] = base;
        p.tasks[i * 4 + 1] = (int32_t)SH;
        p.tasks[i * 4 + 2] = (sL + sH) | (sL << 8) | (sH << 16);
        p.tasks[i * 4 + 3] = 0;
    }
    if (p.fast12) {
        // partial-score entries (S_L, s, i), ordered by (|S_L|, s, channel, i):
        // a warp's entries share |S_L| (the length of their sums) and the i of
        // one (S_L, s) are consecutive, as the combine expects
        std::vector<std::pair<int, uint32_t>> lows;  // (channel base, S_L)
        for (auto &kv : ch_base) lows.push_back({kv.second, kv.first});
        std::sort(lows.begin(), lows.end());
        std::map<std::pair<uint32_t, int>, int> g_of;
        p.gtab.clear();
        for (int sL = 0; sL <= p.ell_eff; ++sL)
            for (int sv = sL; sv <= p.ell_eff; ++sv)
                for (auto &lw : lows) {
                    const uint32_t SL = lw.second;
                    if (popc64(SL) != sL || sv > sL + p.h) continue;
                    g_of[{SL, sv}] = (int)(p.gtab.size() / 2);
                    for (int i = 0; i <= sv - sL; ++i) {
                        p.gtab.push_back((int32_t)lw.first);
                        p.gtab.push_back(sL | (sv << 8) | (i << 16));
                    }
                }
        p.n_g = (int)(p.gtab.size() / 2);
        for (int64_t i = 0; i < p.n_out; ++i) {
            uint64_t S = masks[i];
            uint32_t SL = (uint32_t)(S & low_mask);
            p.tasks[i * 4 + 3] = g_of.at({SL, popc64(S)});
        }
        p.fast12 = p.smem_fast <= smem_budget;
        if (!p.fast12) return TT_FSI_ERR_UNSUPPORTED;  // does not happen for l <= 4
    }

    // ---------------- combined weights omega_s(p, q) ----------------------
    const int S1 = p.ell_eff + 1, P1 = p.h + 1, Q1 = b + 1;
    std::vector<Rational> om((size_t)S1 * P1 * Q1);
    const Pascal &C = pascal();
    for (int s = 0; s < S1; ++s)
        for (int pp = 0; pp < P1; ++pp)
            for (int q = 0; q < Q1; ++q) {
                Rational acc;
                if (!p.mob_only) {
                    for (int n = 0; n <= p.h - pp; ++n) {
                        Rational wv = index_weight(index, ell, s, pp + q + n);
                        if (wv.num == 0) continue;
                        Rational term = rat_mul(wv, rat_make(C(p.h - pp, n), 1));
                        if (n & 1) term.num = -term.num;
                        acc = rat_add(acc, term);
                    }
                }
                om[((size_t)s * P1 + pp) * Q1 + q] = acc;
            }
    p.wf64.resize(om.size());
    p.wf32.resize(om.size());
    for (size_t i = 0; i < om.size(); ++i) {
        p.wf64[i] = (double)om[i].num / (double)om[i].den;
        p.wf32[i] = (float)p.wf64[i];
    }
    p.wnum.assign(om.size(), 0);
    p.wden.assign(S1, 1);
    int max_den_bits = 0;
    for (int s = 0; s < S1; ++s) {
        __int128 L = 1;
        for (int pp = 0; pp < P1; ++pp)
            for (int q = 0; q < Q1; ++q) {
                __int128 dd = om[((size_t)s * P1 + pp) * Q1 + q].den;
                L = L / gcd128(L, dd) * dd;
                if (L > ((__int128)1 << 60)) return TT_FSI_ERR_UNSUPPORTED;
            }
        p.wden[s] = (long long)L;
        int bits = 0;
        while (((__int128)1 << bits) < L) ++bits;
        max_den_bits = std::max(max_den_bits, bits);
        for (int pp = 0; pp < P1; ++pp)
            for (int q = 0; q < Q1; ++q) {
                const Rational &r = om[((size_t)s * P1 + pp) * Q1 + q];
                __int128 v = r.num * (L / r.den);
                if (iabs128(v) >= ((__int128)1 << 62)) return TT_FSI_ERR_UNSUPPORTED;
                p.wnum[((size_t)s * P1 + pp) * Q1 + q] = (long long)v;
            }
    }

    p.winv.resize(S1);
    for (int s = 0; s < S1; ++s) p.winv[s] = 1.0 / (double)p.wden[s];

    // Fixed-point headroom: a tile's ranked sums are bounded by 3^b max|V|
    // (row L1 norm 2^|S_L| C(b-|S_L|, j) 2^j <= 3^b), so |V| < 2^P with
    // P = 62 - ceil(b log2 3) keeps every tile result inside int64.
    p.prec_bits = 62 - (int)std::ceil(b * std::log2(3.0));
    if (p.mob_only) p.prec_bits = 62 - b;
    p.prec_bits = std::min(p.prec_bits, 53);  // never finer than the float64 mantissa
    // the fast tile kernel's branch-free conversion needs P <= 52 (P = 42 at b = 12)
    if (p.fast12 && p.prec_bits > 52) return TT_FSI_ERR_UNSUPPORTED;
    // Cross-tile alignment: a score is at most 2^l max|v| in magnitude (the
    // operator's row L1 norm), so after scaling by 2^shift and the weight
    // denominator it must stay below 2^126.
    p.shift_cap = 124 - p.ell_eff - p.prec_bits - max_den_bits;
    p.shift_cap = std::max(0, std::min(p.shift_cap, 60));

    // Split-product weighting on the fast exact path: a channel Y (|Y| <=
    // 3^12 2^P) is split as Y = Yh 2^31 + Yl, 0 <= Yl < 2^31, so that each
    // weight c times Yh and times Yl is one 32 x 32 -> 64-bit multiply-add.
    // Valid when both int64 sums of at most 13 terms cannot overflow and Yh
    // fits in int32; the weight includes the identity term D_s of j = 0.
    p.g_split31 = false;
    if (p.fast12 && arith == TT_FSI_ARITH_EXACT) {
        long long cmax = 0;
        for (int s = 0; s < S1; ++s)
            for (int pp = 0; pp < P1; ++pp)
                for (int q = 0; q < Q1; ++q) {
                    const long long c = p.wnum[((size_t)s * P1 + pp) * Q1 + q];
                    cmax = std::max(cmax, (c < 0 ? -c : c) + p.wden[s]);
                }
        const __int128 ymax = (__int128)531441 << p.prec_bits;  // 3^12 2^P
        const __int128 yh_max = (ymax >> 31) + 1, lim = (__int128)1 << 63;
        p.g_split31 = cmax < (1ll << 31) && yh_max < ((__int128)1 << 31) &&
                      (__int128)13 * cmax * ((__int128)1 << 31) < lim && (__int128)13 * cmax * yh_max < lim;
    }

    // with the split weighting the rows are int32: the shared-memory size
    // counts them at 4 bytes (three CTAs then share an SM at l <= 3)
    if (p.fast12 && arith == TT_FSI_ARITH_EXACT && p.g_split31)
        p.smem_fast = (size_t)(fast::regT_elems(p.ell_eff, true) + p.n_ch) * elem + 16 +
                      (size_t)fast::n_wcombo(p.ell_eff) * fast::kWRow * 4;

    // Weight rows of the fast path per u_H: row (s, |S_L|, i) holds, for
    // j <= 12 - |S_L|, (-1)^(r - i) [omega_s(u_H + r - i, |S_L| + j) + [i = u_H][j = 0]]
    // (r = s - |S_L|; the identity term is D_s on the exact path), and zeros
    // where no score of such a tile uses the row (i > u_H or r - i > h - u_H).
    p.wstage.clear();
    p.wstage_block = 0;
    if (p.fast12) {
        const int L = p.ell_eff;
        // exact: int32 when the split weighting applies, else int64
        // (|numerator| < 2^62 and D_s < 2^60, so the sum fits)
        const size_t wb = (arith == TT_FSI_ARITH_F32 || (arith == TT_FSI_ARITH_EXACT && p.g_split31)) ? 4 : 8;
        p.wstage_block = (int)((size_t)fast::n_wcombo(L) * fast::kWRow * wb);
        p.wstage.assign((size_t)(p.h + 1) * p.wstage_block, 0);
        for (int uH = 0; uH <= p.h; ++uH)
            for (int s = 0; s <= L; ++s)
                for (int sL = 0; sL <= s; ++sL)
                    for (int i = 0; i <= s - sL; ++i) {
                        const int r = s - sL;
                        if (i > uH || r - i > p.h - uH) continue;
                        const size_t wo = ((size_t)s * P1 + (uH + r - i)) * Q1 + sL;
                        const bool neg = (r - i) & 1, ident = (i == uH);
                        uint8_t *row = p.wstage.data() + (size_t)uH * p.wstage_block +
                                       (size_t)fast::wcombo(s, sL, i) * fast::kWRow * wb;
                        for (int j = 0; j <= b - sL; ++j) {
                            if (arith == TT_FSI_ARITH_EXACT) {
                                long long w = p.wnum[wo + j] + ((j == 0 && ident) ? p.wden[s] : 0);
                                w = neg ? -w : w;
                                if (wb == 4) {
                                    const int32_t c = (int32_t)w;
                                    std::memcpy(row + j * wb, &c, wb);
                                } else {
                                    std::memcpy(row + j * wb, &w, wb);
                                }
                            } else if (arith == TT_FSI_ARITH_F32) {
                                float w = p.wf32[wo + j];
                                if (j == 0 && ident) w += 1.0f;
                                const float c = neg ? -w : w;
                                std::memcpy(row + j * wb, &c, wb);
                            } else {
                                double w = p.wf64[wo + j];
                                if (j == 0 && ident) w += 1.0;
                                const double c = neg ? -w : w;
                                std::memcpy(row + j * wb, &c, wb);
                            }
                        }
                    }
    }
    return TT_FSI_OK;
}

}  // namespace ttfsi

// Host introspection of a plan's combined weights (no device memory).
extern "C" tt_fsi_status tt_fsi_plan_weights(int d, int ell, tt_fsi_index index, int64_t *num, int64_t *den,
                                             int32_t *dims) {
    using namespace ttfsi;
    if (!dims) return TT_FSI_ERR_INVALID_ARG;
    Plan p;
    const tt_fsi_status st = plan_build_host(p, d, ell, TT_FSI_ARITH_EXACT, 1, index);
    if (st != TT_FSI_OK) return st;
    const int S1 = (int)p.wden.size(), P1 = p.h + 1, Q1 = p.b + 1;
    dims[0] = S1;
    dims[1] = P1;
    dims[2] = Q1;
    dims[3] = p.b;
    dims[4] = p.h;
    if (num) std::memcpy(num, p.wnum.data(), p.wnum.size() * sizeof(int64_t));
    if (den) std::memcpy(den, p.wden.data(), p.wden.size() * sizeof(int64_t));
    return TT_FSI_OK;
}
