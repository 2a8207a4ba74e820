// Shared-memory layout of the fast tile path (12-bit tiles, orders l <= 4),
// used by the kernels (as compile-time constants) and by the host plan.
//
// A tile's 12 low bits form three 4-bit groups A (bits 0-3), B (4-7) and
// C (8-11).  The ranked superset sums of Section 3.3 are indexed by the
// absolute rank u = |T n processed bits| (not by |T \ S|), so that each
// group's step is a plain superset sum over 4 bits:
//   level 4:  Z_A(sigma_A, t; tau_B, tau_C)  = sum over tau_A >= sigma_A, |tau_A| = t
//   level 8:  Z_AB(sigma_8, u; tau_C)        = sum over T_8 >= sigma_8, |T_8| = u
//   channels: Z(S_L, u)                      = sum over T_L >= S_L, |T_L| = u
// and the channel of (S_L, j) holds Z(S_L, |S_L| + j).  States are split
// into rounds rd = |sigma_A|; within a round every offset below is a closed
// form in (l, rd, |sigma_B|, |sigma_C|) and the ranks of sigma_A, sigma_B,
// sigma_C among the 4-bit patterns of their popcount.
#pragma once

#if defined(__CUDACC__)
#define TTFSI_HD __host__ __device__
#else
#define TTFSI_HD
#endif

namespace ttfsi {
namespace fast {

constexpr int kBits = 12;

TTFSI_HD constexpr int c4(int k) {
    return k == 0 ? 1 : k == 1 ? 4 : k == 2 ? 6 : k == 3 ? 4 : k == 4 ? 1 : 0;
}
TTFSI_HD constexpr int pc4(int x) { return (x & 1) + ((x >> 1) & 1) + ((x >> 2) & 1) + ((x >> 3) & 1); }
// Rank of a 4-bit pattern among the patterns of its popcount, in increasing
// order (one nibble per pattern: 0,0,1,0,2,1,2,0,3,3,4,1,5,2,3,0).
TTFSI_HD constexpr int rank4(int x) { return (int)((0x0325143302120100ull >> (4 * x)) & 15); }

// level-4 states of round rd: (sigma_A, t), t in [rd, 4]
TTFSI_HD constexpr int n4(int rd) { return c4(rd) * (5 - rd); }

// A round's states can be processed in chunks of consecutive ranks of
// sigma_A, so that only one chunk's level-4 and level-8 states are held in
// shared memory at a time.  Chunk mode CH: 0, every round whole; 1, the
// rounds with 4 or 6 patterns sigma_A (rd = 1, 2) in two chunks; 2, round 1
// in two chunks and round 2 in three, so that a chunk's block-2 items
// (patterns x ranks: 16 and 14) fit one pass of a CTA's 16 half-warps.
// Mode 2 never needs more shared memory than mode 1.
TTFSI_HD constexpr int n_chunks(int rd, int CH) {
    return CH == 0 ? 1 : rd == 1 ? 2 : rd == 2 ? (CH == 2 ? 3 : 2) : 1;
}
TTFSI_HD constexpr int chunk_a(int rd, int CH) { return c4(rd) / n_chunks(rd, CH); }
TTFSI_HD constexpr int n4c_max(int L, int CH) {
    int m = 0;
    for (int rd = 0; rd <= L; ++rd) m = chunk_a(rd, CH) * (5 - rd) > m ? chunk_a(rd, CH) * (5 - rd) : m;
    return m;
}

// level-8 states of round rd, per sigma_A: (sigma_B, u), |sigma_B| = kB <= L - rd,
// u in [rd + kB, 8]; grouped by kB, then rank(sigma_B), then u
TTFSI_HD constexpr int off8(int rd, int kB) {
    return (kB > 0 ? (9 - rd) : 0) + (kB > 1 ? 4 * (8 - rd) : 0) + (kB > 2 ? 6 * (7 - rd) : 0) +
           (kB > 3 ? 4 * (6 - rd) : 0) + (kB > 4 ? (5 - rd) : 0);
}
TTFSI_HD constexpr int s8(int L, int rd) { return off8(rd, L - rd + 1); }
// Row stride of the level-8 region [tau_C][state]: the largest chunk, made
// odd so that both the writes (16 tau_C, one state) and the reads (one
// tau_C, consecutive states) fall on distinct 8-byte bank pairs.
TTFSI_HD constexpr int nst(int L, int CH) {
    int m = 0;
    for (int rd = 0; rd <= L; ++rd) m = chunk_a(rd, CH) * s8(L, rd) > m ? chunk_a(rd, CH) * s8(L, rd) : m;
    return m | 1;
}

// channels: per 8-bit sigma_8 with |sigma_8| = k8 (order O = L - k8 left for
// group C), sigma_C grouped by kC = |sigma_C|, then rank, then j
TTFSI_HD constexpr int offC(int k8, int kC) {
    return (kC > 0 ? (13 - k8) : 0) + (kC > 1 ? 4 * (12 - k8) : 0) + (kC > 2 ? 6 * (11 - k8) : 0) +
           (kC > 3 ? 4 * (10 - k8) : 0) + (kC > 4 ? (9 - k8) : 0);
}
TTFSI_HD constexpr int ch8(int L, int k8) { return offC(k8, L - k8 + 1); }
// channel blocks ordered by round rd, then kB, then (rank sigma_A, rank sigma_B)
TTFSI_HD constexpr int chan_group(int L, int rd, int kB) {
    int o = 0;
    for (int r = 0; r < rd; ++r)
        for (int k = 0; k <= L - r; ++k) o += c4(r) * c4(k) * ch8(L, r + k);
    for (int k = 0; k < kB; ++k) o += c4(rd) * c4(k) * ch8(L, rd + k);
    return o;
}
TTFSI_HD constexpr int n_chan(int L) { return chan_group(L, L + 1, 0); }

// block-3 items of one chunk of round rd and group kB: (rank sigma_A,
// rank sigma_B, u'), u' in [rd + kB, 12]; each group padded to whole warps
TTFSI_HD constexpr int g3(int rd, int kB, int CH) { return chunk_a(rd, CH) * c4(kB) * (13 - rd - kB); }
TTFSI_HD constexpr int pad32(int n) { return (n + 31) & ~31; }

// shared-memory regions in elements: one chunk's level-4 states at offset 0,
// one chunk's level-8 states after them; the tile (4096 elements) overlaps
// both during the Moebius transform; the channels follow.
TTFSI_HD constexpr int reg4_elems(int L, int CH) { return 256 * n4c_max(L, CH); }
TTFSI_HD constexpr int reg8_elems(int L, int CH) { return 16 * nst(L, CH); }
TTFSI_HD constexpr int regT_elems(int L, int CH) {
    return reg4_elems(L, CH) + reg8_elems(L, CH) > 4096 ? reg4_elems(L, CH) + reg8_elems(L, CH) : 4096;
}

// channel of (S_L, j = 0) for a 12-bit low set with |S_L| <= L
TTFSI_HD constexpr int channel_base(int L, int SL) {
    const int a = SL & 15, b = (SL >> 4) & 15, c = (SL >> 8) & 15;
    const int rd = pc4(a), kB = pc4(b), kC = pc4(c), k8 = rd + kB;
    return chan_group(L, rd, kB) + (rank4(a) * c4(kB) + rank4(b)) * ch8(L, k8) + offC(k8, kC) +
           rank4(c) * (13 - k8 - kC);
}

// Per-tile weight rows: one row of kWRow weights per (s, |S_L|, i) with
// s <= L, |S_L| <= s, i <= s - |S_L| (s-major, then |S_L|, then i).
constexpr int kWRow = 16;
TTFSI_HD constexpr int wcombo_base(int s) { return s * (s + 1) * (s + 2) / 6; }
TTFSI_HD constexpr int wcombo(int s, int sL, int i) { return wcombo_base(s) + sL * (s + 1) - sL * (sL - 1) / 2 + i; }
TTFSI_HD constexpr int n_wcombo(int L) { return wcombo_base(L + 1); }

}  // namespace fast
}  // namespace ttfsi
