"""The plan's host arithmetic, on the CPU: every score rebuilt from the tile
decomposition the kernels evaluate, with the plan's own combined weights,
equals the oracle.  A tile of 2^b coalitions with high pattern U_H (u_H set
bits) contributes to S = S_L u S_H (|S| = s, r = |S_H|, i = |U_H n S_H|)
    (-1)^(r - i) sum_j [omega_s(u_H + r - i, |S_L| + j) + [i = u_H][j = 0]] Y(S_L, j),
Y(S_L, j) the sum over T_L >= S_L, |T_L| = |S_L| + j, of the tile's own
Moebius coefficients (over its b low players only; the high players'
Moebius step is folded into omega).  Games with small integer values keep every Moebius
coefficient and channel an exact integer, and Python integers carry the
weighted sums, so the rebuilt scores are exact rationals before the final
division."""
from fractions import Fraction

import numpy as np
import pytest

import paper_2601_01903_gb300 as fsi


def _mobius_int(v, n_bits):
    a = v.astype(np.int64).copy()
    for k in range(n_bits):
        a = a.reshape(-1, 2, 1 << k)
        a[:, 1, :] -= a[:, 0, :]
        a = a.reshape(-1)
    return a


def _rebuilt_scores(v, d, ell, index):
    num, den, b, h = fsi.plan_weights(d, ell, index)
    # games below b players are padded with null players
    n = 1 << (b + h)
    full = np.arange(n)
    v_ext = v[full & ((1 << d) - 1)] if d < b + h else v
    pc = np.array([bin(x).count("1") for x in range(1 << b)])
    T = np.arange(1 << b)
    masks = [int(m) for m in fsi.score_masks(d, ell)]
    low = (1 << b) - 1
    num_py = [[[int(x) for x in row] for row in plane] for plane in num]
    den_py = [int(x) for x in den]
    acc = [0] * len(masks)
    for U in range(1 << h):
        uH = bin(U).count("1")
        tile = _mobius_int(v_ext[U << b:(U + 1) << b], b)
        Y = {}
        for S in masks:
            SL = S & low
            if SL not in Y:
                sel = (T & SL) == SL
                sL = bin(SL).count("1")
                y = np.bincount(pc[sel] - sL, weights=tile[sel].astype(np.float64), minlength=b + 1 - sL)
                Y[SL] = [int(round(x)) for x in y]
        for k, S in enumerate(masks):
            SL, SH = S & low, S >> b
            sL, r, i = bin(SL).count("1"), bin(SH).count("1"), bin(U & SH).count("1")
            s = sL + r
            if i > uH or r - i > h - uH:
                continue
            w = num_py[s][uH + r - i]
            g = sum((w[sL + j] + (den_py[s] if (i == uH and j == 0) else 0)) * Y[SL][j] for j in range(b + 1 - sL))
            acc[k] += -g if (r - i) % 2 else g
    return np.array([float(Fraction(acc[k], den_py[bin(S).count("1")])) for k, S in enumerate(masks)])


@pytest.mark.parametrize("d,ell,index", [
    (10, 2, "fsi"),    # fewer players than a tile: null-player padding, h = 0
    (13, 2, "fsi"), (14, 3, "fsi"), (15, 1, "fsi"), (13, 4, "fsi"),
    (14, 2, "sii"), (14, 2, "bii"), (13, 3, "stii"),
    (14, 3, "ksii"), (13, 2, "ksii"), (12, 4, "ksii"), (15, 1, "ksii"),
])
def test_tile_decomposition_with_plan_weights_equals_oracle(oracle_mod, d, ell, index):
    v = np.random.default_rng(d * 31 + ell).integers(-3, 4, size=1 << d).astype(np.float64)
    got = _rebuilt_scores(v, d, ell, index)
    ref = oracle_mod.interaction(v.reshape(1, -1), d, ell, index)[0]
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(v))


def test_plan_weights_reject_bad_arguments():
    with pytest.raises(RuntimeError):
        fsi.plan_weights(0, 2)
