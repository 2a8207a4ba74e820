"""Pins of the oracle's other interaction indices (Appendix A: SII, Banzhaf
BII, Shapley-Taylor STII), computed there from their definitions over
discrete derivatives.  Each is checked against facts fixed by the
mathematics, not against its own formula:

* unanimity games u_R (u_R(T) = 1 if R is a subset of T): every index is
  linear and is determined by its values on them -- SII_S(u_R) =
  1/(|R|-|S|+1), BII_S(u_R) = 2^-(|R|-|S|) for S inside R (Grabisch 1997);
  STII_S(u_R) = [S = R] for |S| < l and 1/C(|R|, l) for |S| = l inside R
  (Sundararajan, Dhamdhere and Agarwal 2020); 0 when S is not inside R;
* SII on singletons and STII of order 1 are the Shapley value (brute force
  over all player orders);
* STII is efficient: its scores of the non-empty S sum to v(N) - v(empty);
* the Moebius form the CUDA path evaluates, sum over T containing S of
  W(|S|, |T|) a(T), equals the definition on random games;
* k-SII (given in Appendix A by its purpose and its efficiency only): the
  hand-derived values of tests/golden/ksii_cases.json, efficiency, order 1
  = Shapley value, top order = SII, exact recovery of l-additive games.
"""
from fractions import Fraction
from math import comb

import numpy as np
import pytest

pytestmark = pytest.mark.filterwarnings("ignore")


def _unanimity(d, R):
    return np.array([1.0 if (T & R) == R else 0.0 for T in range(1 << d)])


def _pc(x):
    return bin(int(x)).count("1")


def _expected_unanimity(index, R, S, ell):
    r, s = _pc(R), _pc(S)
    if (S & R) != S:
        return 0.0
    if index == "sii":
        return 1.0 / (r - s + 1)
    if index == "bii":
        return 2.0 ** -(r - s)
    if s < ell:
        return 1.0 if S == R else 0.0
    return 1.0 / comb(r, ell)


@pytest.mark.parametrize("index", ["sii", "bii", "stii"])
@pytest.mark.parametrize("d,ell", [(6, 2), (7, 3), (5, 5)])
def test_unanimity_games(oracle_mod, index, d, ell):
    masks = oracle_mod.score_masks(d, ell)
    for R in [0b1, 0b11, 0b101, 0b1011, 0b10111, (1 << d) - 1, 0]:
        R &= (1 << d) - 1
        got = oracle_mod.interaction(_unanimity(d, R), d, ell, index)[0]
        exp = np.array([_expected_unanimity(index, R, int(S), ell) for S in masks])
        assert np.max(np.abs(got - exp)) < 1e-13, (index, R)


def test_sii_singletons_are_shapley_values(oracle_mod):
    d = 6
    v = np.random.default_rng(3).normal(size=1 << d)
    sv = oracle_mod.shapley_permutations(v, d)
    got = oracle_mod.interaction(v, d, 2, "sii")[0]
    assert np.max(np.abs(got[1:d + 1] - sv)) < 1e-12


def test_stii_order_one_is_shapley_value(oracle_mod):
    d = 7
    v = np.random.default_rng(4).normal(size=1 << d)
    sv = oracle_mod.shapley_permutations(v, d)
    got = oracle_mod.interaction(v, d, 1, "stii")[0]
    assert got[0] == v[0]
    assert np.max(np.abs(got[1:] - sv)) < 1e-12


@pytest.mark.parametrize("d,ell", [(6, 2), (8, 3), (7, 4)])
def test_stii_is_efficient(oracle_mod, d, ell):
    v = np.random.default_rng(d * 10 + ell).normal(size=1 << d)
    got = oracle_mod.interaction(v, d, ell, "stii")[0]
    assert abs(got[1:].sum() - (v[-1] - v[0])) < 1e-11


def _mobius_form(a, d, ell, index):
    """sum_{T >= S} W(|S|, |T|) a(T) with the Moebius-form weights, exact."""
    out = []
    for S in range(1 << d):
        s = _pc(S)
        if s > ell:
            continue
        acc = Fraction(0)
        for T in range(1 << d):
            if (T & S) != S:
                continue
            t = _pc(T)
            if index == "sii":
                w = Fraction(1, t - s + 1)
            elif index == "bii":
                w = Fraction(1, 2 ** (t - s))
            elif index == "ksii":
                # W(s, s) = 1; 0 for s < t <= l (the Bernoulli sums cancel);
                # sum_j C(t-s, j) B_j / (t-s-j+1) over j <= l - s for t > l
                B = oracle_mod_bernoulli(ell)
                if t == s:
                    w = Fraction(1)
                elif s == 0 or t <= ell:
                    w = Fraction(0)
                else:
                    w = sum(comb(t - s, j) * B[j] / (t - s - j + 1) for j in range(ell - s + 1))
            else:
                w = Fraction(int(T == S)) if s < ell else Fraction(1, comb(t, ell))
            acc += w * Fraction(a[T])
        out.append((S, float(acc)))
    return dict(out)


def oracle_mod_bernoulli(n):
    import oracle
    return oracle.bernoulli(n)


@pytest.mark.parametrize("index", ["sii", "bii", "stii", "ksii"])
def test_definition_equals_mobius_form(oracle_mod, index):
    d, ell = 6, 3
    v = np.random.default_rng(11).normal(size=1 << d)
    a = oracle_mod.mobius_submask(v, d)
    ref = _mobius_form(a, d, ell, index)
    got = oracle_mod.interaction(v, d, ell, index)[0]
    exp = np.array([ref[int(S)] for S in oracle_mod.score_masks(d, ell)])
    assert np.max(np.abs(got - exp)) < 1e-12


def test_fsi_route_is_the_closed_form(oracle_mod):
    v = np.random.default_rng(5).normal(size=(2, 1 << 7))
    assert np.array_equal(oracle_mod.interaction(v, 7, 2, "fsi"), oracle_mod.fsi(v, 7, 2))


# --------------------------------------------------------------------------
# k-SII (Appendix A): pinned by hand-derived unanimity values, the
# efficiency the paper states for it, its reductions to the Shapley value
# (order 1) and to SII (top order), and exact recovery of l-additive games
# --------------------------------------------------------------------------

def test_bernoulli_numbers_are_the_textbook_values(oracle_mod):
    B = oracle_mod.bernoulli(8)
    assert B == [Fraction(1), Fraction(-1, 2), Fraction(1, 6), 0, Fraction(-1, 30), 0, Fraction(1, 42), 0,
                 Fraction(-1, 30)]


def test_ksii_golden_cases(oracle_mod):
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "ksii_cases.json")) as f:
        cases = json.load(f)
    for c in cases:
        d, ell = c["d"], c["ell"]
        v = np.array([float(Fraction(x)) for x in c["v"]])
        want = np.array([float(Fraction(x)) for x in c["phi"]])
        got = oracle_mod.interaction(v, d, ell, "ksii")[0]
        assert np.max(np.abs(got - want)) < 1e-14, c["name"]
        # the fixtures themselves satisfy the efficiency the paper states
        assert sum(Fraction(x) for x in c["phi"][1:]) == Fraction(c["v"][-1]) - Fraction(c["v"][0])


@pytest.mark.parametrize("d,ell", [(6, 2), (8, 3), (7, 4), (5, 5), (9, 1)])
def test_ksii_is_efficient(oracle_mod, d, ell):
    v = np.random.default_rng(d * 13 + ell).normal(size=(2, 1 << d))
    got = oracle_mod.interaction(v, d, ell, "ksii")
    assert np.array_equal(got[:, 0], v[:, 0])
    assert np.max(np.abs(got[:, 1:].sum(axis=1) - (v[:, -1] - v[:, 0]))) < 1e-11


def test_ksii_order_one_is_shapley_value(oracle_mod):
    d = 7
    v = np.random.default_rng(17).normal(size=1 << d)
    sv = oracle_mod.shapley_permutations(v, d)
    got = oracle_mod.interaction(v, d, 1, "ksii")[0]
    assert np.max(np.abs(got[1:] - sv)) < 1e-12


def test_ksii_top_order_is_sii(oracle_mod):
    d, ell = 7, 3
    v = np.random.default_rng(19).normal(size=1 << d)
    got = oracle_mod.interaction(v, d, ell, "ksii")[0]
    sii = oracle_mod.interaction(v, d, ell, "sii")[0]
    top = [k for k, S in enumerate(oracle_mod.score_masks(d, ell)) if _pc(S) == ell]
    assert np.array_equal(got[top], sii[top])


@pytest.mark.parametrize("ell", [2, 3])
def test_ksii_recovers_l_additive_games(oracle_mod, ell):
    """A game whose Moebius coefficients vanish above order l keeps them as
    its k-SII scores (the Bernoulli sums cancel every lower-order term)."""
    d = 7
    rng = np.random.default_rng(23 + ell)
    m = np.zeros(1 << d)
    for T in range(1, 1 << d):
        if _pc(T) <= ell:
            m[T] = rng.normal()
    v = np.array([sum(m[R] for R in range(1 << d) if (R & T) == R) for T in range(1 << d)])
    got = oracle_mod.interaction(v, d, ell, "ksii")[0]
    want = m[oracle_mod.score_masks(d, ell).astype(np.int64)]
    assert np.max(np.abs(got - want)) < 1e-12
