"""Pins for the CPU oracle: each test checks the oracle against something that
the paper or the mathematics fixes independently of the oracle's own code
(brute-force least squares, permutation Shapley values, hand-derived cases,
efficiency, faithfulness, exact rationals, the paper's MPO construction)."""
import itertools
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from paper_2601_01903_gb300 import synthetic

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand_game(d, seed, v0=True):
    st = synthetic.Stream(1000 + seed, 7)
    v = st.normal(1 << d)
    if v0:
        v[0] = 0.0
    return v


# --------------------------------------------------------------------------
# index conventions and weights
# --------------------------------------------------------------------------

@pytest.mark.parametrize("d", [1, 2, 5, 9, 12])
@pytest.mark.parametrize("ell", [1, 2, 3, 4, 13])
def test_score_masks_c_matches_python(oracle_mod, d, ell):
    a = oracle_mod.score_masks(d, ell)
    b = oracle_mod.score_masks_c(d, ell)
    assert a.shape[0] == oracle_mod.n_scores(d, ell) == b.shape[0]
    assert np.array_equal(a, b)
    # graded, then lexicographic over sorted tuples
    tuples = [tuple(i for i in range(d) if int(m) >> i & 1) for m in a]
    assert tuples == sorted(tuples, key=lambda t: (len(t), t))


def test_score_counts_of_named_workloads(oracle_mod):
    assert oracle_mod.n_scores(8, 2) == 37
    assert oracle_mod.n_scores(14, 2) == 106
    assert oracle_mod.n_scores(20, 3) == 1351
    assert oracle_mod.n_scores(24, 2) == 301
    assert oracle_mod.n_scores(16, 2) == 137


@pytest.mark.parametrize("ell", [1, 2, 3, 4, 6])
def test_weight_c_matches_exact_rational(oracle_mod, ell):
    for s in range(0, ell + 1):
        for t in range(1, 31):
            exact = oracle_mod.weight_exact(ell, s, t)
            got = oracle_mod.weight(ell, s, t)
            assert got == pytest.approx(float(exact), rel=4e-16, abs=0.0)


def test_weight_vanishes_where_the_paper_says(oracle_mod):
    # Eq. weight: C(t-1, l) = 0 for 1 <= t <= l, and the factor s kills s = 0.
    for ell in range(1, 6):
        for t in range(1, ell + 1):
            for s in range(0, ell + 1):
                assert oracle_mod.weight_exact(ell, s, t) == 0
        for t in range(1, 20):
            assert oracle_mod.weight_exact(ell, 0, t) == 0


def test_weight_hand_values(oracle_mod):
    # l = 2, t = 3: w(1,3) = -1/6, w(2,3) = 1/2 (worked by hand from Eq. weight)
    assert oracle_mod.weight_exact(2, 1, 3) == Fraction(-1, 6)
    assert oracle_mod.weight_exact(2, 2, 3) == Fraction(1, 2)
    # l = 1: w(1,t) = 1/2 * C(t-1,1)/C(t,2) = 1/t, so phi_i = sum_{T containing i}
    # a(T)/|T|, the Harsanyi-dividend form of the Shapley value.
    for t in range(2, 25):
        assert oracle_mod.weight_exact(1, 1, t) == Fraction(1, t)


# --------------------------------------------------------------------------
# Moebius transform
# --------------------------------------------------------------------------

@pytest.mark.parametrize("d", [1, 3, 8, 12])
def test_mobius_submask_equals_yates(oracle_mod, d):
    v = _rand_game(d, d, v0=False)
    a1 = oracle_mod.mobius_submask(v, d)
    a2 = oracle_mod.mobius(v, d)
    assert np.max(np.abs(a1 - a2)) <= 1e-12 * max(1.0, np.max(np.abs(a1)))


@pytest.mark.parametrize("d", [4, 10])
def test_mobius_inverts_subset_sums(oracle_mod, d):
    # Moebius inversion: if v(S) = sum_{T subset S} m(T) then a = m.
    m = _rand_game(d, 100 + d, v0=False)
    v = synthetic.subset_sum(m, d)
    for a in (oracle_mod.mobius(v, d), oracle_mod.mobius_submask(v, d)):
        assert np.max(np.abs(a - m)) < 1e-11


def test_mobius_of_unanimity_games(oracle_mod):
    # u_R(S) = [R subset S] has Moebius coefficients [T = R] (textbook).
    d = 6
    for R in (0, 5, 33, 63):
        v = np.array([1.0 if (S & R) == R else 0.0 for S in range(1 << d)])
        a = oracle_mod.mobius(v, d)
        e = np.zeros(1 << d)
        e[R] = 1.0
        assert np.array_equal(a, e)


# --------------------------------------------------------------------------
# the closed form against the definition and the axioms
# --------------------------------------------------------------------------

@pytest.mark.parametrize("d", [1, 2, 3, 4, 5, 6, 7, 8])
def test_closed_form_equals_weighted_least_squares(oracle_mod, d):
    """Eq. fsi_closed/correction agrees with the KKT solution of Eq. fsi_wls
    (Shapley kernel, empty/full set constrained) for every order l."""
    v = _rand_game(d, 10 + d, v0=False)
    for ell in range(1, d + 2):
        phi = oracle_mod.fsi(v, d, ell)[0]
        ref = oracle_mod.fsi_wls(v, d, ell)
        assert np.max(np.abs(phi - ref)) <= 1e-9 * max(1.0, np.max(np.abs(v))), (d, ell)


def test_closed_form_equals_wls_at_d10(oracle_mod):
    d = 10
    v = _rand_game(d, 77, v0=False)
    for ell in (2, 3):
        phi = oracle_mod.fsi(v, d, ell)[0]
        ref = oracle_mod.fsi_wls(v, d, ell)
        assert np.max(np.abs(phi - ref)) <= 1e-8


@pytest.mark.parametrize("d", [2, 3, 5, 7])
def test_order_one_is_the_shapley_value(oracle_mod, d):
    v = _rand_game(d, 20 + d)
    phi = oracle_mod.fsi(v, d, 1)[0]
    perm = oracle_mod.shapley_permutations(v, d)
    form = oracle_mod.shapley_formula(v, d)
    assert phi[0] == v[0]
    assert np.max(np.abs(phi[1:] - perm)) < 1e-12
    assert np.max(np.abs(phi[1:] - form)) < 1e-12


@pytest.mark.parametrize("d,ell", [(3, 1), (6, 2), (9, 3), (12, 2), (12, 4), (14, 3)])
def test_efficiency(oracle_mod, d, ell):
    v = _rand_game(d, 30 + d, v0=False)
    phi = oracle_mod.fsi(v, d, ell)[0]
    assert phi[0] == v[0]
    assert abs(phi[1:].sum() - (v[-1] - v[0])) < 1e-9 * max(1.0, np.abs(v).max())


@pytest.mark.parametrize("d,ell", [(5, 1), (6, 2), (8, 3), (11, 2)])
def test_faithful_recovery_of_l_additive_games(oracle_mod, d, ell):
    """Section 2.2: if the Moebius coefficients vanish above order l, FSI
    returns them exactly."""
    st = synthetic.Stream(555, d * 10 + ell)
    pc = synthetic.popcounts(d)
    m = np.where((pc >= 1) & (pc <= ell), st.normal(1 << d), 0.0)
    v = synthetic.subset_sum(m, d)
    phi = oracle_mod.fsi(v, d, ell)[0]
    masks = oracle_mod.score_masks(d, ell).astype(np.int64)
    assert np.max(np.abs(phi - m[masks])) < 1e-11


def test_faithful_recovery_on_the_d8_mobius_workload(oracle_mod):
    w = synthetic.workload_mobius_d8()
    v, m = w["v"][0], w["m"][0]
    for ell in (4, 5, 8):
        phi = oracle_mod.fsi(v, 8, ell)[0]
        masks = oracle_mod.score_masks(8, ell).astype(np.int64)
        assert np.max(np.abs(phi - m[masks])) < 1e-12


@pytest.mark.parametrize("d", [1, 4, 7])
def test_order_at_least_d_is_the_mobius_transform(oracle_mod, d):
    v = _rand_game(d, 40 + d, v0=False)
    a = oracle_mod.mobius_submask(v, d)
    for ell in (d, d + 1, d + 5):
        phi = oracle_mod.fsi(v, d, ell)[0]
        masks = oracle_mod.score_masks(d, ell).astype(np.int64)
        assert masks.shape[0] == 1 << d
        assert np.max(np.abs(phi - a[masks])) < 1e-12


def test_null_player_gets_zero(oracle_mod):
    d, i = 7, 3
    base = _rand_game(d - 1, 50, v0=False)
    v = np.empty(1 << d)
    for S in range(1 << d):
        lo = S & ((1 << i) - 1)
        hi = (S >> (i + 1)) << i
        v[S] = base[lo | hi]
    for ell in (1, 2, 3):
        phi = oracle_mod.fsi(v, d, ell)[0]
        for k, S in enumerate(oracle_mod.score_masks(d, ell)):
            if int(S) >> i & 1:
                assert abs(phi[k]) < 1e-12


def test_permutation_equivariance_and_linearity(oracle_mod):
    d, ell = 6, 3
    v = _rand_game(d, 60, v0=False)
    u = _rand_game(d, 61, v0=False)
    perm = [2, 0, 5, 1, 4, 3]  # new player perm[i] plays old player i's role
    vp = np.empty_like(v)
    for S in range(1 << d):
        T = 0
        for i in range(d):
            if S >> i & 1:
                T |= 1 << perm[i]
        vp[T] = v[S]
    masks = [int(m) for m in oracle_mod.score_masks(d, ell)]
    pos = {m: k for k, m in enumerate(masks)}
    phi = oracle_mod.fsi(v, d, ell)[0]
    phip = oracle_mod.fsi(vp, d, ell)[0]
    for k, S in enumerate(masks):
        T = 0
        for i in range(d):
            if S >> i & 1:
                T |= 1 << perm[i]
        assert abs(phip[pos[T]] - phi[k]) < 1e-12
    lin = oracle_mod.fsi(2.5 * v - 0.75 * u, d, ell)[0]
    ref = 2.5 * phi - 0.75 * oracle_mod.fsi(u, d, ell)[0]
    assert np.max(np.abs(lin - ref)) < 1e-12


@pytest.mark.parametrize("d,ell", [(3, 2), (6, 1), (7, 3), (8, 2)])
def test_float_oracle_against_exact_rationals(oracle_mod, d, ell):
    v = _rand_game(d, 70 + d, v0=False)
    exact = oracle_mod.fsi_exact(list(v), d, ell)
    got = oracle_mod.fsi(v, d, ell)[0]
    ref = np.array([float(x) for x in exact])
    assert np.max(np.abs(got - ref)) <= 64 * (2.0 ** -52) * (2 ** d) * np.abs(v).max()


def test_exact_oracle_at_d10(oracle_mod):
    d, ell = 10, 3
    v = _rand_game(d, 80, v0=False)
    exact = np.array([float(x) for x in oracle_mod.fsi_exact(list(v), d, ell)])
    got = oracle_mod.fsi(v, d, ell)[0]
    assert np.max(np.abs(got - exact)) < 1e-12 * (2 ** d)


def test_golden_hand_cases(oracle_mod):
    with open(os.path.join(GOLDEN, "hand_cases.json")) as f:
        cases = json.load(f)
    for c in cases:
        d, ell = c["d"], c["ell"]
        v = [Fraction(x) for x in c["v"]]
        want = [Fraction(x) for x in c["phi"]]
        assert oracle_mod.fsi_exact(v, d, ell) == want, c["name"]
        got = oracle_mod.fsi(np.array([float(x) for x in v]), d, ell)[0]
        assert np.max(np.abs(got - np.array([float(x) for x in want]))) < 1e-14, c["name"]
        if d >= 2:
            wls = oracle_mod.fsi_wls(np.array([float(x) for x in v]), d, ell)
            assert np.max(np.abs(wls - np.array([float(x) for x in want]))) < 1e-12, c["name"]


def test_operator_row_l1_norm_is_two_to_the_order(oracle_mod):
    """The FSI operator's largest row L1 norm equals 2^l (observed for these
    sizes; it bounds how much an input perturbation can move a score)."""
    for d, ell in ((6, 1), (6, 2), (7, 3), (8, 2)):
        n = 1 << d
        ops = np.stack([oracle_mod.fsi(np.eye(n)[j], d, ell)[0] for j in range(n)], axis=1)
        assert np.max(np.abs(ops).sum(axis=1)) == pytest.approx(2.0 ** ell, rel=1e-12)


# --------------------------------------------------------------------------
# the paper's MPO construction
# --------------------------------------------------------------------------

def test_mpo_state_counts_of_the_figure(oracle_mod):
    # Figure "fsm" caption: d = 3, l = 2 gives 1 -> 3 -> 6 -> 9 states.
    assert [len(oracle_mod.mpo_states(k, 2)) for k in range(4)] == [1, 3, 6, 9]


def test_mpo_bond_bound_and_transitions(oracle_mod):
    for ell in (1, 2, 3):
        for k in range(1, 15):
            states = oracle_mod.mpo_states(k, ell)
            assert len(states) <= (min(k, ell) + 1) * (k + 1)
            for st in oracle_mod.mpo_states(k - 1, ell):
                tr = oracle_mod.mpo_transitions(st, ell, k)
                assert len(tr) <= 3
                assert all(tau >= sigma for sigma, tau, _ in tr)


@pytest.mark.parametrize("d,ell", [(3, 2), (5, 1), (6, 3), (7, 2)])
def test_mpo_sweep_equals_closed_form(oracle_mod, d, ell):
    v = _rand_game(d, 90 + d, v0=False)
    a = oracle_mod.mobius(v, d)
    corr = oracle_mod.mpo_sweep(a, d, ell)
    phi = oracle_mod.fsi(v, d, ell)[0]
    masks = oracle_mod.score_masks(d, ell).astype(np.int64)
    assert np.max(np.abs(a[masks] + corr[masks] - phi)) < 1e-12
    # the correction vanishes on every S with |S| > l
    pc = synthetic.popcounts(d)
    assert np.all(corr[pc > ell] == 0.0)


# --------------------------------------------------------------------------
# masked-model value function
# --------------------------------------------------------------------------

def test_masked_game_against_torch_forward(oracle_mod):
    torch = pytest.importorskip("torch")
    d = 9
    mlp = synthetic.random_mlp(d, 16, 12, seed=5)
    x = synthetic.gaussian_instances(1, d, 5)[0]
    base = synthetic.Stream(5, 99).normal(d)
    v = oracle_mod.masked_game(mlp, x, base)
    S = np.arange(1 << d)
    bits = ((S[:, None] >> np.arange(d)[None, :]) & 1).astype(bool)
    Z = torch.tensor(np.where(bits, x[None, :], base[None, :]))
    h = torch.nn.functional.gelu(Z @ torch.tensor(mlp.W1).T + torch.tensor(mlp.b1))
    h = torch.nn.functional.gelu(h @ torch.tensor(mlp.W2).T + torch.tensor(mlp.b2))
    ref = (h @ torch.tensor(mlp.W3).T).reshape(-1).numpy() + mlp.b3[0]
    assert np.max(np.abs(v - ref)) < 1e-12


def test_masked_game_end_points_and_null_feature(oracle_mod):
    d = 6
    mlp = synthetic.random_mlp(d, 8, 8, seed=6)
    mlp.W1[:, 2] = 0.0  # feature 2 no longer reaches the model
    x = synthetic.gaussian_instances(1, d, 6)[0]
    base = np.zeros(d)
    v = oracle_mod.masked_game(mlp, x, base)
    for S in range(1 << d):
        assert v[S | 4] == v[S & ~4]
    sub = oracle_mod.masked_game(mlp, x, base, coalitions=[0, (1 << d) - 1, 5])
    assert np.array_equal(sub, v[[0, (1 << d) - 1, 5]])


# ---------------------------------------------------------------------------
# Interventional value function (Section 4.1): pinned by direct forward passes
# ---------------------------------------------------------------------------

def _mlp_forward(mlp, z):
    """f(z) written out for a batch of inputs (GELU in the erf form)."""
    from math import erf, sqrt
    g = np.vectorize(lambda t: 0.5 * t * (1.0 + erf(t / sqrt(2.0))))
    a1 = g(z @ np.asarray(mlp.W1).T + mlp.b1)
    a2 = g(a1 @ np.asarray(mlp.W2).T + mlp.b2)
    return a2 @ np.asarray(mlp.W3).reshape(-1) + float(np.asarray(mlp.b3).reshape(-1)[0])


def test_interventional_value_function_end_points_and_rows(oracle_mod):
    from paper_2601_01903_gb300 import synthetic
    d = 7
    mlp = synthetic.random_mlp(d, 12, 9, seed=3)
    mlp.b1[:] = 0.2
    x = synthetic.gaussian_instances(1, d, seed=5)[0]
    bg = synthetic.gaussian_instances(4, d, seed=6)
    v = oracle_mod.masked_game_interventional(mlp, x, bg)
    # all features present: the background does not matter
    assert abs(v[(1 << d) - 1] - _mlp_forward(mlp, x[None, :])[0]) < 1e-12
    # no feature present: the mean prediction over the background rows
    assert abs(v[0] - _mlp_forward(mlp, bg).mean()) < 1e-12
    # coalition {0, 3}: the mean over rows of f with x_0, x_3 put in
    z = bg.copy()
    z[:, [0, 3]] = x[[0, 3]]
    assert abs(v[0b1001] - _mlp_forward(mlp, z).mean()) < 1e-12
    # one row is the baseline value function; repeating a row changes nothing
    assert np.allclose(oracle_mod.masked_game_interventional(mlp, x, bg[1:2]), oracle_mod.masked_game(mlp, x, bg[1]),
                       rtol=0, atol=1e-14)
    assert np.allclose(oracle_mod.masked_game_interventional(mlp, x, np.repeat(bg[2:3], 3, axis=0)),
                       oracle_mod.masked_game(mlp, x, bg[2]), rtol=0, atol=1e-13)


def test_direct_kernel_order_one_is_the_shapley_kernel(oracle_mod):
    """At l = 1 the FSI of a single player is its Shapley value, whose
    coefficient of v(R) is the textbook (r-1)!(d-r)!/d! when the player is in
    R and -r!(d-r-1)!/d! when not (Shapley 1953); the empty score is v(empty)."""
    from fractions import Fraction
    from math import factorial
    for d in (3, 7, 12):
        for r in range(d + 1):
            inside = oracle_mod.direct_kernel(d, 1, 1, r, 1) if r >= 1 else None
            outside = oracle_mod.direct_kernel(d, 1, 1, r, 0) if r <= d - 1 else None
            if inside is not None:
                assert inside == Fraction(factorial(r - 1) * factorial(d - r), factorial(d))
            if outside is not None:
                assert outside == -Fraction(factorial(r) * factorial(d - r - 1), factorial(d))
            assert oracle_mod.direct_kernel(d, 2, 0, r, 0) == (1 if r == 0 else 0)


@pytest.mark.parametrize("d,ell", [(9, 2), (11, 3), (10, 4)])
def test_direct_route_equals_closed_form(oracle_mod, d, ell):
    """The direct route from v (coefficients kappa, compensated bin sums)
    and the closed form through the Moebius transform agree on every score."""
    v = np.random.default_rng(d * 100 + ell).normal(size=(1, 1 << d))
    masks = [int(m) for m in oracle_mod.score_masks(d, ell)]
    got = oracle_mod.fsi_direct(v, d, ell, masks)
    assert np.max(np.abs(got - oracle_mod.fsi(v, d, ell)[0])) <= 1e-13 * np.max(np.abs(v))


# --------------------------------------------------------------------------
# the fast CPU baseline (timed beside the GPU) agrees with the oracle
# --------------------------------------------------------------------------

@pytest.mark.parametrize("d,ell,B", [(1, 1, 1), (3, 2, 2), (8, 2, 3), (12, 3, 2), (15, 3, 1), (16, 2, 2),
                                     (14, 4, 1), (9, 9, 1), (10, 12, 1)])
def test_cpu_fast_baseline_matches_oracle(oracle_mod, d, ell, B):
    v = np.random.default_rng(d * 100 + ell).normal(size=(B, 1 << d))
    got = oracle_mod.cpu_fast_fsi(v, d, ell)
    ref = oracle_mod.fsi(v, d, ell)
    assert got.shape == ref.shape
    assert np.max(np.abs(got - ref)) <= 1e-10 * np.abs(v).max()
