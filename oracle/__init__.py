"""CPU oracle for Faithful Shapley Interactions -- TEST INFRASTRUCTURE ONLY.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The library (``paper_2601_01903_gb300``)
never imports, links or calls it, and the two share no code: the oracle's C
core (``fsi_oracle.c``) and the pure-Python routines below are written
straight from the paper (Kim & Lee, "TT-FSI: Scalable Faithful Shapley
Interactions via Tensor-Train"), each citing the passage it follows.

What is here:

* ``fsi`` -- the closed form (Eq. fsi_closed with Eq. correction and
  Eq. weight), float64, Moebius by the per-player Kronecker factors and the
  correction by explicit superset enumeration (C, OpenMP over outputs).
* ``fsi_direct`` -- listed scores straight from v: the closed form with
  a = Moebius(v) substituted, phi(S) = sum over R of kappa(|S|, |R|, |S n R|)
  v(R), kappa exact in rationals, v summed per (|R|, |S n R|) bin with
  compensated sums (C).  Accurate at large d, where the float64 Moebius
  coefficients lose digits to cancellation.
* ``fsi_exact`` -- the same closed form in exact rational arithmetic
  (Python ``fractions``), Moebius by explicit submask sums; d <= 10.
* ``fsi_wls`` -- the defining weighted least-squares problem (Eq. fsi_wls)
  solved directly through its KKT system, with the Shapley kernel weights and
  the empty/full-set equality constraints (the paper leaves the weights
  unprinted, "derived from Shapley's axioms"; this reading is pinned by tests
  against the closed form); d <= 10.
* ``shapley_permutations`` -- Shapley values (Section 2.1 equation) by
  enumerating every player order; d <= 8.
* ``interaction`` -- the other indices of Appendix A (SII, Banzhaf BII,
  Shapley-Taylor STII) by their definitions over discrete derivatives (C),
  and k-SII (``ksii``) as the Bernoulli-number aggregation of those SII
  scores (pure Python over the score list).
* ``masked_game`` -- the model value function with absent features set to a
  baseline, one forward pass per coalition (C).
* ``cpu_fast_fsi`` -- not the oracle: the timed fast CPU baseline
  (``fsi_cpu_fast.c``), checked against ``fsi`` by the tests.
* ``mpo_sweep`` -- the paper's own route (Section 3.3 MPO with Algorithm 1's
  left-to-right sweep), pure Python over explicit states; used only to check
  the paper's structural claims (state counts, transitions) and that the
  MPO and the closed form agree.

Parity status: every function above is pinned by tests in ``tests/`` against
something other than itself (brute-force least squares, permutation Shapley
values, hand-derived small cases, efficiency, faithfulness on l-additive
games, exact rationals).  The student-network helpers in ``student.py`` are
pinned by finite differences and closed forms.
"""
from __future__ import annotations

import ctypes
import itertools
import math
import os
import subprocess
import threading
from fractions import Fraction
from typing import List, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fsi_oracle.c")
_FAST_SRC = os.path.join(_HERE, "fsi_cpu_fast.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_FAST_PATH = os.path.join(_BUILD, "libcpufast.so")
_lock = threading.Lock()
_lib = None
_fast = None


def _compile(src: str, out: str, flags, force: bool):
    stale = (not os.path.exists(out)) or os.path.getmtime(out) < os.path.getmtime(src)
    if force or stale:
        tmp = out + f".{os.getpid()}.tmp"
        subprocess.run(["gcc"] + list(flags) + ["-fPIC", "-shared", "-std=c11", "-o", tmp, src, "-lm"],
                       check=True)
        os.replace(tmp, out)


def build(force: bool = False) -> str:
    """Compile the C core with gcc (OpenMP, no fused multiply-add), and the
    fast CPU baseline (fsi_cpu_fast.c, -O3, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    _compile(_SRC, _LIB_PATH, ["-O2", "-fopenmp", "-ffp-contract=off"], force)
    _compile(_FAST_SRC, _FAST_PATH, ["-O3", "-fopenmp"], force)
    return _LIB_PATH


def cpu_fast_fsi(v, d: int, ell: int) -> np.ndarray:
    """FSI scores [B, n_scores] by the fast CPU program of fsi_cpu_fast.c
    (Moebius butterflies, weighted pruned superset sums; float64, OpenMP over
    games) -- the timed CPU baseline, not the oracle; the tests check it
    against ``fsi``."""
    global _fast
    with _lock:
        if _fast is None:
            build()
            lib = ctypes.CDLL(_FAST_PATH)
            lib.cpu_fast_fsi.restype = ctypes.c_int
            lib.cpu_fast_fsi.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p,
                                         ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]
            _fast = lib
    v = _as_games(v, d)
    m = score_masks(d, ell)
    out = np.empty((v.shape[0], m.shape[0]), dtype=np.float64)
    if _fast.cpu_fast_fsi(d, ell, v.shape[0], _ptr(v), m.shape[0], _ptr(m), _ptr(out)) != 0:
        raise RuntimeError("cpu_fast_fsi failed")
    return out


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            d, i, i64, p = ctypes.c_double, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p
            lib.oracle_weight.restype = d
            lib.oracle_weight.argtypes = [i, i, i]
            lib.oracle_bin_sums.restype = None
            lib.oracle_bin_sums.argtypes = [i, i, p, i64, p, p]
            lib.oracle_num_scores.restype = i64
            lib.oracle_num_scores.argtypes = [i, i]
            lib.oracle_score_masks.restype = i64
            lib.oracle_score_masks.argtypes = [i, i, p]
            lib.oracle_mobius_submask.restype = None
            lib.oracle_mobius_submask.argtypes = [i, p, p]
            lib.oracle_mobius_yates.restype = None
            lib.oracle_mobius_yates.argtypes = [i, p, p]
            lib.oracle_fsi_from_mobius.restype = None
            lib.oracle_fsi_from_mobius.argtypes = [i, i, p, i64, p, p]
            lib.oracle_fsi.restype = i
            lib.oracle_fsi.argtypes = [i, i, i64, p, p]
            lib.oracle_masked_game.restype = None
            lib.oracle_masked_game.argtypes = [i, i, i, p, p, p, p, p, d, p, p, i64, p, p]
            lib.oracle_num_threads.restype = i
            lib.oracle_num_threads.argtypes = []
            lib.oracle_index_definition.restype = i
            lib.oracle_index_definition.argtypes = [i, i, i, i64, p, p]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def num_threads() -> int:
    """Threads the C core's parallel loops use on this host."""
    return int(_load().oracle_num_threads())


# ---------------------------------------------------------------------------
# Index conventions
# ---------------------------------------------------------------------------

def n_scores(d: int, ell: int) -> int:
    """sum_{k <= min(l, d)} C(d, k): one score per S with |S| <= l."""
    return sum(math.comb(d, k) for k in range(min(ell, d) + 1))


def score_masks(d: int, ell: int) -> np.ndarray:
    """Coalition masks of the score columns: graded by |S|, lexicographic
    over sorted player tuples inside a grade (pure Python)."""
    out = []
    for k in range(min(ell, d) + 1):
        for comb in itertools.combinations(range(d), k):
            m = 0
            for i in comb:
                m |= 1 << i
            out.append(m)
    return np.array(out, dtype=np.uint64)


def score_masks_c(d: int, ell: int) -> np.ndarray:
    n = int(_load().oracle_num_scores(d, ell))
    out = np.empty(n, dtype=np.uint64)
    _load().oracle_score_masks(d, ell, _ptr(out))
    return out


# ---------------------------------------------------------------------------
# Weights (Eq. weight)
# ---------------------------------------------------------------------------

def weight_exact(ell: int, s: int, t: int) -> Fraction:
    """w(s,t) = (-1)^(l-s) s/(l+s) C(l,s) C(t-1,l)/C(t+l-1,l+s), Eq. weight
    (Section 3.3), as an exact rational."""
    if t < 1 or s == 0 or s > ell or math.comb(t - 1, ell) == 0:
        return Fraction(0)  # factor s, C(l,s) = 0 for s > l, C(t-1,l) = 0 for t <= l
    sign = -1 if (ell - s) % 2 else 1
    return sign * Fraction(s, ell + s) * math.comb(ell, s) * Fraction(
        math.comb(t - 1, ell), math.comb(t + ell - 1, ell + s))


def weight(ell: int, s: int, t: int) -> float:
    """Float64 value of w(s,t) from the C core."""
    return float(_load().oracle_weight(ell, s, t))


# ---------------------------------------------------------------------------
# Moebius transform and FSI (C core)
# ---------------------------------------------------------------------------

def _as_games(v, d: int) -> np.ndarray:
    v = np.ascontiguousarray(v, dtype=np.float64)
    if v.ndim == 1:
        v = v.reshape(1, -1)
    if v.shape[-1] != (1 << d):
        raise ValueError(f"value vectors must have 2^{d} entries")
    return v


def mobius_submask(v, d: int) -> np.ndarray:
    """a(S) = sum_{T subset S} (-1)^(|S|-|T|) v(T) by explicit submask sums
    (Eq. fsi_closed); one game."""
    v = _as_games(v, d)[0]
    a = np.empty_like(v)
    _load().oracle_mobius_submask(d, _ptr(v), _ptr(a))
    return a


def mobius(v, d: int) -> np.ndarray:
    """Moebius transform through the per-player Kronecker factors (Section
    3.2); one game."""
    v = _as_games(v, d)[0]
    a = np.empty_like(v)
    _load().oracle_mobius_yates(d, _ptr(v), _ptr(a))
    return a


def fsi(v, d: int, ell: int) -> np.ndarray:
    """FSI scores [B, n_scores] of games v [B, 2^d] (closed form, float64)."""
    if ell < 1:
        raise ValueError("interaction order must be >= 1")
    v = _as_games(v, d)
    out = np.empty((v.shape[0], n_scores(d, ell)), dtype=np.float64)
    rc = _load().oracle_fsi(d, ell, v.shape[0], _ptr(v), _ptr(out))
    if rc != 0:
        raise RuntimeError("oracle_fsi failed")
    return out


def fsi_at(v, d: int, ell: int, masks: Sequence[int]) -> np.ndarray:
    """Scores of the listed coalitions only (each |S| <= l) for one game."""
    v = _as_games(v, d)[0]
    a = mobius(v, d)
    m = np.ascontiguousarray(np.asarray(masks, dtype=np.uint64))
    out = np.empty(m.shape[0], dtype=np.float64)
    _load().oracle_fsi_from_mobius(d, ell, _ptr(a), m.shape[0], _ptr(m), _ptr(out))
    return out


def direct_kernel(d: int, ell: int, s: int, r: int, q: int) -> Fraction:
    """kappa(s, r, q): the coefficient of v(R) in phi(S) for |S| = s,
    |R| = r, |S n R| = q.  Substituting a(T) = sum over R <= T of
    (-1)^(|T| - |R|) v(R) into phi(S) = sum over T >= S of W(s, |T|) a(T)
    (Eq. fsi_closed with Eq. correction: W(s, s) = 1, W(s, t) = w(s, t) of
    Eq. weight for t > l, 0 otherwise) and counting the C(d - u, m) sets T
    of size u + m that contain S u R (u = s + r - q) gives
        kappa = sum over m of (-1)^(u + m - r) C(d - u, m) W(s, u + m),
    exact in rationals."""
    u = s + r - q
    acc = Fraction(0)
    for m in range(d - u + 1):
        t = u + m
        W = Fraction(1) if t == s else (weight_exact(ell, s, t) if t > ell else Fraction(0))
        if W:
            term = math.comb(d - u, m) * W
            acc += term if (u + m - r) % 2 == 0 else -term
    return acc


def fsi_direct(v, d: int, ell: int, masks: Sequence[int]) -> np.ndarray:
    """Listed scores of one game straight from v, without a Moebius
    transform: phi(S) = sum over (r, q) of kappa(|S|, r, q) times the sum of
    v(R) over |R| = r, |R n S| = q (compensated sums in C, then one
    correctly rounded sum of the weighted bins).  Its error does not grow
    with the cancellation inside the Moebius coefficients, which the
    Moebius route (``fsi_at``) suffers at large d."""
    v = _as_games(v, d)[0]
    m = np.ascontiguousarray(np.asarray(masks, dtype=np.uint64))
    nb = (d + 1) * (ell + 1)
    bins = np.empty((m.shape[0], nb), dtype=np.float64)
    _load().oracle_bin_sums(d, ell, _ptr(v), m.shape[0], _ptr(m), _ptr(bins))
    kap = {}
    out = np.empty(m.shape[0], dtype=np.float64)
    for k in range(m.shape[0]):
        s = _popcount(int(m[k]))
        terms = []
        for r in range(d + 1):
            for q in range(min(s, r) + 1):
                key = (s, r, q)
                if key not in kap:
                    kap[key] = direct_kernel(d, ell, s, r, q)
                if kap[key]:
                    terms.append(float(kap[key] * Fraction(float(bins[k, r * (ell + 1) + q]))))
        out[k] = math.fsum(terms)
    return out


def fsi_from_mobius(a, d: int, ell: int) -> np.ndarray:
    a = _as_games(a, d)[0]
    m = score_masks(d, ell)
    out = np.empty(m.shape[0], dtype=np.float64)
    _load().oracle_fsi_from_mobius(d, ell, _ptr(a), m.shape[0], _ptr(m), _ptr(out))
    return out


INDEX_CODES = {"sii": 1, "bii": 2, "stii": 3}


def bernoulli(n: int) -> List[Fraction]:
    """Bernoulli numbers B_0 .. B_n as exact rationals, from their defining
    recurrence sum_{j=0}^{m} C(m+1, j) B_j = 0 for m >= 1, B_0 = 1 (which
    gives the convention B_1 = -1/2)."""
    B = [Fraction(1)]
    for m in range(1, n + 1):
        B.append(-sum(math.comb(m + 1, j) * B[j] for j in range(m)) / (m + 1))
    return B


def ksii(v, d: int, ell: int) -> np.ndarray:
    """k-SII of order l (Appendix A, "k-SII": higher-order SII terms are
    aggregated into the scores of order <= l so that the scores become
    efficient).  The paper prints no formula; the aggregation taken here is
    the Bernoulli one of the k-SII literature,
        I(S) = sum over T containing S with |T| <= l of B_{|T|-|S|} SII(T)
    for 1 <= |S| <= l (B_1 = -1/2), SII(T) from ``interaction`` (the
    Appendix A definition over discrete derivatives), and I(empty) = v(empty)
    as for FSI, so that the non-empty scores sum to v(N) - v(empty)."""
    if ell < 1:
        raise ValueError("interaction order must be >= 1")
    v = _as_games(v, d)
    sii = interaction(v, d, ell, "sii")
    masks = score_masks(d, ell).astype(np.int64)
    pc = np.array([_popcount(int(m)) for m in masks])
    B = [float(b) for b in bernoulli(min(ell, d))]
    # M[i, j] = B_{|T_j| - |S_i|} where T_j contains S_i
    sup = (masks[None, :] & masks[:, None]) == masks[:, None]
    M = np.zeros((masks.shape[0], masks.shape[0]))
    rows, cols = np.nonzero(sup)
    M[rows, cols] = [B[pc[j] - pc[i]] for i, j in zip(rows, cols)]
    out = sii @ M.T
    out[:, 0] = v[:, 0]
    return out


def interaction(v, d: int, ell: int, index: str) -> np.ndarray:
    """Scores [B, n_scores] of the interaction index ``index`` ("fsi",
    "sii", "bii", "stii" or "ksii") of games v [B, 2^d].  FSI by its closed
    form (``fsi``); SII, BII and STII by their definitions of Appendix A over
    discrete derivatives (C, O(n_scores 2^d) per game, d <= 16 in practice);
    k-SII by ``ksii``."""
    if index == "fsi":
        return fsi(v, d, ell)
    if index == "ksii":
        return ksii(v, d, ell)
    if ell < 1:
        raise ValueError("interaction order must be >= 1")
    v = _as_games(v, d)
    out = np.empty((v.shape[0], n_scores(d, ell)), dtype=np.float64)
    rc = _load().oracle_index_definition(d, ell, INDEX_CODES[index], v.shape[0], _ptr(v), _ptr(out))
    if rc != 0:
        raise RuntimeError("oracle_index_definition failed")
    return out


# ---------------------------------------------------------------------------
# Exact rational closed form (pure Python)
# ---------------------------------------------------------------------------

def _popcount(x: int) -> int:
    return bin(x).count("1")


def fsi_exact(v: Sequence, d: int, ell: int) -> List[Fraction]:
    """Closed form of Eq. fsi_closed / Eq. correction in exact rationals:
    float inputs are taken as the dyadic rationals they are.  Moebius by
    explicit submask sums, correction by explicit superset sums; d <= 10."""
    if d > 10:
        raise ValueError("exact oracle is limited to d <= 10")
    n = 1 << d
    vq = [Fraction(x) for x in v]
    a = [Fraction(0)] * n
    for S in range(n):
        s = _popcount(S)
        acc = Fraction(0)
        T = S
        while True:
            acc += vq[T] if (s - _popcount(T)) % 2 == 0 else -vq[T]
            if T == 0:
                break
            T = (T - 1) & S
        a[S] = acc
    w = {(s, t): weight_exact(ell, s, t) for s in range(d + 1) for t in range(d + 1)}
    out = []
    for S in score_masks(d, ell):
        S = int(S)
        s = _popcount(S)
        val = a[S]
        if s >= 1:
            for T in range(n):
                if T & S == S and T != S and _popcount(T) > ell:
                    val += w[(s, _popcount(T))] * a[T]
        out.append(val)
    return out


# ---------------------------------------------------------------------------
# Weighted least squares definition (Eq. fsi_wls), brute force
# ---------------------------------------------------------------------------

def shapley_kernel(d: int, t: int) -> float:
    """mu(t) = (d - 1) / (C(d, t) t (d - t)) for 0 < t < d."""
    return (d - 1) / (math.comb(d, t) * t * (d - t))


def fsi_wls(v, d: int, ell: int) -> np.ndarray:
    """Solve min sum_T mu(|T|) (v(T) - sum_{S subset T, |S|<=l} I_S)^2 subject
    to the fitted values at the empty and the full coalition equalling v
    there (the infinite-weight end points of the Shapley kernel), Eq. fsi_wls
    (Section 2.2), via its KKT linear system.  d <= 10."""
    if d > 10:
        raise ValueError("brute-force WLS is limited to d <= 10")
    v = np.asarray(v, dtype=np.float64).reshape(-1)
    n = 1 << d
    masks = [int(m) for m in score_masks(d, ell)]
    p = len(masks)
    X = np.zeros((n, p))
    for j, S in enumerate(masks):
        for T in range(n):
            if T & S == S:
                X[T, j] = 1.0
    full = n - 1
    inner = [T for T in range(n) if T != 0 and T != full]
    Xi = X[inner]
    wi = np.array([shapley_kernel(d, _popcount(T)) for T in inner])
    C = X[[0, full]]
    c = v[[0, full]]
    K = np.zeros((p + 2, p + 2))
    K[:p, :p] = Xi.T @ (wi[:, None] * Xi)
    K[:p, p:] = C.T
    K[p:, :p] = C
    rhs = np.concatenate([Xi.T @ (wi * v[inner]), c])
    sol = np.linalg.solve(K, rhs)
    return sol[:p]


# ---------------------------------------------------------------------------
# Shapley values by permutation enumeration (Section 2.1)
# ---------------------------------------------------------------------------

def shapley_permutations(v, d: int) -> np.ndarray:
    """phi_i = average over all d! player orders of v(P u {i}) - v(P), P the
    players before i (equivalent to the Section 2.1 formula); d <= 8."""
    if d > 8:
        raise ValueError("permutation enumeration is limited to d <= 8")
    v = np.asarray(v, dtype=np.float64).reshape(-1)
    phi = np.zeros(d)
    count = 0
    for perm in itertools.permutations(range(d)):
        S = 0
        for i in perm:
            phi[i] += v[S | (1 << i)] - v[S]
            S |= 1 << i
        count += 1
    return phi / count


def shapley_formula(v, d: int) -> np.ndarray:
    """phi_i = sum_{S not containing i} |S|!(d-|S|-1)!/d! [v(S u i) - v(S)]."""
    v = np.asarray(v, dtype=np.float64).reshape(-1)
    phi = np.zeros(d)
    for i in range(d):
        for S in range(1 << d):
            if S >> i & 1:
                continue
            s = _popcount(S)
            wgt = math.factorial(s) * math.factorial(d - s - 1) / math.factorial(d)
            phi[i] += wgt * (v[S | (1 << i)] - v[S])
    return phi


# ---------------------------------------------------------------------------
# Masked-model value function (C core)
# ---------------------------------------------------------------------------

def masked_game(mlp, x, baseline, coalitions=None) -> np.ndarray:
    """v_x(S) = f(x on S, baseline elsewhere) for one instance x; all 2^d
    coalitions unless a list of masks is given."""
    W1 = np.ascontiguousarray(mlp.W1, dtype=np.float64)
    b1 = np.ascontiguousarray(mlp.b1, dtype=np.float64)
    W2 = np.ascontiguousarray(mlp.W2, dtype=np.float64)
    b2 = np.ascontiguousarray(mlp.b2, dtype=np.float64)
    W3 = np.ascontiguousarray(mlp.W3, dtype=np.float64).reshape(-1)
    b3 = float(np.asarray(mlp.b3).reshape(-1)[0])
    h1, d = W1.shape
    h2 = W2.shape[0]
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1)
    base = np.ascontiguousarray(baseline, dtype=np.float64).reshape(-1)
    if coalitions is None:
        coal = np.arange(1 << d, dtype=np.uint64)
    else:
        coal = np.ascontiguousarray(np.asarray(coalitions, dtype=np.uint64))
    out = np.empty(coal.shape[0], dtype=np.float64)
    _load().oracle_masked_game(d, h1, h2, _ptr(W1), _ptr(b1), _ptr(W2), _ptr(b2), _ptr(W3), b3,
                               _ptr(x), _ptr(base), coal.shape[0], _ptr(coal), _ptr(out))
    return out


def masked_game_interventional(mlp, x, background, coalitions=None) -> np.ndarray:
    """Interventional value function of Section 4.1 ("Value Function"):
    v(S) = E over the absent features of f(x_S, X_rest), estimated as the
    mean over the given background rows of the masked game with that row as
    the reference input (rows added in ascending order); one instance."""
    bg = np.atleast_2d(np.asarray(background, dtype=np.float64))
    acc = None
    for row in bg:
        v = masked_game(mlp, x, row, coalitions)
        acc = v if acc is None else acc + v
    return acc / bg.shape[0]


# ---------------------------------------------------------------------------
# The paper's MPO and sweep (Sections 3.2-3.4, Algorithm 1), explicit states
# ---------------------------------------------------------------------------

def mpo_states(k: int, ell: int):
    """Bond states (s, t) after k sites: 0 <= s <= min(k, l), s <= t <= k
    (Section 3.3, "State Space")."""
    return [(s, t) for s in range(min(k, ell) + 1) for t in range(s, k + 1)]


def mpo_transitions(state, ell: int, k: int):
    """Valid (sigma, tau, next) of the site-k core (1-based k): tau >= sigma,
    counters add, next s <= min(k, l) (Section 3.3, "Core Construction")."""
    s, t = state
    out = []
    for sigma in (0, 1):
        for tau in (0, 1):
            if tau < sigma:
                continue
            ns, nt = s + sigma, t + tau
            if ns <= min(k, ell):
                out.append((sigma, tau, (ns, nt)))
    return out


def mpo_sweep(a, d: int, ell: int) -> np.ndarray:
    """Correction C = A_trunc a by the left-to-right sweep of Algorithm 1, with
    the intermediate tensor kept as a dict over (output prefix, state) of
    arrays over the remaining input suffix.  Site k carries player k-1 (the
    paper's site 1 is the most significant index bit in its reshape; the sweep
    here peels players from the high bit down so that the suffix stays a
    contiguous low-bit block).  The last core applies w(s, t) for s <= l,
    t > l.  Returns the correction for every S (zero where |S| > l); small d
    only."""
    a = np.asarray(a, dtype=np.float64).reshape(-1)
    # X[(out_prefix_mask, (s, t))] -> vector over remaining input bits
    X = {(0, (0, 0)): a.copy()}
    for k in range(1, d + 1):
        player = d - k  # high bit first: splitting the top bit of the suffix
        nxt = {}
        for (prefix, state), vec in X.items():
            half = vec.shape[0] // 2
            parts = (vec[:half], vec[half:])  # tau_k = 0, 1 (top bit of the suffix)
            for sigma, tau, ns in mpo_transitions(state, ell, k):
                key = (prefix | (sigma << player), ns)
                contrib = parts[tau]
                if key in nxt:
                    nxt[key] = nxt[key] + contrib
                else:
                    nxt[key] = contrib.copy()
        X = nxt
    out = np.zeros(1 << d)
    for (prefix, (s, t)), vec in X.items():
        if s <= ell and t > ell:
            out[prefix] += float(weight_exact(ell, s, t)) * vec[0]
    return out
