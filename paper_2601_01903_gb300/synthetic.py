"""Seeded synthetic workloads for FSI (shared by the CUDA path's tests, the
bench and the CPU oracle's tests).

This module only draws random numbers and lays them out.  It holds none of
the FSI arithmetic (no Moebius transform, no correction weights, no model
evaluation): the oracle and the CUDA kernels each implement those on their
own and are fed the same arrays from here.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) used in counter mode: draw i of
stream (seed, tag) is mix64(key + (i + 1) * 0x9E3779B97F4A7C15) with
key = mix64(seed * 0x9E3779B97F4A7C15 + tag).  Uniforms take the top 53 bits,
(z >> 11 + 0.5) * 2^-53, which lies strictly inside (0, 1).  Normals use the
Box-Muller transform (Box & Muller 1958) on consecutive uniform pairs and keep
both outputs.

Coalitions are bitmasks: bit i of an index is feature i (feature 0 is the
least significant bit), so a value vector of a d-player game is a float64
array of length 2^d indexed by the coalition mask.

The workloads follow the paper's settings (Section 4 and Appendix D: d from 8
to 20, interaction order 2 or 3, value functions that come from a model
evaluated with absent features replaced) with synthetic models standing in for
the paper's trained ones, which the paper shows only affect the values, not
the running time (Section 4.1, "runtime depends only on d and l").
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_MASK64 = (1 << 64) - 1


def _mix64(z: np.ndarray) -> np.ndarray:
    z = z.astype(np.uint64, copy=True)
    z ^= z >> np.uint64(30)
    z *= _M1
    z ^= z >> np.uint64(27)
    z *= _M2
    z ^= z >> np.uint64(31)
    return z


def _mix64_int(z: int) -> int:
    z &= _MASK64
    z ^= z >> 30
    z = (z * 0xBF58476D1CE4E5B9) & _MASK64
    z ^= z >> 27
    z = (z * 0x94D049BB133111EB) & _MASK64
    z ^= z >> 31
    return z


class Stream:
    """One counter-based SplitMix64 stream, identified by (seed, tag)."""

    def __init__(self, seed: int, tag: int):
        self.key = _mix64_int(seed * 0x9E3779B97F4A7C15 + tag)
        self.counter = 0

    def raw(self, n: int) -> np.ndarray:
        idx = np.arange(self.counter + 1, self.counter + n + 1, dtype=np.uint64)
        self.counter += n
        with np.errstate(over="ignore"):
            z = np.uint64(self.key) + idx * _GAMMA
        return _mix64(z)

    def uniform(self, n: int) -> np.ndarray:
        z = self.raw(n)
        return ((z >> np.uint64(11)).astype(np.float64) + 0.5) * (2.0 ** -53)

    def normal(self, n: int) -> np.ndarray:
        m = (n + 1) // 2
        u = self.uniform(2 * m).reshape(m, 2)
        r = np.sqrt(-2.0 * np.log(u[:, 0]))
        th = 2.0 * math.pi * u[:, 1]
        out = np.empty((m, 2), dtype=np.float64)
        out[:, 0] = r * np.cos(th)
        out[:, 1] = r * np.sin(th)
        return out.reshape(-1)[:n]

    def integers(self, lo: int, hi: int, n: int) -> np.ndarray:
        """Uniform integers in [lo, hi] (inclusive), by floor of a uniform."""
        u = self.uniform(n)
        return (lo + np.floor(u * (hi - lo + 1))).astype(np.int64)


# Stream tags: one per kind of draw, so that adding draws of one kind never
# shifts another kind's numbers.
TAG_MOBIUS = 1
TAG_MLP_W1, TAG_MLP_W2, TAG_MLP_W3 = 11, 12, 13
TAG_X = 21
TAG_GAME_SHAPE = 31
TAG_SUPPORT = 32
TAG_STUDENT = 41
TAG_SHUFFLE = 42
TAG_SPOT = 43


def popcounts(d: int) -> np.ndarray:
    idx = np.arange(1 << d, dtype=np.int64)
    pc = np.zeros(1 << d, dtype=np.int64)
    for i in range(d):
        pc += (idx >> i) & 1
    return pc


def subset_sum(m: np.ndarray, d: int) -> np.ndarray:
    """v(S) = sum over T subset of S of m(T): builds a game from chosen Moebius
    coefficients (the zeta transform, used here only to construct inputs)."""
    v = np.array(m, dtype=np.float64, copy=True)
    lead = v.shape[:-1]
    for i in range(d):
        view = v.reshape(lead + (-1, 2, 1 << i))
        view[..., 1, :] += view[..., 0, :]
    return v


# --------------------------------------------------------------------------
# Moebius-sparse games
# --------------------------------------------------------------------------

def mobius_game_dense(d: int, max_order: int, seed: int, scale_by_factorial: bool = True,
                      stream_tag: int = TAG_MOBIUS):
    """Game with m(T) ~ N(0,1) (divided by |T|! when asked) for 1 <= |T| <=
    max_order and m = 0 elsewhere, m(empty) = 0.  Normals are drawn one per T
    with 1 <= |T| <= max_order in ascending mask order.  Returns (v, m)."""
    st = Stream(seed, stream_tag)
    pc = popcounts(d)
    sel = (pc >= 1) & (pc <= max_order)
    m = np.zeros(1 << d, dtype=np.float64)
    z = st.normal(int(sel.sum()))
    if scale_by_factorial:
        fact = np.array([math.factorial(int(t)) for t in pc[sel]], dtype=np.float64)
        z = z / fact
    m[sel] = z
    return subset_sum(m, d), m


@dataclass
class RaggedGames:
    """A packed batch of games with uneven sizes.  v is one float64 buffer;
    game g occupies v[v_off[g] : v_off[g] + 2**d[g]] and its scores go to
    phi[phi_off[g] : phi_off[g] + n_out(d[g], ell[g])]."""
    d: np.ndarray
    ell: np.ndarray
    v_off: np.ndarray
    phi_off: np.ndarray
    v: np.ndarray
    n_phi: int
    m: Optional[List[np.ndarray]] = field(default=None, repr=False)


def n_scores(d: int, ell: int) -> int:
    return sum(math.comb(d, k) for k in range(0, min(ell, d) + 1))


def sparse_mobius_games(n_games: int, d_lo: int, d_hi: int, ell_lo: int, ell_hi: int,
                        density: float, max_order: int, seed: int, keep_m: bool = False,
                        first: int = 0, count: Optional[int] = None) -> RaggedGames:
    """Batch of uneven Moebius-sparse games: per game d ~ U{d_lo..d_hi} and
    ell ~ U{ell_lo..ell_hi} (drawn first, for all games), then for each game
    every T with 1 <= |T| <= max_order is kept independently with probability
    `density` (one uniform per T in ascending mask order) and a kept T gets
    m(T) ~ N(0,1).  Games [first, first+count) of the batch are built."""
    shape = Stream(seed, TAG_GAME_SHAPE)
    ds = shape.integers(d_lo, d_hi, n_games)
    ells = shape.integers(ell_lo, ell_hi, n_games)
    if count is None:
        count = n_games - first
    sel = slice(first, first + count)
    ds, ells = ds[sel], ells[sel]
    sizes = np.array([1 << int(x) for x in ds], dtype=np.int64)
    outs = np.array([n_scores(int(x), int(l)) for x, l in zip(ds, ells)], dtype=np.int64)
    v_off = np.zeros(len(ds), dtype=np.int64)
    phi_off = np.zeros(len(ds), dtype=np.int64)
    if len(ds):
        v_off[1:] = np.cumsum(sizes)[:-1]
        phi_off[1:] = np.cumsum(outs)[:-1]
    v = np.empty(int(sizes.sum()), dtype=np.float64)
    ms = [] if keep_m else None
    pcache = {}
    for k, g in enumerate(range(first, first + count)):
        d = int(ds[k])
        if d not in pcache:
            pcache[d] = popcounts(d)
        pc = pcache[d]
        st = Stream(seed, TAG_SUPPORT + 1000 * (g + 1))
        cand = (pc >= 1) & (pc <= max_order)
        u = st.uniform(int(cand.sum()))
        keep = np.zeros(1 << d, dtype=bool)
        keep[np.flatnonzero(cand)[u < density]] = True
        m = np.zeros(1 << d, dtype=np.float64)
        m[keep] = st.normal(int(keep.sum()))
        v[v_off[k]:v_off[k] + (1 << d)] = subset_sum(m, d)
        if keep_m:
            ms.append(m)
    return RaggedGames(d=ds.astype(np.int64), ell=ells.astype(np.int64), v_off=v_off,
                       phi_off=phi_off, v=v, n_phi=int(outs.sum()), m=ms)


# --------------------------------------------------------------------------
# Masked-model games: random-init GELU MLPs and instances
# --------------------------------------------------------------------------

@dataclass
class MLP:
    """f(z) = W3 gelu(W2 gelu(W1 z + b1) + b2) + b3, row-major weights
    (W1: [h1, d], W2: [h2, h1], W3: [1, h2]); float64."""
    W1: np.ndarray
    b1: np.ndarray
    W2: np.ndarray
    b2: np.ndarray
    W3: np.ndarray
    b3: np.ndarray

    @property
    def dims(self):
        return self.W1.shape[1], self.W1.shape[0], self.W2.shape[0]


def random_mlp(d: int, h1: int, h2: int, seed: int) -> MLP:
    """Weights N(0, 1/fan_in), biases zero, drawn row-major W1, W2, W3."""
    w1 = Stream(seed, TAG_MLP_W1).normal(h1 * d).reshape(h1, d) / math.sqrt(d)
    w2 = Stream(seed, TAG_MLP_W2).normal(h2 * h1).reshape(h2, h1) / math.sqrt(h1)
    w3 = Stream(seed, TAG_MLP_W3).normal(h2).reshape(1, h2) / math.sqrt(h2)
    return MLP(w1, np.zeros(h1), w2, np.zeros(h2), w3, np.zeros(1))


def gaussian_instances(n: int, d: int, seed: int, ar1_rho: float = 0.0,
                       first: int = 0) -> np.ndarray:
    """x ~ N(0, Sigma) with Sigma_ij = rho^|i-j| (rho = 0 gives N(0, I)),
    sampled exactly as the AR(1) chain x_0 = z_0, x_i = rho x_{i-1} +
    sqrt(1 - rho^2) z_i.  Rows [first, first + n) of the stream."""
    st = Stream(seed, TAG_X)
    # Normal number e of the stream comes from uniform pair e // 2 (cos for
    # even e, sin for odd e), so a slice of rows starts on that pair.
    e0 = first * d
    st.counter = 2 * (e0 // 2)
    z = st.normal(n * d + e0 % 2)[e0 % 2:].reshape(n, d)
    if ar1_rho == 0.0:
        return z
    x = np.empty_like(z)
    x[:, 0] = z[:, 0]
    c = math.sqrt(1.0 - ar1_rho * ar1_rho)
    for i in range(1, d):
        x[:, i] = ar1_rho * x[:, i - 1] + c * z[:, i]
    return x


# --------------------------------------------------------------------------
# Named workloads (the paper's d / l range; seeds fixed)
# --------------------------------------------------------------------------

@dataclass
class MaskedWorkload:
    name: str
    d: int
    ell: int
    B: int
    mlp: MLP
    x: np.ndarray
    baseline: np.ndarray


def workload_mobius_d8():
    """d=8, l=2, one game, m(T) ~ N(0,1)/|T|! for 1 <= |T| <= 4, seed 0."""
    v, m = mobius_game_dense(8, 4, seed=0)
    return dict(name="mobius_d8_l2", d=8, ell=2, B=1, v=v.reshape(1, -1), m=m.reshape(1, -1))


def workload_masked(d: int, ell: int, B: int, hidden: int, seed: int, name: str,
                    ar1_rho: float = 0.0) -> MaskedWorkload:
    mlp = random_mlp(d, hidden, hidden, seed)
    x = gaussian_instances(B, d, seed, ar1_rho)
    return MaskedWorkload(name, d, ell, B, mlp, x, np.zeros(d))


def workload_mlp_d14():
    """d=14, l=2, 64 instances, MLP 14-64-64-1, x ~ N(0, I), seed 1."""
    return workload_masked(14, 2, 64, 64, 1, "mlp_d14_l2_b64")


def workload_mlp_d20():
    """d=20, l=3, 16 instances, MLP 20-128-128-1, x ~ N(0, I), seed 2."""
    return workload_masked(20, 3, 16, 128, 2, "mlp_d20_l3_b16")


def workload_mlp_d24():
    """d=24, l=2, one instance, MLP 24-128-128-1, seed 2 (scale-up case)."""
    return workload_masked(24, 2, 1, 128, 2, "mlp_d24_l2_b1")


def workload_uneven(first: int = 0, count: Optional[int] = None, keep_m: bool = False):
    """1024 Moebius-sparse games, d ~ U{10..20}, l ~ U{1,2,3}, each T with
    1 <= |T| <= 5 kept with probability 0.01, m(T) ~ N(0,1), seed 3."""
    return sparse_mobius_games(1024, 10, 20, 1, 3, 0.01, 5, seed=3, keep_m=keep_m,
                               first=first, count=count)


def workload_student_teacher():
    """Teacher of the amortised explainer: d=16, l=2, MLP 16-128-128-1,
    x ~ N(0, Sigma), Sigma_ij = 0.5^|i-j|, seed 4."""
    return random_mlp(16, 128, 128, 4)


def student_instances(n: int, first: int = 0) -> np.ndarray:
    return gaussian_instances(n, 16, 4, ar1_rho=0.5, first=first)
