"""CPU oracle of the amortised explainer's arithmetic -- TEST INFRASTRUCTURE.

Float64 NumPy forward and backward passes of the student network
x [d] -> H -> H -> n_out (GELU, exact erf form), the projection of its raw
outputs onto the efficiency constraint (sum of the non-empty scores equals
v(N) - v(empty), the empty score equals v(empty); the efficiency axiom of
Section 2.1 carried to interaction scores), the mean squared error against
FSI labels, and one Adam step (Kingma & Ba 2015).  Optionally the BF16
rounding points of the GPU path are reproduced (round to nearest even of the
float32 value), so that GPU results can be compared tightly.  The paper has
no learned component; parity of these functions is pinned by finite
differences, closed forms and library conversions in the tests, not by the
paper.  Only tests/ and bench.py's CPU leg use this module.
"""
from __future__ import annotations

import math

import numpy as np

_SQ2 = math.sqrt(2.0)


def bf16_round(x) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even) after rounding to
    float32, returned as float64; implemented on the IEEE bit pattern."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    r = (u + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)
    out = r.astype(np.uint32).view(np.float32).astype(np.float64)
    nan = np.isnan(f)
    if nan.any():
        out[nan] = np.nan
    return out


def _erf(z):
    from scipy.special import erf  # library routine for erf
    return erf(z)


def gelu(z):
    return 0.5 * z * (1.0 + _erf(z / _SQ2))


def gelu_grad(z):
    return 0.5 * (1.0 + _erf(z / _SQ2)) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def unpack(params, d, H, n_out):
    p = np.asarray(params, dtype=np.float64)
    o = 0
    out = {}
    for name, shape in (("W1", (H, d)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)),
                        ("W3", (n_out, H)), ("b3", (n_out,))):
        n = int(np.prod(shape))
        out[name] = p[o:o + n].reshape(shape)
        o += n
    assert o == p.size
    return out


def pack(tensors) -> np.ndarray:
    return np.concatenate([np.asarray(tensors[k], dtype=np.float64).reshape(-1)
                           for k in ("W1", "b1", "W2", "b2", "W3", "b3")])


def forward(params, x, d, H, n_out, emulate_bf16=False):
    """Raw outputs and the intermediates of the backward pass."""
    P = unpack(params, d, H, n_out)
    r = bf16_round if emulate_bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    X = r(x)
    W1, W2, W3 = r(P["W1"]), r(P["W2"]), r(P["W3"])
    Z1 = X @ W1.T + P["b1"]
    A1 = r(gelu(Z1))
    Z2 = A1 @ W2.T + P["b2"]
    A2 = r(gelu(Z2))
    Y = A2 @ W3.T + P["b3"]
    return dict(X=X, W1=W1, W2=W2, W3=W3, Z1=Z1, A1=A1, Z2=Z2, A2=A2, Y=Y)


def project(Y, target, v_empty):
    """Euclidean projection of the non-empty scores onto the hyperplane
    sum = target (per instance); the empty score is set to v_empty."""
    Y = np.asarray(Y, dtype=np.float64)
    out = Y.copy()
    n = Y.shape[1] - 1
    shift = (np.asarray(target, dtype=np.float64) - Y[:, 1:].sum(axis=1)) / n
    out[:, 1:] = Y[:, 1:] + shift[:, None]
    out[:, 0] = v_empty
    return out


def loss_and_grads(params, x, labels, target, v_empty, d, H, n_out, emulate_bf16=False):
    """Mean squared error (over B * n_out entries) of the projected outputs
    and its gradient with respect to the flat parameter vector."""
    f = forward(params, x, d, H, n_out, emulate_bf16)
    B = f["Y"].shape[0]
    r = bf16_round if emulate_bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    phi = project(f["Y"], target, v_empty)
    err = phi - labels
    loss = float((err * err).sum() / (B * n_out))
    g = 2.0 * err / (B * n_out)
    dY = np.zeros_like(g)
    dY[:, 1:] = g[:, 1:] - g[:, 1:].mean(axis=1, keepdims=True)
    dYr = r(dY)
    gW3 = dYr.T @ f["A2"]
    gb3 = dY.sum(axis=0)
    dH2 = (dYr @ f["W3"]) * gelu_grad(f["Z2"])
    dH2r = r(dH2)
    gW2 = dH2r.T @ f["A1"]
    gb2 = dH2.sum(axis=0)
    dH1 = (dH2r @ f["W2"]) * gelu_grad(f["Z1"])
    gW1 = r(dH1).T @ f["X"]
    gb1 = dH1.sum(axis=0)
    grads = pack(dict(W1=gW1, b1=gb1, W2=gW2, b2=gb2, W3=gW3, b3=gb3))
    return loss, grads


def _forward_scales(params, x, d, H, n_out):
    """Root-sum-square scales of the forward pass with BF16 rounding points
    kept: s(Z1) = sqrt(X^2 (W1^2)^T + b1^2), s(A1) = |A1| + |gelu'(Z1)| s(Z1),
    and so on through layer 2 and the output.  Changing any one rounded
    operand upstream by a relative 2^-8 moves each entry by at most about
    2^-8 times its scale."""
    f = forward(params, x, d, H, n_out, emulate_bf16=True)
    P = unpack(params, d, H, n_out)
    sZ1 = np.sqrt(f["X"] ** 2 @ (f["W1"] ** 2).T + P["b1"] ** 2)
    sA1 = np.abs(f["A1"]) + np.abs(gelu_grad(f["Z1"])) * sZ1
    sZ2 = np.sqrt(sA1 ** 2 @ (f["W2"] ** 2).T + P["b2"] ** 2)
    sA2 = np.abs(f["A2"]) + np.abs(gelu_grad(f["Z2"])) * sZ2
    sY = np.sqrt(sA2 ** 2 @ (f["W3"] ** 2).T + P["b3"] ** 2)
    return f, sA1, sA2, sY


def grad_magnitudes(params, x, labels, target, v_empty, d, H, n_out):
    """Per-entry scale for comparing GPU gradients with ``loss_and_grads``:
    the same backward pass with every sum replaced by the root of the sum of
    its squared terms (BF16 rounding points kept), each forward operand by
    its scale from ``_forward_scales`` and each intermediate carried as that
    root-sum-square scale.  Changing one rounded operand by a relative 2^-8
    (one BF16 ulp) changes one term of each sum it feeds, so it moves
    gradient k by at most about 2^-8 times this scale; FP32 accumulation in
    another order moves it by far less.  Element-wise tolerances are
    multiples of 2^-8 times this value."""
    f, sA1, sA2, sY = _forward_scales(params, x, d, H, n_out)
    B = f["Y"].shape[0]
    phi = project(f["Y"], target, v_empty)
    # |d loss / d Y| and the scale of its changes: the error, plus the
    # output scale (an upstream flip moves Y by 2^-8 of it)
    e = np.abs(phi - labels) + sY
    g = 2.0 * e / (B * n_out)
    dY = np.zeros_like(g)
    dY[:, 1:] = np.sqrt(g[:, 1:] ** 2 + (g[:, 1:] ** 2).mean(axis=1, keepdims=True))
    sq = lambda a: np.asarray(a, dtype=np.float64) ** 2
    gp2, gp1 = np.abs(gelu_grad(f["Z2"])), np.abs(gelu_grad(f["Z1"]))
    mW3 = np.sqrt(sq(dY).T @ sq(sA2))
    mb3 = np.sqrt(sq(dY).sum(axis=0))
    dH2 = np.sqrt(sq(dY) @ sq(f["W3"])) * gp2
    mW2 = np.sqrt(sq(dH2).T @ sq(sA1))
    mb2 = np.sqrt(sq(dH2).sum(axis=0))
    dH1 = np.sqrt(sq(dH2) @ sq(f["W2"])) * gp1
    mW1 = np.sqrt(sq(dH1).T @ sq(f["X"]))
    mb1 = np.sqrt(sq(dH1).sum(axis=0))
    return pack(dict(W1=mW1, b1=mb1, W2=mW2, b2=mb2, W3=mW3, b3=mb3))


def output_magnitudes(params, x, d, H, n_out):
    """Per-entry scale of the raw outputs (``_forward_scales``): the bound on
    how far BF16 rounding flips anywhere in the forward pass can move them,
    in units of 2^-8."""
    return _forward_scales(params, x, d, H, n_out)[3]


def adam_step(p, m, v, g, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update at step t (1-based); returns new (p, m, v)."""
    m = beta1 * m + (1 - beta1) * g
    v = beta2 * v + (1 - beta2) * g * g
    mhat = m / (1 - beta1 ** t)
    vhat = v / (1 - beta2 ** t)
    return p - lr * mhat / (np.sqrt(vhat) + eps), m, v


def surrogate(phi, masks, coalitions):
    """g(T) = sum of phi(S) over the scored S contained in T (the order-l
    surrogate of Eq. fsi_wls), for each instance and coalition."""
    phi = np.asarray(phi, dtype=np.float64)
    masks = np.asarray(masks, dtype=np.uint64)
    coal = np.asarray(coalitions, dtype=np.uint64)
    out = np.zeros(coal.shape)
    for b in range(coal.shape[0]):
        for k in range(coal.shape[1]):
            inside = (masks & coal[b, k]) == masks
            out[b, k] = phi[b, inside].sum()
    return out
