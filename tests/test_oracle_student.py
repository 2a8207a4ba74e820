"""Pins for the student oracle (oracle/student.py): the analytic backward
pass against central finite differences, the projection's closed-form
properties, Adam's first step in closed form, and the BF16 rounding against
PyTorch's conversion."""
import numpy as np
import pytest

from oracle import student as so


def _small(seed=0, d=4, H=6, n_out=5, B=7):
    rng = np.random.default_rng(seed)
    n = H * d + H + H * H + H + n_out * H + n_out
    params = rng.normal(size=n) * 0.5
    x = rng.normal(size=(B, d))
    labels = rng.normal(size=(B, n_out))
    target = rng.normal(size=B)
    v0 = 0.3
    labels[:, 0] = v0
    return params, x, labels, target, v0, d, H, n_out


def test_backward_matches_finite_differences():
    params, x, labels, target, v0, d, H, n_out = _small()
    loss, g = so.loss_and_grads(params, x, labels, target, v0, d, H, n_out)
    eps = 1e-6
    num = np.empty_like(params)
    for i in range(params.size):
        p1 = params.copy()
        p1[i] += eps
        p2 = params.copy()
        p2[i] -= eps
        l1, _ = so.loss_and_grads(p1, x, labels, target, v0, d, H, n_out)
        l2, _ = so.loss_and_grads(p2, x, labels, target, v0, d, H, n_out)
        num[i] = (l1 - l2) / (2 * eps)
    assert np.max(np.abs(num - g)) < 1e-7 * max(1.0, np.abs(g).max())


def test_projection_properties():
    rng = np.random.default_rng(1)
    Y = rng.normal(size=(9, 11))
    t = rng.normal(size=9)
    P = so.project(Y, t, 0.25)
    assert np.allclose(P[:, 1:].sum(axis=1), t, atol=1e-12)
    assert np.all(P[:, 0] == 0.25)
    assert np.allclose(so.project(P, t, 0.25), P, atol=1e-12)           # idempotent
    # orthogonal: the correction is along the all-ones direction only
    d = (P - Y)[:, 1:]
    assert np.allclose(d - d.mean(axis=1, keepdims=True), 0.0, atol=1e-12)


def test_adam_first_step_closed_form():
    g = np.array([3.0, -0.5, 1e-3, 0.0])
    p, m, v = so.adam_step(np.zeros(4), np.zeros(4), np.zeros(4), g, t=1, lr=0.1, eps=1e-8)
    # m_hat = g, v_hat = g^2: step = -lr * g / (|g| + eps)
    assert np.allclose(p, -0.1 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=0)


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(2)
    x = np.concatenate([rng.normal(size=4000) * 10.0 ** rng.integers(-5, 5, size=4000),
                        [0.0, -0.0, 1.0, 3.0e38, 1e-40, 0.1, 1.00390625, 1.01171875]])
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(so.bf16_round(x), ref)


def test_surrogate_matches_definition():
    masks = np.array([0, 1, 2, 4, 3, 5, 6], dtype=np.uint64)  # d = 3, l = 2 layout
    phi = np.array([[0.5, 1.0, 2.0, 3.0, 0.1, 0.2, 0.3]])
    coal = np.array([[0, 1, 3, 7, 6]], dtype=np.uint64)
    g = so.surrogate(phi, masks, coal)
    assert np.allclose(g, [[0.5, 1.5, 3.6, 7.1, 5.8]])
