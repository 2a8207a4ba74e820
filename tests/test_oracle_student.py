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


def test_gradient_scale_separates_rounding_from_mistakes():
    """The element-wise bound used against the GPU (4 BF16 ulps of the
    root-sum-square scale) holds for the same arithmetic done with FP32
    accumulation and perturbed GELU values (as on the GPU), and fails for a
    planted mistake: two rows of the W3 gradient swapped, one b3 entry
    dropped from its sum, one W1 entry with its sign flipped."""
    from paper_2601_01903_gb300 import student as st
    d, H, n_out, B = 16, 64, 137, 256
    params = st.init_params(d, H, n_out, 1).astype(np.float64)
    rng = np.random.default_rng(1)
    x = rng.normal(size=(B, d)).astype(np.float32)
    labels = (rng.normal(size=(B, n_out)) * 0.1).astype(np.float32)
    target = rng.normal(size=B).astype(np.float32)
    _, ref = so.loss_and_grads(params, x, labels, target, 0.2, d, H, n_out, emulate_bf16=True)
    mag = so.grad_magnitudes(params, x, labels, target, 0.2, d, H, n_out)
    # FP32 accumulation of BF16 operands, GELU perturbed by 1e-7 relative
    f32, r = np.float32, (lambda a: so.bf16_round(a).astype(np.float32))
    P = so.unpack(params, d, H, n_out)
    X, W1, W2, W3 = r(x), r(P["W1"]), r(P["W2"]), r(P["W3"])
    Z1 = (X @ W1.T).astype(f32) + P["b1"].astype(f32)
    A1 = r(so.gelu(Z1.astype(np.float64)) * (1 + 1e-7 * rng.normal(size=Z1.shape)))
    Z2 = (A1 @ W2.T).astype(f32) + P["b2"].astype(f32)
    A2 = r(so.gelu(Z2.astype(np.float64)) * (1 + 1e-7 * rng.normal(size=Z2.shape)))
    Y = (A2 @ W3.T).astype(f32) + P["b3"].astype(f32)
    err = so.project(Y.astype(np.float64), target, 0.2).astype(f32) - labels
    g = 2 * err / (B * n_out)
    dY = np.zeros_like(g)
    dY[:, 1:] = g[:, 1:] - g[:, 1:].mean(axis=1, keepdims=True)
    dH2 = (r(dY) @ W3) * so.gelu_grad(Z2.astype(np.float64)).astype(f32)
    dH1 = (r(dH2) @ W2) * so.gelu_grad(Z1.astype(np.float64)).astype(f32)
    got = so.pack(dict(W1=r(dH1).T @ X, b1=dH1.sum(0), W2=r(dH2).T @ A1, b2=dH2.sum(0),
                       W3=r(dY).T @ A2, b3=dY.sum(0)))
    bound = 4 * 2.0 ** -8 * mag
    assert np.all(np.abs(got - ref) <= bound)
    o3 = H * d + H + H * H + H
    ob3 = o3 + n_out * H
    swapped = got.copy()
    swapped[o3 + 5 * H:o3 + 6 * H], swapped[o3 + 9 * H:o3 + 10 * H] = got[o3 + 9 * H:o3 + 10 * H], got[o3 + 5 * H:o3 + 6 * H]
    assert np.any(np.abs(swapped - ref) > bound)
    dropped = got.copy()
    dropped[ob3 + 7] -= dY[int(np.argmax(np.abs(dY[:, 7]))), 7]  # the largest of its 256 terms
    assert np.any(np.abs(dropped - ref) > bound)
    flipped = got.copy()
    k = int(np.argmax(np.abs(ref[:H * d])))
    flipped[k] = -flipped[k]
    assert np.any(np.abs(flipped - ref) > bound)


def test_output_scale_bounds_an_upstream_bf16_flip():
    """Moving one layer-1 activation by one BF16 ulp changes every output of
    its instance; the change stays within 2^-8 times the forward scale."""
    from paper_2601_01903_gb300 import student as st
    d, H, n_out, B = 16, 64, 137, 64
    params = st.init_params(d, H, n_out, 2).astype(np.float64)
    x = np.random.default_rng(2).normal(size=(B, d)).astype(np.float32)
    f = so.forward(params, x, d, H, n_out, emulate_bf16=True)
    mag = so.output_magnitudes(params, x, d, H, n_out)
    P = so.unpack(params, d, H, n_out)
    worst = 0.0
    for b, i in ((0, 0), (5, 17), (40, 63)):
        A1 = f["A1"].copy()
        A1[b, i] *= 1 + 2.0 ** -8
        A2 = so.bf16_round(so.gelu(A1 @ f["W2"].T + P["b2"]))
        Y = A2 @ f["W3"].T + P["b3"]
        worst = max(worst, float(np.max(np.abs(Y - f["Y"]) / mag)))
    assert 0 < worst <= 4 * 2.0 ** -8
