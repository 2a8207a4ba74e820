"""The student explainer on GB300: gradients, Adam and the projection
against the CPU oracle, checkpoint/resume, the sampled value function and
residual, and a small end-to-end training run with the exact-path fallback."""
import numpy as np
import pytest

import paper_2601_01903_gb300 as fsi
from paper_2601_01903_gb300 import student as st
from paper_2601_01903_gb300 import synthetic
from oracle import student as so

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _case(d=16, H=64, n_out=137, B=256, seed=1):
    params = st.init_params(d, H, n_out, seed)
    rng = np.random.default_rng(seed)
    x = rng.normal(size=(B, d)).astype(np.float32)
    labels = (rng.normal(size=(B, n_out)) * 0.1).astype(np.float32)
    v0 = 0.2
    labels[:, 0] = v0
    target = rng.normal(size=B).astype(np.float32)
    return params, x, labels, target, v0


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


# Element-wise tolerance of GPU results against the BF16-emulating oracle.
# The GPU rounds the same operands to BF16 but accumulates in FP32 in another
# order; an FP32 value that lands within a few FP32 ulps of a BF16 rounding
# boundary can round to the neighbouring BF16 value (a relative change of
# 2^-8 in that one operand).  One such flip moves an entry by at most 2^-8
# times its root-sum-square scale (oracle.student.grad_magnitudes and
# output_magnitudes: each sum along the entry's chain replaced by the root of
# its summed squared terms, about the size of the entry itself); FP32
# accumulation moves it by far less.  The bound allows four flips' worth.  A
# wrong index, sign or dropped term moves an entry by about its own size,
# i.e. by about 2^8 / 4 = 64 times the bound.
FLIP = 4 * 2.0 ** -8


def _elementwise(got, ref, mag, name):
    bad = np.abs(got - ref) > FLIP * mag + 1e-30
    assert not bad.any(), (name, int(bad.sum()), float(np.max(np.abs(got - ref) / (mag + 1e-30))))


def test_gradients_match_oracle_with_bf16_rounding():
    d, H, n_out, B = 16, 64, 137, 256
    params, x, labels, target, v0 = _case(d, H, n_out, B)
    s = st.Student(d, H, n_out, B, params)
    loss = s.gradients(_dev(x), _dev(labels), _dev(target), v0)
    s.check()
    g = s.grads().astype(np.float64)
    p64 = params.astype(np.float64)
    ref_loss, ref = so.loss_and_grads(p64, x, labels, target, v0, d, H, n_out, emulate_bf16=True)
    mag = so.grad_magnitudes(p64, x, labels, target, v0, d, H, n_out)
    assert abs(loss.item() - ref_loss) <= 1e-4 * abs(ref_loss)
    o = 0
    for name, n in (("W1", H * d), ("b1", H), ("W2", H * H), ("b2", H), ("W3", n_out * H), ("b3", n_out)):
        gs, rs, ms = g[o:o + n], ref[o:o + n], mag[o:o + n]
        _elementwise(gs, rs, ms, name)
        # whole tensor: a few BF16 flips at most
        assert np.linalg.norm(gs - rs) <= 1e-2 * np.linalg.norm(rs), name
        o += n


def test_adam_step_and_projection_match_oracle():
    d, H, n_out, B = 16, 64, 137, 128
    params, x, labels, target, v0 = _case(d, H, n_out, B, seed=2)
    s = st.Student(d, H, n_out, B, params)
    s.set_adam(lr=1e-2)
    s.train_step(_dev(x), _dev(labels), _dev(target), v0)
    s.check()
    g = s.grads().astype(np.float64)
    p1, m1, v1, step = s.state()
    rp, rm, rv = so.adam_step(params.astype(np.float64), 0.0, 0.0, g, 1, lr=1e-2)
    assert step == 1
    assert np.max(np.abs(p1 - rp)) < 1e-6
    assert np.max(np.abs(m1 - rm)) < 1e-9 + 1e-6 * np.abs(rm).max()
    # projection of the student's output
    phi = s.predict(_dev(x), _dev(target), v0).cpu().numpy().astype(np.float64)
    assert np.all(phi[:, 0] == np.float32(v0))
    assert np.max(np.abs(phi[:, 1:].sum(axis=1) - target)) < 1e-3 * max(1.0, np.abs(target).max())
    f = so.forward(p1.astype(np.float64), x, d, H, n_out, emulate_bf16=True)
    ref = so.project(f["Y"], target, v0)
    # element-wise: the projection shifts every non-empty score by the mean
    # residual, so its scale is the raw outputs' plus their mean
    # (score 0 is v(empty) in float32, checked above)
    mag = so.output_magnitudes(p1.astype(np.float64), x, d, H, n_out)
    mag[:, 1:] += mag[:, 1:].mean(axis=1, keepdims=True)
    _elementwise(phi[:, 1:], ref[:, 1:], mag[:, 1:] + 1e-6 * np.abs(target)[:, None], "projected outputs")


def test_checkpoint_resume_is_bitwise(tmp_path):
    d, H, n_out, B = 16, 64, 137, 128
    params, x, labels, target, v0 = _case(d, H, n_out, B, seed=3)
    X, L, T = _dev(x), _dev(labels), _dev(target)
    a = st.Student(d, H, n_out, B, params)
    for _ in range(3):
        a.train_step(X, L, T, v0)
    path = str(tmp_path / "ckpt.bin")
    a.save(path)
    a.train_step(X, L, T, v0)
    pa = a.state()[0]
    b = st.Student(d, H, n_out, B, params)
    b.load(path)
    b.train_step(X, L, T, v0)
    pb = b.state()[0]
    assert np.array_equal(pa, pb)


def test_sampled_value_function_and_residual(oracle_mod):
    mlp = synthetic.workload_student_teacher()
    dm = fsi.DeviceMLP(mlp)
    x = synthetic.student_instances(6)
    coal = st.sample_coalitions(6, 16, 40, seed=9)
    ex_base = torch.zeros(16, dtype=torch.float64, device="cuda")
    lib = st._declare()
    xd = torch.as_tensor(x, device="cuda")
    c = torch.as_tensor(coal.view(np.int32), device="cuda")
    out = torch.empty(c.shape, dtype=torch.float32, device="cuda")
    assert lib.tt_fsi_masked_game_sampled(st.ctypes.byref(dm.struct), st._p(xd), st._p(ex_base), 6, st._p(c), 40,
                                          st._p(out), fsi._stream_ptr()) == 0
    got = out.cpu().numpy()
    for b in range(6):
        ref = oracle_mod.masked_game(mlp, x[b], np.zeros(16), coalitions=coal[b].astype(np.uint64))
        assert np.max(np.abs(got[b] - ref)) <= 1e-5 * max(1.0, np.abs(ref).max())
    # residual of the exact scores: their surrogate, compared with the values
    v = fsi.masked_game(mlp, x, np.zeros(16))
    phi = fsi.Plan(16, 2, "exact", max_batch=6).apply(v).float()
    masks = torch.as_tensor(fsi.score_masks(16, 2).astype(np.uint32).view(np.int32), device="cuda")
    r = torch.empty(6, dtype=torch.float32, device="cuda")
    assert lib.tt_fsi_surrogate_residual(st._p(phi), 6, 137, st._p(masks), st._p(c), st._p(out), 40, st._p(r),
                                         fsi._stream_ptr()) == 0
    g = so.surrogate(phi.cpu().numpy(), fsi.score_masks(16, 2), coal.astype(np.uint64))
    ref_r = np.sqrt(((g - got) ** 2).mean(axis=1))
    assert np.allclose(r.cpu().numpy(), ref_r, rtol=1e-4, atol=1e-6)


def test_small_training_run_beats_baselines_and_falls_back():
    mlp = synthetic.workload_student_teacher()
    ex = st.Explainer(mlp, ell=2, hidden=256, batch=1024)
    train = ex.dataset(8192, first=0)
    held = ex.dataset(2048, first=200_000)
    losses = ex.train(train, epochs=60, lr=1e-3)
    assert losses[-1] < 0.5 * losses[0]
    phi = ex.predict_raw(held.x, held.target).double()
    err = ((phi - held.labels.double()) ** 2).mean().item()
    base_mean = ((train.labels.double().mean(0) - held.labels.double()) ** 2).mean().item()
    # linear regression baseline on [x, 1]
    Xtr = torch.cat([train.x.double(), torch.ones(train.x.shape[0], 1, device="cuda", dtype=torch.float64)], 1)
    Xh = torch.cat([held.x.double(), torch.ones(held.x.shape[0], 1, device="cuda", dtype=torch.float64)], 1)
    coef = torch.linalg.lstsq(Xtr, train.labels.double()).solution
    base_lin = ((Xh @ coef - held.labels.double()) ** 2).mean().item()
    assert err < 0.5 * base_lin and base_lin < base_mean, (err, base_mean, base_lin)
    # residual check with a calibrated threshold, then a corrupted student
    tau = ex.calibrate(held)
    assert np.isfinite(tau) and tau > 0
    out, fb = ex.explain(held.x[:512], held.target[:512], first=200_000)
    assert fb.float().mean().item() < 0.5
    p, m, v, stp = ex.student.state()
    ex.student.load_state(p * 40.0, m, v, stp)
    out, fb = ex.explain(held.x[:256], held.target[:256], first=200_000)
    assert bool(fb.all())
    # the fallback is the exact transform of the same value path as the labels
    assert torch.equal(out, ex.exact(held.x[:256].double()))
    # those values come from the tensor-core kernel (BF16 layer-2 products):
    # the labels are within a few per mille of labels from FP32 values
    exact32 = ex.exact(held.x[:256].double(), tc=False)
    lab_tc = held.labels[:256].double()
    assert (torch.linalg.norm(lab_tc - exact32) / torch.linalg.norm(exact32)).item() < 2e-2
