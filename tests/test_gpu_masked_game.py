"""Parity of the CUDA masked-model value function against the oracle's
direct forward passes (needs a GB300).  The two sides use their own erf, so
agreement is to a few ulps of the value scale, not bit for bit."""
import numpy as np
import pytest

import paper_2601_01903_gb300 as fsi
from paper_2601_01903_gb300 import synthetic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.mark.parametrize("d,h1,h2,B", [(1, 4, 3, 2), (3, 8, 5, 3), (6, 16, 12, 2), (9, 16, 12, 3),
                                       (11, 33, 7, 2)])
def test_small_models_every_coalition(oracle_mod, d, h1, h2, B):
    mlp = synthetic.random_mlp(d, h1, h2, seed=d)
    mlp.b1[:] = 0.1
    mlp.b2[:] = -0.2
    mlp.b3[:] = 0.3
    x = synthetic.gaussian_instances(B, d, seed=d)
    base = synthetic.Stream(d, 5).normal(d)
    got = fsi.masked_game(mlp, x, base).cpu().numpy()
    for b in range(B):
        assert _rel(got[b], oracle_mod.masked_game(mlp, x[b], base)) <= TOL


def test_mlp_d14_workload_and_chain(oracle_mod):
    w = synthetic.workload_mlp_d14()
    v = fsi.masked_game(w.mlp, w.x, w.baseline)
    vh = v.cpu().numpy()
    for b in (0, 31, 63):
        assert _rel(vh[b], oracle_mod.masked_game(w.mlp, w.x[b], w.baseline)) <= TOL
    phi = fsi.Plan(14, 2, "exact", max_batch=64).apply(v).cpu().numpy()
    ref = oracle_mod.fsi(vh, 14, 2)
    assert np.max(np.abs(phi - ref)) / np.abs(vh).max() <= 1e-10


@pytest.mark.parametrize("maker,d", [(synthetic.workload_mlp_d20, 20), (synthetic.workload_mlp_d24, 24)])
def test_large_workloads_sampled(oracle_mod, maker, d):
    w = maker()
    B = min(w.B, 4)
    v = fsi.masked_game(w.mlp, w.x[:B], w.baseline).cpu().numpy()
    coal = synthetic.Stream(99, d).integers(0, (1 << d) - 1, 3000).astype(np.uint64)
    coal = np.concatenate([coal, np.array([0, (1 << d) - 1, 1, 1 << (d - 1)], dtype=np.uint64)])
    for b in range(B):
        ref = oracle_mod.masked_game(w.mlp, w.x[b], w.baseline, coalitions=coal)
        assert _rel(v[b][coal.astype(np.int64)], ref) <= TOL


def test_float32_output(oracle_mod):
    w = synthetic.workload_mlp_d14()
    v32 = fsi.masked_game(w.mlp, w.x[:2], w.baseline, dtype=torch.float32).cpu().numpy()
    ref = oracle_mod.masked_game(w.mlp, w.x[0], w.baseline)
    assert _rel(v32[0].astype(np.float64), ref) <= 1e-5


# ---------------------------------------------------------------------------
# Tensor-core value function (label path): BF16 layer-2 operands
# ---------------------------------------------------------------------------

# The emulation below rounds the same operands to BF16, but computes layer 1
# in float64 where the GPU uses float32: an activation whose two values sit on
# either side of a BF16 rounding boundary rounds to neighbouring BF16 numbers,
# and each such one-ulp difference (2^-8 relative) moves v by up to ~2e-4 of
# max|v| at these widths.  The bound allows a handful of them per coalition.
TC_EMU_TOL = 5e-3
TC_EXACT_TOL = 3e-2  # against the float64 forward pass: the BF16 precision of this path


def _forward_bf16(mlp, z):
    """The tensor-core path's arithmetic in float64: layer-1 activations and
    W2 rounded to bfloat16 (round to nearest even), everything else exact."""
    from oracle.student import bf16_round, gelu
    a1 = bf16_round(gelu(z @ mlp.W1.T + mlp.b1))
    z2 = a1 @ bf16_round(mlp.W2).T + mlp.b2
    return (gelu(z2) @ np.asarray(mlp.W3).reshape(-1)) + float(np.asarray(mlp.b3).reshape(-1)[0])


def _inputs(x, base, masks, d):
    bits = ((masks[:, None] >> np.arange(d)) & 1).astype(bool)
    return np.where(bits, x[None, :], base[None, :])


@pytest.mark.parametrize("d,B", [(9, 2), (16, 2), (20, 1)])
def test_tensor_core_every_coalition(oracle_mod, d, B):
    mlp = synthetic.random_mlp(d, 128, 128, seed=40 + d)
    mlp.b1[:] = 0.05
    mlp.b2[:] = -0.1
    x = synthetic.gaussian_instances(B, d, seed=d)
    base = synthetic.Stream(d, 9).normal(d) * 0.1
    got = fsi.masked_game_tc(mlp, x, base).cpu().numpy().astype(np.float64)
    masks = np.arange(1 << d, dtype=np.int64)
    for b in range(B):
        if d > 16:  # a sample of rows at d = 20
            masks = synthetic.Stream(d, 11).integers(0, (1 << d) - 1, 4096).astype(np.int64)
        ref = _forward_bf16(mlp, _inputs(x[b], base, masks, d))
        assert _rel(got[b][masks], ref) <= TC_EMU_TOL
        if d <= 16:
            assert _rel(got[b], oracle_mod.masked_game(mlp, x[b], base)) <= TC_EXACT_TOL


def test_tensor_core_listed_coalitions():
    d, B, K = 16, 5, 64
    mlp = synthetic.random_mlp(d, 128, 128, seed=3)
    x = synthetic.gaussian_instances(B, d, seed=7)
    base = np.zeros(d)
    coal = synthetic.Stream(1, 2).integers(0, (1 << d) - 1, B * K).astype(np.uint32).reshape(B, K)
    got = fsi.masked_game_tc(mlp, x, base, coalitions=coal).cpu().numpy().astype(np.float64)
    for b in range(B):
        ref = _forward_bf16(mlp, _inputs(x[b], base, coal[b].astype(np.int64), d))
        assert _rel(got[b], ref) <= TC_EMU_TOL


def test_tensor_core_path_rejects_other_shapes():
    mlp = synthetic.random_mlp(10, 64, 64, seed=1)
    x = synthetic.gaussian_instances(1, 10, seed=1)
    with pytest.raises(fsi.FsiError) as e:
        fsi.masked_game_tc(mlp, x, np.zeros(10))
    assert e.value.status == 2
    small = synthetic.random_mlp(5, 128, 128, seed=1)
    with pytest.raises(fsi.FsiError) as e:
        fsi.masked_game_tc(small, synthetic.gaussian_instances(1, 5, seed=1), np.zeros(5))
    assert e.value.status == 2


# ---------------------------------------------------------------------------
# Interventional value function (mean over background rows, Section 4.1)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("d,h,B,n_bg", [(9, 16, 2, 5), (14, 32, 1, 3)])
def test_interventional_float64(oracle_mod, d, h, B, n_bg):
    mlp = synthetic.random_mlp(d, h, h, seed=d + 50)
    mlp.b2[:] = 0.1
    x = synthetic.gaussian_instances(B, d, seed=d)
    bg = synthetic.gaussian_instances(n_bg, d, seed=d + 1)
    got = fsi.masked_game_interventional(mlp, x, bg).cpu().numpy()
    for b in range(B):
        assert _rel(got[b], oracle_mod.masked_game_interventional(mlp, x[b], bg)) <= TOL


@pytest.mark.parametrize("d,B,n_bg", [(12, 2, 4), (16, 1, 3)])
def test_interventional_tensor_core(oracle_mod, d, B, n_bg):
    mlp = synthetic.random_mlp(d, 128, 128, seed=60 + d)
    x = synthetic.gaussian_instances(B, d, seed=d)
    bg = synthetic.gaussian_instances(n_bg, d, seed=d + 2) * 0.5
    got = fsi.masked_game_tc(mlp, x, bg).cpu().numpy().astype(np.float64)
    masks = np.arange(1 << d, dtype=np.int64)
    for b in range(B):
        ref = np.mean([_forward_bf16(mlp, _inputs(x[b], bg[k], masks, d)) for k in range(n_bg)], axis=0)
        assert _rel(got[b], ref) <= TC_EMU_TOL
        assert _rel(got[b], oracle_mod.masked_game_interventional(mlp, x[b], bg)) <= TC_EXACT_TOL
    # listed coalitions give the same numbers as the dense tiles
    coal = synthetic.Stream(d, 3).integers(0, (1 << d) - 1, B * 64).astype(np.uint32).reshape(B, 64)
    listed = fsi.masked_game_tc(mlp, x, bg, coalitions=coal).cpu().numpy().astype(np.float64)
    for b in range(B):
        assert _rel(listed[b], got[b][coal[b].astype(np.int64)]) <= TC_EMU_TOL


def test_one_background_row_is_the_baseline_path():
    d = 13
    mlp = synthetic.random_mlp(d, 128, 128, seed=2)
    x = synthetic.gaussian_instances(2, d, seed=2)
    base = synthetic.gaussian_instances(1, d, seed=9)
    a = fsi.masked_game_tc(mlp, x, base[0])
    b = fsi.masked_game_tc(mlp, x, base)
    assert torch.equal(a, b)
    c = fsi.masked_game(mlp, x, base[0])
    e = fsi.masked_game_interventional(mlp, x, base)
    assert torch.equal(c, e)
