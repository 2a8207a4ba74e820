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
