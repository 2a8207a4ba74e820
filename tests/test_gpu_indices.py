"""Parity of the CUDA path for the other interaction indices (SII, Banzhaf
BII, Shapley-Taylor STII, k-SII) against the oracle's definitions over
discrete derivatives (k-SII: their Bernoulli aggregation) (needs a GB300).  Same bar as FSI: max |phi_gpu - phi_oracle| /
max |v| <= 1e-10 for the exact and the float64 arithmetic."""
import numpy as np
import pytest

import paper_2601_01903_gb300 as fsi
from paper_2601_01903_gb300 import synthetic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-10
INDICES = ["sii", "bii", "stii", "ksii"]


def _games(d, B, seed):
    return synthetic.Stream(9000 + seed, d).normal(B << d).reshape(B, 1 << d)


def _run(v, d, ell, arith, index):
    dt = torch.float32 if arith == "f32" else torch.float64
    plan = fsi.Plan(d, ell, arith, max_batch=v.shape[0], index=index)
    out = plan.apply(torch.as_tensor(v, dtype=dt, device="cuda"))
    plan.check()
    return out.cpu().numpy().astype(np.float64), plan


def _err(got, ref, v):
    return float(np.max(np.abs(got - ref)) / np.max(np.abs(v)))


@pytest.mark.parametrize("arith", ["exact", "f64"])
@pytest.mark.parametrize("index", INDICES)
@pytest.mark.parametrize("d,ell,B", [
    (14, 2, 2),   # 12-bit tiles, 4 tiles per game
    (16, 3, 1),   # 16 tiles
    (9, 3, 3),    # one tile, null players fill it
    (15, 4, 1),   # order 4 on the fast path
    (11, 5, 2),   # generic tile kernels
])
def test_index_matches_definition(oracle_mod, arith, index, d, ell, B):
    v = _games(d, B, d * 10 + ell)
    got, _ = _run(v, d, ell, arith, index)
    ref = oracle_mod.interaction(v, d, ell, index)
    assert _err(got, ref, v) <= TOL


@pytest.mark.parametrize("index", INDICES)
@pytest.mark.parametrize("d,ell", [(4, 6), (3, 3), (7, 7), (9, 12)])
def test_order_at_least_d(oracle_mod, index, d, ell):
    """l >= d: every subset is scored; SII and BII still sum over supersets,
    STII and k-SII (like FSI) return the Moebius coefficients."""
    v = _games(d, 2, d + ell)
    got, _ = _run(v, d, ell, "exact", index)
    ref = oracle_mod.interaction(v, d, ell, index)
    assert _err(got, ref, v) <= TOL


@pytest.mark.parametrize("index", INDICES)
def test_index_float32_error_is_small(oracle_mod, index):
    d, ell = 13, 3
    v = _games(d, 2, 5)
    got, _ = _run(v, d, ell, "f32", index)
    assert _err(got, oracle_mod.interaction(v, d, ell, index), v) <= 1e-4


@pytest.mark.parametrize("index", INDICES)
def test_index_in_uneven_batch(oracle_mod, index):
    specs = [(12, 3), (6, 2), (14, 1), (10, 4), (8, 5)]
    games, vs, off, poff = [], [], 0, 0
    for i, (d, ell) in enumerate(specs):
        games.append((d, ell, off, poff))
        vs.append(_games(d, 1, 100 + i)[0])
        off += 1 << d
        poff += fsi.num_scores(d, ell)
    b = fsi.Batch(games, index=index)
    phi = torch.zeros(poff, dtype=torch.float64, device="cuda")
    b.apply(torch.as_tensor(np.concatenate(vs), device="cuda"), phi)
    b.check()
    got = phi.cpu().numpy()
    for (d, ell, _, po), v in zip(games, vs):
        ref = oracle_mod.interaction(v, d, ell, index)[0]
        assert _err(got[po:po + len(ref)], ref, v) <= TOL, (index, d, ell)


def test_unknown_index_is_rejected():
    lib = fsi.native.load()
    import ctypes
    h = ctypes.c_void_p()
    assert lib.tt_fsi_plan_create_index(10, 2, 7, 0, 1, ctypes.byref(h)) == 1


@pytest.mark.parametrize("arith", ["exact", "f64"])
def test_ksii_masked_mlp_d20_order3(oracle_mod, arith):
    """k-SII at the headline size (d = 20, l = 3) on a masked-MLP game:
    every score against the oracle, and the efficiency the paper states."""
    w = synthetic.workload_mlp_d20()
    v = oracle_mod.masked_game(w.mlp, w.x[3], w.baseline).reshape(1, -1)
    got, _ = _run(v, 20, 3, arith, "ksii")
    ref = oracle_mod.interaction(v, 20, 3, "ksii")
    assert _err(got, ref, v) <= TOL
    assert abs(got[0, 1:].sum() - (v[0, -1] - v[0, 0])) <= 1e-9 * np.abs(v).max()
