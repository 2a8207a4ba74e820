"""Batched uneven games (one persistent launch) against the oracle, the
per-game and CUDA-graph paths against it, the autotuner, and the bounded
dependency wait (needs a GB300)."""
import numpy as np
import pytest

import paper_2601_01903_gb300 as fsi
from paper_2601_01903_gb300 import synthetic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-10


def _ragged(count=40):
    return synthetic.workload_uneven(count=count)


def _oracle_all(oracle_mod, g):
    out = np.empty(g.n_phi)
    for k in range(len(g.d)):
        d, ell = int(g.d[k]), int(g.ell[k])
        v = g.v[g.v_off[k]:g.v_off[k] + (1 << d)]
        n = oracle_mod.n_scores(d, ell)
        out[g.phi_off[k]:g.phi_off[k] + n] = oracle_mod.fsi(v, d, ell)[0]
    return out


def _check_per_game(g, got, ref):
    for k in range(len(g.d)):
        d = int(g.d[k])
        v = g.v[g.v_off[k]:g.v_off[k] + (1 << d)]
        n = fsi.num_scores(d, int(g.ell[k]))
        sl = slice(int(g.phi_off[k]), int(g.phi_off[k]) + n)
        err = np.max(np.abs(got[sl] - ref[sl])) / max(np.abs(v).max(), 1e-300)
        assert err <= TOL, (k, d, int(g.ell[k]), err)


def test_uneven_batch_all_paths_match_oracle(oracle_mod):
    g = _ragged(40)
    ref = _oracle_all(oracle_mod, g)
    v = torch.as_tensor(g.v, device="cuda")
    b = fsi.Batch.from_ragged(g)
    outs = {}
    for name in ("apply", "apply_per_game", "apply_graph"):
        phi = torch.full((g.n_phi,), np.nan, dtype=torch.float64, device="cuda")
        getattr(b, name)(v, phi)
        b.check()
        outs[name] = phi.cpu().numpy()
        _check_per_game(g, outs[name], ref)
    # the exact arithmetic is order independent: all three paths agree bit for bit
    assert np.array_equal(outs["apply"], outs["apply_per_game"])
    assert np.array_equal(outs["apply"], outs["apply_graph"])


_FULL = {}


@pytest.mark.parametrize("arith", ["exact", "f64"])
def test_uneven_1024_workload_every_game_matches_oracle(oracle_mod, arith):
    """The whole batched workload (1024 Moebius-sparse games, d in 10..20,
    l in 1..3, one persistent launch): every score of every game against
    the oracle, in both arithmetics, and efficiency on every game."""
    if "g" not in _FULL:
        g = synthetic.workload_uneven()
        _FULL["g"] = (g, _oracle_all(oracle_mod, g))
    g, ref = _FULL["g"]
    b = fsi.Batch.from_ragged(g, arith=arith)
    phi = torch.full((g.n_phi,), np.nan, dtype=torch.float64, device="cuda")
    b.apply(torch.as_tensor(g.v, device="cuda"), phi)
    b.check()
    got = phi.cpu().numpy()
    _check_per_game(g, got, ref)
    for k in range(len(g.d)):
        d = int(g.d[k])
        v = g.v[g.v_off[k]:g.v_off[k] + (1 << d)]
        po = int(g.phi_off[k])
        n = fsi.num_scores(d, int(g.ell[k]))
        assert abs(got[po + 1:po + n].sum() - (v[-1] - v[0])) <= 1e-9 * max(np.abs(v).max(), 1e-300)


def test_mixed_batch_with_games_off_the_fast_path(oracle_mod):
    games, vs, off, poff = [], [], 0, 0
    specs = [(12, 3), (5, 5), (9, 4), (14, 2), (3, 1), (13, 13), (16, 1), (11, 5), (15, 4)]
    for i, (d, ell) in enumerate(specs):
        v = synthetic.Stream(300 + i, d).normal(1 << d)
        games.append((d, ell, off, poff))
        vs.append(v)
        off += 1 << d
        poff += fsi.num_scores(d, ell)
    vall = np.concatenate(vs)
    b = fsi.Batch(games)
    phi = torch.zeros(poff, dtype=torch.float64, device="cuda")
    b.apply(torch.as_tensor(vall, device="cuda"), phi)
    b.check()
    got = phi.cpu().numpy()
    for (d, ell, vo, po), v in zip(games, vs):
        ref = oracle_mod.fsi(v, d, ell)[0]
        assert np.max(np.abs(got[po:po + len(ref)] - ref)) / np.abs(v).max() <= TOL, (d, ell)


def test_autotuner_keeps_results(oracle_mod):
    g = _ragged(24)
    ref = _oracle_all(oracle_mod, g)
    v = torch.as_tensor(g.v, device="cuda")
    b = fsi.Batch.from_ragged(g)
    phi = torch.zeros(g.n_phi, dtype=torch.float64, device="cuda")
    t, c = b.autotune(v, phi)
    assert t in (1, 2, 4, 8) and c in (16, 64, 256)
    phi.zero_()
    b.apply(v, phi)
    b.check()
    _check_per_game(g, phi.cpu().numpy(), ref)


def test_float32_batch_error_is_small(oracle_mod):
    g = _ragged(12)
    ref = _oracle_all(oracle_mod, g)
    b = fsi.Batch.from_ragged(g, arith="f32")
    phi = torch.zeros(g.n_phi, dtype=torch.float32, device="cuda")
    b.apply(torch.as_tensor(g.v, device="cuda", dtype=torch.float32), phi)
    b.check()
    got = phi.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(got - ref)) / np.abs(g.v).max() < 1e-4


def test_dependency_wait_times_out_and_reports():
    """A score chunk waits for a tile that is never produced (test hook):
    the wait gives up after its poll limit, the batch reports
    TT_FSI_ERR_TIMEOUT, and the next normal call works."""
    g = _ragged(6)
    v = torch.as_tensor(g.v, device="cuda")
    b = fsi.Batch.from_ragged(g)
    phi = torch.zeros(g.n_phi, dtype=torch.float64, device="cuda")
    b.set_wait_limit(20000, inject_missing_tile=True)
    b.apply(v, phi)
    with pytest.raises(fsi.FsiError) as e:
        b.check()
    assert e.value.status == 5
    b.set_wait_limit(4000000, inject_missing_tile=False)
    b.apply(v, phi)
    b.check()
    assert torch.isfinite(phi).all()
