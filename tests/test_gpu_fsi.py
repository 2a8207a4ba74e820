"""Parity of the CUDA FSI path against the CPU oracle (needs a GB300).

Bar: max |phi_gpu - phi_oracle| / max |v| <= 1e-10 for the exact and the
float64 arithmetic, on the same seeded inputs; the float32 variant's error
is measured and held to a loose bound only.  Every call goes through the
C ABI (via the thin Python binding)."""
import numpy as np
import pytest

import paper_2601_01903_gb300 as fsi
from paper_2601_01903_gb300 import synthetic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-10


def _gpu(x, dtype=None):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dtype or torch.float64, device="cuda")


def _noise_games(d, B, seed, v0=True):
    v = synthetic.Stream(4242 + seed, d).normal(B << d).reshape(B, 1 << d)
    if v0:
        v[:, 0] = 0.0
    return v


def _rel_err(got, ref, v):
    return float(np.max(np.abs(got - ref)) / max(np.max(np.abs(v)), 1e-300))


def _run(v, d, ell, arith):
    plan = fsi.Plan(d, ell, arith, max_batch=v.shape[0])
    dt = torch.float32 if arith == "f32" else torch.float64
    out = plan.apply(_gpu(v, dt))
    plan.check()
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64), plan


@pytest.mark.parametrize("arith", ["exact", "f64"])
def test_mobius_d8_workload(oracle_mod, arith):
    w = synthetic.workload_mobius_d8()
    got, _ = _run(w["v"], 8, 2, arith)
    ref = oracle_mod.fsi(w["v"], 8, 2)
    assert got.shape == (1, 37)
    assert _rel_err(got, ref, w["v"]) <= TOL


@pytest.mark.parametrize("arith", ["exact", "f64"])
@pytest.mark.parametrize("d,ell,B", [
    (1, 1, 1), (2, 1, 3), (3, 2, 2), (5, 3, 4), (6, 1, 1), (7, 2, 5), (9, 3, 3),
    (11, 2, 2), (11, 3, 1), (12, 2, 2), (12, 3, 2), (13, 2, 3), (13, 3, 1), (14, 1, 2),
    (15, 2, 2), (16, 3, 1), (17, 2, 1), (18, 3, 1),
])
def test_random_games_against_oracle(oracle_mod, arith, d, ell, B):
    v = _noise_games(d, B, seed=d * 7 + ell, v0=False)
    got, plan = _run(v, d, ell, arith)
    ref = oracle_mod.fsi(v, d, ell)
    assert got.shape == ref.shape
    assert _rel_err(got, ref, v) <= TOL, (d, ell, plan.tile_bits)


@pytest.mark.parametrize("arith", ["exact", "f64"])
@pytest.mark.parametrize("d,ell", [(1, 3), (4, 4), (6, 9), (9, 9), (13, 13), (14, 15)])
def test_order_at_least_d_gives_moebius(oracle_mod, arith, d, ell):
    v = _noise_games(d, 2, seed=100 + d, v0=False)
    got, _ = _run(v, d, ell, arith)
    ref = oracle_mod.fsi(v, d, ell)
    assert _rel_err(got, ref, v) <= TOL


@pytest.mark.parametrize("arith", ["exact", "f64"])
def test_order_4_and_5(oracle_mod, arith):
    for d, ell in ((10, 4), (13, 5)):
        v = _noise_games(d, 1, seed=200 + d, v0=False)
        got, _ = _run(v, d, ell, arith)
        assert _rel_err(got, oracle_mod.fsi(v, d, ell), v) <= TOL


def test_masked_mlp_d14_batch64(oracle_mod):
    """d=14, l=2, 64 instances of the 14-64-64-1 GELU MLP game."""
    w = synthetic.workload_mlp_d14()
    v = np.stack([oracle_mod.masked_game(w.mlp, w.x[i], w.baseline) for i in range(w.B)])
    ref = oracle_mod.fsi(v, 14, 2)
    for arith in ("exact", "f64"):
        got, _ = _run(v, 14, 2, arith)
        assert _rel_err(got, ref, v) <= TOL, arith
    got32, _ = _run(v, 14, 2, "f32")
    assert _rel_err(got32, ref, v) <= 1e-3


_CACHE = {}


def _d20_batch(oracle_mod):
    """The d = 20, l = 3 batch: two instances of the 20-128-128-1 MLP game
    (oracle-made value vectors) and 14 white-noise games, with the oracle's
    scores of all 16 (computed once per session)."""
    if "d20" not in _CACHE:
        w = synthetic.workload_mlp_d20()
        v = np.empty((16, 1 << 20))
        for i in range(2):
            v[i] = oracle_mod.masked_game(w.mlp, w.x[i], w.baseline)
        v[2:] = _noise_games(20, 14, seed=20)
        _CACHE["d20"] = (v, oracle_mod.fsi(v, 20, 3))
    return _CACHE["d20"]


@pytest.mark.parametrize("arith", ["exact", "f64"])
def test_masked_mlp_d20_order3(oracle_mod, arith):
    """d=20, l=3, 16 games in one call (the headline batch size): every
    score of every game against the oracle, and efficiency on every game."""
    v, ref = _d20_batch(oracle_mod)
    got, _ = _run(v, 20, 3, arith)
    assert got.shape == ref.shape == (16, 1351)
    for k in range(16):
        assert _rel_err(got[k], ref[k], v[k]) <= TOL, (arith, k)
    eff = got[:, 1:].sum(axis=1) - (v[:, -1] - v[:, 0])
    assert np.max(np.abs(eff) / np.abs(v).max(axis=1)) < 1e-9


@pytest.mark.parametrize("arith", ["exact", "f64"])
def test_d24_order2_sampled(oracle_mod, arith):
    """d=24, l=2, one game (2^24 float64 = 128 MiB): every score against the
    oracle's explicit superset sums, and efficiency."""
    if "d24" not in _CACHE:
        v = _noise_games(24, 1, seed=24)
        _CACHE["d24"] = (v, oracle_mod.fsi(v, 24, 2))
    v, ref = _CACHE["d24"]
    got, plan = _run(v, 24, 2, arith)
    assert _rel_err(got, ref, v) <= TOL
    assert abs(got[0, 1:].sum() - (v[0, -1] - v[0, 0])) <= 1e-9 * np.abs(v).max()


@pytest.mark.parametrize("arith", ["exact", "f64"])
def test_teacher_games_d16_order2(oracle_mod, arith):
    """d=16, l=2 on 8 instances of the explainer's teacher (16-128-128-1
    MLP, AR(1) inputs): the exact transform that labels the student."""
    mlp = synthetic.workload_student_teacher()
    x = synthetic.student_instances(8)
    v = np.stack([oracle_mod.masked_game(mlp, x[i], np.zeros(16)) for i in range(8)])
    got, _ = _run(v, 16, 2, arith)
    ref = oracle_mod.fsi(v, 16, 2)
    for k in range(8):
        assert _rel_err(got[k], ref[k], v[k]) <= TOL, (arith, k)


def test_d26_order3_sampled_scores(oracle_mod):
    """d=26, l=3, one game (2^26 float64 = 512 MiB, 2^14 tiles): sampled
    scores of every size, with low and high players, against the oracle's
    direct route from v (at this d the float64 Moebius route itself is off
    by about 2e-10 of max|v| through cancellation in the coefficients)."""
    d, ell = 26, 3
    v = _noise_games(d, 1, seed=26)
    got, plan = _run(v, d, ell, "exact")
    masks = fsi.score_masks(d, ell)
    pick = [0, 1, 2, 12, 25, 26, 27, 40, 200, 300, 351, 352, 353, 1000, 2000, 2601, len(masks) - 1]
    ref = oracle_mod.fsi_direct(v, d, ell, [int(masks[i]) for i in pick])
    assert _rel_err(got[0, pick], ref, v) <= TOL


def test_sparse_games_recover_moebius_coefficients(oracle_mod):
    g = synthetic.workload_uneven(count=6, keep_m=True)
    for k in range(6):
        d, ell = int(g.d[k]), int(g.ell[k])
        v = g.v[g.v_off[k]:g.v_off[k] + (1 << d)].reshape(1, -1)
        got, _ = _run(v, d, 5, "exact")
        masks = oracle_mod.score_masks(d, 5).astype(np.int64)
        assert np.max(np.abs(got[0] - g.m[k][masks])) <= TOL * max(1.0, np.abs(v).max())
        got_l, _ = _run(v, d, ell, "exact")
        assert _rel_err(got_l, oracle_mod.fsi(v, d, ell), v) <= TOL


def test_float32_variant_error_is_reported(oracle_mod):
    v = _noise_games(16, 2, seed=16)
    got, _ = _run(v, 16, 3, "f32")
    err = _rel_err(got, oracle_mod.fsi(v, 16, 3), v)
    assert err < 5e-2  # cancellation on white noise; reported, not a parity claim


def test_scale_invariance_of_exact_path(oracle_mod):
    """Tiles of very different magnitude in one game (per-tile fixed point)."""
    d = 16
    v = _noise_games(d, 1, seed=3, v0=False)
    v[0, : 1 << 12] *= 1e-9
    v[0, 1 << 13: 3 << 12] *= 1e6
    got, _ = _run(v, d, 2, "exact")
    assert _rel_err(got, oracle_mod.fsi(v, d, 2), v) <= TOL


@pytest.mark.parametrize("d,ell,B", [(21, 4, 1), (21, 3, 2), (19, 4, 2), (12, 4, 3), (13, 2, 2)])
def test_scaled_tile_blocks_against_oracle(oracle_mod, d, ell, B):
    """Games from one tile (d = 12) to 2^9 tiles (d = 21) at orders 2 to 4,
    with a block of tiles scaled down so that the combine's alignment
    shifts are not all zero."""
    v = _noise_games(d, B, seed=d + 13 * ell, v0=False)
    v[:, : 1 << min(d, 14)] *= 1e-5
    got, _ = _run(v, d, ell, "exact")
    assert _rel_err(got, oracle_mod.fsi(v, d, ell), v) <= TOL


@pytest.mark.parametrize("d,ell,B,scale", [
    (12, 3, 2, 0), (13, 1, 3, 0), (15, 4, 1, 0), (19, 2, 2, -17), (20, 3, 2, -200),
    (21, 3, 1, 0), (22, 3, 1, -30), (22, 2, 1, -400),
])
def test_split_combine_writes_every_score(oracle_mod, d, ell, B, scale):
    """Games of 1 to 2^10 tiles through the tile-then-combine schedule:
    every score is written (the output starts as NaN), bitwise equal to the
    fused schedule's combine, and within the bar of the oracle -- also with
    a block of tiles 2^scale below the rest, which beyond the alignment cap
    takes rounding right shifts."""
    v = _noise_games(d, B, seed=d * 3 + ell, v0=False)
    if scale:
        v[:, : 1 << min(d, 14)] *= 2.0 ** scale
    vg = _gpu(v)
    plan = fsi.Plan(d, ell, "exact", max_batch=B)
    out = torch.full((B, plan.n_scores), float("nan"), dtype=torch.float64, device="cuda")
    plan.apply(vg, out=out)
    plan.set_schedule(fused=True)
    fused = plan.apply(vg)
    plan.check()
    assert not torch.isnan(out).any()
    assert torch.equal(out, fused)
    ref = oracle_mod.fsi(v, d, ell)
    assert _rel_err(out.cpu().numpy(), ref, v) <= TOL


@pytest.mark.parametrize("d,ell", [(16, 2), (14, 3)])
def test_tiny_tiles_and_subnormals(oracle_mod, d, ell):
    """A tile whose largest value is below 2^-980 (the exact path's general
    conversion) and a tile mixing normal values with zeros and subnormals
    (the branch-free conversion) against the oracle."""
    v = _noise_games(d, 1, seed=11, v0=False)
    v[0, 2 << 12: 3 << 12] *= 2.0 ** -1000
    v[0, 3 << 12: (3 << 12) + 64] = 5e-324
    v[0, (3 << 12) + 64: (3 << 12) + 96] = 0.0
    got, _ = _run(v, d, ell, "exact")
    assert _rel_err(got, oracle_mod.fsi(v, d, ell), v) <= TOL


@pytest.mark.parametrize("k", [-990, -600, 600])
def test_power_of_two_scaling_is_exact(k):
    """Scaling a game by 2^k moves every tile across the conversion's two
    branches (k = -990 leaves only tiny tiles) without changing the integer
    arithmetic: the scores scale by 2^k bit for bit."""
    d, ell = 15, 3
    v = _noise_games(d, 2, seed=12, v0=False)
    got, _ = _run(v, d, ell, "exact")
    got_s, _ = _run(v * 2.0 ** k, d, ell, "exact")
    ref = got * 2.0 ** k
    normal = np.abs(ref) >= 2.0 ** -1022   # a subnormal output loses bits when written
    assert normal.mean() > 0.99
    assert np.array_equal(got_s[normal], ref[normal])


def test_nonfinite_input_is_reported():
    v = _noise_games(10, 1, seed=1)
    v[0, 77] = np.inf
    plan = fsi.Plan(10, 2, "exact", max_batch=1)
    plan.apply(_gpu(v))
    with pytest.raises(fsi.FsiError) as e:
        plan.check()
    assert e.value.status == 6
    plan.check()  # the fault word was cleared


def test_empty_batch_and_bad_arguments():
    plan = fsi.Plan(8, 2, "exact", max_batch=2)
    lib = fsi.native.load()
    assert lib.tt_fsi_apply(plan.handle, None, 0, None, None) == 0
    x = torch.zeros((3, 256), dtype=torch.float64, device="cuda")
    y = torch.zeros((3, 37), dtype=torch.float64, device="cuda")
    assert lib.tt_fsi_apply(plan.handle, x.data_ptr(), 3, y.data_ptr(), None) == 1  # > max_batch


def test_repeated_calls_are_bitwise_identical():
    v = _gpu(_noise_games(18, 2, seed=5))
    plan = fsi.Plan(18, 3, "exact", max_batch=2)
    a = plan.apply(v).clone()
    b = plan.apply(v).clone()
    assert torch.equal(a, b)


@pytest.mark.parametrize("arith", ["exact", "f64", "f32"])
def test_back_to_back_calls_with_different_inputs(arith):
    """The combine is launched as the tile launch's programmatic dependent;
    calls enqueued back to back on one stream with different inputs, and no
    host sync between them, must each see only their own partial scores."""
    d, ell, B = 18, 3, 3
    dt = torch.float32 if arith == "f32" else torch.float64
    vs = [_gpu(_noise_games(d, B, seed=60 + k), dt) for k in range(3)]
    plan = fsi.Plan(d, ell, arith, max_batch=B)
    refs = [plan.apply(v).clone() for v in vs]
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    outs = [torch.empty_like(refs[0]) for _ in range(12)]
    with torch.cuda.stream(s):
        for i in range(12):
            plan.apply(vs[i % 3], out=outs[i], stream=s)
    s.synchronize()
    plan.check()
    for i in range(12):
        assert torch.equal(outs[i], refs[i % 3])


@pytest.mark.parametrize("arith", ["exact", "f64", "f32"])
@pytest.mark.parametrize("d,ell,B", [(14, 3, 5), (20, 2, 2), (9, 3, 7), (16, 1, 3), (13, 3, 1), (17, 4, 2)])
def test_fused_schedule_matches_two_launches(arith, d, ell, B):
    """The fused persistent launch and the tile-then-combine launches run the
    same per-tile and per-score code: results are bitwise identical."""
    dt = torch.float32 if arith == "f32" else torch.float64
    v = _gpu(_noise_games(d, B, seed=d + ell), dt)
    plan = fsi.Plan(d, ell, arith, max_batch=B)
    split = plan.apply(v).clone()  # default schedule: tile launch + combine launch
    plan.set_schedule(fused=True)
    fused = plan.apply(v).clone()
    plan.check()
    assert torch.equal(fused, split)


@pytest.mark.parametrize("tpi,spi", [(1, 1), (3, 64), (8, 1000), (256, 7)])
def test_fused_work_item_sizes(oracle_mod, tpi, spi):
    d, ell, B = 15, 3, 3
    v = _noise_games(d, B, seed=11)
    ref = oracle_mod.fsi(v, d, ell)
    plan = fsi.Plan(d, ell, "exact", max_batch=B)
    plan.set_schedule(fused=True, tiles_per_item=tpi, scores_per_item=spi)
    got = plan.apply(_gpu(v)).cpu().numpy()
    plan.check()
    assert _rel_err(got, ref, v) <= TOL


def test_fused_wait_timeout_is_reported_and_recoverable():
    """Test hook: every combine wait expects one tile more than exists, so
    each wait runs out after a short bound; the timeout is latched, read by
    the host, and the next call with the hook off is correct."""
    d, ell, B = 14, 2, 2
    v = _gpu(_noise_games(d, B, seed=3))
    plan = fsi.Plan(d, ell, "exact", max_batch=B)
    plan.set_schedule(fused=True)
    ref = plan.apply(v).clone()
    plan.check()
    plan.set_wait_limit(20000, inject_missing=True)
    plan.apply(v)
    with pytest.raises(fsi.FsiError) as e:
        plan.check()
    assert e.value.status == 5
    plan.set_wait_limit(4000000, inject_missing=False)
    again = plan.apply(v)
    plan.check()
    assert torch.equal(again, ref)


@pytest.mark.parametrize("arith", ["exact", "f64"])
@pytest.mark.parametrize("d,B", [(16, 2), (14, 3), (7, 4), (5, 2)])
def test_order_4_fast_path(oracle_mod, arith, d, B):
    """Order 4 on the 12-bit-tile path: several tiles (d = 14, 16) and
    games smaller than a tile (d = 5, 7: null players fill the tile)."""
    v = _noise_games(d, B, seed=400 + d, v0=False)
    got, plan = _run(v, d, 4, arith)
    assert plan.tile_bits == 12
    assert _rel_err(got, oracle_mod.fsi(v, d, 4), v) <= TOL


def test_order_4_float32_error_is_small(oracle_mod):
    d = 15
    v = _noise_games(d, 2, seed=77)
    got, _ = _run(v, d, 4, "f32")
    assert _rel_err(got, oracle_mod.fsi(v, d, 4), v) <= 1e-4


@pytest.mark.parametrize("arith", ["exact", "f64"])
@pytest.mark.parametrize("d,ell,B", [(14, 2, 3), (16, 3, 2), (9, 3, 2), (13, 4, 1)])
def test_site_sweep_variant_matches_oracle(oracle_mod, arith, d, ell, B):
    """The site-by-site sweep (comparison variant of the paper's own
    formulation) gives the same scores within the parity bar."""
    v = _noise_games(d, B, seed=700 + d + ell)
    plan = fsi.Plan(d, ell, arith, max_batch=B, site_sweep=True)
    got = plan.apply(_gpu(v)).cpu().numpy()
    plan.check()
    assert _rel_err(got, oracle_mod.fsi(v, d, ell), v) <= TOL


@pytest.mark.parametrize("arith", ["exact", "f64", "f32"])
@pytest.mark.parametrize("d,ell,B", [(14, 2, 3), (16, 3, 2), (9, 3, 2), (13, 4, 1), (11, 5, 2), (5, 6, 2)])
def test_precontracted_sweep_matches_oracle(oracle_mod, arith, d, ell, B):
    """The precontracted operator (Section 3.5) swept site by site on v
    gives the same scores: bit for bit on the exact path (the channels are
    the same integers), within the parity bar in float64, within the float32
    bound in float32; l >= d keeps its Moebius pass."""
    v = _noise_games(d, B, seed=800 + d + ell)
    dt = torch.float32 if arith == "f32" else torch.float64
    plan = fsi.Plan(d, ell, arith, max_batch=B, precontract=True)
    got = plan.apply(_gpu(v, dt)).cpu().numpy().astype(np.float64)
    plan.check()
    assert _rel_err(got, oracle_mod.fsi(v, d, ell), v) <= (1e-4 if arith == "f32" else TOL)
    if arith == "exact":
        ref = fsi.Plan(d, ell, arith, max_batch=B, site_sweep=True)
        assert np.array_equal(got, ref.apply(_gpu(v)).cpu().numpy())


@pytest.mark.parametrize("arith", ["exact", "f32"])
@pytest.mark.parametrize("chunk", [0, 1, 3, 7])
@pytest.mark.parametrize("pinned,zero_copy", [(True, True), (True, False), (False, True)])
def test_host_pipeline_matches_device_apply(oracle_mod, arith, chunk, pinned, zero_copy):
    """tt_fsi_apply_host reads page-locked input in place, or moves the input
    in chunks of whole games on its own copy stream; every route and chunking
    gives the device path's scores bit for bit."""
    d, ell, B = 15, 3, 7
    v = _noise_games(d, B, seed=31)
    dt = torch.float32 if arith == "f32" else torch.float64
    plan = fsi.Plan(d, ell, arith, max_batch=B)
    ref = plan.apply(_gpu(v, dt)).cpu()
    plan.set_host_chunk(chunk)
    plan.set_host_zero_copy(zero_copy)
    vh = torch.as_tensor(v, dtype=dt)
    if pinned:
        vh = vh.pin_memory()
    got = plan.apply_host(vh)
    plan.check()
    assert torch.equal(got, ref)
    if arith == "exact":
        assert _rel_err(got.numpy(), oracle_mod.fsi(v, d, ell), v) <= TOL
    # a smaller batch through the same staging buffers
    got2 = plan.apply_host(vh[2:5])
    assert torch.equal(got2, ref[2:5])


def test_host_pipeline_bad_arguments():
    plan = fsi.Plan(10, 2, "exact", max_batch=2)
    with pytest.raises(RuntimeError):
        plan.set_host_chunk(-1)
    with pytest.raises(ValueError):
        plan.apply_host(torch.zeros((1, 1 << 10), dtype=torch.float64, device="cuda"))
    with pytest.raises(RuntimeError):
        plan.apply_host(torch.zeros((3, 1 << 10), dtype=torch.float64))
    assert plan.apply_host(torch.zeros((0, 1 << 10), dtype=torch.float64)).shape == (0, plan.n_scores)
