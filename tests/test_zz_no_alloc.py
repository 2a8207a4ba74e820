"""The allocation-free entry point, tt_fsi_apply_noalloc, for callers that
cannot allocate device memory (applications that own every byte of device
memory through their own pool, services that must not allocate after
start-up).  It keeps its scratch in one static 64 MiB device array, so it
must give the same scores as the plan-based tt_fsi_apply, call after call,
whether it runs alone in a fresh process or after every other test.  This
file is named to be collected last."""
import ctypes

import numpy as np
import pytest

import paper_2601_01903_gb300 as fsi
from paper_2601_01903_gb300 import native, synthetic

TOL = 1e-10  # max |difference| / max |v|, the parity bar of the exact path


def _games(d, B, seed):
    return synthetic.Stream(777 + seed, d).normal(B << d).reshape(B, 1 << d)


def _noalloc(lib, d, ell, v, out, stream):
    return lib.tt_fsi_apply_noalloc(d, ell, ctypes.c_void_p(v.data_ptr()), v.shape[0],
                                    ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream.cuda_stream))


def test_oversized_requests_are_rejected_before_running():
    lib = native.load()
    dummy = ctypes.c_void_p(256)  # never dereferenced: the size check comes first
    assert lib.tt_fsi_apply_noalloc(20, 3, dummy, 33, dummy, None) == 2  # 33 games > 64 MiB
    assert lib.tt_fsi_apply_noalloc(24, 2, dummy, 10, dummy, None) == 2
    assert lib.tt_fsi_apply_noalloc(20, 0, dummy, 1, dummy, None) == 1  # l = 0
    assert lib.tt_fsi_apply_noalloc(20, 3, None, 1, dummy, None) == 1
    assert lib.tt_fsi_apply_noalloc(20, 3, dummy, 0, dummy, None) == 0   # empty batch


@pytest.mark.gpu
def test_noalloc_matches_plan_based_apply_and_oracle_on_two_calls_in_a_row(oracle_mod):
    torch = pytest.importorskip("torch")
    lib = native.load()
    stream = torch.cuda.current_stream()
    for call, (d, ell, B) in enumerate([(20, 3, 3), (14, 2, 5)]):
        vh = _games(d, B, call)
        v = torch.as_tensor(vh, device="cuda")
        ref = fsi.Plan(d, ell, "exact", max_batch=B).apply(v)
        out = torch.full((B, fsi.num_scores(d, ell)), -7.0, dtype=torch.float64, device="cuda")
        st = _noalloc(lib, d, ell, v, out, stream)
        assert st == 0, fsi.STATUS.get(st)
        torch.cuda.synchronize()
        err = (out - ref).abs().max().item() / v.abs().max().item()
        assert err <= TOL, (call, err)
        got = out.cpu().numpy()
        want = oracle_mod.fsi(vh, d, ell)
        assert np.max(np.abs(got - want)) / np.abs(vh).max() <= TOL, call


@pytest.mark.gpu
def test_noalloc_nonfinite_input_poisons_the_call_and_the_next_call_is_clean():
    """One NaN in v turns every score of that call into NaN (the caller has
    no plan to query); the shared fault word is cleared by the next call,
    which is ordered after it on the same stream with no host sync between."""
    torch = pytest.importorskip("torch")
    lib = native.load()
    stream = torch.cuda.current_stream()
    d, ell, B = 15, 3, 2
    vh = _games(d, B, 5)
    bad = vh.copy()
    bad[1, 1234] = np.nan
    vb = torch.as_tensor(bad, device="cuda")
    vg = torch.as_tensor(vh, device="cuda")
    n = fsi.num_scores(d, ell)
    out_bad = torch.zeros((B, n), dtype=torch.float64, device="cuda")
    out_good = torch.zeros((B, n), dtype=torch.float64, device="cuda")
    assert _noalloc(lib, d, ell, vb, out_bad, stream) == 0
    assert _noalloc(lib, d, ell, vg, out_good, stream) == 0
    torch.cuda.synchronize()
    assert torch.isnan(out_bad).all()
    ref = fsi.Plan(d, ell, "exact", max_batch=B).apply(vg)
    assert (out_good - ref).abs().max().item() / vg.abs().max().item() <= TOL


@pytest.mark.gpu
def test_noalloc_back_to_back_calls_on_one_stream():
    """Two calls of different sizes queued on one stream without a host sync
    between them: each rewrites the shared tables and scratch, and stream
    order keeps the second from touching them before the first is done."""
    torch = pytest.importorskip("torch")
    lib = native.load()
    stream = torch.cuda.current_stream()
    cases = [(20, 3, 4), (14, 2, 7), (20, 3, 2)]
    vs, outs = [], []
    for k, (d, ell, B) in enumerate(cases):
        vs.append(torch.as_tensor(_games(d, B, 40 + k), device="cuda"))
        outs.append(torch.full((B, fsi.num_scores(d, ell)), -1.0, dtype=torch.float64, device="cuda"))
    torch.cuda.synchronize()
    for (d, ell, B), v, out in zip(cases, vs, outs):
        assert _noalloc(lib, d, ell, v, out, stream) == 0
    torch.cuda.synchronize()
    for (d, ell, B), v, out in zip(cases, vs, outs):
        ref = fsi.Plan(d, ell, "exact", max_batch=B).apply(v)
        assert (out - ref).abs().max().item() / v.abs().max().item() <= TOL, (d, ell, B)
