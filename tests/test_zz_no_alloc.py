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


def test_oversized_requests_are_rejected_before_running():
    lib = native.load()
    dummy = ctypes.c_void_p(256)  # never dereferenced: the size check comes first
    assert lib.tt_fsi_apply_noalloc(20, 3, dummy, 33, dummy, None) == 2  # 33 games > 64 MiB
    assert lib.tt_fsi_apply_noalloc(24, 2, dummy, 10, dummy, None) == 2
    assert lib.tt_fsi_apply_noalloc(20, 0, dummy, 1, dummy, None) == 1  # l = 0
    assert lib.tt_fsi_apply_noalloc(20, 3, None, 1, dummy, None) == 1
    assert lib.tt_fsi_apply_noalloc(20, 3, dummy, 0, dummy, None) == 0   # empty batch


@pytest.mark.gpu
def test_noalloc_matches_plan_based_apply_on_two_calls_in_a_row():
    torch = pytest.importorskip("torch")
    lib = native.load()
    stream = torch.cuda.current_stream()
    for call, (d, ell, B) in enumerate([(20, 3, 3), (14, 2, 5)]):
        v = torch.as_tensor(_games(d, B, call), device="cuda")
        ref = fsi.Plan(d, ell, "exact", max_batch=B).apply(v)
        out = torch.full((B, fsi.num_scores(d, ell)), -7.0, dtype=torch.float64, device="cuda")
        st = lib.tt_fsi_apply_noalloc(d, ell, ctypes.c_void_p(v.data_ptr()), B,
                                      ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
        assert st == 0, fsi.STATUS.get(st)
        torch.cuda.synchronize()
        err = (out - ref).abs().max().item() / v.abs().max().item()
        assert err <= TOL, (call, err)
