"""Host-side checks of the C-ABI library (no GPU needed): it builds for
sm_103a, loads, exports every entry point the headers declare, and its
host-only calls agree with the oracle's conventions."""
import ctypes

import numpy as np
import pytest

import paper_2601_01903_gb300 as fsi
from paper_2601_01903_gb300 import native


def test_library_builds_and_exports_every_declared_symbol():
    lib = ctypes.CDLL(native.build())
    declared = native.exported_symbols()
    assert "tt_fsi_apply" in declared and "tt_fsi_plan_create" in declared
    missing = [n for n in declared if not hasattr(lib, n)]
    assert not missing, missing


@pytest.mark.parametrize("d,ell", [(1, 1), (8, 2), (14, 2), (16, 2), (20, 3), (24, 2), (9, 12)])
def test_score_layout_matches_oracle(oracle_mod, d, ell):
    assert fsi.num_scores(d, ell) == oracle_mod.n_scores(d, ell)
    if d <= 20:
        assert np.array_equal(fsi.score_masks(d, ell), oracle_mod.score_masks(d, ell))


def test_invalid_arguments_are_statuses_not_crashes():
    lib = native.load()
    assert lib.tt_fsi_num_scores(0, 2) == -1
    assert lib.tt_fsi_num_scores(5, 0) == -1
    h = ctypes.c_void_p()
    assert lib.tt_fsi_plan_create(8, 0, 0, 1, ctypes.byref(h)) == 1   # l = 0
    assert lib.tt_fsi_plan_create(0, 2, 0, 1, ctypes.byref(h)) == 1   # d = 0
    assert lib.tt_fsi_plan_create(8, 2, 7, 1, ctypes.byref(h)) == 1   # bad arithmetic
    assert lib.tt_fsi_plan_create(31, 2, 0, 1, ctypes.byref(h)) == 2  # beyond the supported sizes
    assert lib.tt_fsi_apply(None, None, 1, None, None) == 1
    assert lib.tt_fsi_score_masks(4, 2, None) == 1
    assert lib.tt_fsi_status_string(6) == b"non-finite input"


def test_unknown_index_rejected_on_host():
    """Plan creation validates the index before touching the GPU."""
    import ctypes
    import paper_2601_01903_gb300 as fsi
    lib = fsi.native.load()
    h = ctypes.c_void_p()
    assert lib.tt_fsi_plan_create_index(10, 2, 9, 0, 1, ctypes.byref(h)) == 1
    assert not h.value


def test_unknown_plan_flag_rejected_on_host():
    import ctypes
    import paper_2601_01903_gb300 as fsi
    lib = fsi.native.load()
    h = ctypes.c_void_p()
    assert lib.tt_fsi_plan_create_ex(10, 2, 0, 0, 1, 4, ctypes.byref(h)) == 1
    assert not h.value


def test_host_chunk_setter_rejects_null_plan_on_host():
    import ctypes
    import paper_2601_01903_gb300 as fsi
    lib = fsi.native.load()
    assert lib.tt_fsi_plan_set_host_chunk(None, 1) == 1
    assert lib.tt_fsi_plan_set_host_zero_copy(None, 1) == 1


def test_peak_microbenchmark_rejects_bad_arguments():
    lib = native.load()
    ops = ctypes.c_int64()
    dummy = ctypes.c_void_p(256)  # never dereferenced: the checks come first
    assert lib.tt_fsi_peak_launch(4, 1, 1, dummy, ctypes.byref(ops), None) == 1   # unknown operation
    assert lib.tt_fsi_peak_launch(0, 0, 1, dummy, ctypes.byref(ops), None) == 1   # no CTA
    assert lib.tt_fsi_peak_launch(0, 1, 0, dummy, ctypes.byref(ops), None) == 1   # no iteration
    assert lib.tt_fsi_peak_launch(0, 1, 1, None, ctypes.byref(ops), None) == 1
    assert lib.tt_fsi_peak_launch(0, 1, 1, dummy, None, None) == 1
