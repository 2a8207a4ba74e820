"""The arithmetic-throughput microbenchmark behind the float64 roofline
(tt_fsi_peak_launch, needs a GB300): every operation kind runs, reports the
operations it performs, and its rate is plausible for the part (float64 far
below integer add; neither above the SM clock times the lanes)."""
import ctypes

import pytest

from paper_2601_01903_gb300 import native

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_every_operation_kind_runs_and_counts_its_operations():
    lib = native.load()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    blocks, iters = sms * 8, 16
    out = torch.zeros(blocks * 256, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    rates = {}
    for kind in range(4):
        ops = ctypes.c_int64()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for rep in range(2):
            e0.record(stream)
            st = lib.tt_fsi_peak_launch(kind, blocks, iters, ctypes.c_void_p(out.data_ptr()), ctypes.byref(ops),
                                        ctypes.c_void_p(stream.cuda_stream))
            e1.record(stream)
            assert st == 0
        torch.cuda.synchronize()
        assert ops.value == blocks * 256 * iters * 16 * 8
        rates[kind] = ops.value / (e0.elapsed_time(e1) * 1e-3)
    lanes_per_s = sms * 128 * 2.1e9  # 128 lanes per SM at the maximum clock
    assert all(r < lanes_per_s for r in rates.values())
    assert rates[0] < rates[2] / 10 and rates[1] < rates[2] / 10
