"""The FP64 throughput probe that gives the solvers' FP64 fractions their
measured denominator: its argument checks, its operation count, and a
throughput in the range the part's FP64 pipe allows (2 FMA lanes per clock
per SM)."""
import ctypes

import pytest
import torch

from paper_2601_13994_b300 import _lib as L
from paper_2601_13994_b300 import sla

pytestmark = pytest.mark.gpu


def test_fp64_probe_rejects_bad_arguments():
    dev = torch.device("cuda", 0)
    out = torch.zeros(1, dtype=torch.float64, device=dev)
    fl = ctypes.c_int64(0)
    st = sla._stream_ptr(dev)
    lib = L.lib()
    assert lib.sla_fp64_probe(0, 8, out.data_ptr(), ctypes.byref(fl), st) == L.SLA_ERR_INVALID
    assert lib.sla_fp64_probe(16, 0, out.data_ptr(), ctypes.byref(fl), st) == L.SLA_ERR_INVALID
    assert lib.sla_fp64_probe(16, 65, out.data_ptr(), ctypes.byref(fl), st) == L.SLA_ERR_INVALID
    assert lib.sla_fp64_probe(16, 8, None, ctypes.byref(fl), st) == L.SLA_ERR_INVALID


def test_fp64_probe_counts_and_rate():
    dev = torch.device("cuda", 0)
    out = torch.zeros(1, dtype=torch.float64, device=dev)
    fl = ctypes.c_int64(0)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    assert L.lib().sla_fp64_probe(100, 2, out.data_ptr(), ctypes.byref(fl), sla._stream_ptr(dev)) == 0
    torch.cuda.synchronize(dev)
    assert fl.value == 2 * 8 * 100 * sms * 2 * 256
    assert float(out[0]) == 0.0  # written only in the impossible case
    tf = sla.fp64_peak_tflops(dev)
    clock_ghz = torch.cuda.get_device_properties(dev).clock_rate / 1e6 if hasattr(
        torch.cuda.get_device_properties(dev), "clock_rate") else 2.032
    bound = 2 * 2 * sms * max(clock_ghz, 2.032) / 1e3 * 1.05  # 2 lanes x 2 flop per clock per SM
    assert 0.2 * bound <= tf <= bound, (tf, bound)
