"""The issue-rate microbenchmark (gs_peak_issue) computes what it claims and measures a plausible rate."""
import pytest
import torch

from paper_2509_12138_gb300 import _lib, peak
from paper_2509_12138_gb300.raster import _ptr, _stream

pytestmark = pytest.mark.gpu


def _run(mode, iters, a, b):
    L = _lib.load()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    out = torch.empty(L.gs_peak_threads(sms), dtype=torch.float32, device="cuda")
    assert L.gs_peak_issue(mode, sms, iters, a, b, _ptr(out), _stream()) == 0
    torch.cuda.synchronize()
    return out


def test_fp32_chains_are_exact():
    # x_j = -j/8 + iters after iters steps of x = x * 1 + 1 (exact in float32); sum over the 8 chains
    iters = 1000
    out = _run(0, iters, 1.0, 1.0)
    assert torch.all(out == float(8 * iters - 3.5))


def test_mufu_chains_reach_the_fixed_point():
    # x = 2^x - 1.5 has the attracting fixed point x = -1 (and a repelling one near 1.66, above the starts)
    out = _run(1, 200, 0.0, 1.5)
    assert torch.allclose(out, torch.full_like(out, -8.0), atol=1e-3)


def test_rates_are_plausible():
    r = peak.issue_rates(iters=20000, repeats=2)
    sms = r["sms"]
    nominal = sms * 128 * 2.07e9 / 1e12  # FP32 lanes x maximum clock
    assert 0.3 * nominal < r["fp32_tops"] < 1.05 * nominal, r
    assert 0.02 * nominal < r["mufu_tops"] < 0.3 * nominal, r


def test_bad_arguments_enqueue_nothing():
    L = _lib.load()
    assert L.gs_peak_issue(2, 1, 1, 0.0, 0.0, None, _stream()) == 1
    assert L.gs_peak_threads(0) == -1
