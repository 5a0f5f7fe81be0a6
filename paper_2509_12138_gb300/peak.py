"""Measured issue rates of the device (gs_peak_issue): FP32 and MUFU lane-operations per second.

The blend kernels are bound by instruction issue, so their roofline divides their algorithmic work
(FP32 issue slots per (pixel, list entry) pair) by the FP32 rate measured here, on the same device and at
the clocks it holds under a saturating load.
"""
from __future__ import annotations

import torch

from . import _lib
from ._lib import check
from .raster import _ptr, _stream

CHAINS = 8  # GS_PEAK_CHAINS


def issue_rates(iters: int = 60000, repeats: int = 3) -> dict:
    """{'fp32_tops', 'mufu_tops'}: lane-operations per second / 1e12 (best of `repeats` timed launches after
    one warm-up launch), with 'sms' and the launch's 'ms'."""
    L = _lib.load()
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    threads = L.gs_peak_threads(sms)
    out = torch.empty(threads, dtype=torch.float32, device="cuda")
    res = {"sms": sms}
    for mode, key, a, b, it in ((0, "fp32", 1.0, 1.0, iters), (1, "mufu", 0.0, 1.5, iters // 8)):
        check(L.gs_peak_issue(mode, sms, it, a, b, _ptr(out), _stream()), "gs_peak_issue")
        best = 0.0
        for _ in range(repeats):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            check(L.gs_peak_issue(mode, sms, it, a, b, _ptr(out), _stream()), "gs_peak_issue")
            e1.record()
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            best = max(best, threads * CHAINS * it / (ms * 1e-3) / 1e12)
            res[key + "_ms"] = ms
        res[key + "_tops"] = best
    return res
