"""gs_bin_sort_static, the bin-sort for callers that cannot allocate device memory.

Callers such as a plugin inside another framework's memory pool, or a program
that must not allocate after start-up, cannot hand gs_bin_sort a workspace.
gs_bin_sort_static keeps its scratch in a fixed array inside the library; this
test checks, through the C ABI, that two calls in a row (different scenes, so
the second call starts from the first call's leftovers in the shared array)
give exactly the lists, ranges and counts of gs_bin_sort, and that inputs above
the stated limit are refused without launching anything.  (Kept in a file of
its own that pytest collects last.)
"""
import ctypes as C

import numpy as np
import pytest
import torch

import paper_2509_12138_gb300 as gs
from paper_2509_12138_gb300 import _lib
from tests import scenes

pytestmark = pytest.mark.gpu

MAX_RECORDS = 131072
MAX_INSTANCES = 524288


def _ptr(t):
    return C.c_void_p(t.data_ptr())


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def test_static_sort_matches_workspace_sort_on_two_calls():
    L = _lib.load()
    for seed, (n, W, H) in enumerate([(40000, 320, 240), (25000, 256, 200)]):
        g, cams = scenes.random_scene(n, 0, 100 + seed, W, H, extent=1.0, log_scale_range=(-5.0, -3.5))
        fr = gs.Frame(n, gs.Units.single(n), W, H, 0, with_backward=False, with_loss=False)
        params = gs.pack_params(g, 0)
        camd = gs.pack_cameras(cams)
        fr.fit_capacity(params, camd)
        fr.preprocess(params, camd)
        fr.sort()  # the entry point with a caller workspace
        torch.cuda.synchronize()
        assert fr.read_status() == 0
        ref_vals, ref_ranges = fr.sorted_lists()
        assert 0 < len(ref_vals) <= MAX_INSTANCES
        vals = torch.full((MAX_INSTANCES,), -1, dtype=torch.int32, device="cuda")
        ranges = torch.full_like(fr.ranges, -1)
        count = torch.zeros(1, dtype=torch.int32, device="cuda")
        status = torch.zeros(1, dtype=torch.int32, device="cuda")
        rc = L.gs_bin_sort_static(C.byref(fr.proj), C.byref(fr.units.struct), W, H, _ptr(vals), _ptr(ranges),
                                  _ptr(count), _ptr(status), _stream())
        assert rc == 0
        torch.cuda.synchronize()
        I = int(count.item())
        assert int(status.item()) == 0
        assert I == len(ref_vals)
        assert np.array_equal(vals[:I].cpu().numpy().astype(np.int64), ref_vals)
        assert np.array_equal(ranges.cpu().numpy().astype(np.int64), ref_ranges)


def test_static_sort_rejects_inputs_above_its_limit():
    L = _lib.load()
    n = MAX_RECORDS + 1
    units = gs.Units.single(n)
    fr_proj = _lib.GsProj(1, 1, 1, 1, 1, 1)  # never dereferenced: the size check comes first
    rc = L.gs_bin_sort_static(C.byref(fr_proj), C.byref(units.struct), 64, 64, None, None, None, None, _stream())
    assert rc == 1
