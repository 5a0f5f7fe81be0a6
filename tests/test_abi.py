"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
function that include/gs.h declares (no compute calls here)."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"^\s*(?:int|size_t|void|double|float)\s+(gs_\w+)\s*\(", src, flags=re.M))
    return names


def test_header_declares_the_hot_path():
    d = _declared()
    for name in ("gs_preprocess", "gs_bin_sort", "gs_render_fwd", "gs_loss", "gs_render_bwd", "gs_adam_step"):
        assert name in d


def test_library_exports_every_declared_symbol():
    from paper_2509_12138_gb300 import _lib, build
    path = build.build()
    L = C.CDLL(path)
    missing = [n for n in sorted(_declared()) if not hasattr(L, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (gs_\w+)", out))
    assert _declared() <= exported
    # the binding declares a signature for every exported entry point
    assert exported <= set(_lib.SIGNATURES) | _lib.OPTIONAL


def test_binding_loads_and_host_checks_without_gpu():
    from paper_2509_12138_gb300 import _lib
    L = _lib.load()
    assert L.gs_param_planes(0) == 4 and L.gs_param_planes(3) == 15 and L.gs_param_planes(7) == -1
    # argument checks run on the host and enqueue nothing
    assert L.gs_preprocess(None, 10, 0, None, None, 8, 8, None, None, None, None) == 1
    assert L.gs_bin_sort_workspace_size(-1, 10) == 0
    assert L.gs_loss_workspace_size(0, 8, 8) == 0


def test_fused_next_projection_refuses_overlapping_units_without_gpu():
    """gs_project_bwd_adam_next writes one record per Gaussian, so a Gaussian in two units is refused
    (GS_ERR_INVALID) by the host check, before any device pointer is used; disjoint units pass the same
    check and reach the zero-Gaussian early return."""
    import numpy as np
    from paper_2509_12138_gb300 import _lib
    L = _lib.load()
    fake = 1 << 20  # never dereferenced: the call returns before any launch
    proj = _lib.GsProj(fake, fake, fake, fake, fake, fake)
    g2d = _lib.GsGrad2d(fake, fake, fake, 0)
    lr = np.zeros(16 * 4, np.float32)

    def call(begin, count, n_gauss, W=64):
        b, c = np.array(begin, np.int64), np.array(count, np.int64)
        units = _lib.GsUnits(len(b), b.ctypes.data_as(_lib.c_i64p), c.ctypes.data_as(_lib.c_i64p))
        lp = lr.ctypes.data_as(_lib.c_f32p)
        return L.gs_project_bwd_adam_next(fake, n_gauss, 0, C.byref(units), fake, C.byref(proj), C.byref(g2d),
                                          fake, fake, lp, lp, 10, 0.9, 0.999, 1e-15, fake, None, 0, fake, W, 48,
                                          None, None)

    assert call([0, 2000], [2500, 2000], 4000) == 1   # [2000, 2500) in both units
    assert call([0, 0], [10, 10], 10) == 1           # the same view twice
    assert call([0, 2500], [2500, 1500], 4000, W=0) == 1  # empty image
    assert call([0, 2500], [2500, 1500], 0) == 1     # units past the Gaussians
    assert call([0], [0], 0) == 0                    # nothing to do: no launch


def test_device_code_is_sm_103a():
    from paper_2509_12138_gb300 import build
    path = build.build()
    out = subprocess.run(["cuobjdump", "--list-elf", path], capture_output=True, text=True)
    if out.returncode != 0:
        pytest.skip("cuobjdump unavailable")
    assert "sm_103a" in out.stdout


def test_struct_layouts_match_the_header(tmp_path):
    """Every struct the binding passes by pointer has the header's size and field offsets (a C program
    compiled with gcc against include/gs.h prints them)."""
    import shutil
    from paper_2509_12138_gb300 import _lib
    if not shutil.which("gcc"):
        pytest.skip("gcc unavailable")
    structs = {"gs_camera": _lib.GsCamera, "gs_proj": _lib.GsProj, "gs_grad2d": _lib.GsGrad2d,
               "gs_schedule": _lib.GsSchedule, "gs_units": _lib.GsUnits, "gs_owned": _lib.GsOwned,
               "gs_densify_cfg": _lib.GsDensifyCfg, "gs_train_batch_desc": _lib.GsTrainBatchDesc}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "gs.h"', 'int main(void) {']
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'  printf("{cname}.{f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("  return 0;\n}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(l.rsplit(" ", 1) for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                        check=True).stdout.split("\n") if l)
    for cname, py in structs.items():
        assert int(got[cname]) == C.sizeof(py), cname
        for f, _ in py._fields_:
            assert int(got[f"{cname}.{f}"]) == getattr(py, f).offset, (cname, f)
