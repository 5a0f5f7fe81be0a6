"""Ghost-cell / background-mask ablation harness on a small scene (needs a GPU).

Two x-slab partitions of the interface, 8 views at 192x108, 200 batched steps per configuration: every
configuration trains, merges with the ghost filter and scores the held-out views; ghost layers add
Gaussians that the merge then drops; the seam band is a non-empty part of the covered pixels; the merged
render of every configuration (including the masked loss with the background-opacity penalty) reaches more
than 20 dB against the whole scene's GT."""
import math

import pytest

from paper_2509_12138_gb300 import experiment as X

pytestmark = pytest.mark.gpu


def test_ghost_mask_ablation_small():
    res = X.ghost_ablation([10_000, 10_000], 4, 8, 192, 108, 200, n_parts=2, ghost=0.05, sh_degree=0, delta=0.01,
                           lambda_bg=0.1)
    keys = ["ghost=on,mask=on", "ghost=on,mask=off", "ghost=off,mask=on", "ghost=off,mask=off",
            "ghost=on,mask=on+bg", "ghost=off,mask=on+bg"]
    for k in keys:
        r = res[k]
        assert math.isfinite(r["psnr_covered"]) and r["psnr_covered"] > 20.0, (k, r)
        assert math.isfinite(r["psnr_seam_band"]), (k, r)
    assert res["ghost=on,mask=on"]["gaussians_with_ghosts"] > res["ghost=off,mask=on"]["gaussians_with_ghosts"]
    assert res["ghost=off,mask=on"]["gaussians_with_ghosts"] == 20_000
    assert 0.0 < res["seam_band_fraction_of_covered"] < 0.5
