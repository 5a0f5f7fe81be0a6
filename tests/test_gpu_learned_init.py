"""What the learned initialiser gains over the plain one (GPU, small scenes).

The MLP is trained on the converged splats of one scene and applied to a scene
it has not seen (another seed of the same isosurface family); held-out-view PSNR
of the learned initialisation must beat the plain kNN initialisation, at the
start and after a short training run of each form."""
import numpy as np
import pytest
import torch

from paper_2509_12138_gb300 import experiment as X
from paper_2509_12138_gb300 import workload

pytestmark = pytest.mark.gpu


def test_learned_init_beats_plain_on_unseen_scene():
    src = workload.isosurface_scene(30000, 8, 24, 256, 192, sh_degree=1, seed=11)
    h_src, trained = X.run_plain(src, steps=400, eval_every=400)
    assert h_src.psnr[-1] > h_src.psnr[0] + 3.0  # the plain form itself trains
    w, losses = X.fit_mlp(src, trained, steps=400)
    assert losses[-1] < 0.5 * losses[0]
    dst = workload.isosurface_scene(30000, 8, 24, 256, 192, sh_degree=1, seed=12)
    h_plain, _ = X.run_plain(dst, steps=60, eval_every=60)
    h_learn, _ = X.run_learned_batched(dst, w, steps=30, eval_every=30, views_per_step=2)
    assert h_learn.psnr[0] >= h_plain.psnr[0] + 1.0, (h_learn.psnr, h_plain.psnr)
    # after the same number of views seen (60), the learned form is still ahead
    assert h_learn.psnr[-1] >= h_plain.psnr[-1], (h_learn.psnr, h_plain.psnr)
