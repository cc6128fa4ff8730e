"""The paper's checkable end-to-end claim (Sec. 4.1): the relaxed reconstruction of a
checkerboard becomes exact once the field is rounded to phases 0/1.

The paper reconstructs a 64 x 64 checkerboard with P = 31 (App. B) and Adam at the
TensorFlow defaults; the loss of the rounded field reaches zero after about 2000
iterations (Sec. 4.1, Fig. convergence), and larger checkerboards become exact with the
multigrid scheme (Fig. checerboardreconstructions).  The descriptor is the quadratic
reduction of Eq. s3 over every pair of half-window shifts (the Gram matrix of the
ensemble); the two-point diagonal alone has relaxed minimisers whose rounding is not
exact, so this test uses the three-point form.  Square side 8 px (the paper does not give
it).  "Exact" means the rounded field's descriptor equals the target's to a relative
error below 1e-6; the rounded field is evaluated by the library every 100 iterations.
"""
import numpy as np
import pytest
import torch

import synthetic

pytestmark = pytest.mark.gpu


def _iterations_to_exact(dm, n, levels, lr, budget):
    p = dm.Params(shape=(n, n), window=(31, 31), levels=levels, descriptor=dm.DMCR_DESC_S3)
    ws = dm.workspace(p)
    D = dm.descriptor(torch.tensor(synthetic.checkerboard(n, 8), dtype=torch.float32, device="cuda"), p, ws)
    f = torch.empty(n, n, device="cuda")
    m = torch.zeros_like(f)
    v = torch.zeros_like(f)
    step = 0
    while step < budget:
        init = dm.DMCR_INIT_UNIFORM_SEEDED if step == 0 else dm.DMCR_INIT_CALLER
        rep, step = dm.dmcr_reconstruct(p, dm.ReconOpts(max_iters=100, lr=lr, seed=1, init=init), D, f, m, v,
                                        step=step, ws=ws)
        assert rep["status"] == 0
        if rep["rounded_rel_err"] < 1e-6:
            # the rounded field is the target up to a periodic translation (Sec. 4.2)
            r = (f >= 0.5).cpu().numpy().astype(np.float64)
            T = synthetic.checkerboard(n, 8)
            assert any(np.array_equal(np.roll(r, (dy, dx), axis=(0, 1)), T)
                       for dy in range(16) for dx in range(16))
            return step
    return None


def test_checkerboard_64_becomes_exact_at_the_paper_settings(cuda_lib):
    """64 x 64, P = 31, one level, Adam lr 1e-3: exact within 4000 iterations (the paper:
    about 2000; this build reaches it at 2500 with the uniform start of seed 1)."""
    it = _iterations_to_exact(cuda_lib, 64, 1, 1e-3, 4000)
    assert it is not None and it <= 4000


def test_checkerboard_128_becomes_exact_with_two_levels(cuda_lib):
    """128 x 128 with the simultaneous multigrid of Sec. 3.3 (levels 128 and 64, P = 31):
    exact within 3000 iterations at Adam lr 1e-2 (the paper reports fewer than 2000
    iterations for its multigrid run)."""
    it = _iterations_to_exact(cuda_lib, 128, 2, 1e-2, 3000)
    assert it is not None and it <= 3000
