"""Autotuner: shapes are valid, cached, and change results only within rounding."""
import json

import numpy as np
import pytest
import torch

import synthetic

pytestmark = pytest.mark.gpu


def test_tuner_picks_valid_shape_and_caches(cuda_lib, tmp_path):
    dm = cuda_lib
    from paper_2103_09686_gb300 import tune
    p = dm.Params(shape=(128, 128), window=(16, 16), levels=2)
    cache = str(tmp_path / "tune.json")
    pt = tune.tuned(p, cache)
    table = json.load(open(cache))
    assert len(table) == 1 and list(table.values())[0]["tune"] == list(pt.tune)
    assert tune.tuned(p, cache).tune == pt.tune            # second call: from the cache
    f = torch.tensor(synthetic.uniform_field((128, 128), 3), dtype=torch.float32, device="cuda")
    a = dm.descriptor(f, p).cpu().numpy()
    b = dm.descriptor(f, pt).cpu().numpy()
    np.testing.assert_allclose(b, a, rtol=1e-5, atol=1e-9)


@pytest.mark.parametrize("tune_", [(8, 2, 8, 1), (32, 16, 64, 0), (16, 1, 1, 2), (0, 3, 0, 32)])
def test_explicit_shapes_agree(cuda_lib, tune_):
    dm = cuda_lib
    p = dm.Params(shape=(96, 64), window=(12, 9), levels=2)
    f = torch.tensor(synthetic.uniform_field((96, 64), 4), dtype=torch.float32, device="cuda")
    T = torch.tensor((np.random.default_rng(1).random((96, 64)) < 0.4).astype(np.float32), device="cuda")
    import dataclasses
    q = dataclasses.replace(p, tune=tune_)
    d0 = dm.descriptor(T, p)
    l0, g0 = dm.loss_grad(f, d0, p)
    l1, g1 = dm.loss_grad(f, d0, q)
    np.testing.assert_allclose(dm.descriptor(T, q).cpu().numpy(), d0.cpu().numpy(), rtol=1e-5, atol=1e-9)
    np.testing.assert_allclose(l1.cpu().numpy(), l0.cpu().numpy(), rtol=1e-5)
    assert float(torch.linalg.norm(g1 - g0) / torch.linalg.norm(g0)) < 1e-5
