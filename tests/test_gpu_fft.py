"""The FFT path (hand-written FP64 mixed-radix transforms) against the FP64 oracle:
identity-threshold descriptor and adjoint on any field, soft-threshold descriptor on
binary fields (App. A), and agreement with the direct kernels."""
import numpy as np
import pytest
import torch

import oracle
import synthetic

pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.tensor(np.asarray(a, dtype=np.float32), device="cuda")


def _f64(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


CASES = [((64, 64), (16, 16), 1), ((96, 80), (10, 12), 1), ((60, 64), (6, 8), 2), ((30, 24, 20), (5, 6, 4), 1),
         ((24, 24, 24), (4, 4, 4), 2), ((16, 16), (8, 8), 1), ((1024, 1024), (31, 31), 1)]


@pytest.mark.parametrize("shape,window,levels", CASES)
def test_fft_identity_descriptor_and_vjp(cuda_lib, shape, window, levels):
    dm = cuda_lib
    M = np.random.default_rng(4).uniform(-0.3, 1.3, shape)
    p = dm.Params(shape=shape, window=window, levels=levels, threshold=dm.DMCR_IDENTITY, path=dm.DMCR_PATH_FFT)
    op = oracle.Params(ndim=len(shape), window=window, levels=levels, threshold="identity")
    got = dm.descriptor(_dev(M), p).cpu().numpy().astype(np.float64)
    if np.prod(shape) <= 1 << 16:
        want = oracle.descriptor(_f64(M), op)
    else:   # large field: sampled shifts (each O(N))
        H = oracle.half_window(len(shape), window)
        idx = np.sort(np.random.default_rng(1).choice(H.shape[0], 24, replace=False))
        want, got = oracle.descriptor_shifts(_f64(M), op, 0, H[idx]), got[idx]
    np.testing.assert_allclose(got, want, rtol=1e-5, atol=1e-9)
    G = np.random.default_rng(5).standard_normal(dm.dmcr_descriptor_length(p))
    g = dm.descriptor_vjp(_dev(M), _dev(G), p).cpu().numpy().astype(np.float64).ravel()
    if np.prod(shape) <= 1 << 16:
        g_ref = oracle.descriptor_vjp(_f64(M), op, _f64(G)).ravel()
        assert np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref) < 1e-5
    else:
        pos = np.random.default_rng(2).choice(M.size, 64, replace=False)
        g_ref = oracle.level_vjp(_f64(M), op, _f64(G), pos)
        assert np.linalg.norm(g[pos] - g_ref) / np.linalg.norm(g_ref) < 1e-5


def test_fft_equals_direct_identity(cuda_lib):
    dm = cuda_lib
    shape, window = (64, 96), (12, 16)
    M = _dev(np.random.default_rng(6).uniform(0, 1, shape))
    T = _dev((np.random.default_rng(7).random(shape) < 0.3).astype(np.float32))
    out = {}
    for path in (dm.DMCR_PATH_DIRECT, dm.DMCR_PATH_FFT):
        p = dm.Params(shape=shape, window=window, levels=2, threshold=dm.DMCR_IDENTITY, path=path)
        d = dm.descriptor(T, p)
        out[path] = (d, *dm.loss_grad(M, d, p))
    (d1, l1, g1), (d2, l2, g2) = out[dm.DMCR_PATH_DIRECT], out[dm.DMCR_PATH_FFT]
    np.testing.assert_allclose(d2.cpu().numpy(), d1.cpu().numpy(), rtol=1e-5, atol=1e-9)
    np.testing.assert_allclose(l2.cpu().numpy(), l1.cpu().numpy(), rtol=1e-5)
    assert float(torch.linalg.norm(g2 - g1) / torch.linalg.norm(g1)) < 1e-5


@pytest.mark.parametrize("shape,window,levels", [((128, 128), (31, 31), 1), ((40, 30, 20), (6, 6, 4), 1)])
def test_fft_soft_threshold_on_binary_targets(cuda_lib, shape, window, levels):
    """App. A: the soft descriptor of a binary field is an affine map of its exact S2."""
    dm = cuda_lib
    if len(shape) == 2:
        T = synthetic.target_2d_grf(shape[0], 4.0, 0.35, 8)
    else:
        T = synthetic.threshold_count(synthetic.gaussian_random_field(shape, 3.0, 8), 0.3)
    p = dm.Params(shape=shape, window=window, levels=levels, path=dm.DMCR_PATH_FFT)
    got = dm.descriptor(_dev(T), p).cpu().numpy().astype(np.float64)
    want = oracle.descriptor(T, oracle.Params(ndim=len(shape), window=window, levels=levels))
    np.testing.assert_allclose(got, want, rtol=1e-5, atol=1e-9)
    direct = dm.descriptor(_dev(T), dm.Params(shape=shape, window=window, levels=levels)).cpu().numpy()
    np.testing.assert_allclose(got, direct, rtol=1e-5, atol=1e-9)


def test_fft_path_limits(cuda_lib):
    dm = cuda_lib
    p = dm.Params(shape=(64, 64), window=(8, 8), path=dm.DMCR_PATH_FFT)       # soft: descriptor only
    f = torch.zeros(64, 64, device="cuda")
    d = dm.descriptor(f, p)
    with pytest.raises(dm.DmcrError) as e:
        dm.loss_grad(f, d, p)
    assert e.value.status == 6
    with pytest.raises(dm.DmcrError) as e:
        dm.dmcr_descriptor_length(dm.Params(shape=(14, 14), window=(3, 3), threshold=dm.DMCR_IDENTITY,
                                            path=dm.DMCR_PATH_FFT))
    assert e.value.status == 6
