"""Corrected two-point descriptor (App. A, Eq. s2rfroms2rbar) on the GPU against the FP64
oracle, through the C ABI."""
import numpy as np
import pytest
import torch

import oracle
import synthetic

pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.tensor(np.asarray(a, dtype=np.float32), device="cuda")


def _op(p):
    return oracle.Params(ndim=len(p.shape), window=tuple(p.window), levels=p.levels,
                         threshold="identity" if p.threshold == 1 else "soft", alpha=p.alpha)


CASES = [
    ((64, 64), (16, 16), 1, 0, 0),        # shape, window, levels, identity, path
    ((48, 40), (5, 7), 2, 0, 0),
    ((16, 16, 16), (3, 3, 3), 2, 0, 0),
    ((32, 48), (4, 6), 2, 1, 0),          # f(x) = x, direct
    ((32, 48), (4, 6), 2, 1, 2),          # f(x) = x, FFT path
]


def _params(dm, shape, window, levels, ident, path):
    return dm.Params(shape=shape, window=window, levels=levels, descriptor=dm.DMCR_DESC_S2_TILDE, path=path,
                     threshold=dm.DMCR_IDENTITY if ident else dm.DMCR_SOFT)


@pytest.mark.parametrize("shape,window,levels,ident,path", CASES)
def test_tilde_descriptor_parity(cuda_lib, shape, window, levels, ident, path):
    dm = cuda_lib
    p = _params(dm, shape, window, levels, ident, path)
    M = np.random.default_rng(3).uniform(-0.2, 1.2, shape)
    got = dm.descriptor(_dev(M), p).cpu().numpy().astype(np.float64)
    want = oracle.descriptor_tilde(M, _op(p))
    np.testing.assert_allclose(got, want, rtol=1e-5, atol=1e-6 * np.max(np.abs(want)))


def test_tilde_descriptor_of_a_binary_field_is_the_counted_two_point_function(cuda_lib):
    dm = cuda_lib
    T = synthetic.target_small_2d(1000)
    p = dm.Params(shape=T.shape, window=(8, 8), descriptor=dm.DMCR_DESC_S2_TILDE)
    got = dm.descriptor(_dev(T), p).cpu().numpy()
    H = oracle.half_window(2, (8, 8))
    want = np.array([oracle.s2_count(T, r) for r in H])
    assert np.max(np.abs(got - want)) < 2e-6


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("shape,window,levels,ident,path", CASES)
def test_tilde_loss_grad_parity(cuda_lib, mode, shape, window, levels, ident, path):
    dm = cuda_lib
    p = _params(dm, shape, window, levels, ident, path)
    rng = np.random.default_rng(21)
    T = (rng.random(shape) < 0.35).astype(np.float64)
    M = rng.uniform(-0.2, 1.2, shape)
    D_des = oracle.descriptor_tilde(T, _op(p))
    loss, g = dm.loss_grad(_dev(M), _dev(D_des), p, dm.LossOpts(mode=mode))
    ref, g_ref = oracle.tilde_loss_grad(M, D_des, _op(p), mode="norm" if mode == 0 else "squared")
    l = loss.cpu().numpy()
    assert abs(l[0] - ref["E"]) <= 1e-5 * ref["E"]
    assert abs(l[4] - ref["L"]) <= 1e-5 * ref["L"]
    g = g.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref) < 1e-5


def test_tilde_vjp_parity(cuda_lib):
    dm = cuda_lib
    shape, window = (48, 40), (5, 7)
    p = dm.Params(shape=shape, window=window, levels=2, descriptor=dm.DMCR_DESC_S2_TILDE)
    M = np.random.default_rng(5).uniform(-0.2, 1.2, shape)
    op = _op(p)
    K = oracle.half_window(2, window).shape[0]
    G = np.random.default_rng(6).standard_normal(2 * K)
    g = dm.descriptor_vjp(_dev(M), _dev(G), p).cpu().numpy().astype(np.float64)
    A = oracle.s2tilde_map(K, oracle.half_value(op))
    gbar = np.concatenate([A.T @ G[l * K:(l + 1) * K] for l in range(2)])
    g_ref = oracle.descriptor_vjp(M, op, gbar)
    assert np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref) < 1e-5
