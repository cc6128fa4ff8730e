"""Three-point descriptor on the GPU (tensor-core Gram of the ensemble) against the FP64
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


def _field(shape, seed, kind="uniform"):
    rng = np.random.default_rng(seed)
    if kind == "binary":
        return (rng.random(shape) < 0.4).astype(np.float64)
    if kind == "relaxed":
        return rng.uniform(-0.3, 1.3, shape)
    return synthetic.uniform_field(shape, seed)


CASES = [
    ((16, 16), (3, 3), 1, "uniform", 0),      # K = 25: one 128 x 128 tile
    ((32, 32), (8, 8), 1, "relaxed", 0),      # K = 145: 2 x 2 tiles, mirrored triangle
    ((24, 20), (4, 2), 2, "uniform", 0),      # two levels, ragged position count
    ((8, 8, 8), (1, 1, 2), 1, "binary", 0),   # 3-D
    ((20, 24), (3, 4), 1, "relaxed", 1),      # identity threshold
]


def _params(dm, shape, window, levels, ident):
    return dm.Params(shape=shape, window=window, levels=levels, descriptor=dm.DMCR_DESC_S3,
                     threshold=dm.DMCR_IDENTITY if ident else dm.DMCR_SOFT)


@pytest.mark.parametrize("shape,window,levels,kind,ident", CASES)
def test_s3_descriptor_parity(cuda_lib, shape, window, levels, kind, ident):
    dm = cuda_lib
    p = _params(dm, shape, window, levels, ident)
    M = _field(shape, 11, kind)
    got = dm.descriptor(_dev(M), p).cpu().numpy().astype(np.float64)
    want = oracle.s3_descriptor(M, _op(p))
    assert got.shape == want.shape
    np.testing.assert_allclose(got, want, rtol=1e-5, atol=1e-6 * np.max(np.abs(want)))


def test_s3_diagonal_is_the_two_point_descriptor(cuda_lib):
    dm = cuda_lib
    shape, window = (48, 40), (6, 5)
    M = _field(shape, 3)
    p3 = dm.Params(shape=shape, window=window, levels=2, descriptor=dm.DMCR_DESC_S3)
    p2 = dm.Params(shape=shape, window=window, levels=2)
    d3 = dm.descriptor(_dev(M), p3).cpu().numpy()
    d2 = dm.descriptor(_dev(M), p2).cpu().numpy()
    K = d2.size // 2
    for l in range(2):
        np.testing.assert_allclose(np.diag(d3[l * K * K:(l + 1) * K * K].reshape(K, K)), d2[l * K:(l + 1) * K],
                                   rtol=2e-5)


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("shape,window,levels,kind,ident", CASES[:4])
def test_s3_loss_grad_parity(cuda_lib, mode, shape, window, levels, kind, ident):
    dm = cuda_lib
    p = _params(dm, shape, window, levels, ident)
    rng = np.random.default_rng(21)
    T = (rng.random(shape) < 0.35).astype(np.float64)
    M = rng.uniform(-0.2, 1.2, shape)
    D_des = oracle.s3_descriptor(T, _op(p))
    loss, g = dm.loss_grad(_dev(M), _dev(D_des), p, dm.LossOpts(mode=mode))
    ref, g_ref = oracle.s3_loss_grad(M, D_des, _op(p), mode="norm" if mode == 0 else "squared")
    l = loss.cpu().numpy()
    assert abs(l[0] - ref["E"]) <= 1e-5 * ref["E"]
    assert abs(l[4] - ref["L"]) <= 1e-5 * ref["L"]
    g = g.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref) < 1e-5


def test_s3_vjp_parity(cuda_lib):
    dm = cuda_lib
    shape, window = (24, 24), (5, 4)
    p = dm.Params(shape=shape, window=window, levels=2, descriptor=dm.DMCR_DESC_S3)
    M = _field(shape, 5, "relaxed")
    K = oracle.half_window(2, window).shape[0]
    G = np.random.default_rng(6).standard_normal(2 * K * K)
    g = dm.descriptor_vjp(_dev(M), _dev(G), p).cpu().numpy().astype(np.float64)
    op = _op(p)
    pyr = oracle.pyramid(M, 2)
    w = op.weights()
    g1 = oracle.s3_level_vjp(pyr[1], op, w[1] * G[K * K:].reshape(K, K))
    g_ref = oracle.s3_level_vjp(pyr[0], op, w[0] * G[:K * K].reshape(K, K)) + oracle.prolongate_adjoint(g1)
    assert np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref) < 1e-5


def test_s3_adam_steps_reduce_the_loss(cuda_lib):
    dm = cuda_lib
    n, P = 32, (6, 6)
    p = dm.Params(shape=(n, n), window=P, descriptor=dm.DMCR_DESC_S3)
    D = dm.descriptor(_dev(synthetic.checkerboard(n, 4)), p)
    f = _dev(synthetic.uniform_field((n, n), 9))
    m = torch.zeros_like(f)
    v = torch.zeros_like(f)
    rep, step = dm.dmcr_reconstruct(p, dm.ReconOpts(max_iters=200, lr=1e-2), D, f, m, v)
    assert rep["status"] == 0 and step == 200
    assert rep["rel_err"] < 0.5
    first, _ = dm.loss_grad(_dev(synthetic.uniform_field((n, n), 9)), D, p)
    assert rep["L"] < 0.5 * float(first[4])
    Dr = dm.descriptor((f >= 0.5).float(), p).double()
    want = float(torch.linalg.norm(Dr - D.double()) / torch.linalg.norm(D.double()))
    np.testing.assert_allclose(rep["rounded_rel_err"], want, rtol=1e-4, atol=1e-7)


def test_s3_identity_values_beyond_the_fp16_range(cuda_lib):
    # f(x) = x: e = (M_x + M_{x+r}) / 2 reaches 2e5, beyond FP16; the ensemble is scaled by a
    # power of two before the split and the Gram is scaled back
    dm = cuda_lib
    shape, window = (24, 20), (3, 4)
    p = dm.Params(shape=shape, window=window, descriptor=dm.DMCR_DESC_S3, threshold=dm.DMCR_IDENTITY)
    M = np.random.default_rng(13).uniform(-1e5, 2e5, shape)
    got = dm.descriptor(_dev(M), p).cpu().numpy().astype(np.float64)
    want = oracle.s3_descriptor(M, _op(p))
    np.testing.assert_allclose(got, want, rtol=1e-5, atol=1e-6 * np.max(np.abs(want)))


@pytest.mark.parametrize("gscale", [1e-12, 1e6])
def test_s3_vjp_of_tiny_and_large_upstream_gradients(cuda_lib, gscale):
    # G far below or above the FP16 range: scaled into [1/2, 1) before the split
    dm = cuda_lib
    shape, window = (24, 24), (5, 4)
    p = dm.Params(shape=shape, window=window, descriptor=dm.DMCR_DESC_S3)
    M = _field(shape, 15, "relaxed")
    K = oracle.half_window(2, window).shape[0]
    G = gscale * np.random.default_rng(16).standard_normal(K * K)
    g = dm.descriptor_vjp(_dev(M), _dev(G), p).cpu().numpy().astype(np.float64)
    g_ref = oracle.s3_level_vjp(M, _op(p), G.reshape(K, K))
    assert np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref) < 1e-5


def test_s3_full_size_paper_configuration_64_p31(cuda_lib):
    # the configuration the three-point bench times: 64^2, P = 31 (K = 1985, padded to 2048),
    # checked entry by entry against the oracle, with the gradient of a random upstream
    dm = cuda_lib
    n, P = 64, 31
    p = dm.Params(shape=(n, n), window=(P, P), descriptor=dm.DMCR_DESC_S3)
    M = _field((n, n), 17, "relaxed")
    got = dm.descriptor(_dev(M), p).cpu().numpy().astype(np.float64)
    want = oracle.s3_descriptor(M, _op(p))
    np.testing.assert_allclose(got, want, rtol=1e-5, atol=1e-6 * np.max(np.abs(want)))
    K = oracle.half_window(2, (P, P)).shape[0]
    G = np.random.default_rng(18).standard_normal(K * K)
    g = dm.descriptor_vjp(_dev(M), _dev(G), p).cpu().numpy().astype(np.float64)
    g_ref = oracle.s3_level_vjp(M, _op(p), G.reshape(K, K))
    assert np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref) < 1e-5
