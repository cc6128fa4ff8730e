"""Multi-phase descriptor (cross-correlations of every ordered phase pair through the
two-point chain of Sec. 3.2.2-3.2.4) on the GPU against the FP64 oracle, through the C ABI."""
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
    # shape, window, levels, phases, identity
    ((64, 64), (16, 16), 1, 2, 0),
    ((48, 40), (5, 7), 2, 3, 0),        # ragged tiles, two levels
    ((96, 72), (9, 6), 2, 3, 0),        # several forward and adjoint tiles per axis
    ((16, 16, 16), (3, 3, 3), 2, 2, 0),
    ((32, 48), (4, 6), 2, 3, 1),        # f(x) = x
]


def _params(dm, shape, window, levels, phases, ident):
    return dm.Params(shape=shape, window=window, levels=levels, phases=phases,
                     threshold=dm.DMCR_IDENTITY if ident else dm.DMCR_SOFT)


@pytest.mark.parametrize("shape,window,levels,phases,ident", CASES)
def test_multiphase_descriptor_parity(cuda_lib, shape, window, levels, phases, ident):
    dm = cuda_lib
    p = _params(dm, shape, window, levels, phases, ident)
    F = np.random.default_rng(3).uniform(-0.2, 1.2, (phases,) + shape)
    got = dm.descriptor(_dev(F), p).cpu().numpy().astype(np.float64)
    want = oracle.multiphase_descriptor(F, _op(p))
    assert got.shape == want.shape
    np.testing.assert_allclose(got, want, rtol=1e-5, atol=1e-6 * np.max(np.abs(want)))


def test_partition_descriptor_maps_to_counted_cross_probabilities(cuda_lib):
    dm = cuda_lib
    F = synthetic.multiphase_grf((48, 48), 3.0, (0.3, 0.25), 11)
    p = dm.Params(shape=(48, 48), window=(6, 6), phases=3)
    D = dm.descriptor(_dev(F), p).cpu().numpy().astype(np.float64)
    H = oracle.half_window(2, (6, 6))
    K = H.shape[0]
    fh = oracle.half_value(_op(p))
    phi = F.reshape(3, -1).mean(axis=1)
    rng = np.random.default_rng(12)
    for a in range(3):
        for b in range(3):
            for k in rng.choice(K, 6, replace=False):
                want = oracle.cross_count(F[a], F[b], H[k])
                got = (D[(3 * a + b) * K + k] - fh * fh * (phi[a] + phi[b])) / (1 - 2 * fh * fh)
                assert abs(got - want) < 3e-6


def test_swapping_phases_permutes_the_blocks_bitwise(cuda_lib):
    dm = cuda_lib
    shape = (40, 56)
    p = dm.Params(shape=shape, window=(6, 9), levels=2, phases=2)
    F = _dev(np.random.default_rng(4).random((2,) + shape))
    K = oracle.half_window(2, (6, 9)).shape[0]
    d = dm.descriptor(F, p).view(2, 2, 2, K)
    e = dm.descriptor(F.flip(0).contiguous(), p).view(2, 2, 2, K)
    assert torch.equal(d, e.flip(1).flip(2))


def test_one_phase_is_the_single_field_descriptor_bitwise(cuda_lib):
    dm = cuda_lib
    shape = (64, 48)
    M = _dev(np.random.default_rng(5).random(shape))
    p1 = dm.Params(shape=shape, window=(8, 8), levels=2, phases=1)
    p0 = dm.Params(shape=shape, window=(8, 8), levels=2)
    assert torch.equal(dm.descriptor(M, p1), dm.descriptor(M, p0))
    D = dm.descriptor(M, p0)
    l1, g1 = dm.loss_grad(M * 0.9, D, p1)
    l0, g0 = dm.loss_grad(M * 0.9, D, p0)
    assert torch.equal(l1, l0) and torch.equal(g1, g0)


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("shape,window,levels,phases,ident", CASES)
def test_multiphase_loss_grad_parity(cuda_lib, mode, shape, window, levels, phases, ident):
    dm = cuda_lib
    p = _params(dm, shape, window, levels, phases, ident)
    T = synthetic.multiphase_grf(shape, 2.0, tuple([0.8 / phases] * (phases - 1)), 21)
    F = np.random.default_rng(21).uniform(-0.2, 1.2, (phases,) + shape)
    D_des = oracle.multiphase_descriptor(T, _op(p))
    loss, g = dm.loss_grad(_dev(F), _dev(D_des), p, dm.LossOpts(mode=mode))
    ref, g_ref = oracle.multiphase_loss_grad(F, D_des, _op(p), mode="norm" if mode == 0 else "squared")
    l = loss.cpu().numpy()
    assert abs(l[0] - ref["E"]) <= 1e-5 * ref["E"]
    assert abs(l[2] - ref["Ebc"]) <= 1e-5 * ref["Ebc"]
    assert abs(l[4] - ref["L"]) <= 1e-5 * ref["L"]
    g = g.cpu().numpy().astype(np.float64)
    assert g.shape == g_ref.shape
    assert np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref) < 1e-5


def test_multiphase_vjp_parity(cuda_lib):
    dm = cuda_lib
    shape, window = (48, 40), (5, 7)
    p = dm.Params(shape=shape, window=window, levels=2, phases=3)
    F = np.random.default_rng(6).uniform(-0.2, 1.2, (3,) + shape)
    K = oracle.half_window(2, window).shape[0]
    G = np.random.default_rng(7).standard_normal(2 * 9 * K)
    g = dm.descriptor_vjp(_dev(F), _dev(G), p).cpu().numpy().astype(np.float64)
    g_ref = oracle.multiphase_descriptor_vjp(F, _op(p), G)
    assert np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref) < 1e-5


def test_full_size_three_phases_512_window64_three_levels(cuda_lib):
    """Three phases of 512^2, +-64, 3 levels: sampled shifts of every block and level, and
    the gradient at sampled positions."""
    dm = cuda_lib
    shape, window, levels = (512, 512), (64, 64), 3
    p = dm.Params(shape=shape, window=window, levels=levels, phases=3)
    op = _op(p)
    F = 0.8 * synthetic.multiphase_grf(shape, 12.0, (0.3, 0.3), 2101) + 0.1 * np.stack(
        [synthetic.uniform_field(shape, seed=2102 + a) for a in range(3)])
    Fd = _dev(F)
    D = dm.descriptor(Fd, p).cpu().numpy().astype(np.float64)
    H = oracle.half_window(2, window)
    K = H.shape[0]
    rng = np.random.default_rng(8)
    pyrs = [oracle.pyramid(np.asarray(F[a], dtype=np.float32).astype(np.float64), levels) for a in range(3)]
    w = op.weights()
    for l in range(levels):
        for a in range(3):
            for b in range(3):
                idx = rng.choice(K, 4, replace=False)
                want = w[l] * oracle.cross_sbar(pyrs[a][l], pyrs[b][l], H[idx])
                got = D[(l * 9 + 3 * a + b) * K + idx]
                np.testing.assert_allclose(got, want, rtol=1e-5)
    G = rng.standard_normal(D.size)
    g = dm.descriptor_vjp(Fd, _dev(G), p).cpu().numpy().astype(np.float64).reshape(3, -1)
    pos = rng.choice(F[0].size, 8, replace=False)
    want = oracle.multiphase_vjp_at(np.asarray(F, dtype=np.float32).astype(np.float64), op, G, pos)
    got = g[:, pos]
    scale = np.linalg.norm(want) / np.sqrt(want.size)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-4 * scale)
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < 1e-5


def test_multiphase_reconstruction_reduces_the_loss(cuda_lib):
    dm = cuda_lib
    n = 48
    p = dm.Params(shape=(n, n), window=(8, 8), levels=2, phases=3)
    T = synthetic.multiphase_grf((n, n), 3.0, (0.3, 0.3), 31)
    D = dm.descriptor(_dev(T), p)
    f = torch.empty(3, n, n, device="cuda")
    m = torch.zeros_like(f)
    v = torch.zeros_like(f)
    rep, step = dm.dmcr_reconstruct(p, dm.ReconOpts(max_iters=300, lr=1e-2, seed=3, init=dm.DMCR_INIT_UNIFORM_SEEDED),
                                    D, f, m, v)
    assert rep["status"] == 0 and step == 300
    f0 = _dev(synthetic.uniform_field((3, n, n), 3))
    first, _ = dm.loss_grad(f0, D, p)
    assert rep["L"] < 0.2 * float(first[4])
    Dr = dm.descriptor((f >= 0.5).float(), p).double()
    want = float(torch.linalg.norm(Dr - D.double()) / torch.linalg.norm(D.double()))
    np.testing.assert_allclose(rep["rounded_rel_err"], want, rtol=1e-4, atol=1e-7)


def test_multiphase_rejections(cuda_lib):
    dm = cuda_lib
    f = torch.zeros(2, 32, 32, device="cuda")
    for kw in (dict(descriptor=dm.DMCR_DESC_S3), dict(descriptor=dm.DMCR_DESC_S2_TILDE),
               dict(path=dm.DMCR_PATH_FFT, threshold=dm.DMCR_IDENTITY)):
        p = dm.Params(shape=(32, 32), window=(4, 4), phases=2, **kw)
        with pytest.raises(dm.DmcrError):
            dm.descriptor(f, p)
    with pytest.raises(dm.DmcrError):
        dm.dmcr_descriptor_length(dm.Params(shape=(32, 32), window=(4, 4), phases=9))
