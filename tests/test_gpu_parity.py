"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances: descriptor entries within 1e-5 relative (plus 1e-9 absolute for entries that
are exactly 0 in the oracle); gradients within 1e-5 normwise on unconverged fields, since
the residual rho cancels near convergence and a per-pixel relative error is ill-posed.
Inputs are FP32 on the device; the oracle receives the same FP32 values in FP64.
"""
import numpy as np
import pytest
import torch

import oracle
import synthetic

pytestmark = pytest.mark.gpu

RTOL = 1e-5
GTOL = 1e-5


def _dev(a):
    return torch.tensor(np.asarray(a, dtype=np.float32), device="cuda")


def _f64(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def _oparams(p):
    return oracle.Params(ndim=len(p.shape), window=tuple(p.window), levels=p.levels,
                         threshold="identity" if p.threshold == 1 else "soft", alpha=p.alpha)


CASES = [
    # shape, window, levels, field kind
    ((64, 64), (16, 16), 1, "uniform"),       # the 64x64, +-16 workload
    ((48, 40), (5, 7), 2, "uniform"),         # ragged tiles on both axes
    ((32, 96), (8, 3), 2, "binary"),
    ((16, 16), (8, 8), 1, "uniform"),         # window = n/2 (aliased +-P)
    ((8, 8), (2, 3), 1, "uniform"),
    ((16, 16, 16), (3, 3, 3), 2, "uniform"),
    ((12, 16, 24), (2, 4, 5), 1, "binary"),   # ragged 3-D
    ((64, 64), (16, 16), 1, "extreme"),       # values far outside [0, 1]: exact slow path
    ((40, 64), (6, 6), 1, "relaxed"),
    ((33, 40), (9, 7), 1, "uniform"),         # odd row count: the last row pair is half
    ((7, 9), (3, 4), 1, "relaxed"),           # tile larger than the field, ragged columns
    ((9, 11, 13), (2, 3, 4), 1, "uniform"),   # odd 3-D
    ((64, 64), (16, 16), 1, "mid"),           # |M| up to 3: the two-pair product form
    ((96, 64), (12, 9), 2, "mixed"),          # a few out-of-range pixels: per-block mode mix
    ((80, 96), (10, 44), 1, "uniform"),       # 12 rx blocks: adjoint chunks split the rx range
    ((32, 32), (0, 0), 2, "uniform"),         # window 0: S(0) alone per level
    ((24, 40), (0, 5), 1, "uniform"),         # shifts along one axis only
    ((40, 24), (6, 0), 1, "binary"),
    ((8, 8, 16), (0, 2, 0), 1, "relaxed"),    # 3-D, one axis of shifts
    ((1, 1), (0, 0), 1, "relaxed"),           # a single pixel
]


def _field(kind, shape, seed):
    rng = np.random.default_rng(seed)
    if kind == "uniform":
        return synthetic.uniform_field(shape, seed)
    if kind == "binary":
        return (rng.random(shape) < 0.35).astype(np.float64)
    if kind == "extreme":
        return rng.uniform(-30, 30, shape)
    if kind == "mid":
        return rng.uniform(-3, 3, shape)
    if kind == "mixed":
        M = synthetic.uniform_field(shape, seed).copy()
        flat = M.reshape(-1)
        idx = rng.choice(flat.size, 6, replace=False)
        flat[idx] = [2.5, -2.0, 3.0, 9.0, -6.0, 2.2]
        return M
    return rng.uniform(-0.4, 1.4, shape)


@pytest.mark.parametrize("shape,window,levels,kind", CASES)
def test_descriptor_parity(cuda_lib, shape, window, levels, kind):
    dm = cuda_lib
    M = _field(kind, shape, 100 + len(shape))
    p = dm.Params(shape=shape, window=window, levels=levels)
    got = dm.descriptor(_dev(M), p).cpu().numpy().astype(np.float64)
    want = oracle.descriptor(_f64(M), _oparams(p))
    np.testing.assert_allclose(got, want, rtol=RTOL, atol=1e-9)


@pytest.mark.parametrize("shape,window,levels", [((64, 64), (16, 16), 1), ((32, 48), (4, 6), 2),
                                                 ((8, 16, 32), (2, 3, 3), 2)])
def test_identity_threshold_parity(cuda_lib, shape, window, levels):
    dm = cuda_lib
    M = _field("relaxed", shape, 7)
    p = dm.Params(shape=shape, window=window, levels=levels, threshold=dm.DMCR_IDENTITY)
    got = dm.descriptor(_dev(M), p).cpu().numpy().astype(np.float64)
    want = oracle.descriptor(_f64(M), _oparams(p))
    np.testing.assert_allclose(got, want, rtol=RTOL, atol=1e-9)
    G = np.random.default_rng(3).standard_normal(got.size)
    g = dm.descriptor_vjp(_dev(M), _dev(G), p).cpu().numpy().astype(np.float64)
    g_ref = oracle.descriptor_vjp(_f64(M), _oparams(p), _f64(G))
    assert np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref) < GTOL


def test_all_zero_field_gives_zero_descriptor(cuda_lib):
    dm = cuda_lib
    p = dm.Params(shape=(32, 32), window=(4, 4))
    got = dm.descriptor(torch.zeros(32, 32, device="cuda"), p).cpu().numpy()
    assert np.all(np.abs(got) < 1e-9)


@pytest.mark.parametrize("shape,window,levels,kind", CASES)
def test_vjp_parity(cuda_lib, shape, window, levels, kind):
    dm = cuda_lib
    M = _field(kind, shape, 200 + len(shape))
    p = dm.Params(shape=shape, window=window, levels=levels)
    K = dm.dmcr_descriptor_length(p)
    G = np.random.default_rng(5).standard_normal(K)
    g = dm.descriptor_vjp(_dev(M), _dev(G), p).cpu().numpy().astype(np.float64)
    g_ref = oracle.descriptor_vjp(_f64(M), _oparams(p), _f64(G))
    assert np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref) < GTOL


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("shape,window,levels", [((64, 64), (16, 16), 1), ((64, 48), (6, 5), 3),
                                                 ((16, 16, 32), (3, 2, 4), 2)])
def test_loss_grad_parity(cuda_lib, mode, shape, window, levels):
    dm = cuda_lib
    rng = np.random.default_rng(17)
    T = (rng.random(shape) < 0.3).astype(np.float64)
    M = rng.uniform(-0.2, 1.2, shape)           # exercises the box penalty on both sides
    p = dm.Params(shape=shape, window=window, levels=levels)
    op = _oparams(p)
    D_des = oracle.descriptor(T, op)
    lam0 = float(np.prod(shape))
    opts = dm.LossOpts(mode=mode)
    loss, g = dm.loss_grad(_dev(M), _dev(D_des), p, opts)
    out, g_ref = oracle.loss_grad(_f64(M), _f64(D_des), op, mode="norm" if mode == 0 else "squared", lambda0=lam0)
    loss = loss.cpu().numpy().astype(np.float64)
    for i, k in enumerate(dm.OUT_NAMES):
        np.testing.assert_allclose(loss[i], out[k], rtol=RTOL, err_msg=k)
    g = g.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref) < GTOL


def test_restrict_prolongate_parity(cuda_lib):
    dm = cuda_lib
    rng = np.random.default_rng(1)
    for shape in [(64, 48), (8, 16, 12)]:
        x = rng.standard_normal(shape)
        c = torch.empty([s // 2 for s in shape], device="cuda")
        dm.dmcr_restrict(_dev(x), c)
        np.testing.assert_allclose(c.cpu().numpy(), oracle.restrict(_f64(x)), rtol=1e-6, atol=1e-7)
        y = rng.standard_normal([s // 2 for s in shape])
        f = _dev(np.ones(shape))
        dm.dmcr_prolongate(_dev(y), f, dm.DMCR_PROLONG_ADJOINT_ACCUMULATE)
        np.testing.assert_allclose(f.cpu().numpy(), 1.0 + oracle.prolongate_adjoint(_f64(y)), rtol=1e-6, atol=1e-7)
        f2 = torch.zeros(shape, device="cuda")
        dm.dmcr_prolongate(_dev(y), f2, dm.DMCR_PROLONG_INJECT)
        want = _f64(y)
        for ax in range(len(shape)):
            want = np.repeat(want, 2, axis=ax)
        np.testing.assert_array_equal(f2.cpu().numpy(), want.astype(np.float32))


def test_init_uniform_is_bit_exact(cuda_lib):
    dm = cuda_lib
    f = torch.empty(37, 53, device="cuda")
    dm.dmcr_init_uniform(f, seed=123456789)
    want = synthetic.uniform_field((37, 53), 123456789).astype(np.float32)
    np.testing.assert_array_equal(f.cpu().numpy(), want)


def test_results_are_deterministic(cuda_lib):
    dm = cuda_lib
    M = _dev(_field("uniform", (128, 128), 3))
    T = _dev((np.random.default_rng(4).random((128, 128)) < 0.4).astype(np.float64))
    p = dm.Params(shape=(128, 128), window=(16, 16), levels=2)
    d = dm.descriptor(T, p)
    l1, g1 = dm.loss_grad(M, d, p)
    l2, g2 = dm.loss_grad(M, d, p)
    assert torch.equal(l1, l2) and torch.equal(g1, g2)


# ------------------------------------------------------------------ full-size sampled parity

def _sampled_descriptor_check(dm, M, p, nshift, seed):
    op = _oparams(p)
    got = dm.descriptor(_dev(M), p).cpu().numpy().astype(np.float64)
    H = oracle.half_window(len(p.shape), p.window)
    K = H.shape[0]
    rng = np.random.default_rng(seed)
    for l in range(p.levels):
        idx = np.sort(rng.choice(K, size=nshift, replace=False))
        idx[0] = 0                                   # always include r = 0
        want = oracle.descriptor_shifts(_f64(M), op, l, H[idx])
        np.testing.assert_allclose(got[l * K + idx], want, rtol=RTOL, err_msg="level %d" % l)


def _sampled_vjp_check(dm, M, p, npos, seed):
    """The VJP through every level (Sec. 3.3) for a random upstream gradient, at sampled
    finest positions: the oracle's gather form (``vjp_at``) costs O(levels K_half) per
    position, so it runs at the full sizes."""
    op = _oparams(p)
    rng = np.random.default_rng(seed)
    G = rng.standard_normal(dm.dmcr_descriptor_length(p))
    g = dm.descriptor_vjp(_dev(M), _dev(G), p).cpu().numpy().astype(np.float64).ravel()
    pos = rng.choice(M.size, size=npos, replace=False)
    want = oracle.vjp_at(_f64(M), op, _f64(G), pos)
    assert np.linalg.norm(g[pos] - want) / np.linalg.norm(want) < GTOL


@pytest.fixture(scope="module")
def grf512_full():
    """The 512^2, +-64, 3-level workload (levels 512, 256, 128): a relaxed field with values
    in [-0.2, 1.2) (the box penalty is active) and the GRF + discs target, both with their
    FULL oracle descriptors (3 x 8321 entries, about 2.9e9 FP64 pair evaluations each)."""
    M = synthetic.uniform_field((512, 512), seed=2001) * 1.4 - 0.2
    T = synthetic.target_large_2d(2000)
    op = oracle.Params(ndim=2, window=(64, 64), levels=3)
    return M, T, oracle.descriptor(_f64(M), op), oracle.descriptor(_f64(T), op)


def test_full_size_2d_512_window64_three_levels(cuda_lib, grf512_full):
    """Every descriptor entry of the 512^2, +-64, 3-level workload against the oracle."""
    dm = cuda_lib
    M, _, D_M, _ = grf512_full
    p = dm.Params(shape=(512, 512), window=(64, 64), levels=3)
    got = dm.descriptor(_dev(M), p).cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(got, D_M, rtol=RTOL)


@pytest.mark.parametrize("mode", [0, 1])
def test_full_size_2d_512_window64_loss_and_gradient(cuda_lib, grf512_full, mode):
    """The loss scalars and the loss gradient of the 512^2, +-64, 3-level workload (the
    configuration the benchmark times): E, E^2, E_bc, lambda, L and rel_err within 1e-5 of
    the oracle's full evaluation, and the gradient through all three levels plus the box
    penalty at 256 sampled positions within 1e-5 normwise."""
    dm = cuda_lib
    M, _, D_M, D_des = grf512_full
    p = dm.Params(shape=(512, 512), window=(64, 64), levels=3)
    op = _oparams(p)
    loss, g = dm.loss_grad(_dev(M), _dev(D_des), p, dm.LossOpts(mode=mode))
    Mf = _f64(M)
    out = oracle.loss(Mf, _f64(D_des), op, mode="norm" if mode == 0 else "squared", D=D_M)
    loss = loss.cpu().numpy().astype(np.float64)
    for i, k in enumerate(dm.OUT_NAMES):
        np.testing.assert_allclose(loss[i], out[k], rtol=RTOL, err_msg=k)
    # dL/dM = phi'(E) (1 + lambda0 E_bc) (dD/dM)^T (rho / |rho| or 2 rho) + lambda0 phi dE_bc/dM
    lam0, E, Ebc = out["lambda0"], out["E"], out["Ebc"]
    gD = (out["rho"] / E if mode == 0 else 2.0 * out["rho"]) * (1.0 + lam0 * Ebc)
    phi = E if mode == 0 else out["E2"]
    pos = np.random.default_rng(7).choice(M.size, size=256, replace=False)
    N = M.size
    ex, Mp = oracle.box_excess(Mf).ravel()[pos], Mf.ravel()[pos]
    dex = np.where(Mp > 1.0, 1.0, 0.0) - np.where(Mp < 0.0, 1.0, 0.0)
    want = oracle.vjp_at(Mf, op, gD, pos) + lam0 * phi * 2.0 * ex * dex / (N * N)
    got = g.cpu().numpy().astype(np.float64).ravel()[pos]
    assert np.any(dex != 0)                       # the penalty term is exercised
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < GTOL


def test_full_size_2d_512_window64_vjp_sampled(cuda_lib):
    """The VJP of the 512^2, +-64 workload through all three levels at sampled positions."""
    dm = cuda_lib
    M = synthetic.target_large_2d(2000) * 0.8 + 0.1 * synthetic.uniform_field((512, 512), seed=5)
    p = dm.Params(shape=(512, 512), window=(64, 64), levels=3)
    _sampled_vjp_check(dm, M, p, npos=96, seed=2)


def test_full_size_3d_128_window24(cuda_lib):
    """The 128^3, +-24, 2-level workload: sampled shifts per level, and the VJP through both
    levels at sampled positions."""
    dm = cuda_lib
    M = synthetic.uniform_field((128, 128, 128), seed=3001)
    p = dm.Params(shape=(128, 128, 128), window=(24, 24, 24), levels=2)
    _sampled_descriptor_check(dm, M, p, nshift=12, seed=3)
    _sampled_vjp_check(dm, M, p, npos=32, seed=4)


# ------------------------------------------------------------------ reconstruction

def test_reconstruction_trajectory_matches_oracle(cuda_lib):
    """First iterations of the Adam reconstruction follow the oracle's loss curve (Adam's
    normalisation amplifies rounding differences later on, so only the start is compared
    step by step)."""
    dm = cuda_lib
    n, P = 32, 6
    T = synthetic.target_2d_grf(n, 3.0, 0.3, seed=41)
    M0 = synthetic.uniform_field((n, n), seed=42)
    p = dm.Params(shape=(n, n), window=(P, P))
    op = _oparams(p)
    D_des = oracle.descriptor(T, op)
    iters = 30
    _, hist = oracle.reconstruct(M0, D_des, op, iters=iters, lr=1e-2)
    f = _dev(M0)
    m = torch.zeros_like(f)
    v = torch.zeros_like(f)
    h = torch.zeros(iters * 3, device="cuda")
    rep, step = dm.dmcr_reconstruct(p, dm.ReconOpts(max_iters=iters, lr=1e-2), _dev(D_des), f, m, v, history=h)
    assert rep["iterations"] == iters and step == iters
    h = h.cpu().numpy().reshape(iters, 3)
    want = np.array([x["L"] for x in hist])
    np.testing.assert_allclose(h[:, 1], want, rtol=1e-4)


def test_reconstruction_64_window16_matches_oracle_over_200_iterations(cuda_lib):
    """The 64^2, +-16, one-level reconstruction (GRF target thresholded to 0.30, uniform
    start): the loss follows the oracle's for the first 50 iterations within 1e-4, and the
    relative descriptor error after 200 iterations agrees within 5%."""
    dm = cuda_lib
    n, P, iters = 64, 16, 200
    T = synthetic.target_small_2d(1000)
    M0 = synthetic.uniform_field((n, n), seed=1001)
    p = dm.Params(shape=(n, n), window=(P, P))
    op = _oparams(p)
    D_des = oracle.descriptor(T, op)
    _, hist = oracle.reconstruct(M0, D_des, op, iters=iters, lr=1e-2)
    f = _dev(M0)
    m = torch.zeros_like(f)
    v = torch.zeros_like(f)
    h = torch.zeros(iters * 3, device="cuda")
    rep, step = dm.dmcr_reconstruct(p, dm.ReconOpts(max_iters=iters, lr=1e-2), _dev(D_des), f, m, v, history=h)
    assert rep["iterations"] == iters and step == iters
    h = h.cpu().numpy().reshape(iters, 3)
    want_L = np.array([x["L"] for x in hist])
    np.testing.assert_allclose(h[:50, 1], want_L[:50], rtol=1e-4)
    want_rel = hist[-1]["rel_err"]
    assert want_rel < 0.1 * hist[0]["rel_err"]              # the run did converge a long way
    assert abs(h[-1, 2] - want_rel) <= 0.05 * want_rel


def test_adam_step_matches_oracle(cuda_lib):
    """Two single iterations through dmcr_adam_step: the loss, the moments and the field
    update follow the oracle's gradient and Adam step (Keras form)."""
    dm = cuda_lib
    shape, window, levels = (48, 40), (5, 7), 2
    rng = np.random.default_rng(23)
    T = (rng.random(shape) < 0.35).astype(np.float64)
    M = rng.uniform(-0.2, 1.2, shape)
    p = dm.Params(shape=shape, window=window, levels=levels)
    op = _oparams(p)
    D_des = oracle.descriptor(T, op)
    opts = dm.ReconOpts(lr=1e-2)
    f = _dev(M)
    m = torch.zeros_like(f)
    v = torch.zeros_like(f)
    loss = torch.zeros(len(dm.OUT_NAMES), device="cuda")
    Mr, mr, vr = _f64(M), np.zeros(shape), np.zeros(shape)
    step = 0
    for t in (1, 2):
        f_before = f.cpu().numpy().astype(np.float64)
        step = dm.dmcr_adam_step(p, opts, _dev(D_des), f, m, v, step, loss_out=loss)
        out, g = oracle.loss_grad(Mr, _f64(D_des), op)
        Mn, mr, vr = oracle.adam_step(Mr, g, mr, vr, t, lr=1e-2)
        assert step == t
        np.testing.assert_allclose(loss.cpu().numpy().astype(np.float64), [out[k] for k in dm.OUT_NAMES],
                                   rtol=RTOL)
        for got, want, tol in ((m, mr, 2e-5), (v, vr, 4e-5)):
            got = got.cpu().numpy().astype(np.float64)
            assert np.linalg.norm(got - want) / np.linalg.norm(want) < tol
        dM = f.cpu().numpy().astype(np.float64) - f_before
        assert np.linalg.norm(dM - (Mn - Mr)) / np.linalg.norm(Mn - Mr) < 1e-4
        Mr = f.cpu().numpy().astype(np.float64)     # continue from the GPU's FP32 iterate


def test_reconstruction_converges_and_resume_is_exact(cuda_lib):
    dm = cuda_lib
    n, P = 64, 16
    T = synthetic.target_small_2d(1000)
    p = dm.Params(shape=(n, n), window=(P, P))
    d_des = dm.descriptor(_dev(T), p)
    opts = dm.ReconOpts(max_iters=200, init=dm.DMCR_INIT_UNIFORM_SEEDED, seed=1001, lr=1e-2)
    f = torch.empty(n, n, device="cuda")
    m = torch.zeros_like(f)
    v = torch.zeros_like(f)
    rep, step = dm.dmcr_reconstruct(p, opts, d_des, f, m, v)
    assert rep["iterations"] == 200 and rep["rel_err"] < 0.5
    # 120 + 80 iterations with a checkpoint in between equal 200 in one go, bitwise
    f2 = torch.empty(n, n, device="cuda")
    m2 = torch.zeros_like(f2)
    v2 = torch.zeros_like(f2)
    _, s1 = dm.dmcr_reconstruct(p, dm.ReconOpts(max_iters=120, init=dm.DMCR_INIT_UNIFORM_SEEDED, seed=1001, lr=1e-2),
                                d_des, f2, m2, v2)
    ck = (f2.clone(), m2.clone(), v2.clone(), s1)
    f3, m3, v3 = ck[0].clone(), ck[1].clone(), ck[2].clone()
    _, s2 = dm.dmcr_reconstruct(p, dm.ReconOpts(max_iters=80, lr=1e-2), d_des, f3, m3, v3, step=ck[3])
    assert s2 == 200
    assert torch.equal(f3, f) and torch.equal(m3, m) and torch.equal(v3, v)


def test_reconstruction_stops_at_tolerance(cuda_lib):
    dm = cuda_lib
    n, P = 32, 4
    T = synthetic.target_2d_grf(n, 3.0, 0.4, seed=9)
    p = dm.Params(shape=(n, n), window=(P, P))
    d_des = dm.descriptor(_dev(T), p)
    f = torch.empty(n, n, device="cuda")
    m = torch.zeros_like(f)
    v = torch.zeros_like(f)
    rep, _ = dm.dmcr_reconstruct(p, dm.ReconOpts(max_iters=3000, tol_rel=0.05, lr=1e-2, check_every=10,
                                                 init=dm.DMCR_INIT_UNIFORM_SEEDED, seed=3), d_des, f, m, v)
    assert rep["converged"] and rep["iterations"] < 3000 and rep["iterations"] % 10 == 0
    assert rep["rel_err"] < 0.05 * 1.5


def test_report_gives_the_rounded_field_error(cuda_lib):
    """report.rounded_rel_err is the relative descriptor error of the returned field rounded
    to phases 0/1 (M >= 1/2 -> 1, Sec. 4.1), against the oracle's descriptor of that field."""
    dm = cuda_lib
    n, P = 32, 4
    T = synthetic.target_2d_grf(n, 3.0, 0.4, seed=19)
    p = dm.Params(shape=(n, n), window=(P, P), levels=2)
    op = _oparams(p)
    D_des = oracle.descriptor(T, op)
    f = torch.empty(n, n, device="cuda")
    m = torch.zeros_like(f)
    v = torch.zeros_like(f)
    rep, _ = dm.dmcr_reconstruct(p, dm.ReconOpts(max_iters=150, lr=1e-2, init=dm.DMCR_INIT_UNIFORM_SEEDED, seed=4),
                                 _dev(D_des), f, m, v)
    Mr = oracle.round_field(f.cpu().numpy().astype(np.float64))
    want = np.linalg.norm(oracle.descriptor(Mr, op) - D_des) / np.linalg.norm(D_des)
    assert want > 1e-3                                     # not yet exact: a non-trivial value
    np.testing.assert_allclose(rep["rounded_rel_err"], want, rtol=1e-3)
    # the rounded error of the exact target is zero
    f = _dev(T)
    rep, _ = dm.dmcr_reconstruct(p, dm.ReconOpts(max_iters=0), _dev(D_des), f, m, v)
    assert rep["rounded_rel_err"] < 1e-6
    rep, _ = dm.dmcr_reconstruct(p, dm.ReconOpts(max_iters=0, report_rounded=False), _dev(D_des), f, m, v)
    assert np.isnan(rep["rounded_rel_err"])


def test_workspace_too_small_is_enomem(cuda_lib):
    dm = cuda_lib
    p = dm.Params(shape=(64, 64), window=(8, 8))
    ws = torch.empty(1024, dtype=torch.uint8, device="cuda")
    with pytest.raises(dm.DmcrError) as e:
        dm.dmcr_descriptor(p, torch.zeros(64, 64, device="cuda"), torch.empty(dm.dmcr_descriptor_length(p),
                                                                                device="cuda"), ws=ws)
    assert e.value.status == 2
