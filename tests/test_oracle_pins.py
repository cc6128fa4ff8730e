"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a value printed in the
paper, a closed form, brute-force counting, an explicit-mask convolution, a library FFT,
a quadrature, a finite difference, or an invariant.  Together they are chosen so that a
dropped term, a wrong sign or index, or a transposed operand fails at least one of them.
"""
import os

import numpy as np
import pytest

import oracle
import synthetic

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    vals = {}
    for line in open(os.path.join(GOLDEN, name)):
        line = line.split("#", 1)[0].strip()
        if line:
            k, v = [s.strip() for s in line.split("=")]
            vals[k] = float(v)
    return vals


PAPER = _golden("paper_parameters.txt")


# --------------------------------------------------------------------------- threshold

def test_soft_threshold_defining_conditions():
    """Sec. 3.2.4: f(0)=0, f(1)=1, f''(0.75)=0 with alpha = 10."""
    a = PAPER["alpha"]
    f, _ = oracle.threshold(np.array([0.0, 1.0]), "soft", a)
    assert abs(f[0] - PAPER["f_at_0"]) < 1e-15
    assert abs(f[1] - PAPER["f_at_1"]) < 1e-15
    h = 1e-4
    x = np.array([0.75 - h, 0.75, 0.75 + h])
    fx, _ = oracle.threshold(x, "soft", a)
    fpp = (fx[0] - 2 * fx[1] + fx[2]) / h**2
    assert abs(fpp - PAPER["fpp_at_0.75"]) < 1e-4
    # away from the inflection the curvature is large (so the check above is not vacuous)
    y = np.array([0.6 - h, 0.6, 0.6 + h])
    fy, _ = oracle.threshold(y, "soft", a)
    assert (fy[0] - 2 * fy[1] + fy[2]) / h**2 > 1.0


def test_soft_threshold_derivative_and_monotonicity():
    """Sec. 3.2.4 requirement f' > 0 on (0,1) (hence f(1/2) > 0); f' against central FD."""
    x = np.linspace(-0.5, 1.5, 201)
    f, df = oracle.threshold(x, "soft", 10.0)
    h = 1e-6
    fp, _ = oracle.threshold(x + h, "soft", 10.0)
    fm, _ = oracle.threshold(x - h, "soft", 10.0)
    np.testing.assert_allclose(df, (fp - fm) / (2 * h), rtol=1e-7, atol=1e-9)
    inside = (x > 0) & (x < 1)
    assert np.all(df[inside] > 0)
    fh, _ = oracle.threshold(np.array([0.5]), "soft", 10.0)
    assert fh[0] > 0


def test_tanh_special_case_of_logistic_form():
    """Sec. 3.2.4 footnote: c1 = alpha = 2, c2 = 0, c3 = -1 gives tanh."""
    x = np.linspace(-3, 3, 61)
    f = oracle.threshold_custom(x, PAPER["tanh_alpha"], PAPER["tanh_c1"], PAPER["tanh_c2"], PAPER["tanh_c3"])
    np.testing.assert_allclose(f, np.tanh(x), rtol=0, atol=1e-15)


def test_soft_threshold_tends_to_hard_threshold():
    """Sec. 3.2.4: lim alpha->inf of the soft threshold is H(x - 0.75)."""
    x = np.array([0.0, 0.5, 0.7, 0.8, 1.0])
    f, _ = oracle.threshold(x, "soft", 400.0)
    hard, _ = oracle.threshold(x, "hard")
    np.testing.assert_allclose(f, hard, atol=1e-8)
    np.testing.assert_array_equal(hard, (x > PAPER["hard_threshold_at"]).astype(float))


# --------------------------------------------------------------------------- windows

def test_half_window_counts_and_symmetry():
    for ndim, P in [(2, (3, 5)), (2, (16, 16)), (3, (2, 3, 1)), (3, (24, 24, 24))]:
        H = oracle.half_window(ndim, P)
        F = oracle.full_window(ndim, P)
        kf = int(np.prod([2 * p + 1 for p in P]))
        assert F.shape == (kf, ndim)
        assert H.shape == ((kf + 1) // 2, ndim)
        # H and -H cover the full window exactly once except r = 0 (shared)
        keys = {tuple(r) for r in H} | {tuple(-r) for r in H}
        assert keys == {tuple(r) for r in F}
        assert tuple(H[0]) == (0,) * ndim


# --------------------------------------------------------------------------- descriptor pins

def _s2_count(M, r):
    """Exact two-point probability S2(r) by counting pairs (both ends in phase 1)."""
    M = np.asarray(M)
    n = M.shape
    cnt = 0
    for x in np.ndindex(*n):
        y = tuple((x[a] + r[a]) % n[a] for a in range(len(n)))
        cnt += int(M[x] == 1 and M[y] == 1)
    return cnt / M.size


@pytest.mark.parametrize("shape,P", [((8, 8), (3, 3)), ((6, 10), (2, 4)), ((4, 4, 6), (1, 2, 2))])
def test_hard_linear_pipeline_is_exact_s2(shape, P):
    """Sec. 3.2.3: convolve -> hard threshold -> (linear) reduce gives the exact S2 on
    binary fields; checked against pair counting."""
    rng = np.random.default_rng(7)
    M = (rng.random(shape) < 0.4).astype(float)
    H = oracle.half_window(len(shape), P)
    got = oracle.sbar(M, H, "hard", linear=True)
    got_q = oracle.sbar(M, H, "hard", linear=False)
    want = np.array([_s2_count(M, r) for r in H])
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-15)
    np.testing.assert_allclose(got_q, want, rtol=0, atol=1e-15)


@pytest.mark.parametrize("shape,P", [((16, 16), (5, 5)), ((8, 8, 8), (2, 2, 2))])
def test_appendix_a_identity_on_binary_fields(shape, P):
    """App. A: on binary fields S_bar(r) = (1 - 2 f(1/2)^2) S2(r) + 2 f(1/2)^2 S2(0)
    for r != 0, and S_bar(0) = S2(0) (the volume fraction)."""
    rng = np.random.default_rng(11)
    M = (rng.random(shape) < 0.35).astype(float)
    H = oracle.half_window(len(shape), P)
    sb = oracle.sbar(M, H, "soft")
    s2 = np.array([_s2_count(M, r) for r in H])
    fh = oracle.threshold(np.array([0.5]), "soft")[0][0]
    want = (1 - 2 * fh**2) * s2 + 2 * fh**2 * s2[0]
    want[0] = s2[0]
    np.testing.assert_allclose(sb, want, rtol=0, atol=2e-15)
    assert abs(s2[0] - M.mean()) < 1e-15


@pytest.mark.parametrize("kind", ["soft", "identity"])
def test_shift_form_equals_explicit_mask_convolution(kind):
    """Sec. 3.2.3 with the masks m_pqrs built explicitly (1/2 at tail and tip, 1 at r=0)."""
    rng = np.random.default_rng(3)
    M = rng.uniform(-0.3, 1.3, (8, 8))
    P = (3, 3)
    H = oracle.half_window(2, P)
    np.testing.assert_allclose(oracle.sbar(M, H, kind), oracle.sbar_masks(M, P, H, kind), rtol=1e-14, atol=1e-16)
    M3 = rng.uniform(0, 1, (4, 4, 4))
    H3 = oracle.half_window(3, (1, 1, 1))
    np.testing.assert_allclose(oracle.sbar(M3, H3, kind), oracle.sbar_masks(M3, (1, 1, 1), H3, kind), rtol=1e-14)


def test_point_symmetry_and_periodic_aliasing():
    rng = np.random.default_rng(5)
    M = rng.uniform(0, 1, (12, 10))
    F = oracle.full_window(2, (4, 4))
    s = oracle.sbar(M, F)
    s_neg = oracle.sbar(M, -F)
    np.testing.assert_allclose(s, s_neg, rtol=1e-13)
    alias = F + np.array([12, -10])
    np.testing.assert_allclose(oracle.sbar(M, alias), s, rtol=1e-13)
    # translation invariance of the whole descriptor
    Mt = np.roll(M, (3, -2), axis=(0, 1))
    np.testing.assert_allclose(oracle.sbar(Mt, F), s, rtol=1e-13)


def test_identity_threshold_equals_autocorrelation_algebra():
    """With f(x) = x (Sec. 4.1 ablation) S_bar(r) = (<M^2> + C(r)) / 2, C the periodic
    autocorrelation -- checked against numpy's FFT."""
    rng = np.random.default_rng(9)
    for shape, P in [((16, 12), (5, 4)), ((8, 6, 10), (2, 2, 3))]:
        M = rng.uniform(-0.2, 1.2, shape)
        H = oracle.half_window(len(shape), P)
        FM = np.fft.fftn(M)
        C = np.real(np.fft.ifftn(np.conj(FM) * FM)) / M.size   # C(r) = mean M_x M_{x+r}
        want = np.array([0.5 * (np.mean(M * M) + C[tuple(r)]) for r in H])
        np.testing.assert_allclose(oracle.sbar(M, H, "identity"), want, rtol=1e-12, atol=1e-15)


def test_checkerboard_closed_form():
    """Exact S2 of a checkerboard with squares of side a (2a | n):
    S2(p, q) = 1/2 [al(p) al(q) + (1 - al(p))(1 - al(q))], al(p) = 1 - min(u, 2a-u)/a,
    u = p mod 2a (derived independently from the geometry)."""
    n, a = 32, 4
    M = synthetic.checkerboard(n, a)
    H = oracle.half_window(2, (9, 9))
    got = oracle.sbar(M, H, "hard", linear=True)

    def al(p):
        u = p % (2 * a)
        return 1.0 - min(u, 2 * a - u) / a

    want = np.array([0.5 * (al(p) * al(q) + (1 - al(p)) * (1 - al(q))) for p, q in H])
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-15)


def test_uncorrelated_uniform_field_expectation():
    """For i.i.d. U(0,1) pixels, S_bar(r != 0) -> E[f((U+V)/2)^2] (triangular density of
    the mean); statistical tolerance ~ 6 sigma of a mean over N pairs."""
    from scipy import integrate
    M = synthetic.uniform_field((256, 256), seed=77)
    shifts = np.array([[0, 9], [5, 7], [20, -3], [31, 31]])
    got = oracle.sbar(M, shifts, "soft")

    def dens(a):
        return 4 * a if a < 0.5 else 4 * (1 - a)

    def integrand(a):
        return oracle.threshold(np.array([a]), "soft")[0][0] ** 2 * dens(a)

    mean, _ = integrate.quad(integrand, 0, 1, points=[0.5, 0.75], limit=200)
    def integrand2(a):
        return oracle.threshold(np.array([a]), "soft")[0][0] ** 4 * dens(a)
    m2, _ = integrate.quad(integrand2, 0, 1, points=[0.5, 0.75], limit=200)
    sigma = np.sqrt(m2 - mean**2) / np.sqrt(M.size)
    assert np.all(np.abs(got - mean) < 6 * sigma), (got, mean, sigma)
    # S_bar(0) is the mean of f(U)^2
    m0, _ = integrate.quad(lambda a: oracle.threshold(np.array([a]), "soft")[0][0] ** 2, 0, 1, points=[0.75])
    s0 = oracle.sbar(M, np.array([[0, 0]]))[0]
    assert abs(s0 - m0) < 6 * np.sqrt(0.25 / M.size)


# --------------------------------------------------------------------------- multigrid

def test_restrict_prolongate_are_transposes():
    rng = np.random.default_rng(1)
    for shape in [(8, 12), (4, 6, 8)]:
        x = rng.standard_normal(shape)
        cshape = tuple(s // 2 for s in shape)
        y = rng.standard_normal(cshape)
        lhs = np.sum(oracle.restrict(x) * y)
        rhs = np.sum(x * oracle.prolongate_adjoint(y))
        assert abs(lhs - rhs) < 1e-13 * (1 + abs(lhs))
        np.testing.assert_allclose(oracle.restrict(np.full(shape, 0.3)), np.full(cshape, 0.3), rtol=1e-15)
        assert abs(oracle.restrict(x).mean() - x.mean()) < 1e-14


def test_block_constant_field_relates_levels():
    """A field constant on 2x2 blocks, F = upsample(C): S_bar_F(2r) = S_bar_C(r), and
    the second multigrid level of F is w_2 S_bar_C with w_2 = 2 in 2-D (Eq. mg)."""
    rng = np.random.default_rng(2)
    C = rng.uniform(0, 1, (8, 8))
    F = np.repeat(np.repeat(C, 2, axis=0), 2, axis=1)
    H = oracle.half_window(2, (3, 3))
    np.testing.assert_allclose(oracle.sbar(F, 2 * H), oracle.sbar(C, H), rtol=1e-13)
    p = oracle.Params(ndim=2, window=(3, 3), levels=2)
    D = oracle.descriptor(F, p)
    K = H.shape[0]
    assert p.weights()[1] == PAPER["level_weight_base"] ** 1
    np.testing.assert_allclose(D[K:], PAPER["level_weight_base"] * oracle.sbar(C, H), rtol=1e-13)
    np.testing.assert_allclose(D[:K], oracle.sbar(F, H), rtol=1e-15)


def test_level_count_rule_of_the_paper():
    """App. B: P = 31 gives 1 level at 64, 2 at 128, 3 at 256 -- coarsest level 2(P+1)."""
    P = int(PAPER["window_P"])
    for n in (64, 128, 256):
        levels = int(np.log2(n // (2 * (P + 1)))) + 1
        assert levels == PAPER["levels_at_%d" % n]


# --------------------------------------------------------------------------- loss and gradient

def test_box_penalty_worked_example():
    """Sec. 3.1: E_bc = sum_x [((M-1) H(M-1) - M H(-M)) / N]^2, H(0) = 0."""
    M = np.full((4, 4), 0.5)
    M[0, 0] = 1.5      # above the box by 0.5
    M[1, 1] = -0.25    # below by 0.25
    M[2, 2] = 1.0      # on the boundary: H(0) = 0, no penalty
    M[3, 3] = 0.0
    p = oracle.Params(ndim=2, window=(1, 1))
    D_des = oracle.descriptor(np.full((4, 4), 0.5), p)
    out = oracle.loss(M, D_des, p, lambda0=3.0)
    assert abs(out["Ebc"] - ((0.5 / 16) ** 2 + (0.25 / 16) ** 2)) < 1e-16
    assert abs(out["lambda"] - 3.0 * out["E"]) < 1e-15
    assert abs(out["L"] - (out["E"] + out["lambda"] * out["Ebc"])) < 1e-15
    assert oracle.loss(np.clip(M, 0, 1), D_des, p)["Ebc"] == 0.0


@pytest.mark.parametrize("mode", ["norm", "squared"])
@pytest.mark.parametrize("case", ["2d_soft_2lev", "2d_identity", "3d_soft"])
def test_gradient_matches_central_differences(mode, case):
    """The analytic adjoint through every level (Sec. 3.3) and the penalty against FP64
    central differences of the loss, h = 1e-5."""
    rng = np.random.default_rng(13)
    if case == "2d_soft_2lev":
        p = oracle.Params(ndim=2, window=(3, 2), levels=2)
        M = rng.uniform(-0.15, 1.15, (12, 8))
        T = (rng.random((12, 8)) < 0.4).astype(float)
    elif case == "2d_identity":
        p = oracle.Params(ndim=2, window=(2, 3), levels=1, threshold="identity")
        M = rng.uniform(-0.15, 1.15, (6, 8))
        T = (rng.random((6, 8)) < 0.5).astype(float)
    else:
        p = oracle.Params(ndim=3, window=(1, 1, 2), levels=2)
        M = rng.uniform(-0.15, 1.15, (4, 4, 8))
        T = (rng.random((4, 4, 8)) < 0.3).astype(float)
    D_des = oracle.descriptor(T, p)
    lam0 = 5.0
    out, g = oracle.loss_grad(M, D_des, p, mode=mode, lambda0=lam0)
    h = 1e-5
    fd = np.zeros(M.size)
    flat = M.ravel()
    for i in range(M.size):
        e = np.zeros(M.size)
        e[i] = h
        Lp = oracle.loss((flat + e).reshape(M.shape), D_des, p, mode=mode, lambda0=lam0)["L"]
        Lm = oracle.loss((flat - e).reshape(M.shape), D_des, p, mode=mode, lambda0=lam0)["L"]
        fd[i] = (Lp - Lm) / (2 * h)
    err = np.linalg.norm(g.ravel() - fd) / np.linalg.norm(fd)
    assert err < 1e-6, err


def test_vjp_linear_in_upstream_and_sampled_positions():
    rng = np.random.default_rng(21)
    p = oracle.Params(ndim=2, window=(2, 2), levels=1)
    M = rng.uniform(0, 1, (8, 8))
    K = oracle.half_window(2, (2, 2)).shape[0]
    G1, G2 = rng.standard_normal(K), rng.standard_normal(K)
    g1 = oracle.descriptor_vjp(M, p, G1)
    g2 = oracle.descriptor_vjp(M, p, G2)
    np.testing.assert_allclose(oracle.descriptor_vjp(M, p, 2 * G1 - G2), 2 * g1 - g2, rtol=1e-12, atol=1e-15)
    pos = np.array([0, 7, 33, 63])
    np.testing.assert_allclose(oracle.level_vjp(M, p, G1, pos), g1.ravel()[pos], rtol=1e-14)
    # VJP = J^T G checked against forward directional derivatives <G, J v> = <J^T G, v>
    v = rng.standard_normal(M.shape)
    h = 1e-6
    Jv = (oracle.descriptor(M + h * v, p) - oracle.descriptor(M - h * v, p)) / (2 * h)
    assert abs(np.dot(G1, Jv) - np.sum(g1 * v)) < 1e-7 * (1 + abs(np.dot(G1, Jv)))


@pytest.mark.parametrize("case", ["2d_3lev", "3d_2lev", "2d_identity_2lev"])
def test_sampled_gather_vjp_through_every_level(case):
    """``vjp_at`` (the gradient through every level at sampled finest positions, Sec. 3.3)
    against FP64 central differences of <G, D(M)> at those positions, and against the
    scatter form ``descriptor_vjp`` at every position."""
    rng = np.random.default_rng(31)
    if case == "2d_3lev":
        p = oracle.Params(ndim=2, window=(2, 3), levels=3)
        M = rng.uniform(-0.2, 1.2, (16, 24))
    elif case == "3d_2lev":
        p = oracle.Params(ndim=3, window=(1, 2, 1), levels=2)
        M = rng.uniform(-0.2, 1.2, (4, 8, 6))
    else:
        p = oracle.Params(ndim=2, window=(3, 1), levels=2, threshold="identity")
        M = rng.uniform(-0.2, 1.2, (12, 8))
    G = rng.standard_normal(oracle.descriptor(M, p).size)
    pos = rng.choice(M.size, size=10, replace=False)
    got = oracle.vjp_at(M, p, G, pos)
    h = 1e-5
    fd = np.zeros(pos.size)
    for i, q in enumerate(pos):
        e = np.zeros(M.size)
        e[q] = h
        fd[i] = (np.dot(G, oracle.descriptor(M + e.reshape(M.shape), p)) -
                 np.dot(G, oracle.descriptor(M - e.reshape(M.shape), p))) / (2 * h)
    assert np.linalg.norm(got - fd) / np.linalg.norm(fd) < 1e-7
    full = oracle.descriptor_vjp(M, p, G).ravel()
    np.testing.assert_allclose(oracle.vjp_at(M, p, G, np.arange(M.size)), full, rtol=1e-12, atol=1e-15)


# --------------------------------------------------------------------------- optimiser

def test_adam_constant_gradient_steps_by_lr():
    """With a constant gradient the bias corrections make every Adam step move each
    parameter by lr * g / (|g| + eps') -- i.e. by ~lr, whatever |g| (Kingma & Ba, Sec. 2.1)."""
    lr = PAPER["adam_lr"]
    M = np.zeros(2)
    m = np.zeros(2)
    v = np.zeros(2)
    g = np.array([3.0, -0.5])
    for t in range(1, 6):
        M_new, m, v = oracle.adam_step(M, g, m, v, t, lr, PAPER["adam_beta1"], PAPER["adam_beta2"])
        np.testing.assert_allclose(M_new - M, -lr * np.sign(g), rtol=1e-5)
        M = M_new


def test_adam_two_steps_where_eps_matters():
    """Two steps by hand on one parameter with gradients 1e-6 then -2e-6, beta = (0.9, 0.999),
    eps = 1e-7, in the efficient form of Kingma & Ba (Sec. 2: step size
    lr * sqrt(1 - beta2^t) / (1 - beta1^t), eps added to the uncorrected sqrt(v)):
      t = 1: m = 1e-7, v = 1e-15, sqrt(v) = 3.16227766e-8,
             move = lr * 0.316227766 * 1e-7 / 1.316227766e-7   = 0.240253073 lr;
      t = 2: m = -1.1e-7, v = 4.999e-15, sqrt(v) = 7.0703607e-8,
             move = lr * 0.235317 * -1.1e-7 / 1.70703607e-7  = -0.151636162 lr.
    At |g| ~ eps these differ from the bias-corrected-eps placement (0.909 lr at t = 1)."""
    lr = 0.01
    M = np.zeros(1)
    m = np.zeros(1)
    v = np.zeros(1)
    M1, m, v = oracle.adam_step(M, np.array([1e-6]), m, v, 1, lr, 0.9, 0.999, 1e-7)
    np.testing.assert_allclose(M1, -0.240253073352042 * lr, rtol=1e-12)
    M2, m, v = oracle.adam_step(M1, np.array([-2e-6]), m, v, 2, lr, 0.9, 0.999, 1e-7)
    np.testing.assert_allclose(M2 - M1, 0.151636162157530 * lr, rtol=1e-12)


def test_rounding_for_evaluation():
    """Sec. 4.1 rounds the relaxed field to phases 0/1; the tie 1/2 goes to phase 1 and
    values outside [0, 1] round to the nearer phase."""
    M = np.array([[0.49999999, 0.5, 0.50000001], [-3.0, 7.0, 0.0]])
    np.testing.assert_array_equal(oracle.round_field(M), [[0, 1, 1], [0, 1, 0]])
    B = (np.random.default_rng(2).random((9, 7)) < 0.4).astype(np.float64)
    np.testing.assert_array_equal(oracle.round_field(B), B)     # binary fields are fixed points


def test_oracle_reconstruction_lowers_loss_on_small_checkerboard():
    """Flow chart of Sec. 3 on a 16x16 checkerboard: the loss falls."""
    T = synthetic.checkerboard(16, 4)
    p = oracle.Params(ndim=2, window=(4, 4), levels=1)
    D_des = oracle.descriptor(T, p)
    M0 = synthetic.uniform_field((16, 16), seed=5)
    M, hist = oracle.reconstruct(M0, D_des, p, iters=150, lr=0.01)
    assert hist[-1]["L"] < 0.5 * hist[0]["L"]
