"""Pins of the three-point oracle (the quadratic reduction of the ensemble, Eq. s3) and of
the corrected two-point descriptor (App. A, Eq. s2rfroms2rbar), on the CPU, checked
against quantities that do not go through them."""
import itertools

import numpy as np
import pytest

import oracle


def _rel(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


@pytest.mark.parametrize("shape,window", [((10, 12), (3, 2)), ((6, 8, 6), (1, 2, 2))])
def test_diagonal_is_the_two_point_descriptor(shape, window):
    # S_bar3(r, r) = S_bar2(r) (Eq. s3 with p = r, q = s); sbar() is the C code of the
    # two-point pipeline, which shares nothing with the ensemble matrix
    M = np.random.default_rng(1).uniform(-0.2, 1.2, shape)
    H = oracle.half_window(len(shape), window)
    S3 = oracle.s3bar(M, H)
    assert _rel(np.diag(S3), oracle.sbar(M, H)) < 1e-13
    assert _rel(S3, S3.T) == 0.0


def test_multigrid_blocks_match_the_two_point_descriptor():
    M = np.random.default_rng(2).random((16, 16))
    p = oracle.Params(ndim=2, window=(2, 3), levels=2)
    D2 = oracle.descriptor(M, p)
    _, blocks = oracle.s3_descriptor(M, p, levels_out=True)
    K = oracle.half_window(2, p.window).shape[0]
    for l, B in enumerate(blocks):
        assert _rel(np.diag(B), D2[l * K:(l + 1) * K]) < 1e-13


@pytest.mark.parametrize("seed,vf", [(3, 0.4), (4, 0.6)])
def test_app_a_mapping_recovers_counted_three_point_probabilities(seed, vf):
    # binary field: a in {0, 1/2, 1}, so S_bar3 mixes S3 with two-point terms weighted by
    # f(1/2) and f(1/2)^2; App. A (Eq. s3rfroms3rbar) undoes that, which must give the
    # probabilities counted directly
    M = (np.random.default_rng(seed).random((12, 14)) < vf).astype(np.float64)
    H = oracle.half_window(2, (3, 3))
    S3b = oracle.s3bar(M, H)
    fh = float(oracle.threshold(np.array([0.5]))[0][0])
    s20 = oracle.s2_count(M, (0, 0))
    checked = 0
    for a, b in itertools.product(range(len(H)), repeat=2):
        ra, rb = H[a], H[b]
        if not ra.any() or not rb.any() or (ra == rb).all():
            continue
        got = oracle.s3_from_s3bar(S3b[a, b], oracle.s2_count(M, ra), oracle.s2_count(M, rb), s20,
                                   oracle.s2_count(M, ra - rb), fh)
        assert abs(got - oracle.s3_count(M, ra, rb)) < 1e-12
        checked += 1
    assert checked == len(H) * (len(H) - 1) - 2 * (len(H) - 1)
    # the diagonal follows App. A's two-point mapping
    for k, r in enumerate(H[1:], start=1):
        want = (1 - 2 * fh * fh) * oracle.s2_count(M, r) + 2 * fh * fh * s20
        assert abs(S3b[k, k] - want) < 1e-12


def test_identity_threshold_closed_form_by_fft():
    # f(x) = x: e_x(r) = (M_x + M_{x+r}) / 2, so
    # S_bar3(a, b) = (<M^2> + C(r_a) + C(r_b) + C(r_b - r_a)) / 4 for r_a, r_b != 0 with the
    # periodic autocorrelation C(r) = <M_x M_{x+r}>, here from numpy's FFT
    M = np.random.default_rng(5).random((9, 12))
    H = oracle.half_window(2, (2, 3))
    S3 = oracle.s3bar(M, H, kind="identity")
    F = np.fft.fft2(M)
    C = np.real(np.fft.ifft2(F * np.conj(F))) / M.size

    def c(r):
        return C[(-r[0]) % M.shape[0], (-r[1]) % M.shape[1]]

    m2 = float(np.mean(M * M))
    for a, b in itertools.product(range(1, len(H)), repeat=2):
        want = (m2 + c(H[a]) + c(H[b]) + c(H[b] - H[a])) / 4.0
        assert abs(S3[a, b] - want) < 1e-13
    for b in range(1, len(H)):
        assert abs(S3[0, b] - (m2 + c(H[b])) / 2.0) < 1e-13


def test_translation_invariance():
    M = np.random.default_rng(6).random((8, 10))
    H = oracle.half_window(2, (2, 2))
    S3 = oracle.s3bar(M, H)
    assert _rel(oracle.s3bar(np.roll(M, (3, -4), axis=(0, 1)), H), S3) < 1e-13


@pytest.mark.parametrize("mode", ["norm", "squared"])
@pytest.mark.parametrize("shape,window,levels", [((8, 8), (2, 2), 2), ((4, 6, 4), (1, 1, 2), 1)])
def test_gradient_matches_central_differences(mode, shape, window, levels):
    rng = np.random.default_rng(7)
    p = oracle.Params(ndim=len(shape), window=window, levels=levels)
    T = (rng.random(shape) < 0.4).astype(np.float64)
    D_des = oracle.s3_descriptor(T, p)
    M = rng.uniform(-0.2, 1.2, shape)            # exercises the box penalty on both sides
    _, g = oracle.s3_loss_grad(M, D_des, p, mode=mode)
    h = 1e-5
    flat = M.ravel()
    for i in rng.choice(flat.size, 8, replace=False):
        Mp, Mm = flat.copy(), flat.copy()
        Mp[i] += h
        Mm[i] -= h
        Lp = oracle.loss(Mp.reshape(shape), D_des, p, mode, D=oracle.s3_descriptor(Mp.reshape(shape), p))["L"]
        Lm = oracle.loss(Mm.reshape(shape), D_des, p, mode, D=oracle.s3_descriptor(Mm.reshape(shape), p))["L"]
        fd = (Lp - Lm) / (2 * h)
        assert abs(g.ravel()[i] - fd) <= 1e-6 * max(1.0, abs(fd)), (i, g.ravel()[i], fd)


# ----------------------------------------------------------------------------- corrected S2

@pytest.mark.parametrize("kind", ["soft", "identity"])
@pytest.mark.parametrize("seed", [8, 9])
def test_corrected_descriptor_recovers_counted_two_point_probabilities(kind, seed):
    # App. A: on binary fields S_tilde(r) equals the exact S2(r) counted directly, for the
    # soft threshold and (the paper's footnote) for f(x) = x
    shape = (14, 12)
    M = (np.random.default_rng(seed).random(shape) < 0.45).astype(np.float64)
    p = oracle.Params(ndim=2, window=(3, 4), threshold=kind)
    Dt = oracle.descriptor_tilde(M, p)
    H = oracle.half_window(2, p.window)
    want = np.array([oracle.s2_count(M, r) for r in H])
    assert np.max(np.abs(Dt - want)) < 1e-13


def test_corrected_descriptor_multigrid_blocks_and_weights():
    M = np.random.default_rng(10).random((16, 16))
    p = oracle.Params(ndim=2, window=(2, 2), levels=2)
    K = oracle.half_window(2, p.window).shape[0]
    Dt = oracle.descriptor_tilde(M, p)
    D = oracle.descriptor(M, p)
    fh = oracle.half_value(p)
    q = 2 * fh * fh
    for l in range(2):
        b, t = D[l * K:(l + 1) * K], Dt[l * K:(l + 1) * K]
        assert abs(t[0] - b[0]) < 1e-15
        np.testing.assert_allclose(t[1:], (b[1:] - q * b[0]) / (1 - q), rtol=1e-13)


@pytest.mark.parametrize("mode", ["norm", "squared"])
def test_corrected_gradient_matches_central_differences(mode):
    rng = np.random.default_rng(11)
    shape = (8, 8)
    p = oracle.Params(ndim=2, window=(2, 3), levels=2)
    T = (rng.random(shape) < 0.4).astype(np.float64)
    D_des = oracle.descriptor_tilde(T, p)
    M = rng.uniform(-0.2, 1.2, shape)
    _, g = oracle.tilde_loss_grad(M, D_des, p, mode=mode)
    h = 1e-5
    flat = M.ravel()
    for i in rng.choice(flat.size, 8, replace=False):
        Mp, Mm = flat.copy(), flat.copy()
        Mp[i] += h
        Mm[i] -= h
        Lp = oracle.loss(Mp.reshape(shape), D_des, p, mode, D=oracle.descriptor_tilde(Mp.reshape(shape), p))["L"]
        Lm = oracle.loss(Mm.reshape(shape), D_des, p, mode, D=oracle.descriptor_tilde(Mm.reshape(shape), p))["L"]
        fd = (Lp - Lm) / (2 * h)
        assert abs(g.ravel()[i] - fd) <= 1e-6 * max(1.0, abs(fd)), (i, g.ravel()[i], fd)
