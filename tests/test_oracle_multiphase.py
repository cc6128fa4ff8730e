"""Pins of the multi-phase oracle (cross-correlations S2^{a->b} through the two-point
chain of Sec. 3.2.2-3.2.4, every ordered phase pair on every level), on the CPU, checked
against quantities that do not go through it."""
import numpy as np
import pytest

import oracle
import synthetic


def _rel(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


@pytest.mark.parametrize("shape,window,levels", [((16, 12), (3, 2), 2), ((8, 8, 8), (1, 2, 1), 2)])
def test_same_phase_blocks_are_the_two_point_descriptor(shape, window, levels):
    # blocks (a, a) against descriptor(), whose S_bar comes from the C code of the
    # single-field pipeline and shares nothing with the cross reduction
    F = np.random.default_rng(1).uniform(-0.2, 1.2, (3,) + shape)
    p = oracle.Params(ndim=len(shape), window=window, levels=levels)
    K = oracle.half_window(p.ndim, window).shape[0]
    D = oracle.multiphase_descriptor(F, p)
    assert D.size == levels * 9 * K
    for a in range(3):
        single = oracle.descriptor(F[a], p)
        for l in range(levels):
            blk = D[(l * 9 + 4 * a) * K:(l * 9 + 4 * a + 1) * K]
            assert _rel(blk, single[l * K:(l + 1) * K]) < 1e-13


@pytest.mark.parametrize("kind", ["soft", "identity"])
@pytest.mark.parametrize("seed", [2, 3])
def test_partition_maps_to_counted_cross_probabilities(kind, seed):
    # binary indicators: (Ma_x + Mb_{x+r}) / 2 takes 0, 1/2 or 1, so
    # S_bar^{a->b} = S2^{a->b} (1 - 2 f(1/2)^2) + f(1/2)^2 (phi_a + phi_b) (App. A's argument);
    # undoing it must give the probabilities counted position by position, which are not
    # symmetric in r for a != b and so fix the direction of the shift
    F = synthetic.multiphase_grf((10, 12), 2.0, (0.3, 0.25), seed)
    p = oracle.Params(ndim=2, window=(3, 4), threshold=kind)
    H = oracle.half_window(2, p.window)
    K = H.shape[0]
    D = oracle.multiphase_descriptor(F, p)
    fh = oracle.half_value(p)
    phi = F.reshape(3, -1).mean(axis=1)
    asym = 0
    for a in range(3):
        for b in range(3):
            blk = D[(3 * a + b) * K:(3 * a + b + 1) * K]
            for k, r in enumerate(H):
                want = oracle.cross_count(F[a], F[b], r)
                got = (blk[k] - fh * fh * (phi[a] + phi[b])) / (1.0 - 2.0 * fh * fh)
                assert abs(got - want) < 1e-12, (a, b, tuple(r))
                asym += abs(want - oracle.cross_count(F[a], F[b], -r)) > 0
    assert asym > 0          # the field really distinguishes r from -r


def test_swapped_pair_is_the_reflected_shift():
    F = np.random.default_rng(4).random((2, 9, 11))
    H = oracle.half_window(2, (2, 3))
    assert _rel(oracle.cross_sbar(F[0], F[1], H), oracle.cross_sbar(F[1], F[0], -H)) < 1e-14


def test_identity_two_phase_partition_closed_form_by_fft():
    # M1 = 1 - M0 and f(x) = x: with C(r) = <M0_x M0_{x+r}> from numpy's FFT,
    #   S^{0->1}(r) = (1 + 2<M0^2> - 2 C(r)) / 4,  S^{1->1}(r) = (4 - 8<M0> + 2<M0^2> + 2 C(r)) / 4
    M = np.random.default_rng(5).random((12, 10))
    F = np.stack([M, 1.0 - M])
    p = oracle.Params(ndim=2, window=(3, 3), threshold="identity")
    H = oracle.half_window(2, p.window)
    K = H.shape[0]
    D = oracle.multiphase_descriptor(F, p)
    Fm = np.fft.fft2(M)
    C = np.real(np.fft.ifft2(Fm * np.conj(Fm))) / M.size

    def c(r):
        return C[(-r[0]) % M.shape[0], (-r[1]) % M.shape[1]]

    m1, m2 = float(M.mean()), float(np.mean(M * M))
    for k, r in enumerate(H):
        assert abs(D[1 * K + k] - (1 + 2 * m2 - 2 * c(r)) / 4) < 1e-13
        assert abs(D[2 * K + k] - (1 + 2 * m2 - 2 * c(r)) / 4) < 1e-13
        assert abs(D[3 * K + k] - (4 - 8 * m1 + 2 * m2 + 2 * c(r)) / 4) < 1e-13


def test_one_phase_gradient_is_the_two_point_gradient():
    # one phase: the term-by-term chain rule against the C adjoint of the single-field oracle
    rng = np.random.default_rng(6)
    M = rng.uniform(-0.2, 1.2, (12, 16))
    p = oracle.Params(ndim=2, window=(2, 3), levels=2)
    K = oracle.half_window(2, p.window).shape[0]
    G = rng.standard_normal(2 * K)
    g1 = oracle.multiphase_descriptor_vjp(M[None], p, G)[0]
    g2 = oracle.descriptor_vjp(M, p, G)
    assert _rel(g1, g2) < 1e-12


@pytest.mark.parametrize("mode", ["norm", "squared"])
@pytest.mark.parametrize("shape,window,levels", [((8, 8), (2, 2), 2), ((4, 4, 6), (1, 1, 2), 1)])
def test_gradient_matches_central_differences(mode, shape, window, levels):
    rng = np.random.default_rng(7)
    p = oracle.Params(ndim=len(shape), window=window, levels=levels)
    T = synthetic.multiphase_grf(shape, 1.5, (0.35, 0.3), 8)
    D_des = oracle.multiphase_descriptor(T, p)
    F = rng.uniform(-0.2, 1.2, (3,) + shape)          # exercises the box penalty on both sides
    _, g = oracle.multiphase_loss_grad(F, D_des, p, mode=mode)
    h = 1e-5
    flat = F.ravel()
    for i in rng.choice(flat.size, 10, replace=False):
        Fp, Fm = flat.copy(), flat.copy()
        Fp[i] += h
        Fm[i] -= h
        Lp = oracle.multiphase_loss_grad(Fp.reshape(F.shape), D_des, p, mode=mode)[0]["L"]
        Lm = oracle.multiphase_loss_grad(Fm.reshape(F.shape), D_des, p, mode=mode)[0]["L"]
        fd = (Lp - Lm) / (2 * h)
        assert abs(g.ravel()[i] - fd) <= 1e-6 * max(1.0, abs(fd)), (i, g.ravel()[i], fd)


def test_partition_generator():
    F = synthetic.multiphase_grf((16, 20), 3.0, (0.2, 0.5), 9)
    assert F.shape == (3, 16, 20)
    assert np.array_equal(F.sum(axis=0), np.ones((16, 20)))
    assert [int(F[a].sum()) for a in range(3)] == [64, 160, 96]


def test_sampled_gradient_equals_the_full_gradient():
    # gather form at sampled positions against the scatter form of the full VJP
    rng = np.random.default_rng(10)
    shape = (16, 12)
    p = oracle.Params(ndim=2, window=(3, 2), levels=2)
    K = oracle.half_window(2, p.window).shape[0]
    F = rng.uniform(-0.2, 1.2, (3,) + shape)
    G = rng.standard_normal(2 * 9 * K)
    full = oracle.multiphase_descriptor_vjp(F, p, G).reshape(3, -1)
    pos = rng.choice(F[0].size, 12, replace=False)
    got = oracle.multiphase_vjp_at(F, p, G, pos)
    assert _rel(got, full[:, pos]) < 1e-12
