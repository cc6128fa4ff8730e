"""torch.autograd wrappers: the backward is the library adjoint (checked against the
single-call VJP, the FP64 oracle and FP64 central finite differences, h = 1e-3)."""
import numpy as np
import pytest
import torch

import oracle
import synthetic

pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.tensor(np.asarray(a, dtype=np.float32), device="cuda")


def test_descriptor_autograd_matches_vjp(cuda_lib):
    dm = cuda_lib
    from paper_2103_09686_gb300.autograd import s2_descriptor
    p = dm.Params(shape=(64, 64), window=(16, 16), levels=2)
    f = _dev(synthetic.uniform_field((64, 64), 3)).requires_grad_(True)
    D = s2_descriptor(f, p)
    w = torch.randn_like(D)
    (D * w).sum().backward()
    assert torch.equal(f.grad, dm.descriptor_vjp(f.detach(), w, p))


def test_loss_autograd_matches_loss_grad(cuda_lib):
    dm = cuda_lib
    from paper_2103_09686_gb300.autograd import dmcr_loss
    p = dm.Params(shape=(48, 64), window=(6, 8))
    T = _dev((np.random.default_rng(2).random((48, 64)) < 0.3).astype(np.float32))
    d = dm.descriptor(T, p)
    f = _dev(np.random.default_rng(3).uniform(-0.2, 1.2, (48, 64))).requires_grad_(True)
    L = dmcr_loss(f, d, p)
    (3.0 * L).backward()
    loss, g = dm.loss_grad(f.detach(), d, p)
    assert float(L.detach()) == float(loss[4])
    assert torch.equal(f.grad, 3.0 * g)


def _instances(n, seed):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        size = int(rng.choice([64, 128, 256, 512]))
        P = int(min(rng.integers(16, 65), size // 2))
        vf = float(rng.uniform(0.1, 0.5))
        out.append((size, P, vf, seed + i))
    return out


def test_batched_autograd_mixed_sizes(cuda_lib):
    """Mixed 2-D instances {64..512}^2, windows 16..64, vf in [0.1, 0.5]: one fused launch
    per phase; the backward equals each instance's own VJP, and sampled gradient entries
    equal the FP64 oracle's."""
    dm = cuda_lib
    from paper_2103_09686_gb300.autograd import s2_descriptor_batched
    inst = _instances(12, 40)
    params = [dm.Params(shape=(n, n), window=(P, P)) for n, P, _, _ in inst]
    fields = [_dev(synthetic.target_2d_grf(n, max(n / 32, 2), vf, s) * 0.8 + 0.1).requires_grad_(True)
              for n, P, vf, s in inst]
    descs = s2_descriptor_batched(fields, params)
    ups = [torch.randn_like(d) for d in descs]
    sum((d * u).sum() for d, u in zip(descs, ups)).backward()
    rng = np.random.default_rng(0)
    for i, (p, f, u) in enumerate(zip(params, fields, ups)):
        assert torch.equal(f.grad, dm.descriptor_vjp(f.detach(), u, p))
        if i < 4:   # sampled oracle check (O(K) per position)
            M = f.detach().cpu().numpy().astype(np.float64)
            op = oracle.Params(ndim=2, window=p.window)
            pos = rng.choice(M.size, 32, replace=False)
            want = oracle.level_vjp(M, op, u.cpu().numpy().astype(np.float64), pos)
            got = f.grad.cpu().numpy().ravel()[pos].astype(np.float64)
            assert np.linalg.norm(got - want) / np.linalg.norm(want) < 1e-5


def test_batched_autograd_against_fp64_finite_differences(cuda_lib):
    """Central differences h = 1e-3 in FP64 (oracle descriptor) of J(M) = <u, D(M)> on 32
    random pixels of each small instance; FP32 differences of the GPU loss would be
    dominated by rounding (eps |J| / h)."""
    dm = cuda_lib
    from paper_2103_09686_gb300.autograd import s2_descriptor_batched
    specs = [((64, 64), (16, 16)), ((32, 48), (6, 10)), ((64, 64), (8, 8))]
    params = [dm.Params(shape=s, window=w) for s, w in specs]
    fields = [_dev(synthetic.uniform_field(s, 70 + i)).requires_grad_(True) for i, (s, _) in enumerate(specs)]
    descs = s2_descriptor_batched(fields, params)
    ups = [torch.randn_like(d) for d in descs]
    sum((d * u).sum() for d, u in zip(descs, ups)).backward()
    h = 1e-3
    rng = np.random.default_rng(9)
    for p, f, u in zip(params, fields, ups):
        M = f.detach().cpu().numpy().astype(np.float64)
        uu = u.cpu().numpy().astype(np.float64)
        op = oracle.Params(ndim=2, window=p.window)
        pos = rng.choice(M.size, 32, replace=False)
        fd = []
        for q in pos:
            e = np.zeros(M.size)
            e[q] = h
            Jp = np.dot(uu, oracle.descriptor((M.ravel() + e).reshape(M.shape), op))
            Jm = np.dot(uu, oracle.descriptor((M.ravel() - e).reshape(M.shape), op))
            fd.append((Jp - Jm) / (2 * h))
        fd = np.array(fd)
        got = f.grad.cpu().numpy().ravel()[pos].astype(np.float64)
        # FD truncation ~ h^2 |f'''| / 6 relative to the gradient: ~1e-4
        assert np.linalg.norm(got - fd) / np.linalg.norm(fd) < 1e-3
