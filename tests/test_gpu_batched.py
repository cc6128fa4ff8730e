"""Batched (fused, mixed-size) calls through the C ABI: every instance must give exactly the
result of its single-instance call -- same tiles, same summation order, bitwise -- and the
reconstruction of a job must be the same alone and in a mix."""
import numpy as np
import pytest
import torch

import oracle
import synthetic

pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.tensor(np.asarray(a, dtype=np.float32), device="cuda")


def _mix(dm):
    specs = [((64, 64), (16, 16), 1), ((128, 128), (12, 10), 2), ((48, 80), (6, 9), 1),
             ((32, 32, 32), (3, 4, 5), 2), ((256, 256), (31, 31), 3), ((16, 24), (4, 5), 1)]
    params, fields, targets = [], [], []
    for i, (shape, win, lev) in enumerate(specs):
        params.append(dm.Params(shape=shape, window=win, levels=lev))
        fields.append(_dev(synthetic.uniform_field(shape, 50 + i)))
        rng = np.random.default_rng(60 + i)
        targets.append(_dev((rng.random(shape) < 0.3).astype(np.float32)))
    return params, fields, targets


def test_descriptor_batched_equals_single_calls(cuda_lib):
    dm = cuda_lib
    params, fields, _ = _mix(dm)
    descs = [torch.empty(dm.dmcr_descriptor_length(p), device="cuda") for p in params]
    dm.dmcr_descriptor_batched(params, fields, descs)
    for p, f, d in zip(params, fields, descs):
        assert torch.equal(d, dm.descriptor(f, p))
    # and against the oracle for one 3-D instance
    p, f, d = params[3], fields[3], descs[3]
    op = oracle.Params(ndim=3, window=p.window, levels=p.levels)
    np.testing.assert_allclose(d.cpu().numpy(), oracle.descriptor(f.cpu().numpy().astype(np.float64), op), rtol=1e-5)


def test_loss_grad_and_vjp_batched_equal_single_calls(cuda_lib):
    dm = cuda_lib
    params, fields, targets = _mix(dm)
    d_des = [dm.descriptor(t, p) for p, t in zip(params, targets)]
    n = len(params)
    loss = torch.empty(n * 6, device="cuda")
    grads = [torch.empty_like(f) for f in fields]
    dm.dmcr_loss_grad_batched(params, dm.LossOpts(), fields, d_des, loss, grads)
    for i in range(n):
        l1, g1 = dm.loss_grad(fields[i], d_des[i], params[i])
        assert torch.equal(loss[6 * i:6 * i + 6], l1)
        assert torch.equal(grads[i], g1)
    up = [torch.randn(dm.dmcr_descriptor_length(p), device="cuda") for p in params]
    gf = [torch.empty_like(f) for f in fields]
    dm.dmcr_descriptor_vjp_batched(params, fields, up, gf)
    for i in range(n):
        assert torch.equal(gf[i], dm.descriptor_vjp(fields[i], up[i], params[i]))


def test_adam_step_batched_equals_single_steps(cuda_lib):
    dm = cuda_lib
    params, fields, targets = _mix(dm)
    d_des = [dm.descriptor(t, p) for p, t in zip(params, targets)]
    opts = dm.ReconOpts(lr=1e-2)
    fa = [f.clone() for f in fields]
    ma = [torch.zeros_like(f) for f in fields]
    va = [torch.zeros_like(f) for f in fields]
    steps = [0] * len(params)
    for _ in range(3):
        steps = dm.dmcr_adam_step_batched(params, opts, d_des, fa, ma, va, steps)
    assert steps == [3] * len(params)
    for i, p in enumerate(params):
        f = fields[i].clone()
        m = torch.zeros_like(f)
        v = torch.zeros_like(f)
        s = 0
        for _ in range(3):
            s = dm.dmcr_adam_step(p, opts, d_des[i], f, m, v, s)
        assert torch.equal(f, fa[i]) and torch.equal(m, ma[i]) and torch.equal(v, va[i])


def test_reconstruction_same_alone_and_in_the_mix(cuda_lib):
    dm = cuda_lib
    params, fields, targets = _mix(dm)
    d_des = [dm.descriptor(t, p) for p, t in zip(params, targets)]
    opts = [dm.ReconOpts(max_iters=40 + 10 * i, lr=1e-2, tol_rel=0.0 if i % 2 else 0.2, check_every=5)
            for i in range(len(params))]
    fb = [f.clone() for f in fields]
    mb = [torch.zeros_like(f) for f in fields]
    vb = [torch.zeros_like(f) for f in fields]
    reps, steps = dm.dmcr_reconstruct_batched(params, opts, d_des, fb, mb, vb, [0] * len(params))
    for i, p in enumerate(params):
        f = fields[i].clone()
        m = torch.zeros_like(f)
        v = torch.zeros_like(f)
        rep, st = dm.dmcr_reconstruct(p, opts[i], d_des[i], f, m, v)
        assert st == steps[i] and rep["iterations"] == reps[i]["iterations"]
        assert rep["converged"] == reps[i]["converged"]
        assert torch.equal(f, fb[i]), i
        assert rep["rel_err"] == reps[i]["rel_err"]
        assert rep["rounded_rel_err"] == reps[i]["rounded_rel_err"]


def test_nan_poisoned_instance_is_isolated(cuda_lib):
    """A NaN-poisoned job stops with DMCR_ENONFINITE; the other jobs of the batch finish
    exactly as they would alone, and the single-instance call reports the error."""
    dm = cuda_lib
    params, fields, targets = _mix(dm)
    params, fields, targets = params[:3], fields[:3], targets[:3]
    d_des = [dm.descriptor(t, p) for p, t in zip(params, targets)]
    fields[1] = fields[1].clone()
    fields[1].view(-1)[5] = float("nan")
    opts = dm.ReconOpts(max_iters=30, lr=1e-2)
    fb = [f.clone() for f in fields]
    mb = [torch.zeros_like(f) for f in fields]
    vb = [torch.zeros_like(f) for f in fields]
    reps, steps = dm.dmcr_reconstruct_batched(params, opts, d_des, fb, mb, vb, [0, 0, 0])
    assert reps[1]["status"] == 4 and steps[1] == 0
    for i in (0, 2):
        assert reps[i]["status"] == 0 and steps[i] == 30
        f = fields[i].clone()
        m = torch.zeros_like(f)
        v = torch.zeros_like(f)
        dm.dmcr_reconstruct(params[i], opts, d_des[i], f, m, v)
        assert torch.equal(f, fb[i])
    f = fields[1].clone()
    with pytest.raises(dm.DmcrError) as e:
        dm.dmcr_reconstruct(params[1], opts, d_des[1], f, torch.zeros_like(f), torch.zeros_like(f))
    assert e.value.status == 4


def test_batched_mix_of_descriptor_kinds_and_phases_equals_single_calls(cuda_lib):
    # one batch holding two-point, three-point, corrected and three-phase instances
    dm = cuda_lib
    specs = [dict(shape=(48, 40), window=(5, 4), levels=2),
             dict(shape=(32, 32), window=(6, 6), descriptor=dm.DMCR_DESC_S3),
             dict(shape=(40, 48), window=(4, 7), levels=2, descriptor=dm.DMCR_DESC_S2_TILDE),
             dict(shape=(64, 48), window=(7, 5), levels=2, phases=3),
             dict(shape=(16, 16, 16), window=(2, 2, 2), phases=2)]
    params = [dm.Params(**s) for s in specs]
    fields, targets = [], []
    for i, p in enumerate(params):
        shape = tuple(p.shape) if p.phases == 1 else (p.phases,) + tuple(p.shape)
        fields.append(_dev(np.random.default_rng(70 + i).uniform(-0.2, 1.2, shape)))
        targets.append(_dev((np.random.default_rng(80 + i).random(shape) < 0.35).astype(np.float32)))
    descs = [torch.empty(dm.dmcr_descriptor_length(p), device="cuda") for p in params]
    dm.dmcr_descriptor_batched(params, fields, descs)
    for p, f, d in zip(params, fields, descs):
        assert torch.equal(d, dm.descriptor(f, p))
    d_des = [dm.descriptor(t, p) for p, t in zip(params, targets)]
    n = len(params)
    loss = torch.empty(n * 6, device="cuda")
    grads = [torch.empty_like(f) for f in fields]
    dm.dmcr_loss_grad_batched(params, dm.LossOpts(), fields, d_des, loss, grads)
    for i in range(n):
        l1, g1 = dm.loss_grad(fields[i], d_des[i], params[i])
        assert torch.equal(loss[6 * i:6 * i + 6], l1), i
        assert torch.equal(grads[i], g1), i
