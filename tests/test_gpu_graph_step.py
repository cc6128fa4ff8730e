"""dmcr_adam_step(_batched) replays a cached CUDA graph of the iteration when it is called
again with the same arguments.  The replay must give exactly (bitwise) what the direct
launches give -- the library's per-kernel timers force the direct path -- including after
a jump in the Adam step count (a resume) and with calls of other kinds on the same
workspace in between."""
import numpy as np
import pytest
import torch

import synthetic

pytestmark = pytest.mark.gpu


def _run(dm, p, D, steps, direct, step0=0, interleave=False):
    f = torch.tensor(synthetic.uniform_field(p.shape, 3), dtype=torch.float32, device="cuda")
    m, v = torch.zeros_like(f), torch.zeros_like(f)
    ws = dm.workspace(p)
    loss = torch.zeros(6, device="cuda")
    losses = []
    dm.dmcr_profile_enable(direct)
    try:
        st = step0
        for k in range(steps):
            st = dm.dmcr_adam_step(p, dm.ReconOpts(lr=1e-2), D, f, m, v, st, loss, ws)
            losses.append(loss.clone())
            if interleave and k == 2:
                dm.dmcr_loss_grad(p, dm.LossOpts(), f, D, torch.empty(6, device="cuda"), torch.empty_like(f), None, ws)
        torch.cuda.synchronize()
    finally:
        dm.dmcr_profile_enable(False)
        dm.dmcr_profile_reset()
    assert st == step0 + steps
    return f, m, v, torch.stack(losses)


@pytest.mark.parametrize("shape,window,levels", [((64, 64), (16, 16), 1), ((48, 40), (5, 7), 2),
                                                 ((16, 16, 16), (3, 2, 3), 2)])
def test_cached_graph_steps_equal_direct_steps(cuda_lib, shape, window, levels):
    dm = cuda_lib
    p = dm.Params(shape=shape, window=window, levels=levels)
    T = torch.tensor((np.random.default_rng(1).random(shape) < 0.3).astype(np.float32), device="cuda")
    D = dm.descriptor(T, p)
    for kw in (dict(), dict(step0=57), dict(interleave=True)):
        a = _run(dm, p, D, 6, direct=False, **kw)
        b = _run(dm, p, D, 6, direct=True, **kw)
        for x, y in zip(a, b):
            assert torch.equal(x, y), kw


def test_cached_graph_batched_steps_equal_direct_steps(cuda_lib):
    dm = cuda_lib
    params = [dm.Params(shape=(64, 64), window=(8, 8), levels=2), dm.Params(shape=(32, 48), window=(4, 6)),
              dm.Params(shape=(16, 16, 16), window=(2, 2, 2))]
    targets = [dm.descriptor(torch.tensor((np.random.default_rng(i).random(p.shape) < 0.4).astype(np.float32),
                                          device="cuda"), p) for i, p in enumerate(params)]

    def run(direct):
        fields = [torch.tensor(synthetic.uniform_field(p.shape, 9 + i), dtype=torch.float32, device="cuda")
                  for i, p in enumerate(params)]
        ms = [torch.zeros_like(f) for f in fields]
        vs = [torch.zeros_like(f) for f in fields]
        ws = dm.batch_workspace(params)
        loss = torch.zeros(6 * len(params), device="cuda")
        steps = [0, 10, 3]
        dm.dmcr_profile_enable(direct)
        try:
            for _ in range(5):
                steps = dm.dmcr_adam_step_batched(params, dm.ReconOpts(lr=1e-2), targets, fields, ms, vs, steps, loss,
                                                  ws)
            torch.cuda.synchronize()
        finally:
            dm.dmcr_profile_enable(False)
            dm.dmcr_profile_reset()
        assert steps == [5, 15, 8]
        return fields + ms + vs + [loss]

    for x, y in zip(run(False), run(True)):
        assert torch.equal(x, y)
