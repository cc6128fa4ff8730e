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


def test_graph_caches_evict_and_recapture(cuda_lib):
    """More argument sets than the caches hold (16 step graphs, 32 reconstruction graphs):
    the least recently used graphs are evicted (after their last replay has run) and a later
    call with evicted arguments captures again; every result equals the direct launches."""
    dm = cuda_lib
    p = dm.Params(shape=(32, 32), window=(4, 4))
    D = dm.descriptor(torch.tensor((np.random.default_rng(2).random((32, 32)) < 0.4).astype(np.float32),
                                   device="cuda"), p)

    def fresh(k):
        f = torch.tensor(synthetic.uniform_field((32, 32), 100 + k), dtype=torch.float32, device="cuda")
        return f, torch.zeros_like(f), torch.zeros_like(f)

    def steps(k, direct, n=3):
        f, m, v = fresh(k)
        dm.dmcr_profile_enable(direct)
        try:
            st = 0
            for _ in range(n):
                st = dm.dmcr_adam_step(p, dm.ReconOpts(lr=1e-2), D, f, m, v, st, None, wss[k])
        finally:
            dm.dmcr_profile_enable(False)
            dm.dmcr_profile_reset()
        return f

    wss = [dm.workspace(p) for _ in range(20)]       # distinct workspaces: distinct argument sets
    graph = [steps(k, False) for k in range(20)] + [steps(0, False)]      # set 0 evicted by now
    direct = [steps(k, True) for k in range(20)] + [steps(0, True)]
    for a, b in zip(graph, direct):
        assert torch.equal(a, b)

    rws = [dm.workspace(p) for _ in range(40)]     # 40 table addresses: 40 distinct launch sequences

    def recon(k):
        f, m, v = fresh(k)
        rep, _ = dm.dmcr_reconstruct(p, dm.ReconOpts(max_iters=3 + k % 4, lr=1e-2, check_every=1), D, f, m, v,
                                     ws=rws[k])
        return f, rep["iterations"]

    first = [recon(k) for k in range(40)]          # more than the 32 cached: evictions
    again = [recon(k) for k in (0, 1, 39)]
    for (fa, ia), (fb, ib) in zip([first[0], first[1], first[39]], again):
        assert ia == ib and torch.equal(fa, fb)
