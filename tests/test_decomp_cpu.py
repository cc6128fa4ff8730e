"""Domain decomposition of one reconstruction over CPU ranks (gloo, world sizes 1-3).

Every rank owns a slab of rows (2-D) or planes (3-D), receives a halo of P_0 rows from
its neighbours, pools its slab (coarse levels replicated by one sum-allreduce), sums its
own pairs, and one sum-allreduce of the sum_l K_half partial sums (with the box-penalty
sum) gives every rank the descriptor.  The adjoint and Adam are local.  The per-slab pair
arithmetic runs the oracle's threshold on each rank's own positions; descriptor, loss,
gradient and two Adam steps must equal the UNSHARDED oracle to FP64 rounding."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import synthetic
from paper_2103_09686_gb300 import decomp


class OracleSlabBackend:
    """The per-slab pair arithmetic from the oracle's threshold (FP64): f(a)^2 summed over
    the own positions, and the gather-form gradient sum_r G(r) [h(a_y(r)) + h(a_{y-r}(r))],
    h = f f', with the halo supplying the rows beyond the slab."""

    def __init__(self, kind="soft", alpha=10.0):
        self.kind, self.alpha = kind, alpha

    @staticmethod
    def _tip(ext, p0, rows, r):
        t = ext[p0 + int(r[0]):p0 + int(r[0]) + rows]
        return np.roll(t, shift=tuple(-int(c) for c in r[1:]), axis=tuple(range(1, ext.ndim)))

    def _fh(self, a):
        f, df = oracle.threshold(a.ravel(), self.kind, self.alpha)
        return f.reshape(a.shape), (f * df).reshape(a.shape)

    def level_sums(self, ext, p0, rows, shifts):
        own = ext[p0:p0 + rows]
        out = np.empty(len(shifts))
        for k, r in enumerate(shifts):
            a = own if not np.any(r) else 0.5 * (own + self._tip(ext, p0, rows, r))
            f, _ = self._fh(a)
            out[k] = np.sum(f * f)
        return out

    def level_vjp(self, ext, p0, rows, shifts, G):
        own = ext[p0:p0 + rows]
        g = np.zeros(own.shape)
        for k, r in enumerate(shifts):
            if not np.any(r):
                g += 2.0 * G[k] * self._fh(own)[1]
            else:
                g += G[k] * (self._fh(0.5 * (own + self._tip(ext, p0, rows, r)))[1] +
                             self._fh(0.5 * (own + self._tip(ext, p0, rows, -r)))[1])
        return g


CASES = {
    "2d": dict(shape=(24, 16), window=(3, 2), levels=2, kind="soft"),
    "2d_identity": dict(shape=(24, 16), window=(2, 3), levels=1, kind="identity"),
    "3d": dict(shape=(16, 8, 8), window=(2, 1, 2), levels=2, kind="soft"),
}


def _problem(case):
    c = CASES[case]
    shape = c["shape"]
    M = synthetic.uniform_field(shape, 71) * 1.4 - 0.2            # box penalty active
    T = (np.random.default_rng(72).random(shape) < 0.35).astype(np.float64)
    op = oracle.Params(ndim=len(shape), window=c["window"], levels=c["levels"], threshold=c["kind"])
    return c, M, oracle.descriptor(T, op), op


def _run_rank(case, rank, world, mode):
    c, M, D_des, _ = _problem(case)
    plan = decomp.SlabPlan(c["shape"], c["window"], c["levels"], rank, world)
    lo, hi = plan.rows
    rec = decomp.SlabReconstruction(plan, OracleSlabBackend(c["kind"]), M[lo:hi], D_des, mode=mode)
    out, g = rec.loss_grad()
    losses = [rec.adam_step(lr=1e-2)["L"], rec.adam_step(lr=1e-2)["L"]]
    return out, g, losses, rec.M


def _rank_main(case, rank, world, port, mode, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        q.put((rank, _run_rank(case, rank, world, mode)))
    finally:
        dist.destroy_process_group()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _sharded(case, world, mode):
    if world == 1:
        return [_run_rank(case, 0, 1, mode)]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(case, r, world, port, mode, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return [res[r] for r in range(world)]


@pytest.mark.parametrize("case,world,mode", [("2d", 2, "norm"), ("2d", 3, "squared"), ("2d_identity", 2, "norm"),
                                             ("3d", 2, "norm"), ("3d", 3, "norm"), ("2d", 1, "norm")])
def test_sharded_evaluation_equals_the_unsharded_oracle(case, world, mode):
    c, M, D_des, op = _problem(case)
    ranks = _sharded(case, world, mode)
    want, g_ref = oracle.loss_grad(M, D_des, op, mode=mode)
    for out, _, _, _ in ranks:          # every rank holds the same descriptor and loss
        np.testing.assert_allclose(out["D"], oracle.descriptor(M, op), rtol=1e-12, atol=1e-15)
        for k in ("E", "E2", "Ebc", "lambda", "L", "rel_err"):
            np.testing.assert_allclose(out[k], want[k], rtol=1e-12, err_msg=k)
    g = np.concatenate([r[1] for r in ranks], axis=0)
    assert g.shape == M.shape
    assert np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref) < 1e-12
    # two Adam steps (Keras form, the library's) on the slabs = two on the whole field
    M2, hist = oracle.reconstruct(M, D_des, op, iters=3, lr=1e-2, mode=mode)
    np.testing.assert_allclose([ranks[0][2][0], ranks[0][2][1]], [hist[0]["L"], hist[1]["L"]], rtol=1e-12)
    Mr = np.concatenate([r[3] for r in ranks], axis=0)
    # oracle.reconstruct took a third step after evaluating iteration 3; redo two steps here
    Mo, m, v = np.array(M), np.zeros_like(M), np.zeros_like(M)
    for t in (1, 2):
        _, gt = oracle.loss_grad(Mo, D_des, op, mode=mode)
        Mo, m, v = oracle.adam_step(Mo, gt, m, v, t, lr=1e-2)
    np.testing.assert_allclose(Mr, Mo, rtol=1e-12, atol=1e-14)


def test_slab_plan_rows_align_to_the_coarsest_level():
    plan = [decomp.SlabPlan((40, 16), (2, 2), 3, r, 3) for r in range(3)]
    rows = [p.rows for p in plan]
    assert rows[0][0] == 0 and rows[-1][1] == 40
    assert all(a[1] == b[0] for a, b in zip(rows, rows[1:]))      # contiguous, no overlap
    assert all(lo % 4 == 0 and hi % 4 == 0 for lo, hi in rows)     # 2^(levels-1) = 4
    assert plan[1].rows_of(1, 2) == (rows[1][0] >> 2, rows[1][1] >> 2)


@pytest.mark.parametrize("kw", [dict(shape=(16, 16), window=(3, 2), levels=2, world=8),   # slabs of 2 rows < P_0
                                dict(shape=(16, 16), window=(2, 2), levels=3, world=5),   # 4 units for 5 ranks
                                dict(shape=(18, 16), window=(2, 2), levels=3, world=2),   # 18 not divisible by 4
                                dict(shape=(16, 16), window=(5, 2), levels=2, world=1)])  # window > level size / 2
def test_slab_plan_rejections(kw):
    world = kw.pop("world")
    with pytest.raises(ValueError):
        decomp.SlabPlan(rank=0, world=world, **kw)
