"""Host logic of the reconstruction server on the CPU: admission by slots and HBM budget,
cost classes, ticks of at most tick_iters iterations, retirement and the order in which
waiting jobs are admitted.  The library's device calls are replaced by a fake that only
counts iterations (no GPU is touched); the sizes and lengths come from the real library."""
import dataclasses

import numpy as np
import pytest
import torch

import paper_2103_09686_gb300 as dm
from paper_2103_09686_gb300 import _lib, serve


class FakeDevice:
    """Stands in for the device calls: a job converges after `need` iterations."""

    def __init__(self, need):
        self.need = need          # job_id -> iterations to convergence
        self.calls = []           # (job ids of the tick, iterations asked per job)
        self.ids = {}

    def init_uniform(self, field, seed, stream=None):
        field.fill_(0.5)

    def descriptor_batched(self, params, fields, descs, ws=None, stream=None):
        for d in descs:
            d.fill_(1.0)
        return descs

    def reconstruct_batched(self, params, opts, targets, fields, ms, vs, steps, ws=None, stream=None):
        ids = [self.ids[id(f)] for f in fields]
        self.calls.append((ids, [o.max_iters for o in opts]))
        reps, out = [], []
        for jid, o, s in zip(ids, opts, steps):
            left = self.need[jid] - s
            take = min(o.max_iters, max(left, 0))
            conv = left <= o.max_iters
            reps.append({"iterations": take, "converged": conv, "status": 0, "E": 0.0, "E2": 0.0, "Ebc": 0.0,
                         "lambda": 0.0, "L": 0.0, "rel_err": 1e-4 if conv else 1.0})
            out.append(s + take)
        return reps, out


@pytest.fixture()
def fake(monkeypatch):
    _lib.load(build_if_missing=True)   # lengths and workspace sizes: host-side queries of the library
    dev = FakeDevice({})
    monkeypatch.setattr(_lib, "dmcr_init_uniform", dev.init_uniform)
    monkeypatch.setattr(_lib, "dmcr_descriptor_batched", dev.descriptor_batched)
    monkeypatch.setattr(_lib, "dmcr_reconstruct_batched", dev.reconstruct_batched)
    orig_empty = torch.empty

    def empty(shape, dtype=None, device=None, **kw):
        t = orig_empty(shape, dtype=dtype, device="cpu", **kw)
        return t

    monkeypatch.setattr(serve.torch, "empty", empty)
    return dev


def _job(i, shape=(64, 64), window=(8, 8), levels=1, max_iters=400, phases=1):
    p = dm.Params(shape=shape, window=window, levels=levels, phases=phases)
    tshape = tuple(shape) if phases == 1 else (phases,) + tuple(shape)
    return serve.Job(job_id=i, params=p, target=np.zeros(tshape, np.float32),
                     opts=dm.ReconOpts(max_iters=max_iters, tol_rel=1e-3, check_every=10))


def _run(srv, dev, jobs):
    orig_admit = srv._admit

    def admit(cls):
        orig_admit(cls)
        for j in cls.active:
            dev.ids[id(j.field)] = j.job_id

    srv._admit = admit
    for j in jobs:
        srv.submit(j)
    for _ in range(1000):
        if srv.idle():
            break
        srv.tick()
    assert srv.idle()


def test_slots_bound_the_active_jobs_and_jobs_retire_when_converged(fake):
    jobs = [_job(i) for i in range(5)]
    fake.need.update({0: 30, 1: 120, 2: 60, 3: 10, 4: 90})
    srv = serve.Server(device="cpu", max_slots=2, tick_iters=50)
    _run(srv, fake, jobs)
    assert all(len(ids) <= 2 for ids, _ in fake.calls)
    assert all(all(it <= 50 for it in its) for _, its in fake.calls)
    assert {j.job_id: j.iters_done for j in srv.done} == {0: 30, 1: 120, 2: 60, 3: 10, 4: 90}
    # first come, first admitted
    first = [ids for ids, _ in fake.calls][0]
    assert first == [0, 1]


def test_hbm_budget_limits_admission(fake):
    jobs = [_job(i, shape=(256, 256), window=(16, 16), levels=2) for i in range(4)]
    fake.need.update({i: 100 for i in range(4)})
    per_job = jobs[0].bytes_estimate()
    srv = serve.Server(device="cpu", hbm_budget_bytes=int(2.5 * per_job), max_slots=64, tick_iters=50)
    _run(srv, fake, jobs)
    assert max(len(ids) for ids, _ in fake.calls) == 2
    assert len(srv.done) == 4


def test_a_job_larger_than_the_budget_is_refused(fake):
    job = _job(0, shape=(256, 256), window=(16, 16))
    fake.need[0] = 10
    srv = serve.Server(device="cpu", hbm_budget_bytes=job.bytes_estimate() // 2, tick_iters=50)
    srv.submit(job)
    with pytest.raises(MemoryError):
        srv.tick()


def test_cost_classes_tick_separately(fake):
    small = [_job(i, shape=(64, 64), window=(4, 4)) for i in range(3)]
    large = [_job(10 + i, shape=(256, 256), window=(32, 32), levels=2) for i in range(2)]
    fake.need.update({j.job_id: 100 for j in small + large})
    cap = serve.iteration_units(small[0].params) * 10
    srv = serve.Server(device="cpu", max_slots=64, tick_iters=50, class_caps=(cap, float("inf")))
    _run(srv, fake, small + large)
    for ids, _ in fake.calls:
        assert all(i < 10 for i in ids) or all(i >= 10 for i in ids)
    assert len(srv.done) == 5


def test_phase_stacks_are_sized_by_their_phases(fake):
    one = _job(0, shape=(64, 64), window=(8, 8))
    three = _job(1, shape=(64, 64), window=(8, 8), phases=3)
    assert serve.field_shape(three.params) == (3, 64, 64)
    assert serve.iteration_units(three.params) == 9 * serve.iteration_units(one.params)
    assert three.bytes_estimate() > 3 * (one.bytes_estimate() - dm.dmcr_workspace_size(one.params))


def test_tick_iters_must_be_a_multiple_of_check_every(fake):
    srv = serve.Server(device="cpu", tick_iters=50)
    job = _job(0)
    job.opts = dataclasses.replace(job.opts, check_every=7)
    with pytest.raises(ValueError):
        srv.submit(job)


def test_class_slots_serve_heavy_jobs_one_at_a_time(fake):
    """A class limited to one active job serves its jobs in arrival order, one per tick set,
    while a cheap class keeps several active."""
    small = [_job(i, shape=(64, 64), window=(4, 4)) for i in range(3)]
    large = [_job(10 + i, shape=(256, 256), window=(32, 32), levels=2) for i in range(3)]
    fake.need.update({j.job_id: 100 for j in small + large})
    cap = serve.iteration_units(small[0].params) * 10
    srv = serve.Server(device="cpu", max_slots=64, tick_iters=50, class_caps=(float("inf"), cap),
                       class_slots=(1, None))
    _run(srv, fake, small + large)
    heavy = [ids for ids, _ in fake.calls if ids and ids[0] >= 10]
    assert all(len(ids) == 1 for ids in heavy)
    assert [ids[0] for ids in heavy] == [10, 10, 11, 11, 12, 12]        # arrival order, 2 ticks each
    assert max(len(ids) for ids, _ in fake.calls if ids[0] < 10) == 3
    assert len(srv.done) == 6
    with pytest.raises(ValueError):
        serve.Server(device="cpu", class_caps=(1.0, 2.0), class_slots=(1,))


def test_exclusive_top_class_pauses_the_others(fake):
    """With exclusive_top, no tick of a cheaper class runs while a job of the most expensive
    class is waiting or active."""
    small = [_job(i, shape=(64, 64), window=(4, 4)) for i in range(2)]
    large = [_job(10, shape=(256, 256), window=(32, 32), levels=2)]
    fake.need.update({0: 100, 1: 100, 10: 150})
    cap = serve.iteration_units(small[0].params) * 10
    srv = serve.Server(device="cpu", max_slots=64, tick_iters=50, class_caps=(cap, float("inf")),
                       exclusive_top=True)
    _run(srv, fake, small + large)
    kinds = ["large" if ids[0] >= 10 else "small" for ids, _ in fake.calls]
    assert kinds == ["large"] * 3 + ["small"] * 2        # the large job first, alone, then the small ones
    assert len(srv.done) == 3
