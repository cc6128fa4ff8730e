"""Continuous batching: jobs of mixed 2-D/3-D sizes admitted while others run, limited by
slots and an HBM budget; every job's result must be the same alone and in the mix."""
import numpy as np
import pytest
import torch

import synthetic

pytestmark = pytest.mark.gpu


def _jobs(dm, serve):
    specs = [((64, 64), (8, 8), 2, 0.3), ((48, 48), (6, 6), 1, 0.4), ((32, 32, 32), (3, 3, 3), 2, 0.25),
             ((128, 128), (12, 12), 2, 0.35), ((64, 64), (16, 16), 1, 0.2), ((16, 24, 32), (2, 3, 4), 1, 0.3),
             ((96, 96), (8, 8), 3, 0.45)]
    jobs = []
    for i, (shape, win, lev, vf) in enumerate(specs):
        if len(shape) == 2:
            tgt = synthetic.target_2d_grf(shape[0], 3.0, vf, 500 + i) if shape[0] == shape[1] else \
                synthetic.threshold_count(synthetic.gaussian_random_field(shape, 3.0, 500 + i), vf)
        else:
            tgt = synthetic.threshold_count(synthetic.gaussian_random_field(shape, 2.0, 500 + i), vf)
        opts = dm.ReconOpts(max_iters=60 + 20 * i, lr=1e-2, tol_rel=0.05 if i % 3 == 0 else 0.0, check_every=10,
                            seed=900 + i)
        jobs.append(serve.Job(job_id=i, params=dm.Params(shape=shape, window=win, levels=lev), target=tgt, opts=opts,
                              arrival=0.0))
    return jobs


def test_serve_results_equal_alone(cuda_lib):
    dm = cuda_lib
    from paper_2103_09686_gb300 import serve
    srv = serve.Server(max_slots=3, tick_iters=20)
    jobs = _jobs(dm, serve)
    # staggered submission: some jobs arrive while others are mid-flight
    srv.submit(jobs[0])
    srv.submit(jobs[1])
    srv.tick()
    for j in jobs[2:5]:
        srv.submit(j)
    srv.tick()
    srv.tick()
    for j in jobs[5:]:
        srv.submit(j)
    while not srv.idle():
        srv.tick()
    assert len(srv.done) == len(jobs)
    for j in jobs:
        alone = serve.reconstruct_alone(_jobs(dm, serve)[j.job_id])
        assert j.iters_done == alone.iters_done, j.job_id
        assert j.report["converged"] == alone.report["converged"]
        np.testing.assert_array_equal(j.result, alone.result)
        assert j.report["rel_err"] == alone.report["rel_err"]


def test_serve_respects_hbm_budget(cuda_lib):
    dm = cuda_lib
    from paper_2103_09686_gb300 import serve
    base = _jobs(dm, serve)[0]
    jobs = [serve.Job(job_id=k, params=base.params, target=base.target, opts=base.opts) for k in range(3)]
    one = jobs[0].bytes_estimate()
    srv = serve.Server(hbm_budget_bytes=int(one * 1.5), max_slots=8, tick_iters=20)
    for j in jobs:
        srv.submit(j)
    peak = 0
    while not srv.idle():
        srv.tick()
        peak = max(peak, len(srv.active))
        assert srv.in_use <= srv.budget
    assert peak == 1 and len(srv.done) == 3
    tiny = serve.Server(hbm_budget_bytes=1024, tick_iters=20)
    tiny.submit(_jobs(dm, serve)[0])
    with pytest.raises(MemoryError):
        tiny.tick()


def test_threaded_classes_results_equal_alone(cuda_lib):
    """Cost classes ticking on their own threads and streams, jobs submitted while the
    workers run: each result equals the job's reconstruction alone."""
    dm = cuda_lib
    from paper_2103_09686_gb300 import serve
    jobs = _jobs(dm, serve)
    srv = serve.Server(max_slots=4, tick_iters=20, class_caps=(5e6, 5e7, float("inf")))
    srv.start()
    try:
        for j in jobs:
            srv.submit(j)
        srv.wait_idle(timeout=300)
    finally:
        srv.stop()
    assert len(srv.done) == len(jobs)
    for j in jobs:
        alone = serve.reconstruct_alone(_jobs(dm, serve)[j.job_id])
        assert j.iters_done == alone.iters_done
        np.testing.assert_array_equal(j.result, alone.result)


def test_serve_multiphase_job_equals_alone(cuda_lib):
    # a three-phase job (field stack 3 x 48 x 48) batched with a one-field job
    dm = cuda_lib
    from paper_2103_09686_gb300 import serve

    def jobs():
        mp = serve.Job(job_id=0, params=dm.Params(shape=(48, 48), window=(6, 6), levels=2, phases=3),
                       target=synthetic.multiphase_grf((48, 48), 3.0, (0.3, 0.3), 77),
                       opts=dm.ReconOpts(max_iters=80, lr=1e-2, check_every=10, seed=5))
        one = serve.Job(job_id=1, params=dm.Params(shape=(64, 64), window=(8, 8), levels=2),
                        target=synthetic.target_2d_grf(64, 3.0, 0.3, 78),
                        opts=dm.ReconOpts(max_iters=60, lr=1e-2, check_every=10, seed=6))
        return [mp, one]

    srv = serve.Server(max_slots=4, tick_iters=20)
    js = jobs()
    for j in js:
        srv.submit(j)
    while not srv.idle():
        srv.tick()
    assert js[0].result.shape == (3, 48, 48)
    for j, a in zip(js, jobs()):
        alone = serve.reconstruct_alone(a)
        assert j.iters_done == alone.iters_done
        np.testing.assert_array_equal(j.result, alone.result)
