"""The autotuner's coordinate descent and cache on the CPU, with a synthetic cost model in
place of the CUDA-event timer."""
import json

import numpy as np

import paper_2103_09686_gb300 as dm
from paper_2103_09686_gb300 import tune


def _cost(target):
    # a bowl around `target` in every coordinate, with invalid shapes (inf) mixed in
    def timer(p, field, tgt):
        t = p.tune
        if t[1] == 12:
            return float("inf")
        return 1.0 + sum(abs(a - b) for a, b in zip(t, target)) / 100.0
    return timer


def test_coordinate_descent_finds_the_best_value_of_every_axis():
    p = dm.Params(shape=(32, 32), window=(4, 4))
    best, ms, trials = tune.search(p, device="cpu", timer=_cost((16, 8, 64, 5)))
    assert best == (16, 8, 64, 5)
    assert ms == 1.0
    # one trial per candidate value and axis, the start shape once
    n = 1 + sum(len(v) - (1 if 0 in v else 0) for v in (tune.FWD_ROWS, tune.ADJ_XBLOCKS, tune.ADJ_ROWS,
                                                          tune.ADJ_CHUNKS))
    assert len(trials) == n


def test_search_builds_phase_stacks():
    seen = []

    def timer(p, field, tgt):
        seen.append(tuple(field.shape))
        return 1.0
    tune.search(dm.Params(shape=(16, 16), window=(2, 2), phases=3), device="cpu", timer=timer)
    assert set(seen) == {(3, 16, 16)}


def test_cache_is_keyed_by_problem_descriptor_and_phases(tmp_path, monkeypatch):
    calls = []

    def fake_search(p, seed=0, device="cuda", timer=None):
        calls.append(p.phases)
        return (8, 2, 0, 3), 1.0, []
    key = tune._key
    monkeypatch.setattr(tune, "search", fake_search)
    monkeypatch.setattr(tune, "_key", lambda p: key(p, "GPU"))
    cache = str(tmp_path / "tune.json")
    p = dm.Params(shape=(64, 64), window=(8, 8))
    assert tune.tuned(p, cache).tune == (8, 2, 0, 3)
    assert tune.tuned(p, cache).tune == (8, 2, 0, 3)          # cached: no second search
    tune.tuned(dm.Params(shape=(64, 64), window=(8, 8), phases=2), cache)
    assert calls == [1, 2]
    table = json.load(open(cache))
    assert len(table) == 2
    # the three-point descriptor does not use the tuned kernels
    p3 = dm.Params(shape=(64, 64), window=(8, 8), descriptor=dm.DMCR_DESC_S3)
    assert tune.tuned(p3, cache) is p3

