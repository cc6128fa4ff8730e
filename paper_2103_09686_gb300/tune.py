"""Autotuner for the launch shapes of the fused correlation kernels.

The plan's built-in choices (forward tile rows; adjoint rx blocks, ry rows and count of the
shift chunks) are heuristics.  ``tuned(params)`` measures one descriptor + loss + gradient
evaluation (``dmcr_loss_grad``, CUDA events, median of 3 after a warm-up) for candidate
shapes by coordinate descent -- forward tile rows first (they only affect the forward
kernel), then the adjoint's rx blocks per chunk (they set how many ry rows fit in shared
memory), its ry rows, and its chunk limit -- and returns the params with the fastest shape
in ``tune``.  Results are cached in a JSON file keyed by the problem class and the GPU, so a
shape is measured once per machine.  Shapes change only the blocking and summation order:
results agree to rounding.
"""
from __future__ import annotations

import dataclasses
import json
import os
import threading

import numpy as np
import torch

from . import _lib

FWD_ROWS = (4, 8, 16, 32)
ADJ_ROWS = (0, 2, 4, 8, 12, 16)
ADJ_CHUNKS = (0, 8, 16, 64)
ADJ_XBLOCKS = (0, 3, 5, 12, 32)
_lock = threading.Lock()


def _cache_path(path: str | None) -> str:
    if path:
        return path
    return os.environ.get("DMCR_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "dmcr_tune.json"))


def _key(p: _lib.Params, device_name: str | None = None) -> str:
    name = device_name if device_name is not None else torch.cuda.get_device_name()
    return "|".join(map(str, (name, tuple(p.shape), tuple(p.window), p.levels, p.threshold, p.alpha, p.path,
                              p.descriptor, p.phases)))


def _field_shape(p: _lib.Params) -> tuple:
    return tuple(p.shape) if p.phases == 1 else (p.phases,) + tuple(p.shape)


def _time(p: _lib.Params, field, target, reps: int = 3) -> float:
    try:
        ws = _lib.workspace(p, field.device)
        desc = _lib.descriptor(target, p, ws)
    except _lib.DmcrError:
        return float("inf")          # shape not valid for this problem (e.g. shared memory)
    loss = torch.empty(6, device=field.device)
    grad = torch.empty_like(field)
    _lib.dmcr_loss_grad(p, _lib.LossOpts(), field, desc, loss, grad, None, ws)
    times = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        _lib.dmcr_loss_grad(p, _lib.LossOpts(), field, desc, loss, grad, None, ws)
        b.record()
        torch.cuda.synchronize()
        times.append(a.elapsed_time(b))
    return float(np.median(times))


def search(p: _lib.Params, seed: int = 0, device="cuda", timer=None) -> tuple[tuple, float, list]:
    """Coordinate descent over the launch shapes; returns (best tune, its ms, trials).
    ``timer(params, field, target)`` measures one shape (default: CUDA events)."""
    rng = np.random.default_rng(seed)
    shape = _field_shape(p)
    field = torch.tensor(rng.uniform(0.0, 1.0, shape), dtype=torch.float32, device=device)
    target = torch.tensor((rng.random(shape) < 0.35).astype(np.float32), device=device)
    trials = []
    timer = timer or _time

    def run(t):
        ms = timer(dataclasses.replace(p, tune=t), field, target)
        trials.append((t, ms))
        return ms

    best = (0, 0, 0, 0)
    best_ms = run(best)
    for axis, values in ((0, FWD_ROWS), (3, ADJ_XBLOCKS), (1, ADJ_ROWS), (2, ADJ_CHUNKS)):
        for v in values:
            t = list(best)
            t[axis] = v
            t = tuple(t)
            if t == best:
                continue
            ms = run(t)
            if ms < best_ms:
                best, best_ms = t, ms
    return best, best_ms, trials


def tuned(p: _lib.Params, cache: str | None = None) -> _lib.Params:
    """params with the cached (or freshly measured) fastest launch shape.  The three-point
    descriptor does not run the tuned kernels: its params come back unchanged."""
    if p.descriptor == _lib.DMCR_DESC_S3:
        return p
    path = _cache_path(cache)
    key = _key(p)
    with _lock:
        table = {}
        if os.path.exists(path):
            try:
                table = json.load(open(path))
            except (OSError, ValueError):
                table = {}
        if key not in table:
            best, ms, _ = search(p)
            table[key] = {"tune": list(best), "ms": ms}
            os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
            tmp = path + ".tmp.%d" % os.getpid()
            with open(tmp, "w") as f:
                json.dump(table, f, indent=1, sort_keys=True)
            os.replace(tmp, path)
        return dataclasses.replace(p, tune=tuple(table[key]["tune"]))
