"""Continuous-batching reconstruction server.

Jobs (target image + problem statement + optimiser options) arrive at any time.  The
server keeps every admitted job resident on the device -- its field, Adam moments and
step count, its target descriptor -- and advances them in ticks: one tick of a class is
one ``dmcr_reconstruct_batched`` call (one fused launch per phase over every active job
and level of the class, replayed as a captured CUDA graph) of at most ``tick_iters``
iterations.  Jobs are grouped in cost classes by their work per iteration; in threaded
mode every class ticks on its own host thread and CUDA stream, so cheap, latency-bound
jobs are not held to the iteration time of expensive ones and the classes' kernels
overlap on the device.  A class may cap how many of its jobs are active at once: jobs
large enough to fill the device each are then served one after another in arrival order,
which finishes each sooner than sharing the device among them.  Between ticks, finished
jobs retire (result copied to the host) and waiting jobs are admitted while a slot and the
HBM budget allow.  Because the
per-instance arithmetic of a batched call equals that of a single call bitwise, and a tick
boundary only re-evaluates the loss of the current field, a job's result is the same
alone and in any mix (tested).

``run_trace`` replays an arrival trace against the server (``serve``) or against plain
one-job-at-a-time reconstructions (``plain``) and reports per-job time from arrival to
completion (p50/p99) and reconstructions per second.
"""
from __future__ import annotations

import collections
import dataclasses
import threading
import time

import numpy as np
import torch

from . import _lib


@dataclasses.dataclass
class Job:
    job_id: int
    params: _lib.Params
    target: np.ndarray                 # host target image (the target descriptor is computed on admission)
    opts: _lib.ReconOpts
    arrival: float = 0.0               # seconds on the trace clock
    # filled in by the server
    field: torch.Tensor | None = None
    m: torch.Tensor | None = None
    v: torch.Tensor | None = None
    desc: torch.Tensor | None = None
    step: int = 0
    iters_done: int = 0
    admitted: float | None = None
    finished: float | None = None
    result: np.ndarray | None = None
    report: dict | None = None

    def bytes_estimate(self) -> int:
        """Device bytes held while resident: field, moments, target, descriptors and the
        job's share of the batch workspace."""
        n = int(np.prod(field_shape(self.params)))
        k = _lib.dmcr_descriptor_length(self.params)
        return 4 * (4 * n + 2 * k) + _lib.dmcr_workspace_size(self.params)


def field_shape(params: _lib.Params) -> tuple:
    """Shape of a job's field: the phase stack (phases, *shape) when there are several."""
    return tuple(params.shape) if params.phases == 1 else (params.phases,) + tuple(params.shape)


def iteration_units(params: _lib.Params) -> int:
    """Voxel-shift pairs of one iteration: phases^2 sum_l N_l prod_a (2 P_a + 1)."""
    kfull = int(np.prod([2 * w + 1 for w in params.window]))
    return params.phases ** 2 * sum(int(np.prod([s >> l for s in params.shape])) * kfull
                                    for l in range(params.levels))


class _Class:
    def __init__(self, cap, slots):
        self.cap = cap
        self.slots = slots        # most jobs of this class active at once
        self.pending: collections.deque[Job] = collections.deque()
        self.active: list[Job] = []
        self.stream = None
        self.tick_s: list[float] = []
        self.tick_jobs: list[int] = []


class Server:
    def __init__(self, device="cuda", hbm_budget_bytes: int = 150 << 30, max_slots: int = 64, tick_iters: int = 50,
                 class_caps=(float("inf"),), class_slots=None, priorities: str = "cheap_first",
                 exclusive_top: bool = False, clock=time.perf_counter):
        self.dev = torch.device(device)
        self.budget = int(hbm_budget_bytes)
        self.max_slots = int(max_slots)
        self.tick_iters = int(tick_iters)
        self.clock = clock
        self.t0 = None
        # class_slots[i]: most active jobs of the class with cap class_caps[i] (None: only the
        # server-wide max_slots).  Jobs of one class that could each fill the device run better
        # one after another in arrival order than side by side: sharing the device delays all
        # of them, while serial service finishes the first at full speed.
        slots = [None] * len(class_caps) if class_slots is None else list(class_slots)
        if len(slots) != len(class_caps):
            raise ValueError("class_slots needs one entry per class cap")
        self.classes = [_Class(c, n if n is not None else self.max_slots)
                        for c, n in sorted(zip(class_caps, slots), key=lambda cs: cs[0])]
        if priorities not in ("cheap_first", "equal", "heavy_first"):
            raise ValueError("priorities: 'cheap_first', 'equal' or 'heavy_first'")
        self.priorities = priorities
        # exclusive_top: while a job of the most expensive class is active, the other classes
        # pause at their next tick boundary, so that job has the device to itself
        self.exclusive_top = bool(exclusive_top)
        self.done: list[Job] = []
        self.in_use = 0
        self.ticks = 0
        self._lock = threading.Lock()
        self._wake = threading.Condition(self._lock)
        self._threads = []
        self._stop = False
        self.error = None

    @property
    def active(self):
        return [j for c in self.classes for j in c.active]

    @property
    def pending(self):
        return [j for c in self.classes for j in c.pending]

    def now(self) -> float:
        return self.clock() - self.t0

    def _class_of(self, job):
        u = iteration_units(job.params)
        for c in self.classes:
            if u <= c.cap:
                return c
        return self.classes[-1]

    def submit(self, job: Job):
        if job.opts.check_every < 1 or self.tick_iters % job.opts.check_every:
            raise ValueError("tick_iters must be a multiple of every job's check_every")
        with self._wake:
            self._class_of(job).pending.append(job)
            self._wake.notify_all()

    def _admit(self, cls):
        new = []
        with self._lock:
            while (cls.pending and sum(len(c.active) for c in self.classes) + len(new) < self.max_slots
                   and len(cls.active) + len(new) < cls.slots):
                job = cls.pending[0]
                need = job.bytes_estimate()
                if self.in_use + need > self.budget:
                    if not any(c.active for c in self.classes) and not new:
                        raise MemoryError("job %d needs %d bytes, more than the HBM budget" % (job.job_id, need))
                    break
                cls.pending.popleft()
                self.in_use += need
                new.append(job)
        if not new:
            return
        for job in new:
            p = job.params
            job._tgt = torch.tensor(np.asarray(job.target, dtype=np.float32), device=self.dev)
            job.desc = torch.empty(_lib.dmcr_descriptor_length(p), dtype=torch.float32, device=self.dev)
            job.field = torch.empty(field_shape(p), dtype=torch.float32, device=self.dev)
            _lib.dmcr_init_uniform(job.field, job.opts.seed)
            job.m = torch.zeros_like(job.field)
            job.v = torch.zeros_like(job.field)
            job.admitted = self.now()
        _lib.dmcr_descriptor_batched([j.params for j in new], [j._tgt for j in new], [j.desc for j in new])
        for j in new:
            del j._tgt
        with self._lock:
            cls.active.extend(new)

    def _paused(self, cls) -> bool:
        top = self.classes[-1]
        return self.exclusive_top and cls is not top and bool(top.active or top.pending)

    def _tick_class(self, cls) -> int:
        if self._paused(cls):
            return 0
        self._admit(cls)
        jobs = list(cls.active)
        if not jobs:
            return 0
        opts = []
        for j in jobs:
            left = j.opts.max_iters - j.iters_done
            opts.append(dataclasses.replace(j.opts, max_iters=min(self.tick_iters, left), init=_lib.DMCR_INIT_CALLER,
                                            report_rounded=False))
        t_tick = time.perf_counter()
        reps, steps = _lib.dmcr_reconstruct_batched([j.params for j in jobs], opts, [j.desc for j in jobs],
                                                    [j.field for j in jobs], [j.m for j in jobs],
                                                    [j.v for j in jobs], [j.step for j in jobs])
        cls.tick_s.append(time.perf_counter() - t_tick)
        cls.tick_jobs.append(len(jobs))
        keep, finished = [], []
        for j, r, s in zip(jobs, reps, steps):
            j.iters_done += s - j.step
            j.step = s
            j.report = r
            if r["converged"] or j.iters_done >= j.opts.max_iters or r["status"] != 0:
                j.finished = self.now()
                j.result = j.field.cpu().numpy()
                j.field = j.m = j.v = j.desc = None
                finished.append(j)
            else:
                keep.append(j)
        with self._wake:
            cls.active = keep
            for j in finished:
                self.in_use -= j.bytes_estimate()
                self.done.append(j)
            self.ticks += 1
            self._wake.notify_all()
        return len(finished)

    def tick(self) -> int:
        """Synchronous mode: advance every class once, in order.  Returns jobs retired."""
        if self.t0 is None:
            self.t0 = self.clock()
        return sum(self._tick_class(c) for c in self.classes)

    def idle(self) -> bool:
        with self._lock:
            return not any(c.pending or c.active for c in self.classes)

    # ---- threaded mode: one worker thread and CUDA stream per class
    def start(self):
        if self.t0 is None:
            self.t0 = self.clock()
        self._stop = False
        # "cheap_first": cheaper classes get higher stream priority, so their short kernels are
        # scheduled ahead of the long-running blocks of expensive classes as SMs free up;
        # "heavy_first": the reverse -- the longest jobs run at nearly full speed and the cheap
        # classes fill the SMs they leave; "equal": every class stream has the default priority
        lo, hi = torch.cuda.Stream.priority_range()      # least, greatest (numerically lower = higher)
        last = len(self.classes) - 1
        for i, c in enumerate(self.classes):
            if self.priorities == "cheap_first":
                prio = min(lo, hi + i)
            elif self.priorities == "heavy_first":
                prio = min(lo, hi + (last - i))
            else:
                prio = 0
            c.stream = torch.cuda.Stream(device=self.dev, priority=prio)
            t = threading.Thread(target=self._worker, args=(c,), daemon=True)
            t.start()
            self._threads.append(t)

    def _worker(self, cls):
        try:
            with torch.cuda.stream(cls.stream):
                while True:
                    with self._wake:
                        while not self._stop and not cls.pending and not cls.active:
                            self._wake.wait(0.05)
                        if self._stop and not cls.pending and not cls.active:
                            return
                    self._tick_class(cls)
                    if not cls.active or self._paused(cls):   # waiting for memory, slots or the top class
                        with self._wake:
                            self._wake.wait(0.01)
        except BaseException as e:     # surfaced by stop()
            self.error = e
            with self._wake:
                self._wake.notify_all()

    def wait_idle(self, timeout: float | None = None):
        end = None if timeout is None else time.perf_counter() + timeout
        with self._wake:
            while any(c.pending or c.active for c in self.classes) and self.error is None:
                left = None if end is None else end - time.perf_counter()
                if left is not None and left <= 0:
                    raise TimeoutError("server did not drain")
                self._wake.wait(0.05 if left is None else min(0.05, left))
        if self.error is not None:
            raise self.error

    def stop(self):
        with self._wake:
            self._stop = True
            self._wake.notify_all()
        for t in self._threads:
            t.join()
        self._threads = []
        if self.error is not None:
            raise self.error


def reconstruct_alone(job: Job, device="cuda") -> Job:
    """The plain form: one job, one dmcr_reconstruct call."""
    dev = torch.device(device)
    p = job.params
    tgt = torch.tensor(np.asarray(job.target, dtype=np.float32), device=dev)
    desc = _lib.descriptor(tgt, p)
    field = torch.empty(field_shape(p), dtype=torch.float32, device=dev)
    _lib.dmcr_init_uniform(field, job.opts.seed)
    m = torch.zeros_like(field)
    v = torch.zeros_like(field)
    rep, step = _lib.dmcr_reconstruct(p, dataclasses.replace(job.opts, init=_lib.DMCR_INIT_CALLER), desc, field, m, v)
    job.report = rep
    job.step = job.iters_done = step
    job.result = field.cpu().numpy()
    return job


def poisson_trace(n_jobs: int, rate_per_s: float, seed: int, make_job) -> list[Job]:
    """n_jobs arrivals of a Poisson process of the given rate; make_job(i, rng) builds job i."""
    rng = np.random.default_rng(seed)
    t = 0.0
    jobs = []
    for i in range(n_jobs):
        t += float(rng.exponential(1.0 / rate_per_s))
        job = make_job(i, rng)
        job.arrival = t
        jobs.append(job)
    return jobs


def run_trace(jobs: list[Job], mode: str = "serve", **server_kw) -> dict:
    """Replays the arrivals in real time (a job is submitted once the trace clock passes its
    arrival) and returns latency percentiles and throughput."""
    jobs = sorted(jobs, key=lambda j: j.arrival)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    if mode == "serve":
        srv = Server(**server_kw)
        srv.t0 = t0
        srv.start()
        try:
            for j in jobs:
                now = time.perf_counter() - t0
                if j.arrival > now:
                    time.sleep(j.arrival - now)
                srv.submit(j)
            srv.wait_idle()
        finally:
            srv.stop()
        torch.cuda.synchronize()
        ticks = [{"cap": c.cap, "ticks": len(c.tick_s), "mean_tick_s": float(np.mean(c.tick_s)) if c.tick_s else 0.0,
                  "mean_jobs": float(np.mean(c.tick_jobs)) if c.tick_jobs else 0.0} for c in srv.classes]
    else:
        for j in jobs:
            now = time.perf_counter() - t0
            if j.arrival > now:
                time.sleep(j.arrival - now)
            j.admitted = time.perf_counter() - t0
            reconstruct_alone(j)
            j.finished = time.perf_counter() - t0
    if mode != "serve":
        ticks = None
    wall = time.perf_counter() - t0
    lat = np.array([j.finished - j.arrival for j in jobs])
    by = collections.defaultdict(list)
    for j in jobs:
        by["%dD %s" % (len(j.params.shape), "x".join(map(str, j.params.shape)))].append(
            (j.finished - j.arrival, j.iters_done))
    breakdown = {k: {"jobs": len(v), "p50_s": float(np.percentile([a for a, _ in v], 50)),
                     "max_s": float(max(a for a, _ in v)), "mean_iters": float(np.mean([b for _, b in v]))}
                 for k, v in sorted(by.items())}
    conv = sum(bool(j.report and j.report["converged"]) for j in jobs)
    return {"mode": mode, "jobs": len(jobs), "converged": conv, "wall_s": wall,
            "reconstructions_per_s": len(jobs) / wall, "p50_s": float(np.percentile(lat, 50)),
            "p99_s": float(np.percentile(lat, 99)), "mean_s": float(lat.mean()),
            "final_rel_err_max": float(max(j.report["rel_err"] for j in jobs)), "by_shape": breakdown, "classes": ticks}
