"""Domain decomposition of ONE reconstruction over several ranks (slabs with halos).

The paper runs one field on one worker (App. B).  A field too large for one device can be
split into slabs along its slowest axis (rows of a 2-D field, planes of a 3-D one); the
method then needs exactly one exchange step and one reduction per iteration, because the
field is fixed within an iteration:

  * halo exchange: every rank receives the P_0 rows before and after its slab from its two
    neighbours (the window reaches P_0 rows along the split axis, Sec. 3.3);
  * coarse levels (Sec. 3.3: level l pools 2^d children) are REPLICATED: every rank pools
    its own slab (slab boundaries are multiples of 2^(levels-1) rows, so pooling never
    crosses them) and one sum-allreduce of the zero-padded coarse slabs gives every rank
    every coarse level, bit for bit (each entry is one value plus zeros);
  * forward: every rank sums f(a_x(r))^2 over its own positions x of every level (the
    coarse positions are split along the same rows), and ONE sum-allreduce of the
    sum_l K_half partial sums, together with the box-penalty sum, gives every rank the full
    descriptor D = [w_l S_bar_l] (Eq. mg) and E_bc;
  * loss and the adjoint coefficients G_l = dL/dS_bar_l are then identical on every rank
    (Eq. L_func_dMCR); the gather-form adjoint of an own position needs only positions
    within the window, i.e. the slab and its halo (or the replicated coarse level), so it
    is local; the pooling transposes map every level's own rows onto the own finest rows;
  * Adam (Eq. M-update, App. B) is local.

The rank-local pair arithmetic comes from a backend (``SlabBackend``): sums and gradients
over the own rows of a halo-extended slab, periodic along the other axes.  Communication
uses torch.distributed (gloo on CPU ranks, where this is tested; the process group is the
caller's).  All host arithmetic here is FP64.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Protocol

import numpy as np
import torch
import torch.distributed as dist


class SlabBackend(Protocol):
    """Pair arithmetic over the own rows of a slab.

    ``ext`` holds the slab's rows [lo - P_0, hi + P_0) along axis 0 (the halo included; not
    periodic along axis 0) and the whole extent of the other axes (periodic there); own
    rows are ext rows [P_0, P_0 + rows).  ``shifts`` is the (K, ndim) half window.
    """

    def level_sums(self, ext: np.ndarray, p0: int, rows: int, shifts: np.ndarray) -> np.ndarray:
        """sum over own positions x of f(a_x(r))^2 for every shift r (not normalised)."""

    def level_vjp(self, ext: np.ndarray, p0: int, rows: int, shifts: np.ndarray, G: np.ndarray) -> np.ndarray:
        """g_y = sum_r G(r) [h(a_y(r)) + h(a_{y-r}(r))] for r != 0 and 2 G(0) h(M_y) at r = 0,
        h = f f', at the own positions y (shape: (rows,) + other axes)."""


def half_window(ndim: int, P) -> np.ndarray:
    """The canonical half window of the library (include/dmcr.h): 2-D (0, 0..P1), then
    (1..P0, -P1..P1); 3-D (0, 0, 0..P2), (0, 1..P1, -P2..P2), (1..P0, -P1..P1, -P2..P2)."""
    P = [int(p) for p in P]
    out = []
    if ndim == 2:
        out += [(0, q) for q in range(P[1] + 1)]
        out += [(p, q) for p in range(1, P[0] + 1) for q in range(-P[1], P[1] + 1)]
    else:
        out += [(0, 0, s) for s in range(P[2] + 1)]
        out += [(0, q, s) for q in range(1, P[1] + 1) for s in range(-P[2], P[2] + 1)]
        out += [(p, q, s) for p in range(1, P[0] + 1) for q in range(-P[1], P[1] + 1) for s in range(-P[2], P[2] + 1)]
    return np.array(out, dtype=np.int64).reshape(-1, ndim)


def _pool(M: np.ndarray) -> np.ndarray:
    """One coarsening: the mean of every 2^d block of children (Sec. 3.3)."""
    shape = []
    for s in M.shape:
        shape += [s // 2, 2]
    return M.reshape(shape).mean(axis=tuple(range(1, 2 * M.ndim, 2)))


def _expand(g: np.ndarray, l: int) -> np.ndarray:
    """Transpose of l poolings: every finest descendant receives g / 2^(d l)."""
    for ax in range(g.ndim):
        g = np.repeat(g, 1 << l, axis=ax)
    return g / float(2 ** (g.ndim * l))


@dataclasses.dataclass(frozen=True)
class SlabPlan:
    """Rows [lo, hi) of the finest level owned by ``rank`` of ``world``: contiguous, at
    multiples of 2^(levels-1), as even as that allows.  Raises when a rank would own no
    rows or fewer than P_0 (the halo then would have to come from beyond a neighbour)."""
    shape: tuple
    window: tuple
    levels: int
    rank: int
    world: int

    def __post_init__(self):
        unit = 1 << (self.levels - 1)
        n0 = int(self.shape[0])
        if n0 % unit:
            raise ValueError("axis 0 (%d) is not divisible by 2^(levels-1) = %d" % (n0, unit))
        for l in range(self.levels):
            for a, (n, p) in enumerate(zip(self.shape, self.window)):
                if 2 * int(p) > (int(n) >> l):
                    raise ValueError("window %d exceeds half the level-%d size on axis %d" % (p, l + 1, a))
        for r in range(self.world):
            lo, hi = self.rows_of(r)
            if hi - lo < max(1, int(self.window[0])):
                raise ValueError("rank %d would own %d rows: every slab needs at least max(1, P_0 = %d) rows; "
                                 "use fewer ranks" % (r, hi - lo, self.window[0]))

    def rows_of(self, r: int, level: int = 0):
        unit = 1 << (self.levels - 1)
        units = int(self.shape[0]) // unit
        lo = (r * units // self.world) * unit
        hi = ((r + 1) * units // self.world) * unit
        return lo >> level, hi >> level

    @property
    def rows(self):
        return self.rows_of(self.rank)


class SlabReconstruction:
    """One rank's part of a decomposed reconstruction: its slab of the field, its Adam
    moments, and the per-iteration exchange, reduction, loss, adjoint and Adam step.

    ``field`` is this rank's slab (rows ``plan.rows`` of the finest field).  Loss options
    follow the library (include/dmcr.h): mode "norm" (the paper's L = E (1 + lambda0 E_bc))
    or "squared"; lambda0 defaults to the finest position count N; the level weights are
    w_l = 2^((d/2)(l-1)).
    """

    def __init__(self, plan: SlabPlan, backend: SlabBackend, field: np.ndarray, target_desc: np.ndarray,
                 mode: str = "norm", lambda0: float | None = None, bc: bool = True, group=None):
        self.plan = plan
        self.backend = backend
        self.group = group
        self.ndim = len(plan.shape)
        lo, hi = plan.rows
        want = (hi - lo,) + tuple(int(s) for s in plan.shape[1:])
        self.M = np.array(field, dtype=np.float64).reshape(want)
        self.target = np.asarray(target_desc, dtype=np.float64)
        self.H = half_window(self.ndim, plan.window)
        self.K = self.H.shape[0]
        if self.target.size != plan.levels * self.K:
            raise ValueError("target descriptor: %d entries, expected %d" % (self.target.size, plan.levels * self.K))
        self.N = int(np.prod(plan.shape))
        self.mode = mode
        self.lam0 = (float(self.N) if lambda0 is None else float(lambda0)) if bc else 0.0
        self.w = np.array([2.0 ** (self.ndim / 2.0 * l) for l in range(plan.levels)])
        self.m = np.zeros_like(self.M)
        self.v = np.zeros_like(self.M)
        self.step = 0

    # ------------------------------------------------------------------ communication

    def _neighbours(self):
        W, r = self.plan.world, self.plan.rank
        return (r - 1) % W, (r + 1) % W

    def halo(self) -> np.ndarray:
        """The own slab with P_0 rows of each neighbour before and after it (the one
        exchange step of an iteration: point-to-point with the two neighbours)."""
        P0 = int(self.plan.window[0])
        if P0 == 0:
            return self.M
        if self.plan.world == 1:
            return np.concatenate([self.M[-P0:], self.M, self.M[:P0]], axis=0)
        prev, nxt = self._neighbours()
        head = torch.from_numpy(np.ascontiguousarray(self.M[:P0]))
        tail = torch.from_numpy(np.ascontiguousarray(self.M[-P0:]))
        before = torch.empty_like(tail)
        after = torch.empty_like(head)
        # tag 0: a slab's first rows (the previous rank's "after" halo); tag 1: its last rows
        reqs = [dist.isend(head, dst=prev, tag=0, group=self.group), dist.isend(tail, dst=nxt, tag=1, group=self.group),
                dist.irecv(before, src=prev, tag=1, group=self.group),
                dist.irecv(after, src=nxt, tag=0, group=self.group)]
        for q in reqs:
            q.wait()
        return np.concatenate([before.numpy(), self.M, after.numpy()], axis=0)

    def _allreduce(self, x: np.ndarray) -> np.ndarray:
        if self.plan.world == 1:
            return x
        t = torch.from_numpy(np.ascontiguousarray(x))
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=self.group)
        return t.numpy()

    def coarse_levels(self) -> list:
        """Every coarse level, replicated: own pooled slabs, one sum-allreduce of all of
        them zero-padded to the full level sizes."""
        plan = self.plan
        own = [self.M]
        for l in range(1, plan.levels):
            own.append(_pool(own[-1]))
        full_shapes = [tuple(int(s) >> l for s in plan.shape) for l in range(1, plan.levels)]
        if not full_shapes:
            return []
        buf = np.zeros(sum(int(np.prod(s)) for s in full_shapes))
        off = 0
        for l, sh in enumerate(full_shapes, start=1):
            lo, hi = plan.rows_of(plan.rank, l)
            blk = np.zeros(sh)
            blk[lo:hi] = own[l]
            buf[off:off + blk.size] = blk.ravel()
            off += blk.size
        buf = self._allreduce(buf)
        out, off = [], 0
        for sh in full_shapes:
            n = int(np.prod(sh))
            out.append(buf[off:off + n].reshape(sh))
            off += n
        return out

    # ------------------------------------------------------------------ one evaluation

    def _levels(self):
        """(ext, p0, rows) of every level: level 1 is the exchanged halo slab; coarse levels
        are the replicated fields extended periodically by P_0 rows, own rows at their
        slab's position."""
        P0 = int(self.plan.window[0])
        out = [(self.halo(), P0, self.M.shape[0])]
        for l, full in enumerate(self.coarse_levels(), start=1):
            lo, hi = self.plan.rows_of(self.plan.rank, l)
            ext = np.concatenate([full[full.shape[0] - P0:], full, full[:P0]], axis=0) if P0 else full
            out.append((ext, P0 + lo, hi - lo))
        return out

    def loss_grad(self):
        """Loss scalars (dict, as the library's loss_out: E, E2, Ebc, lambda, L, rel_err, plus
        the descriptor D) and the gradient of the own slab."""
        plan = self.plan
        levels = self._levels()
        sums = [self.backend.level_sums(ext, p0, rows, self.H) for ext, p0, rows in levels]
        ex = np.where(self.M > 1.0, self.M - 1.0, 0.0) + np.where(self.M < 0.0, -self.M, 0.0)
        vec = self._allreduce(np.concatenate(sums + [np.array([float(np.sum(ex * ex))])]))
        Nl = [self.N >> (self.ndim * l) for l in range(plan.levels)]
        D = np.concatenate([self.w[l] * vec[l * self.K:(l + 1) * self.K] / Nl[l] for l in range(plan.levels)])
        rho = D - self.target
        E2 = float(np.dot(rho, rho))
        E = math.sqrt(E2)
        Ebc = float(vec[-1]) / (self.N * self.N)
        phi = E if self.mode == "norm" else E2
        lam = self.lam0 * phi
        ref = math.sqrt(float(np.dot(self.target, self.target)))
        out = {"E": E, "E2": E2, "Ebc": Ebc, "lambda": lam, "L": phi + lam * Ebc,
               "rel_err": E / ref if ref > 0 else math.inf, "D": D}
        # dL/dD, then G_l = dL/dS_bar_l per level
        if self.mode == "norm":
            gD = (rho / E if E > 0 else np.zeros_like(rho)) * (1.0 + self.lam0 * Ebc)
        else:
            gD = 2.0 * rho * (1.0 + self.lam0 * Ebc)
        g = np.zeros_like(self.M)
        for l, (ext, p0, rows) in enumerate(levels):
            G = self.w[l] * gD[l * self.K:(l + 1) * self.K] / Nl[l]
            gl = self.backend.level_vjp(ext, p0, rows, self.H, G)
            g += _expand(gl, l) if l else gl
        dex = np.where(self.M > 1.0, 1.0, 0.0) - np.where(self.M < 0.0, 1.0, 0.0)
        g += self.lam0 * phi * 2.0 * ex * dex / (self.N * self.N)
        return out, g

    def adam_step(self, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-7):
        """One iteration: loss and gradient at the current field, then a local Adam step in
        the Keras form (the library's).  Returns the loss dict of the evaluated field."""
        out, g = self.loss_grad()
        self.step += 1
        t = self.step
        self.m = beta1 * self.m + (1.0 - beta1) * g
        self.v = beta2 * self.v + (1.0 - beta2) * g * g
        lr_t = lr * math.sqrt(1.0 - beta2 ** t) / (1.0 - beta1 ** t)
        self.M = self.M - lr_t * self.m / (np.sqrt(self.v) + eps)
        return out
