"""FP64 CPU oracle for differentiable microstructure reconstruction (arXiv 2103.09686).

TEST INFRASTRUCTURE ONLY: the plain, slow, obviously correct restatement of what the
method computes.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline /
reference leg of ``bench.py`` may import it; the library never does, and this module
imports nothing from the library.  Heavy loops live in ``dmcr_oracle.c`` (plain C,
double precision); everything else is numpy float64 written in the paper's order.

What each function follows (sections and equations of the paper):

* ``soft_constants``, ``threshold`` -- Sec. 3.2.4, Eq. softthreshold and its three
  defining conditions f(0)=0, f(1)=1, f''(0.75)=0, alpha = 10.
* ``sbar`` -- Sec. 3.2.2/3.2.3: convolve (Eq. convdef) -> threshold -> reduce
  (Eq. s3 with p=r, q=s; the linear reduction of Sec. 3.2.2 on request).
* ``sbar_masks`` -- the same with the masks m_pqrs built explicitly (Sec. 3.2.3).
* ``half_window`` / ``full_window`` -- the shift sets |r_a| <= P_a of Sec. 3.3, halved by
  the point symmetry of App. B.
* ``restrict`` / ``prolongate_adjoint`` / ``descriptor`` -- Sec. 3.3, Eq. mg: each level
  summarises 2^d children (read: arithmetic mean), weights w_l = 2^{(d/2)(l-1)}
  (= 2^{l-1} in 2-D as in the paper's footnote), all levels active at once.
* ``loss`` -- Sec. 3.1, Eq. L_func_dMCR: E = ||D - D_des||_2, E_bc with H(0)=0,
  lambda = lambda0 * E.
* ``loss_grad`` / ``descriptor_vjp`` -- the exact gradient by the chain rule through all
  levels simultaneously (Sec. 3.1, Sec. 3.3); ``vjp_at`` the same gradient at sampled
  finest positions (gather form, for full-size problems).
* ``round_field`` -- the rounding used to evaluate a reconstruction (Sec. 4.1): values
  >= 1/2 become phase 1 (the tie goes to phase 1), the rest phase 0.
* ``adam_step`` / ``reconstruct`` -- Eq. M-update with Adam at the TensorFlow defaults
  (App. B): lr 1e-3, beta1 0.9, beta2 0.999; epsilon 1e-7 (Keras form; the paper does
  not print epsilon).
* ``ensemble`` / ``s3bar`` / ``s3_descriptor`` / ``s3_loss_grad`` -- the ensemble
  e_x(r) = f(a_x(r)) of Sec. 3.2.2-3.2.4 as an explicit N x K matrix and its quadratic
  reduction, Eq. s3: S_bar3(r_a, r_b) = (1/N) sum_x e_x(r_a) e_x(r_b), the Gram matrix of
  the ensemble (Sec. 3.4's footnote), on the half window of every level; the exact gradient
  of a loss on it by the chain rule.
* ``s2tilde_map`` / ``descriptor_tilde`` / ``tilde_loss_grad`` -- the corrected two-point
  descriptor of App. A, Eq. s2rfroms2rbar: S_tilde(0) = S_bar(0) and
  S_tilde(r) = (S_bar(r) - 2 f(1/2)^2 S_bar(0)) / (1 - 2 f(1/2)^2), a linear map of every
  level's block, and the gradient of a loss on it (the map's transpose, then the S_bar
  gradient).
* ``s2_count`` / ``s3_count`` / ``s3_from_s3bar`` -- exact two- and three-point
  probabilities of a binary field by counting (Sec. 3.2.1) and App. A's mapping from
  S_bar3 back to S3 (Eq. s3rfroms3rbar).
* ``cross_sbar`` / ``multiphase_descriptor`` / ``multiphase_loss_grad`` -- the two-point
  chain of Sec. 3.2.2-3.2.4 with the pair's tail and tip in two different phase fields:
  the cross-correlations S2^{a->b} of the multi-phase outlook (Sec. 5), every ordered
  phase pair on the half window of every level, and the exact gradient with respect to
  every phase field.  ``cross_count`` counts S2^{a->b} of binary indicators (Sec. 3.2.1).
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dmcr_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None
_lock = threading.Lock()

TH_SOFT, TH_IDENTITY, TH_HARD = 0, 1, 2
_KIND = {"soft": TH_SOFT, "identity": TH_IDENTITY, "hard": TH_HARD}


def build(force: bool = False) -> str:
    """Compile the C part of the oracle (gcc, -O2, OpenMP) next to its source."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + ".tmp.%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c99",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            P = ctypes.POINTER
            d, i64, i32 = ctypes.c_double, ctypes.c_int64, ctypes.c_int
            lib.oracle_soft_constants.argtypes = [d, P(d), P(d), P(d)]
            lib.oracle_threshold.argtypes = [i32, d, P(d), i64, P(d), P(d)]
            lib.oracle_threshold_custom.argtypes = [d, d, d, d, P(d), i64, P(d)]
            lib.oracle_sbar.argtypes = [P(d), P(i64), P(i32), i64, i32, d, i32, P(d)]
            lib.oracle_sbar_masks.argtypes = [P(d), P(i64), P(i32), P(i32), i64, i32, d, P(d)]
            lib.oracle_vjp_level.argtypes = [P(d), P(i64), P(i32), i64, P(d), i32, d, P(i64), i64, P(d)]
            _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _i64p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def _i32p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def set_threads(n: int | None) -> None:
    """Number of OpenMP threads the C loops use (None: leave the runtime default)."""
    if n is not None:
        os.environ["OMP_NUM_THREADS"] = str(int(n))
        try:
            ctypes.CDLL("libgomp.so.1").omp_set_num_threads(int(n))
        except OSError:
            pass


# ----------------------------------------------------------------------------- threshold

def soft_constants(alpha: float = 10.0):
    """(c1, c2, c3) of Eq. softthreshold from f(0)=0, f(1)=1, f''(0.75)=0."""
    lib = _load()
    c1, c2, c3 = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    lib.oracle_soft_constants(alpha, ctypes.byref(c1), ctypes.byref(c2), ctypes.byref(c3))
    return c1.value, c2.value, c3.value


def threshold(x, kind: str = "soft", alpha: float = 10.0):
    """f(x) and f'(x) elementwise."""
    lib = _load()
    x = np.ascontiguousarray(x, dtype=np.float64).ravel()
    f = np.empty_like(x)
    df = np.empty_like(x)
    lib.oracle_threshold(_KIND[kind], alpha, _dp(x), x.size, _dp(f), _dp(df))
    return f, df


def threshold_custom(x, alpha, c1, c2, c3):
    """The logistic of Eq. softthreshold with explicit constants."""
    lib = _load()
    x = np.ascontiguousarray(x, dtype=np.float64).ravel()
    f = np.empty_like(x)
    lib.oracle_threshold_custom(alpha, c1, c2, c3, _dp(x), x.size, _dp(f))
    return f


# ----------------------------------------------------------------------------- windows

def half_window(ndim: int, P) -> np.ndarray:
    """Unique shifts under r <-> -r, r = 0 once, as (K_half, ndim) int array.

    Order: 2-D  (0, 0..P1), then (1..P0, -P1..P1) row-major;
           3-D  (0, 0, 0..P2), (0, 1..P1, -P2..P2), (1..P0, -P1..P1, -P2..P2).
    """
    P = [int(p) for p in P][:ndim]
    out = []
    if ndim == 2:
        for q in range(0, P[1] + 1):
            out.append((0, q))
        for p in range(1, P[0] + 1):
            for q in range(-P[1], P[1] + 1):
                out.append((p, q))
    elif ndim == 3:
        for s in range(0, P[2] + 1):
            out.append((0, 0, s))
        for q in range(1, P[1] + 1):
            for s in range(-P[2], P[2] + 1):
                out.append((0, q, s))
        for p in range(1, P[0] + 1):
            for q in range(-P[1], P[1] + 1):
                for s in range(-P[2], P[2] + 1):
                    out.append((p, q, s))
    else:
        raise ValueError("ndim must be 2 or 3")
    return np.array(out, dtype=np.int64).reshape(-1, ndim)


def full_window(ndim: int, P) -> np.ndarray:
    """All shifts |r_a| <= P_a, row-major, as (K_full, ndim)."""
    P = [int(p) for p in P][:ndim]
    axes = [np.arange(-p, p + 1) for p in P]
    grid = np.meshgrid(*axes, indexing="ij")
    return np.stack([g.ravel() for g in grid], axis=1).astype(np.int64)


def _as3(M: np.ndarray):
    M = np.ascontiguousarray(M, dtype=np.float64)
    if M.ndim == 2:
        n = np.array([1, M.shape[0], M.shape[1]], dtype=np.int64)
    elif M.ndim == 3:
        n = np.array(M.shape, dtype=np.int64)
    else:
        raise ValueError("field must be 2-D or 3-D")
    return M, n


def _shifts3(shifts: np.ndarray, ndim: int) -> np.ndarray:
    shifts = np.asarray(shifts, dtype=np.int64).reshape(-1, ndim)
    s3 = np.zeros((shifts.shape[0], 3), dtype=np.int32)
    s3[:, 3 - ndim:] = shifts
    return np.ascontiguousarray(s3)


# ----------------------------------------------------------------------------- descriptor

def sbar(M, shifts, kind: str = "soft", alpha: float = 10.0, linear: bool = False) -> np.ndarray:
    """One level: S_bar(r) = mean_x f(a_x(r))^2 (or mean_x f(a_x(r)) if linear)."""
    lib = _load()
    M, n = _as3(M)
    s3 = _shifts3(shifts, M.ndim)
    out = np.empty(s3.shape[0], dtype=np.float64)
    lib.oracle_sbar(_dp(M), _i64p(n), _i32p(s3), s3.shape[0], _KIND[kind], alpha, int(linear), _dp(out))
    return out


def sbar_masks(M, P, shifts, kind: str = "soft", alpha: float = 10.0) -> np.ndarray:
    """Same as ``sbar`` but through explicitly built masks (small fields only)."""
    lib = _load()
    M, n = _as3(M)
    s3 = _shifts3(shifts, M.ndim)
    P3 = np.zeros(3, dtype=np.int32)
    P3[3 - M.ndim:] = [int(p) for p in P][:M.ndim]
    out = np.empty(s3.shape[0], dtype=np.float64)
    lib.oracle_sbar_masks(_dp(M), _i64p(n), _i32p(P3), _i32p(s3), s3.shape[0], _KIND[kind], alpha, _dp(out))
    return out


def restrict(M: np.ndarray) -> np.ndarray:
    """One multigrid coarsening: each coarse cell is the mean of its 2^d children."""
    M = np.asarray(M, dtype=np.float64)
    d = M.ndim
    shape = []
    for s in M.shape:
        if s % 2:
            raise ValueError("size not divisible by 2")
        shape += [s // 2, 2]
    return M.reshape(shape).mean(axis=tuple(range(1, 2 * d, 2)))


def prolongate_adjoint(C: np.ndarray) -> np.ndarray:
    """Transpose of ``restrict``: every child receives its parent's value / 2^d."""
    C = np.asarray(C, dtype=np.float64)
    d = C.ndim
    F = C
    for ax in range(d):
        F = np.repeat(F, 2, axis=ax)
    return F / float(2 ** d)


@dataclasses.dataclass
class Params:
    """Problem statement (Sec. 3.3): window P_a per axis, number of levels, threshold."""
    ndim: int
    window: tuple
    levels: int = 1
    threshold: str = "soft"
    alpha: float = 10.0
    weight_exp: float | None = None   # w_l = 2^{weight_exp (l-1)}; None -> d/2

    def weights(self) -> np.ndarray:
        e = self.ndim / 2.0 if self.weight_exp is None else self.weight_exp
        return np.array([2.0 ** (e * l) for l in range(self.levels)])


def pyramid(M: np.ndarray, levels: int):
    out = [np.asarray(M, dtype=np.float64)]
    for _ in range(1, levels):
        out.append(restrict(out[-1]))
    return out


def descriptor(M, p: Params, levels_out: bool = False):
    """Eq. mg: D = [w_1 S_bar_1, w_2 S_bar_2, ...] on the half window of every level."""
    H = half_window(p.ndim, p.window)
    pyr = pyramid(M, p.levels)
    w = p.weights()
    blocks = [w[l] * sbar(pyr[l], H, p.threshold, p.alpha) for l in range(p.levels)]
    D = np.concatenate(blocks)
    return (D, blocks) if levels_out else D


def descriptor_shifts(M, p: Params, level: int, shifts) -> np.ndarray:
    """Sampled entries: w_l * S_bar_l(r) for an explicit shift list at one level."""
    pyr = pyramid(M, level + 1)
    return p.weights()[level] * sbar(pyr[level], shifts, p.threshold, p.alpha)


# ----------------------------------------------------------------------------- loss

def box_excess(M: np.ndarray) -> np.ndarray:
    """(M-1) H(M-1) - M H(-M) with H(0) = 0 (Sec. 3.1)."""
    M = np.asarray(M, dtype=np.float64)
    return np.where(M - 1.0 > 0, M - 1.0, 0.0) - np.where(-M > 0, M, 0.0)


def loss(M, D_des, p: Params, mode: str = "norm", lambda0: float | None = None, bc: bool = True,
         D=None) -> dict:
    """Eq. L_func_dMCR.  mode 'norm': L = E + lambda E_bc, lambda = lambda0 E (the paper);
    mode 'squared': L = E^2 + lambda0 E^2 E_bc.  lambda0 defaults to the finest pixel count.
    """
    M = np.asarray(M, dtype=np.float64)
    N = M.size
    if lambda0 is None:
        lambda0 = float(N)
    if not bc:
        lambda0 = 0.0
    if D is None:
        D = descriptor(M, p)
    rho = D - np.asarray(D_des, dtype=np.float64)
    E2 = float(np.sum(rho * rho))
    E = float(np.sqrt(E2))
    Ebc = float(np.sum((box_excess(M) / N) ** 2))
    phi = E if mode == "norm" else E2
    lam = lambda0 * phi
    L = phi + lam * Ebc
    ref = float(np.sqrt(np.sum(np.asarray(D_des, dtype=np.float64) ** 2)))
    return {"E": E, "E2": E2, "Ebc": Ebc, "lambda": lam, "L": L,
            "rel_err": E / ref if ref > 0 else float("inf"), "rho": rho, "lambda0": lambda0}


def level_vjp(M_level, p: Params, G_half, positions=None) -> np.ndarray:
    """g_y = sum_r G(r) dS_bar(r)/dM_y for one level (positions: flat indices or all)."""
    lib = _load()
    M3, n = _as3(M_level)
    s3 = _shifts3(half_window(p.ndim, p.window), M_level.ndim)
    G = np.ascontiguousarray(G_half, dtype=np.float64)
    if positions is None:
        npos = int(np.prod(n))
        out = np.empty(npos, dtype=np.float64)
        lib.oracle_vjp_level(_dp(M3), _i64p(n), _i32p(s3), s3.shape[0], _dp(G), _KIND[p.threshold],
                             p.alpha, None, npos, _dp(out))
        return out.reshape(M_level.shape)
    pos = np.ascontiguousarray(positions, dtype=np.int64)
    out = np.empty(pos.size, dtype=np.float64)
    lib.oracle_vjp_level(_dp(M3), _i64p(n), _i32p(s3), s3.shape[0], _dp(G), _KIND[p.threshold],
                         p.alpha, _i64p(pos), pos.size, _dp(out))
    return out


def descriptor_vjp(M, p: Params, grad_D) -> np.ndarray:
    """Gradient of <grad_D, D(M)> w.r.t. the finest field, back-propagated through every
    level at once (Sec. 3.3): per-level VJP, then the transpose of the pooling chain."""
    M = np.asarray(M, dtype=np.float64)
    K = half_window(p.ndim, p.window).shape[0]
    pyr = pyramid(M, p.levels)
    w = p.weights()
    g = None
    for l in reversed(range(p.levels)):
        gl = level_vjp(pyr[l], p, w[l] * np.asarray(grad_D[l * K:(l + 1) * K], dtype=np.float64))
        g = gl if g is None else gl + prolongate_adjoint(g)
    return g


def vjp_at(M, p: Params, grad_D, positions) -> np.ndarray:
    """``descriptor_vjp`` at sampled finest positions (flat indices), in gather form: the
    finest position x receives, from every level l, the level-l gradient of its ancestor
    (coordinates x >> l, the cell that pools x at level l, Sec. 3.3) times 2^{-d l}, the
    product of the l pooling transposes on the way down (each gives a child 1/2^d of its
    parent).  O(levels * K_half) pair evaluations per position, so it serves full-size
    problems where the scatter form of ``descriptor_vjp`` would be too slow."""
    M = np.asarray(M, dtype=np.float64)
    d = M.ndim
    K = half_window(p.ndim, p.window).shape[0]
    pyr = pyramid(M, p.levels)
    w = p.weights()
    coords = np.stack(np.unravel_index(np.asarray(positions, dtype=np.int64), M.shape), axis=1)
    out = np.zeros(coords.shape[0])
    for l in range(p.levels):
        n_l = np.array(pyr[l].shape, dtype=np.int64)
        anc = coords >> l
        flat = np.ravel_multi_index(tuple(anc.T), tuple(n_l))
        G = w[l] * np.asarray(grad_D[l * K:(l + 1) * K], dtype=np.float64)
        out += level_vjp(pyr[l], p, G, flat) / float(2 ** (d * l))
    return out


def loss_grad(M, D_des, p: Params, mode: str = "norm", lambda0: float | None = None, bc: bool = True):
    """Loss (as ``loss``) and dL/dM by the chain rule:
    dL/dM = phi'(E) (1 + lambda0 E_bc) dE/dM + lambda0 phi(E) dE_bc/dM."""
    M = np.asarray(M, dtype=np.float64)
    N = M.size
    out = loss(M, D_des, p, mode, lambda0, bc)
    lam0 = out["lambda0"]
    rho, E, Ebc = out["rho"], out["E"], out["Ebc"]
    if mode == "norm":
        dphi_dD = rho / E if E > 0 else np.zeros_like(rho)
        phi = E
    else:
        dphi_dD = 2.0 * rho
        phi = out["E2"]
    g = descriptor_vjp(M, p, dphi_dD * (1.0 + lam0 * Ebc))
    ex = box_excess(M)
    dex = np.where(M - 1.0 > 0, 1.0, 0.0) - np.where(-M > 0, 1.0, 0.0)
    g = g + lam0 * phi * 2.0 * (ex / N) * dex / N
    return out, g


# ----------------------------------------------------------------------------- optimiser

def adam_step(M, g, m, v, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-7):
    """One Adam step in the TensorFlow/Keras form; t is the 1-based step count."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    lr_t = lr * np.sqrt(1.0 - beta2 ** t) / (1.0 - beta1 ** t)
    M = M - lr_t * m / (np.sqrt(v) + eps)
    return M, m, v


def reconstruct(M0, D_des, p: Params, iters: int, tol_rel: float = 0.0, lr=1e-3, beta1=0.9,
                beta2=0.999, eps=1e-7, mode="norm", lambda0=None, bc=True, check_every=1):
    """Flow chart of Sec. 3: evaluate L and dL/dM, stop when rel_err < tol_rel (tested every
    ``check_every`` iterations), otherwise take one Adam step.  Returns the field and the
    per-iteration loss records."""
    M = np.array(M0, dtype=np.float64)
    m = np.zeros_like(M)
    v = np.zeros_like(M)
    hist = []
    for t in range(1, iters + 1):
        out, g = loss_grad(M, D_des, p, mode, lambda0, bc)
        hist.append({k: out[k] for k in ("E", "E2", "Ebc", "lambda", "L", "rel_err")})
        if tol_rel > 0 and (t - 1) % check_every == 0 and out["rel_err"] < tol_rel:
            break
        M, m, v = adam_step(M, g, m, v, t, lr, beta1, beta2, eps)
    return M, hist


def round_field(M) -> np.ndarray:
    """Rounding for evaluation (Sec. 4.1): values >= 0.5 become phase 1."""
    return (np.asarray(M) >= 0.5).astype(np.float64)


# ----------------------------------------------------------------------------- three-point

def ensemble(M_level, shifts, kind: str = "soft", alpha: float = 10.0):
    """The ensemble of one level as explicit (N, K) arrays: e_x(r) = f(a_x(r)) and f'(a_x(r)),
    a_x(r) = (M_x + M_{x+r}) / 2 for r != 0 and a_x(0) = M_x (the masks of Sec. 3.2.3 hold
    1/2 at tip and tail, a single 1 at r = 0), periodic in every axis; x in C order."""
    M = np.asarray(M_level, dtype=np.float64)
    shifts = np.asarray(shifts, dtype=np.int64).reshape(-1, M.ndim)
    N = M.size
    E = np.empty((N, shifts.shape[0]))
    dE = np.empty((N, shifts.shape[0]))
    for k, r in enumerate(shifts):
        if np.any(r != 0):
            tip = np.roll(M, shift=tuple(-int(c) for c in r), axis=tuple(range(M.ndim)))
            a = 0.5 * (M + tip)
        else:
            a = M
        f, df = threshold(a.ravel(), kind, alpha)
        E[:, k] = f
        dE[:, k] = df
    return E, dE


def s3bar(M_level, shifts, kind: str = "soft", alpha: float = 10.0) -> np.ndarray:
    """Eq. s3 on one level: the K x K matrix S_bar3(r_a, r_b) = (1/N) sum_x e_x(r_a) e_x(r_b)."""
    E, _ = ensemble(M_level, shifts, kind, alpha)
    return (E.T @ E) / E.shape[0]


def s3_descriptor(M, p: Params, levels_out: bool = False):
    """Multigrid form (Eq. mg) of the three-point descriptor: per level the K x K matrix on
    the half window, multiplied by w_l; flattened row-major and concatenated, finest first."""
    H = half_window(p.ndim, p.window)
    pyr = pyramid(M, p.levels)
    w = p.weights()
    blocks = [w[l] * s3bar(pyr[l], H, p.threshold, p.alpha) for l in range(p.levels)]
    D = np.concatenate([b.ravel() for b in blocks])
    return (D, blocks) if levels_out else D


def s3_level_vjp(M_level, p: Params, G) -> np.ndarray:
    """g_y = sum_{a,b} G[a, b] dS_bar3(r_a, r_b)/dM_y for one level: with
    V = f'(a) * (E (G + G^T) / N), every entry a_x(r) depends on M_x and M_{x+r} with
    weight 1/2 (weight 1 for r = 0)."""
    M = np.asarray(M_level, dtype=np.float64)
    H = half_window(p.ndim, p.window)
    E, dE = ensemble(M, H, p.threshold, p.alpha)
    G = np.asarray(G, dtype=np.float64)
    V = dE * ((E @ (G + G.T)) / E.shape[0])
    g = np.zeros(M.shape)
    axes = tuple(range(M.ndim))
    for k, r in enumerate(H):
        Vk = V[:, k].reshape(M.shape)
        if np.any(r != 0):
            g += 0.5 * Vk + 0.5 * np.roll(Vk, shift=tuple(int(c) for c in r), axis=axes)
        else:
            g += Vk
    return g


def s3_loss_grad(M, D_des, p: Params, mode: str = "norm", lambda0: float | None = None, bc: bool = True):
    """Eq. L_func_dMCR with the three-point descriptor (Frobenius norm over every level's
    K x K matrix) and its gradient, through all levels at once (Sec. 3.3)."""
    M = np.asarray(M, dtype=np.float64)
    N = M.size
    D = s3_descriptor(M, p)
    out = loss(M, D_des, p, mode, lambda0, bc, D=D)
    lam0 = out["lambda0"]
    rho, E, Ebc = out["rho"], out["E"], out["Ebc"]
    if mode == "norm":
        dphi_dD = rho / E if E > 0 else np.zeros_like(rho)
        phi = E
    else:
        dphi_dD = 2.0 * rho
        phi = out["E2"]
    gD = dphi_dD * (1.0 + lam0 * Ebc)
    K = half_window(p.ndim, p.window).shape[0]
    pyr = pyramid(M, p.levels)
    w = p.weights()
    g = None
    for l in reversed(range(p.levels)):
        Gl = w[l] * gD[l * K * K:(l + 1) * K * K].reshape(K, K)
        gl = s3_level_vjp(pyr[l], p, Gl)
        g = gl if g is None else gl + prolongate_adjoint(g)
    ex = box_excess(M)
    dex = np.where(M - 1.0 > 0, 1.0, 0.0) - np.where(-M > 0, 1.0, 0.0)
    g = g + lam0 * phi * 2.0 * (ex / N) * dex / N
    return out, g


def s2_count(M, r) -> float:
    """Binary field: the probability that x and x + r are both in phase 1 (any vector r)."""
    M = np.asarray(M)
    tip = np.roll(M, shift=tuple(-int(c) for c in r), axis=tuple(range(M.ndim)))
    return float(np.mean((M == 1) & (tip == 1)))


def s3_count(M, ra, rb) -> float:
    """Binary field: the probability that x, x + r_a and x + r_b are all in phase 1."""
    M = np.asarray(M)
    axes = tuple(range(M.ndim))
    ta = np.roll(M, shift=tuple(-int(c) for c in ra), axis=axes)
    tb = np.roll(M, shift=tuple(-int(c) for c in rb), axis=axes)
    return float(np.mean((M == 1) & (ta == 1) & (tb == 1)))


def s3_from_s3bar(s3b: float, s2a: float, s2b: float, s20: float, s2ab: float, fh: float) -> float:
    """App. A, Eq. s3rfroms3rbar, general case 0 != r_a != r_b != 0: S3 from S_bar3 and the
    exact two-point values S2(r_a), S2(r_b), S2(0) and S2(r_a - r_b), with fh = f(1/2)."""
    return (s3b - fh * (s2a + s2b) - fh * fh * (s20 - s2a - s2b + s2ab)) / (1.0 - 2.0 * fh)


# ----------------------------------------------------------------------------- corrected S2

def half_value(p: Params) -> float:
    """f(1/2) of the threshold (1/2 for f(x) = x)."""
    return float(threshold(np.array([0.5]), p.threshold, p.alpha)[0][0])


def s2tilde_map(K: int, fh: float) -> np.ndarray:
    """The K x K matrix A of App. A (Eq. s2rfroms2rbar) on one level's half-window block,
    S_tilde = A S_bar: row 0 keeps S_bar(0); row k >= 1 is (e_k - 2 fh^2 e_0) / (1 - 2 fh^2)."""
    q = 2.0 * fh * fh
    A = np.eye(K) / (1.0 - q)
    A[0, 0] = 1.0
    A[1:, 0] = -q / (1.0 - q)
    return A


def descriptor_tilde(M, p: Params) -> np.ndarray:
    """The corrected descriptor: every level block of ``descriptor`` mapped by A."""
    D = descriptor(M, p)
    K = half_window(p.ndim, p.window).shape[0]
    A = s2tilde_map(K, half_value(p))
    return np.concatenate([A @ D[l * K:(l + 1) * K] for l in range(p.levels)])


def tilde_loss_grad(M, D_des, p: Params, mode: str = "norm", lambda0: float | None = None, bc: bool = True):
    """Eq. L_func_dMCR on the corrected descriptor and its gradient: dL/dS_bar = A^T dL/dS_tilde
    per level, then the two-point chain rule through all levels."""
    M = np.asarray(M, dtype=np.float64)
    N = M.size
    D = descriptor_tilde(M, p)
    out = loss(M, D_des, p, mode, lambda0, bc, D=D)
    lam0 = out["lambda0"]
    rho, E, Ebc = out["rho"], out["E"], out["Ebc"]
    if mode == "norm":
        dphi_dD = rho / E if E > 0 else np.zeros_like(rho)
        phi = E
    else:
        dphi_dD = 2.0 * rho
        phi = out["E2"]
    gD = dphi_dD * (1.0 + lam0 * Ebc)
    K = half_window(p.ndim, p.window).shape[0]
    A = s2tilde_map(K, half_value(p))
    gbar = np.concatenate([A.T @ gD[l * K:(l + 1) * K] for l in range(p.levels)])
    g = descriptor_vjp(M, p, gbar)
    ex = box_excess(M)
    dex = np.where(M - 1.0 > 0, 1.0, 0.0) - np.where(-M > 0, 1.0, 0.0)
    g = g + lam0 * phi * 2.0 * (ex / N) * dex / N
    return out, g


# ----------------------------------------------------------------------------- multi-phase

def cross_sbar(Ma, Mb, shifts, kind: str = "soft", alpha: float = 10.0) -> np.ndarray:
    """Two-point reduction with the pair's tail in one phase field and its tip in another:
    S_bar^{a->b}(r) = (1/N) sum_x f((Ma_x + Mb_{x+r}) / 2)^2, the convolve -> threshold ->
    reduce chain of Sec. 3.2.2-3.2.4 applied to the cross-correlation S2^{a->b} that the
    outlook (Sec. 5) names for microstructures of more than two phases.  Ma = Mb gives
    S_bar2."""
    Ma = np.asarray(Ma, dtype=np.float64)
    Mb = np.asarray(Mb, dtype=np.float64)
    axes = tuple(range(Ma.ndim))
    out = np.empty(len(shifts))
    for k, r in enumerate(shifts):
        tip = np.roll(Mb, shift=tuple(-int(c) for c in r), axis=axes)   # tip[x] = Mb[x + r]
        e = threshold(0.5 * (Ma + tip), kind, alpha)[0]
        out[k] = float(np.mean(e * e))
    return out


def multiphase_descriptor(F, p: Params, levels_out: bool = False):
    """Eq. mg for a stack F of phase fields (n_phase, *shape): per level l (pyramid of every
    field) and per ordered phase pair (a, b) in row-major order, w_l S_bar_l^{a->b}(r) on the
    half window.  The pairs (a, b) and (b, a) together give S^{a->b} on the full window
    (S^{a->b}(-r) = S^{b->a}(r)); both hold the r = 0 value."""
    F = np.asarray(F, dtype=np.float64)
    nph = F.shape[0]
    H = half_window(p.ndim, p.window)
    pyrs = [pyramid(F[a], p.levels) for a in range(nph)]
    w = p.weights()
    blocks = [w[l] * cross_sbar(pyrs[a][l], pyrs[b][l], H, p.threshold, p.alpha)
              for l in range(p.levels) for a in range(nph) for b in range(nph)]
    D = np.concatenate(blocks)
    return (D, blocks) if levels_out else D


def multiphase_level_vjp(Ml, p: Params, G) -> np.ndarray:
    """Chain rule of one level, term by term: G[a, b, k] weighs S_bar^{a->b}(r_k), whose
    summand f(u)^2, u = (Ma_x + Mb_{x+r}) / 2, has the derivative f(u) f'(u) / N with
    respect to Ma_x and to Mb_{x+r}.  Ml: the level's fields (n_phase, *shape)."""
    Ml = np.asarray(Ml, dtype=np.float64)
    nph = Ml.shape[0]
    H = half_window(p.ndim, p.window)
    axes = tuple(range(Ml.ndim - 1))
    N = Ml[0].size
    g = np.zeros_like(Ml)
    for a in range(nph):
        for b in range(nph):
            for k, r in enumerate(H):
                tip = np.roll(Ml[b], shift=tuple(-int(c) for c in r), axis=axes)
                f, df = threshold(0.5 * (Ml[a] + tip), p.threshold, p.alpha)
                t = G[a, b, k] * (f * df).reshape(Ml[a].shape) / N
                g[a] += t                                                      # d/dMa_x
                g[b] += np.roll(t, shift=tuple(int(c) for c in r), axis=axes)  # d/dMb_{x+r}
    return g


def multiphase_descriptor_vjp(F, p: Params, grad_D) -> np.ndarray:
    """Gradient of <grad_D, D(F)> with respect to every finest phase field: per-level VJP,
    then the transpose of each field's pooling chain (Sec. 3.3)."""
    F = np.asarray(F, dtype=np.float64)
    nph = F.shape[0]
    K = half_window(p.ndim, p.window).shape[0]
    pyrs = [pyramid(F[a], p.levels) for a in range(nph)]
    w = p.weights()
    g = None
    for l in reversed(range(p.levels)):
        blk = np.asarray(grad_D[l * nph * nph * K:(l + 1) * nph * nph * K], dtype=np.float64)
        Ml = np.stack([pyrs[a][l] for a in range(nph)])
        gl = multiphase_level_vjp(Ml, p, w[l] * blk.reshape(nph, nph, K))
        g = gl if g is None else gl + np.stack([prolongate_adjoint(g[a]) for a in range(nph)])
    return g


def multiphase_loss_grad(F, D_des, p: Params, mode: str = "norm", lambda0: float | None = None,
                         bc: bool = True):
    """Eq. L_func_dMCR on the multi-phase descriptor and its gradient.  E_bc sums the box
    excess of every phase field, each normalised by the finest pixel count N of one field;
    lambda0 defaults to N."""
    F = np.asarray(F, dtype=np.float64)
    N = F[0].size
    if lambda0 is None:
        lambda0 = float(N)
    if not bc:
        lambda0 = 0.0
    D = multiphase_descriptor(F, p)
    rho = D - np.asarray(D_des, dtype=np.float64)
    E2 = float(np.sum(rho * rho))
    E = float(np.sqrt(E2))
    Ebc = float(np.sum((box_excess(F) / N) ** 2))
    phi = E if mode == "norm" else E2
    lam = lambda0 * phi
    ref = float(np.sqrt(np.sum(np.asarray(D_des, dtype=np.float64) ** 2)))
    out = {"E": E, "E2": E2, "Ebc": Ebc, "lambda": lam, "L": phi + lam * Ebc,
           "rel_err": E / ref if ref > 0 else float("inf"), "rho": rho, "lambda0": lambda0}
    dphi_dD = (rho / E if E > 0 else np.zeros_like(rho)) if mode == "norm" else 2.0 * rho
    g = multiphase_descriptor_vjp(F, p, dphi_dD * (1.0 + lambda0 * Ebc))
    dex = np.where(F - 1.0 > 0, 1.0, 0.0) - np.where(-F > 0, 1.0, 0.0)
    g = g + lambda0 * phi * 2.0 * (box_excess(F) / N) * dex / N
    return out, g


def cross_count(A, B, r) -> float:
    """Binary phase indicators: the probability that x lies in phase a and x + r in phase b,
    counted position by position."""
    A = np.asarray(A)
    B = np.asarray(B)
    hits = 0
    for x in np.ndindex(A.shape):
        y = tuple((x[i] + int(r[i])) % A.shape[i] for i in range(A.ndim))
        hits += int(A[x] == 1 and B[y] == 1)
    return hits / A.size


def multiphase_vjp_at(F, p: Params, grad_D, positions) -> np.ndarray:
    """``multiphase_descriptor_vjp`` at sampled finest positions (flat indices), written in
    gather form: at level l the position's ancestor y (coordinates >> l) collects, for every
    phase b and shift r_k, G[a, b, k] h((Ma_y + Mb_{y+r}) / 2) + G[b, a, k] h((Mb_{y-r} + Ma_y) / 2)
    over N_l, h = f f'; the pooling transpose scales level l by 2^{-d l}.  Returns
    (n_phase, len(positions))."""
    F = np.asarray(F, dtype=np.float64)
    nph = F.shape[0]
    shape = F.shape[1:]
    d = len(shape)
    H = half_window(p.ndim, p.window)
    K = H.shape[0]
    pyrs = [pyramid(F[a], p.levels) for a in range(nph)]
    w = p.weights()
    coords = np.stack(np.unravel_index(np.asarray(positions, dtype=np.int64), shape), axis=1)
    out = np.zeros((nph, coords.shape[0]))
    for l in range(p.levels):
        G = w[l] * np.asarray(grad_D[l * nph * nph * K:(l + 1) * nph * nph * K], dtype=np.float64)
        G = G.reshape(nph, nph, K)
        n = np.array(pyrs[0][l].shape)
        Nl = int(np.prod(n))
        for i, c in enumerate(coords):
            y = c >> l
            fwd = tuple(((y + H) % n).T)          # y + r_k
            bwd = tuple(((y - H) % n).T)          # y - r_k
            for a in range(nph):
                ma = pyrs[a][l][tuple(y)]
                acc = 0.0
                for b in range(nph):
                    f1, d1 = threshold(0.5 * (ma + pyrs[b][l][fwd]), p.threshold, p.alpha)
                    f2, d2 = threshold(0.5 * (pyrs[b][l][bwd] + ma), p.threshold, p.alpha)
                    acc += float(np.dot(G[a, b], f1 * d1) + np.dot(G[b, a], f2 * d2))
                out[a, i] += acc / Nl / float(2 ** (d * l))
    return out
