"""Thin ctypes binding of libdmcr (include/dmcr.h): argument marshalling only.

Every function named ``dmcr_*`` here calls the C entry point of the same name with the
device pointers of CUDA tensors and the current PyTorch stream; all arithmetic runs in
the library's kernels.  The library must be built (``__graft_entry__.build()`` or
``python -m paper_2103_09686_gb300._build``); nothing here falls back to another
implementation when it is missing.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import threading

import torch

from . import _build

c_int, c_int64, c_float, c_void_p, c_uint64, c_size_t = (ctypes.c_int, ctypes.c_int64, ctypes.c_float,
                                                        ctypes.c_void_p, ctypes.c_uint64, ctypes.c_size_t)

DMCR_OK, DMCR_EINVAL, DMCR_ENOMEM, DMCR_ECUDA, DMCR_ENONFINITE, DMCR_ETIMEOUT, DMCR_ENOTSUP = range(7)
DMCR_SOFT, DMCR_IDENTITY = 0, 1
DMCR_PATH_AUTO, DMCR_PATH_DIRECT, DMCR_PATH_FFT = 0, 1, 2
DMCR_DESC_S2, DMCR_DESC_S3, DMCR_DESC_S2_TILDE = 0, 1, 2
DMCR_LOSS_NORM, DMCR_LOSS_SQUARED = 0, 1
DMCR_PROLONG_ADJOINT_ACCUMULATE, DMCR_PROLONG_INJECT = 0, 1
DMCR_INIT_CALLER, DMCR_INIT_UNIFORM_SEEDED = 0, 1
OUT_NAMES = ("E", "E2", "Ebc", "lambda", "L", "rel_err")
DMCR_OUT_COUNT = len(OUT_NAMES)


class dmcr_params(ctypes.Structure):
    _fields_ = [("ndim", c_int), ("n", c_int64 * 3), ("window", c_int * 3), ("levels", c_int),
                ("threshold", c_int), ("alpha", c_float), ("level_weight_exp", c_float), ("path", c_int),
                ("tune", c_int * 4), ("descriptor", c_int), ("phases", c_int)]


class dmcr_loss_opts(ctypes.Structure):
    _fields_ = [("mode", c_int), ("lambda0", c_float), ("bc_on", c_int)]


class dmcr_recon_opts(ctypes.Structure):
    _fields_ = [("max_iters", c_int), ("tol_rel", c_float), ("lr", c_float), ("beta1", c_float),
                ("beta2", c_float), ("eps", c_float), ("loss", dmcr_loss_opts), ("init", c_int),
                ("seed", c_uint64), ("check_every", c_int), ("report_rounded", c_int)]


class dmcr_adam_state(ctypes.Structure):
    _fields_ = [("m", c_void_p), ("v", c_void_p), ("step", c_int64)]


class dmcr_recon_report(ctypes.Structure):
    _fields_ = [("iterations", c_int), ("converged", c_int), ("loss", c_float * 6), ("status", c_int),
                ("rounded_rel_err", c_float)]


class DmcrError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("dmcr status %d: %s" % (status, msg))
        self.status = status


_lib = None
_lock = threading.Lock()


def load(build_if_missing: bool = False):
    """Load libdmcr.so from the package directory (raises when it is missing)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build_if_missing or not os.path.exists(_build.LIB):
            if not build_if_missing:
                raise RuntimeError("libdmcr.so is not built: run __graft_entry__.build() or "
                                   "python -m paper_2103_09686_gb300._build")
            _build.build()
        lib = ctypes.CDLL(_build.LIB)
        P = ctypes.POINTER
        lib.dmcr_version.restype = c_int
        lib.dmcr_last_error.restype = ctypes.c_char_p
        lib.dmcr_descriptor_length.argtypes = [P(dmcr_params), P(c_int64)]
        lib.dmcr_workspace_size.argtypes = [P(dmcr_params), P(c_size_t)]
        lib.dmcr_descriptor.argtypes = [P(dmcr_params), c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]
        lib.dmcr_loss_grad.argtypes = [P(dmcr_params), P(dmcr_loss_opts), c_void_p, c_void_p, c_void_p, c_void_p,
                                       c_void_p, c_void_p, c_size_t, c_void_p]
        lib.dmcr_descriptor_vjp.argtypes = [P(dmcr_params), c_void_p, c_void_p, c_void_p, c_void_p, c_size_t,
                                            c_void_p]
        lib.dmcr_restrict.argtypes = [c_int, P(c_int64), c_void_p, c_void_p, c_void_p]
        lib.dmcr_prolongate.argtypes = [c_int, P(c_int64), c_void_p, c_void_p, c_int, c_void_p]
        lib.dmcr_init_uniform.argtypes = [c_void_p, c_int64, c_uint64, c_void_p]
        lib.dmcr_reconstruct.argtypes = [P(dmcr_params), P(dmcr_recon_opts), c_void_p, c_void_p, P(dmcr_adam_state),
                                         c_void_p, P(dmcr_recon_report), c_void_p, c_size_t, c_void_p]
        lib.dmcr_adam_step.argtypes = [P(dmcr_params), P(dmcr_recon_opts), c_void_p, c_void_p, P(dmcr_adam_state),
                                       c_void_p, c_void_p, c_size_t, c_void_p]
        lib.dmcr_descriptor_noalloc.argtypes = [P(dmcr_params), c_void_p, c_void_p, c_void_p]
        PP = P(c_void_p)
        lib.dmcr_batch_workspace_size.argtypes = [c_int, P(dmcr_params), P(c_size_t)]
        lib.dmcr_descriptor_batched.argtypes = [c_int, P(dmcr_params), PP, PP, c_void_p, c_size_t, c_void_p]
        lib.dmcr_loss_grad_batched.argtypes = [c_int, P(dmcr_params), P(dmcr_loss_opts), PP, PP, c_void_p, PP,
                                               c_void_p, c_size_t, c_void_p]
        lib.dmcr_descriptor_vjp_batched.argtypes = [c_int, P(dmcr_params), PP, PP, PP, c_void_p, c_size_t, c_void_p]
        lib.dmcr_adam_step_batched.argtypes = [c_int, P(dmcr_params), P(dmcr_recon_opts), PP, PP, P(dmcr_adam_state),
                                               c_void_p, c_void_p, c_size_t, c_void_p]
        lib.dmcr_reconstruct_batched.argtypes = [c_int, P(dmcr_params), P(dmcr_recon_opts), PP, PP,
                                                 P(dmcr_adam_state), P(dmcr_recon_report), c_void_p, c_size_t,
                                                 c_void_p]
        lib.dmcr_profile_enable.argtypes = [c_int]
        lib.dmcr_profile_reset.argtypes = []
        lib.dmcr_profile_read.argtypes = [c_int, ctypes.c_char_p, c_int, P(ctypes.c_double), P(c_int64)]
        for name in ("dmcr_descriptor_length", "dmcr_workspace_size", "dmcr_descriptor", "dmcr_loss_grad",
                     "dmcr_descriptor_vjp", "dmcr_restrict", "dmcr_prolongate", "dmcr_init_uniform",
                     "dmcr_reconstruct", "dmcr_adam_step", "dmcr_profile_enable", "dmcr_profile_reset",
                     "dmcr_profile_read", "dmcr_descriptor_noalloc", "dmcr_batch_workspace_size",
                     "dmcr_descriptor_batched", "dmcr_loss_grad_batched", "dmcr_descriptor_vjp_batched",
                     "dmcr_adam_step_batched", "dmcr_reconstruct_batched"):
            getattr(lib, name).restype = c_int
        _lib = lib
        return lib


def _check(st: int):
    if st != DMCR_OK:
        raise DmcrError(st, load().dmcr_last_error().decode(errors="replace"))


def _stream(stream=None) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _check_device(t, what: str = "tensor"):
    """The library launches on the current CUDA device, so every pointer must belong to it:
    a tensor on another device would hand foreign addresses to the kernels."""
    index = getattr(t.device, "index", None)
    if isinstance(index, int) and index != torch.cuda.current_device():
        raise ValueError("%s is on cuda:%d but the current device is cuda:%d (make its device current, e.g. "
                         "with torch.cuda.device(...))" % (what, index, torch.cuda.current_device()))


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("tensor must be on a CUDA device")
    if t.dtype != torch.float32 or not t.is_contiguous():
        raise ValueError("tensor must be contiguous float32")
    _check_device(t)
    return t.data_ptr()


# The C calls take bare device pointers and trust their sizes; the binding checks every
# tensor against the sizes the parameters imply before anything is launched, so that a
# wrong tensor raises here instead of reaching the device.

def _sized(t, n: int, what: str, at_least: bool = False):
    """Pointer of a float32 CUDA tensor holding exactly (or at least) n elements."""
    ptr = _ptr(t)
    if t is not None and (t.numel() < n if at_least else t.numel() != n):
        raise ValueError("%s must hold %s%d float32 elements (has %d)" % (what, "at least " if at_least else "", n,
                                                                          t.numel()))
    return ptr


def _ws(ws):
    """(pointer, bytes) of a workspace tensor."""
    if not ws.is_cuda or not ws.is_contiguous():
        raise ValueError("workspace must be a contiguous CUDA tensor")
    _check_device(ws, "workspace")
    return ws.data_ptr(), ws.numel() * ws.element_size()


def _lengths(p) -> tuple:
    """(field elements, descriptor length) of a problem: N * phases and sum_l K."""
    n = 1
    for a in p.shape:
        n *= int(a)
    return n * max(int(p.phases), 1), dmcr_descriptor_length(p)


# ----------------------------------------------------------------------------- params

@dataclasses.dataclass(frozen=True)
class Params:
    """Problem statement (Sec. 3.3): field shape, window P_a per axis, multigrid levels."""
    shape: tuple
    window: tuple
    levels: int = 1
    threshold: int = DMCR_SOFT
    alpha: float = 10.0
    level_weight_exp: float = -1.0
    path: int = DMCR_PATH_AUTO
    tune: tuple = (0, 0, 0, 0)     # launch shape; 0 = built-in choice (see tune.py)
    descriptor: int = DMCR_DESC_S2  # DMCR_DESC_S3: K x K three-point matrix; S2_TILDE: App. A corrected S2
    phases: int = 1                 # > 1: fields are (phases, *shape) stacks; cross-correlations of every pair

    @property
    def ndim(self) -> int:
        return len(self.shape)

    def c(self) -> dmcr_params:
        if len(self.shape) not in (2, 3) or len(self.window) != len(self.shape) or len(self.tune) > 4:
            raise DmcrError(DMCR_EINVAL, "shape and window must both have 2 or 3 entries (got %d and %d),"
                            " tune at most 4" % (len(self.shape), len(self.window)))
        p = dmcr_params()
        p.ndim = len(self.shape)
        for a, s in enumerate(self.shape):
            p.n[a] = int(s)
        for a, w in enumerate(self.window):
            p.window[a] = int(w)
        p.levels = int(self.levels)
        p.threshold = int(self.threshold)
        p.alpha = float(self.alpha)
        p.level_weight_exp = float(self.level_weight_exp)
        p.path = int(self.path)
        for i, t in enumerate(self.tune):
            p.tune[i] = int(t)
        p.descriptor = int(self.descriptor)
        p.phases = int(self.phases)
        return p


@dataclasses.dataclass(frozen=True)
class LossOpts:
    mode: int = DMCR_LOSS_NORM
    lambda0: float = -1.0      # <0: finest pixel count
    bc_on: bool = True

    def c(self) -> dmcr_loss_opts:
        return dmcr_loss_opts(int(self.mode), float(self.lambda0), int(bool(self.bc_on)))


@dataclasses.dataclass(frozen=True)
class ReconOpts:
    max_iters: int = 200
    tol_rel: float = 0.0
    lr: float = 1e-3
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-7
    loss: LossOpts = LossOpts()
    init: int = DMCR_INIT_CALLER
    seed: int = 0
    check_every: int = 1
    report_rounded: bool = True   # evaluate the rounded result once more (report["rounded_rel_err"])

    def c(self) -> dmcr_recon_opts:
        o = dmcr_recon_opts()
        o.max_iters = int(self.max_iters)
        o.tol_rel = float(self.tol_rel)
        o.lr, o.beta1, o.beta2, o.eps = float(self.lr), float(self.beta1), float(self.beta2), float(self.eps)
        o.loss = self.loss.c()
        o.init = int(self.init)
        o.seed = int(self.seed) & ((1 << 64) - 1)
        o.check_every = int(self.check_every)
        o.report_rounded = int(bool(self.report_rounded))
        return o


# ----------------------------------------------------------------------------- raw C entry points

def dmcr_version() -> int:
    return load().dmcr_version()


def dmcr_descriptor_length(p: Params) -> int:
    out = c_int64()
    _check(load().dmcr_descriptor_length(ctypes.byref(p.c()), ctypes.byref(out)))
    return out.value


def dmcr_workspace_size(p: Params) -> int:
    out = c_size_t()
    _check(load().dmcr_workspace_size(ctypes.byref(p.c()), ctypes.byref(out)))
    return out.value


def workspace(p: Params, device=None) -> torch.Tensor:
    n = dmcr_workspace_size(p)
    return torch.empty(max(n, 256), dtype=torch.uint8, device=device or "cuda")


def dmcr_descriptor(p: Params, field, desc, ws=None, stream=None):
    N, K = _lengths(p)
    fp, dp = _sized(field, N, "field"), _sized(desc, K, "desc")
    ws = workspace(p, field.device) if ws is None else ws
    _check(load().dmcr_descriptor(ctypes.byref(p.c()), fp, dp, *_ws(ws), _stream(stream)))
    return desc


def dmcr_loss_grad(p: Params, opts: LossOpts, field, target_desc, loss_out, grad=None, desc_out=None, ws=None,
                   stream=None):
    N, K = _lengths(p)
    ptrs = (_sized(field, N, "field"), _sized(target_desc, K, "target_desc"),
            _sized(loss_out, DMCR_OUT_COUNT, "loss_out", at_least=True), _sized(grad, N, "grad"),
            _sized(desc_out, K, "desc_out"))
    ws = workspace(p, field.device) if ws is None else ws
    _check(load().dmcr_loss_grad(ctypes.byref(p.c()), ctypes.byref(opts.c()), *ptrs, *_ws(ws), _stream(stream)))


def dmcr_descriptor_vjp(p: Params, field, grad_desc, grad_field, ws=None, stream=None):
    N, K = _lengths(p)
    ptrs = (_sized(field, N, "field"), _sized(grad_desc, K, "grad_desc"), _sized(grad_field, N, "grad_field"))
    ws = workspace(p, field.device) if ws is None else ws
    _check(load().dmcr_descriptor_vjp(ctypes.byref(p.c()), *ptrs, *_ws(ws), _stream(stream)))
    return grad_field


def dmcr_restrict(fine, coarse, stream=None):
    n = (c_int64 * 3)(*list(fine.shape) + [0] * (3 - fine.dim()))
    fp = _ptr(fine)
    cp = _sized(coarse, fine.numel() >> fine.dim(), "coarse")
    _check(load().dmcr_restrict(fine.dim(), n, fp, cp, _stream(stream)))
    return coarse


def dmcr_prolongate(coarse, fine, mode=DMCR_PROLONG_ADJOINT_ACCUMULATE, stream=None):
    n = (c_int64 * 3)(*list(coarse.shape) + [0] * (3 - coarse.dim()))
    cp = _ptr(coarse)
    fp = _sized(fine, coarse.numel() << coarse.dim(), "fine")
    _check(load().dmcr_prolongate(coarse.dim(), n, cp, fp, int(mode), _stream(stream)))
    return fine


def dmcr_init_uniform(field, seed: int, stream=None):
    _check(load().dmcr_init_uniform(_ptr(field), field.numel(), int(seed) & ((1 << 64) - 1), _stream(stream)))
    return field


def dmcr_reconstruct(p: Params, opts: ReconOpts, target_desc, field, m, v, step: int = 0, history=None, ws=None,
                     stream=None):
    """Runs the reconstruction (synchronous).  Returns (report dict, new Adam step)."""
    N, K = _lengths(p)
    tp, fp = _sized(target_desc, K, "target_desc"), _sized(field, N, "field")
    hp = _sized(history, 3 * max(int(opts.max_iters), 0), "history", at_least=True)
    st = dmcr_adam_state(_sized(m, N, "m"), _sized(v, N, "v"), int(step))
    ws = workspace(p, field.device) if ws is None else ws
    rep = dmcr_recon_report()
    status = load().dmcr_reconstruct(ctypes.byref(p.c()), ctypes.byref(opts.c()), tp, fp, ctypes.byref(st), hp,
                                     ctypes.byref(rep), *_ws(ws), _stream(stream))
    _check(status)
    report = {"iterations": rep.iterations, "converged": bool(rep.converged), "status": rep.status,
              "rounded_rel_err": float(rep.rounded_rel_err)}
    report.update({k: float(rep.loss[i]) for i, k in enumerate(OUT_NAMES)})
    return report, st.step


def dmcr_adam_step(p: Params, opts: ReconOpts, target_desc, field, m, v, step: int, loss_out=None, ws=None,
                   stream=None) -> int:
    """One asynchronous iteration (loss, gradient, Adam step).  Returns the new step count."""
    N, K = _lengths(p)
    tp, fp = _sized(target_desc, K, "target_desc"), _sized(field, N, "field")
    lp = _sized(loss_out, DMCR_OUT_COUNT, "loss_out", at_least=True)
    st = dmcr_adam_state(_sized(m, N, "m"), _sized(v, N, "v"), int(step))
    ws = workspace(p, field.device) if ws is None else ws
    _check(load().dmcr_adam_step(ctypes.byref(p.c()), ctypes.byref(opts.c()), tp, fp, ctypes.byref(st), lp,
                                 *_ws(ws), _stream(stream)))
    return st.step


def dmcr_descriptor_noalloc(p: Params, field, desc, stream=None):
    """dmcr_descriptor without a workspace: scratch from the library's fixed device array."""
    N, K = _lengths(p)
    _check(load().dmcr_descriptor_noalloc(ctypes.byref(p.c()), _sized(field, N, "field"), _sized(desc, K, "desc"),
                                          _stream(stream)))
    return desc


# ----------------------------------------------------------------------------- batched calls

def _params_array(params):
    arr = (dmcr_params * len(params))()
    for i, p in enumerate(params):
        arr[i] = p.c()
    return arr


def _ptr_array(tensors, sizes=None, what="tensor"):
    """Host array of device pointers; tensor i must hold sizes[i] elements when given."""
    if tensors is None:
        return None
    if sizes is not None and len(tensors) != len(sizes):
        raise ValueError("%s: %d tensors for %d instances" % (what, len(tensors), len(sizes)))
    ptrs = [_sized(t, sizes[i], "%s[%d]" % (what, i)) if sizes is not None else _ptr(t)
            for i, t in enumerate(tensors)]
    return (c_void_p * len(tensors))(*ptrs)


def _adam_states(ms, vs, steps, Ns):
    n = len(Ns)
    if len(ms) != n or len(vs) != n or len(steps) != n:
        raise ValueError("ms, vs and steps need one entry per instance (%d)" % n)
    st = (dmcr_adam_state * n)()
    for i in range(n):
        st[i] = dmcr_adam_state(_sized(ms[i], Ns[i], "ms[%d]" % i), _sized(vs[i], Ns[i], "vs[%d]" % i), int(steps[i]))
    return st


def _batch_lengths(params):
    ln = [_lengths(p) for p in params]
    return [a for a, _ in ln], [b for _, b in ln]


def dmcr_batch_workspace_size(params) -> int:
    out = c_size_t()
    _check(load().dmcr_batch_workspace_size(len(params), _params_array(params), ctypes.byref(out)))
    return out.value


def batch_workspace(params, device=None) -> torch.Tensor:
    return torch.empty(max(dmcr_batch_workspace_size(params), 256), dtype=torch.uint8, device=device or "cuda")


def dmcr_descriptor_batched(params, fields, descs, ws=None, stream=None):
    Ns, Ks = _batch_lengths(params)
    fa, da = _ptr_array(fields, Ns, "fields"), _ptr_array(descs, Ks, "descs")
    ws = batch_workspace(params, fields[0].device) if ws is None else ws
    _check(load().dmcr_descriptor_batched(len(params), _params_array(params), fa, da, *_ws(ws), _stream(stream)))
    return descs


def dmcr_loss_grad_batched(params, opts: LossOpts, fields, targets, loss_out, grads=None, ws=None, stream=None):
    Ns, Ks = _batch_lengths(params)
    fa, ta = _ptr_array(fields, Ns, "fields"), _ptr_array(targets, Ks, "targets")
    lo = _sized(loss_out, DMCR_OUT_COUNT * len(params), "loss_out", at_least=True)
    ga = _ptr_array(grads, Ns, "grads")
    ws = batch_workspace(params, fields[0].device) if ws is None else ws
    _check(load().dmcr_loss_grad_batched(len(params), _params_array(params), ctypes.byref(opts.c()), fa, ta, lo, ga,
                                         *_ws(ws), _stream(stream)))


def dmcr_descriptor_vjp_batched(params, fields, grad_descs, grad_fields, ws=None, stream=None):
    Ns, Ks = _batch_lengths(params)
    fa, ga = _ptr_array(fields, Ns, "fields"), _ptr_array(grad_descs, Ks, "grad_descs")
    gf = _ptr_array(grad_fields, Ns, "grad_fields")
    ws = batch_workspace(params, fields[0].device) if ws is None else ws
    _check(load().dmcr_descriptor_vjp_batched(len(params), _params_array(params), fa, ga, gf, *_ws(ws),
                                              _stream(stream)))
    return grad_fields


def dmcr_adam_step_batched(params, opts: ReconOpts, targets, fields, ms, vs, steps, loss_out=None, ws=None,
                           stream=None):
    """One Adam iteration of every instance; returns the new step counts."""
    n = len(params)
    Ns, Ks = _batch_lengths(params)
    ta, fa = _ptr_array(targets, Ks, "targets"), _ptr_array(fields, Ns, "fields")
    lo = _sized(loss_out, DMCR_OUT_COUNT * n, "loss_out", at_least=True)
    st = _adam_states(ms, vs, steps, Ns)
    ws = batch_workspace(params, fields[0].device) if ws is None else ws
    _check(load().dmcr_adam_step_batched(n, _params_array(params), ctypes.byref(opts.c()), ta, fa, st, lo, *_ws(ws),
                                         _stream(stream)))
    return [st[i].step for i in range(n)]


def dmcr_reconstruct_batched(params, opts, targets, fields, ms, vs, steps, ws=None, stream=None):
    """Graph-captured reconstruction of every instance (synchronous).  ``opts`` is one
    ReconOpts or a list.  Returns (list of report dicts, list of new step counts)."""
    n = len(params)
    if isinstance(opts, ReconOpts):
        opts = [opts] * n
    if len(opts) != n:
        raise ValueError("opts: %d entries for %d instances" % (len(opts), n))
    Ns, Ks = _batch_lengths(params)
    ta, fa = _ptr_array(targets, Ks, "targets"), _ptr_array(fields, Ns, "fields")
    oa = (dmcr_recon_opts * n)()
    for i in range(n):
        oa[i] = opts[i].c()
    st = _adam_states(ms, vs, steps, Ns)
    ws = batch_workspace(params, fields[0].device) if ws is None else ws
    reps = (dmcr_recon_report * n)()
    status = load().dmcr_reconstruct_batched(n, _params_array(params), oa, ta, fa, st, reps, *_ws(ws),
                                             _stream(stream))
    _check(status)
    out = []
    for i in range(n):
        r = {"iterations": reps[i].iterations, "converged": bool(reps[i].converged), "status": reps[i].status,
             "rounded_rel_err": float(reps[i].rounded_rel_err)}
        r.update({k: float(reps[i].loss[j]) for j, k in enumerate(OUT_NAMES)})
        out.append(r)
    return out, [st[i].step for i in range(n)]


def dmcr_profile_enable(on: bool = True):
    _check(load().dmcr_profile_enable(int(bool(on))))


def dmcr_profile_reset():
    _check(load().dmcr_profile_reset())


def dmcr_profile_read() -> dict:
    """{kernel name: (total ms, launches)} of the launches recorded since the last reset."""
    lib = load()
    out = {}
    i = 0
    buf = ctypes.create_string_buffer(64)
    ms = ctypes.c_double()
    cnt = c_int64()
    while lib.dmcr_profile_read(i, buf, 64, ctypes.byref(ms), ctypes.byref(cnt)) == DMCR_OK:
        out[buf.value.decode()] = (ms.value, cnt.value)
        i += 1
    return out


# ----------------------------------------------------------------------------- conveniences

def descriptor(field: torch.Tensor, p: Params, ws=None) -> torch.Tensor:
    desc = torch.empty(dmcr_descriptor_length(p), dtype=torch.float32, device=field.device)
    return dmcr_descriptor(p, field, desc, ws)


def loss_grad(field: torch.Tensor, target_desc: torch.Tensor, p: Params, opts: LossOpts = LossOpts(),
              want_grad: bool = True, ws=None):
    loss = torch.empty(6, dtype=torch.float32, device=field.device)
    grad = torch.empty_like(field) if want_grad else None
    dmcr_loss_grad(p, opts, field, target_desc, loss, grad, None, ws)
    return loss, grad


def descriptor_vjp(field: torch.Tensor, grad_desc: torch.Tensor, p: Params, ws=None) -> torch.Tensor:
    g = torch.empty_like(field)
    return dmcr_descriptor_vjp(p, field, grad_desc, g, ws)
