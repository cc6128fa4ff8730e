"""CPU-side checks of the C ABI: the library builds for sm_103a, loads, exports every
symbol include/dmcr.h declares, and validates arguments without touching a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2103_09686_gb300 import _build, _lib
    _build.build()
    return _lib.load()


def _declared_symbols():
    src = open(os.path.join(ROOT, "include", "dmcr.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dmcr_[a-z_]+)\s*\(", src)))


def test_header_declares_the_four_named_calls():
    syms = _declared_symbols()
    for name in ("dmcr_descriptor", "dmcr_loss_grad", "dmcr_prolongate", "dmcr_reconstruct"):
        assert name in syms


def test_library_exports_every_declared_symbol(lib):
    for name in _declared_symbols():
        assert hasattr(lib, name), name
        assert getattr(lib, name) is not None


def test_version_and_lengths(lib):
    import paper_2103_09686_gb300 as dm
    assert dm.dmcr_version() >= 100
    # K_half per level, summed over levels (Sec. 3.3)
    assert dm.dmcr_descriptor_length(dm.Params((64, 64), (16, 16))) == 545
    assert dm.dmcr_descriptor_length(dm.Params((512, 512), (64, 64), levels=3)) == 3 * 8321
    assert dm.dmcr_descriptor_length(dm.Params((128, 128, 128), (24, 24, 24), levels=2)) == 2 * 58825
    assert dm.dmcr_descriptor_length(dm.Params((64, 64), (31, 31))) == 1985
    assert dm.dmcr_workspace_size(dm.Params((512, 512), (64, 64), levels=3)) > 0


@pytest.mark.parametrize("kw,status", [
    (dict(shape=(64, 64), window=(40, 16)), 1),            # window > n/2
    (dict(shape=(64, 64), window=(16, 16), levels=4), 1),  # 8x8 coarsest level < 2P
    (dict(shape=(60, 64), window=(4, 4), levels=4), 1),    # 60 not divisible by 8
    (dict(shape=(64, 64), window=(4, 4), threshold=7), 1),
    (dict(shape=(64, 64), window=(4, 4), alpha=-1.0), 1),
    (dict(shape=(64, 64), window=(4, 4), path=3), 1),      # unknown path
    (dict(shape=(14, 14), window=(3, 3), path=2), 6),      # FFT path: sizes must factor into 2, 3, 5
    (dict(shape=(64, 60), window=(4, 4), threshold=1), 6),  # identity needs n % 8 == 0
    (dict(shape=(64, 64), window=(4, 4), tune=(12, 0, 0, 0)), 1),   # forward tile rows must be 8/16/32
    (dict(shape=(0, 64), window=(0, 0)), 1),               # empty field
    (dict(shape=(64, 64), window=(-1, 4)), 1),
    (dict(shape=(64,), window=(4,)), 1),                   # 1-D
    (dict(shape=(8, 8, 8, 8), window=(1, 1, 1, 1)), 1),    # 4-D
    (dict(shape=(64, 64), window=(4, 4, 4)), 1),           # window rank differs from the field's
    (dict(shape=(64, 64), window=(4, 4), levels=0), 1),
    (dict(shape=(64, 64), window=(4, 4), levels=9), 1),
    (dict(shape=(64, 64), window=(4, 4), alpha=float("nan")), 1),
    (dict(shape=(64, 64), window=(4, 4), level_weight_exp=float("inf")), 1),
    (dict(shape=(1 << 18, 1 << 17), window=(1, 1)), 1),   # more than 2^34 elements
    (dict(shape=(1 << 31, 4), window=(1, 1)), 1),         # an axis above 2^30
    (dict(shape=(1 << 17, 1 << 17), window=(128, 1 << 16)), 1),   # a workspace above 2^50 bytes
    # three axes of 2^30 (and two with 16): the product of the axes passes 2^63 or wraps to
    # 0 in 64-bit integers; the element count must still be rejected as too large
    (dict(shape=(1 << 30, 1 << 30, 1 << 30), window=(0, 0, 0)), 1),
    (dict(shape=(1 << 30, 1 << 30, 16), window=(0, 0, 0)), 1),
    (dict(shape=(1 << 30, 1 << 30, 1 << 30), window=(1, 1, 1), phases=8), 1),
    (dict(shape=(1 << 12, 1 << 11, 1 << 11), window=(1, 1, 1), phases=3), 1),   # 2^34 cells x 3 phases
])
def test_argument_validation(lib, kw, status):
    import paper_2103_09686_gb300 as dm
    with pytest.raises(dm.DmcrError) as e:
        dm.dmcr_descriptor_length(dm.Params(**kw))
    assert e.value.status == status
    assert len(lib.dmcr_last_error()) > 0


def test_degenerate_windows_are_valid():
    import paper_2103_09686_gb300 as dm
    # window 0: only S(0) per level; a 1 x 1 field; a window of exactly half the size
    assert dm.dmcr_descriptor_length(dm.Params((64, 64), (0, 0), levels=2)) == 2
    assert dm.dmcr_descriptor_length(dm.Params((1, 1), (0, 0))) == 1
    assert dm.dmcr_descriptor_length(dm.Params((8, 8), (4, 4))) == (9 * 9 + 1) // 2
    assert dm.dmcr_descriptor_length(dm.Params((8, 8, 8), (0, 0, 4))) == 5


def test_null_workspace_is_rejected_before_any_launch(lib):
    import paper_2103_09686_gb300 as dm
    from paper_2103_09686_gb300 import _lib
    p = dm.Params((64, 64), (4, 4)).c()
    st = lib.dmcr_descriptor(ctypes.byref(p), 1 << 20, 1 << 21, None, 0, None)
    assert st == _lib.DMCR_EINVAL
    st = lib.dmcr_descriptor(ctypes.byref(p), 1 << 20, 1 << 21, 1 << 22, 16, None)
    assert st == _lib.DMCR_ENOMEM


def test_lengths_of_the_other_descriptors(lib):
    import paper_2103_09686_gb300 as dm
    # three-point: K_half^2 per level; corrected two-point: K_half; P phases: P^2 K_half
    assert dm.dmcr_descriptor_length(dm.Params((64, 64), (31, 31), descriptor=dm.DMCR_DESC_S3)) == 1985 ** 2
    assert dm.dmcr_descriptor_length(dm.Params((64, 64), (4, 4), levels=2, descriptor=dm.DMCR_DESC_S3)) == 2 * 41 ** 2
    assert dm.dmcr_descriptor_length(dm.Params((64, 64), (16, 16), descriptor=dm.DMCR_DESC_S2_TILDE)) == 545
    assert dm.dmcr_descriptor_length(dm.Params((512, 512), (64, 64), levels=3, phases=3)) == 3 * 9 * 8321
    assert dm.dmcr_descriptor_length(dm.Params((64, 64), (16, 16), phases=1)) == 545
    one = dm.dmcr_workspace_size(dm.Params((256, 256), (16, 16), levels=2))
    three = dm.dmcr_workspace_size(dm.Params((256, 256), (16, 16), levels=2, phases=3))
    # nine forward-partial and coefficient blocks per level; the adjoint partials grow less
    # than nine-fold (a chunk of a multi-phase problem covers up to 9 times the ry rows)
    assert three > 2 * one


@pytest.mark.parametrize("kw,status", [
    (dict(shape=(64, 64), window=(4, 4), descriptor=7), 1),                       # unknown descriptor
    (dict(shape=(64, 64), window=(4, 4), descriptor=1, path=2), 6),               # S3 has no FFT path
    (dict(shape=(64, 64), window=(4, 4), phases=9), 1),                           # at most 8 phases
    (dict(shape=(64, 64), window=(4, 4), phases=-1), 1),
    (dict(shape=(64, 64), window=(4, 4), phases=2, descriptor=1), 6),             # phases: S2 only
    (dict(shape=(64, 64), window=(4, 4), phases=2, descriptor=2), 6),
    (dict(shape=(64, 64), window=(4, 4), phases=2, path=2, threshold=1), 6),      # phases: direct only
])
def test_validation_of_descriptor_kinds_and_phases(lib, kw, status):
    import paper_2103_09686_gb300 as dm
    with pytest.raises(dm.DmcrError) as e:
        dm.dmcr_descriptor_length(dm.Params(**kw))
    assert e.value.status == status


class _FakeCudaTensor:
    """Stands in for a CUDA float32 tensor in the binding's argument checks (which run
    before any call into the library); its pointer is never dereferenced."""

    def __init__(self, n):
        import torch
        self.n = n
        self.dtype = torch.float32
        self.is_cuda = True
        self.device = "cuda"

    def numel(self):
        return self.n

    def is_contiguous(self):
        return True

    def data_ptr(self):
        return 1 << 40

    def element_size(self):
        return 4


@pytest.mark.parametrize("call", ["descriptor_field", "descriptor_desc", "loss_target", "loss_out", "loss_grad",
                                  "vjp_grad", "adam_m", "recon_history", "restrict", "prolongate",
                                  "batched_count", "batched_field", "batched_loss_out", "noalloc"])
def test_binding_rejects_wrongly_sized_tensors_before_any_launch(lib, call):
    import paper_2103_09686_gb300 as dm
    from paper_2103_09686_gb300 import _lib
    T = _FakeCudaTensor
    p = dm.Params((32, 24), (4, 3), levels=2)
    N, K = 32 * 24, dm.dmcr_descriptor_length(p)
    q = dm.Params((16, 16), (2, 2), phases=2)
    Nq, Kq = 2 * 256, dm.dmcr_descriptor_length(q)
    ws = T(1 << 20)
    calls = {
        "descriptor_field": lambda: _lib.dmcr_descriptor(p, T(N + 1), T(K), ws),
        "descriptor_desc": lambda: _lib.dmcr_descriptor(p, T(N), T(K - 1), ws),
        "loss_target": lambda: _lib.dmcr_loss_grad(p, dm.LossOpts(), T(N), T(2 * K), T(6), None, None, ws),
        "loss_out": lambda: _lib.dmcr_loss_grad(p, dm.LossOpts(), T(N), T(K), T(5), None, None, ws),
        "loss_grad": lambda: _lib.dmcr_loss_grad(p, dm.LossOpts(), T(N), T(K), T(6), T(N // 2), None, ws),
        "vjp_grad": lambda: _lib.dmcr_descriptor_vjp(p, T(N), T(K), T(N - 1), ws),
        "adam_m": lambda: _lib.dmcr_adam_step(p, dm.ReconOpts(), T(K), T(N), T(N - 1), T(N), 0, None, ws),
        "recon_history": lambda: _lib.dmcr_reconstruct(p, dm.ReconOpts(max_iters=10), T(K), T(N), T(N), T(N),
                                                       history=T(29), ws=ws),
        "restrict": lambda: _lib.dmcr_restrict(_Shaped((32, 24)), T(16 * 12 + 1)),
        "prolongate": lambda: _lib.dmcr_prolongate(_Shaped((16, 12)), T(32 * 24 - 4)),
        "batched_count": lambda: _lib.dmcr_descriptor_batched([p, q], [T(N)], [T(K), T(Kq)], ws),
        "batched_field": lambda: _lib.dmcr_descriptor_batched([p, q], [T(N), T(Nq // 2)], [T(K), T(Kq)], ws),
        "batched_loss_out": lambda: _lib.dmcr_loss_grad_batched([p, q], dm.LossOpts(), [T(N), T(Nq)], [T(K), T(Kq)],
                                                                T(11), None, ws),
        "noalloc": lambda: _lib.dmcr_descriptor_noalloc(q, T(Nq), T(Kq + 1)),
    }
    with pytest.raises(ValueError):
        calls[call]()


class _Dev:
    def __init__(self, index):
        self.index = index


def test_binding_rejects_tensors_on_another_device(lib, monkeypatch):
    """A tensor on a device other than the current one is rejected on the host: the library
    launches on the current device and would otherwise receive a foreign pointer."""
    import torch
    import paper_2103_09686_gb300 as dm
    from paper_2103_09686_gb300 import _lib
    monkeypatch.setattr(torch.cuda, "current_device", lambda: 0)
    p = dm.Params((32, 24), (4, 3))
    N, K = 32 * 24, dm.dmcr_descriptor_length(p)
    here, there = _FakeCudaTensor(N), _FakeCudaTensor(N)
    here.device, there.device = _Dev(0), _Dev(1)
    desc = _FakeCudaTensor(K)
    desc.device = _Dev(0)
    ws = _FakeCudaTensor(1 << 20)
    ws.device = _Dev(1)
    with pytest.raises(ValueError, match="cuda:1"):
        _lib.dmcr_descriptor(p, there, desc)
    with pytest.raises(ValueError, match="workspace"):
        _lib.dmcr_descriptor(p, here, desc, ws)


class _Shaped(_FakeCudaTensor):
    def __init__(self, shape):
        n = 1
        for s in shape:
            n *= s
        super().__init__(n)
        self.shape = shape

    def dim(self):
        return len(self.shape)


class _RecordingLib:
    """The real library for the host-side queries; every other entry point is recorded
    and answers DMCR_OK without running."""

    HOST = ("dmcr_descriptor_length", "dmcr_workspace_size", "dmcr_batch_workspace_size", "dmcr_last_error")

    def __init__(self, real):
        self.real = real
        self.calls = []

    def __getattr__(self, name):
        if name in self.HOST:
            return getattr(self.real, name)

        def record(*args):
            self.calls.append(name)
            return 0
        return record


def test_binding_passes_correctly_sized_tensors_through(lib, monkeypatch):
    import paper_2103_09686_gb300 as dm
    from paper_2103_09686_gb300 import _lib
    rec = _RecordingLib(lib)
    monkeypatch.setattr(_lib, "load", lambda build_if_missing=False: rec)
    monkeypatch.setattr(_lib, "_stream", lambda stream=None: 0)
    T = _FakeCudaTensor
    p = dm.Params((32, 24), (4, 3), levels=2)
    q = dm.Params((16, 16), (2, 2), phases=2)
    s3 = dm.Params((16, 16), (3, 3), descriptor=dm.DMCR_DESC_S3)
    N, K = 32 * 24, dm.dmcr_descriptor_length(p)
    Nq, Kq = 2 * 256, dm.dmcr_descriptor_length(q)
    N3, K3 = 256, dm.dmcr_descriptor_length(s3)
    ws = T(1 << 20)
    _lib.dmcr_descriptor(p, T(N), T(K), ws)
    _lib.dmcr_descriptor(q, T(Nq), T(Kq), ws)
    _lib.dmcr_descriptor(s3, T(N3), T(K3), ws)
    _lib.dmcr_loss_grad(p, dm.LossOpts(), T(N), T(K), T(6), T(N), None, ws)
    _lib.dmcr_loss_grad(q, dm.LossOpts(), T(Nq), T(Kq), T(6), None, T(Kq), ws)
    _lib.dmcr_descriptor_vjp(s3, T(N3), T(K3), T(N3), ws)
    _lib.dmcr_restrict(_Shaped((32, 24)), T(16 * 12))
    _lib.dmcr_prolongate(_Shaped((4, 6, 8)), T(8 * 12 * 16))
    _lib.dmcr_reconstruct(p, dm.ReconOpts(max_iters=10), T(K), T(N), T(N), T(N), history=T(30), ws=ws)
    _lib.dmcr_reconstruct(q, dm.ReconOpts(max_iters=10), T(Kq), T(Nq), T(Nq), T(Nq), ws=ws)
    _lib.dmcr_adam_step(p, dm.ReconOpts(), T(K), T(N), T(N), T(N), 0, T(6), ws)
    _lib.dmcr_descriptor_noalloc(p, T(N), T(K))
    params = [p, q, s3]
    Ns, Ks = [N, Nq, N3], [K, Kq, K3]
    F = lambda sizes: [T(n) for n in sizes]  # noqa: E731
    _lib.dmcr_descriptor_batched(params, F(Ns), F(Ks), ws)
    _lib.dmcr_loss_grad_batched(params, dm.LossOpts(), F(Ns), F(Ks), T(18), F(Ns), ws)
    _lib.dmcr_descriptor_vjp_batched(params, F(Ns), F(Ks), F(Ns), ws)
    _lib.dmcr_adam_step_batched(params, dm.ReconOpts(), F(Ks), F(Ns), F(Ns), F(Ns), [0, 0, 0], T(18), ws)
    _lib.dmcr_reconstruct_batched(params, dm.ReconOpts(), F(Ks), F(Ns), F(Ns), F(Ns), [0, 0, 0], ws)
    assert rec.calls == ["dmcr_descriptor"] * 3 + ["dmcr_loss_grad"] * 2 + [
        "dmcr_descriptor_vjp", "dmcr_restrict", "dmcr_prolongate", "dmcr_reconstruct", "dmcr_reconstruct",
        "dmcr_adam_step", "dmcr_descriptor_noalloc", "dmcr_descriptor_batched", "dmcr_loss_grad_batched",
        "dmcr_descriptor_vjp_batched", "dmcr_adam_step_batched", "dmcr_reconstruct_batched"]
