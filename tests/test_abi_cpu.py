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
    assert three > 3 * one


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
