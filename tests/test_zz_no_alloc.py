"""dmcr_descriptor_noalloc against dmcr_descriptor, through the C ABI.

The allocation-free entry point serves callers that cannot allocate device memory during
the call (host callbacks, real-time loops, deployments that reserve all memory at
start-up); it takes its scratch from one fixed device array in the library.  This file is
collected last on purpose so that a run stopping at its first failure has already run
every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

import synthetic

pytestmark = pytest.mark.gpu

RTOL = 1e-5


def _call_noalloc(dm, p, field, desc):
    from paper_2103_09686_gb300 import _lib
    lib = _lib.load()
    st = lib.dmcr_descriptor_noalloc(ctypes.byref(p.c()), field.data_ptr(), desc.data_ptr(),
                                     torch.cuda.current_stream().cuda_stream)
    return st, lib.dmcr_last_error().decode()


@pytest.mark.parametrize("shape,window,levels", [((64, 64), (16, 16), 1), ((128, 128), (16, 16), 2),
                                                 ((32, 32, 32), (4, 4, 4), 2)])
def test_noalloc_matches_workspace_entry_point_twice(cuda_lib, shape, window, levels):
    dm = cuda_lib
    p = dm.Params(shape=shape, window=window, levels=levels)
    K = dm.dmcr_descriptor_length(p)
    for call, seed in enumerate((11, 12)):            # two calls in a row share the scratch array
        field = torch.tensor(synthetic.uniform_field(shape, seed).astype(np.float32), device="cuda")
        want = dm.descriptor(field, p)
        got = torch.full((K,), float("nan"), device="cuda")
        st, err = _call_noalloc(dm, p, field, got)
        assert st == 0, err
        torch.cuda.synchronize()
        np.testing.assert_allclose(got.cpu().numpy(), want.cpu().numpy(), rtol=RTOL, atol=1e-9,
                                   err_msg="call %d" % call)


def test_noalloc_rejects_problems_beyond_its_scratch(cuda_lib):
    dm = cuda_lib
    # 1024^2 +-64: 1024 forward tiles x 8321 shifts of partial sums alone exceed 16 MiB
    p = dm.Params(shape=(1024, 1024), window=(64, 64), levels=1)
    field = torch.zeros(1024, 1024, device="cuda")
    desc = torch.empty(dm.dmcr_descriptor_length(p), device="cuda")
    st, err = _call_noalloc(dm, p, field, desc)
    assert st == 2 and "scratch" in err
