"""GB300-native differentiable microstructure reconstruction (arXiv 2103.09686).

The compute path is libdmcr.so (hand-written CUDA for sm_103a behind the C ABI of
``include/dmcr.h``); this package is its thin Python binding plus the autograd wrapper.
"""
from ._lib import (  # noqa: F401
    DMCR_DESC_S2, DMCR_DESC_S2_TILDE, DMCR_DESC_S3, DMCR_IDENTITY, DMCR_INIT_CALLER, DMCR_INIT_UNIFORM_SEEDED, DMCR_LOSS_NORM, DMCR_LOSS_SQUARED,
    DMCR_PATH_AUTO, DMCR_PATH_DIRECT, DMCR_PATH_FFT, DMCR_PROLONG_ADJOINT_ACCUMULATE, DMCR_PROLONG_INJECT, DMCR_SOFT,
    OUT_NAMES, DmcrError, LossOpts, Params, ReconOpts, descriptor, descriptor_vjp, dmcr_descriptor,
    dmcr_adam_step, dmcr_descriptor_length, dmcr_descriptor_noalloc, dmcr_descriptor_vjp,
    dmcr_profile_enable, dmcr_profile_read, dmcr_profile_reset, dmcr_init_uniform, dmcr_loss_grad, dmcr_prolongate,
    dmcr_reconstruct, dmcr_restrict, dmcr_version, dmcr_workspace_size, load, loss_grad, workspace,
    batch_workspace, dmcr_adam_step_batched, dmcr_batch_workspace_size, dmcr_descriptor_batched,
    dmcr_descriptor_vjp_batched, dmcr_loss_grad_batched, dmcr_reconstruct_batched,
)
