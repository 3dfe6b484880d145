"""GB300-native (sm_103a) differentiable 3D Gaussian Splatting training step.

The compute lives in libgs.so (include/gs.h); this package binds it:
  _lib      ctypes declarations of the C ABI
  api       torch-facing wrappers with the ABI's names, Plan, Gaussians
  trainer   one full training step (preprocess .. Adam) per call
  autograd  torch.autograd.Function over the forward and backward kernels
  build     nvcc build of libgs.so for sm_103a
"""
from ._lib import GsError, load  # noqa: F401
from .api import (  # noqa: F401
    Gaussians,
    Plan,
    camera_struct,
    gs_adam_step,
    gs_adam_step_multi,
    gs_adam_step_multi_dev,
    gs_bin_sort,
    gs_loss,
    gs_loss_scratch,
    gs_preprocess,
    gs_preprocess_bwd_adam,
    gs_render_bwd,
    gs_render_fwd,
    gs_sort_pairs_u32,
    NgParams,
    gs_ng_decode_bwd,
    gs_ng_decode_fwd,
    gs_ng_workspace,
    ng_children,
)
