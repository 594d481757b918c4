"""B300-native (sm_103a) Magnetic Gaussian slice renderer: the hot path of
M-Gaussian (arxiv 2603.00145) as a C-ABI CUDA library with a thin torch binding.

Submodules: ``ops`` (binding with the C entry-point names, SliceRenderer,
RenderSlices autograd Function, VolumeSampler), ``build`` (nvcc build of
``_lib/libmgauss.so``), ``_lib`` (ctypes signatures).
"""
from .ops import (NRF, NRFFunction, mg_nrf_bwd, mg_nrf_bwd_at, mg_nrf_fwd, mg_nrf_fwd_at, mg_nrf_param_count, DeviceStacks, RenderSlices, SliceRenderer, VolumeSampler, mg_loss_l1l2, mg_reduce_workspace_size,
                  mg_render_bwd, mg_render_fwd, mg_render_stats_get, mg_render_workspace_size, mg_sample_volume,
                  mg_sample_workspace_size, mg_sq_diff_sum, mg_version, render_slices)

__all__ = ["NRF", "NRFFunction", "mg_nrf_bwd", "mg_nrf_bwd_at", "mg_nrf_fwd", "mg_nrf_fwd_at", "mg_nrf_param_count", "DeviceStacks", "RenderSlices", "SliceRenderer", "VolumeSampler", "mg_loss_l1l2",
           "mg_reduce_workspace_size", "mg_render_bwd", "mg_render_fwd", "mg_render_stats_get",
           "mg_render_workspace_size", "mg_sample_volume", "mg_sample_workspace_size", "mg_sq_diff_sum", "mg_version",
           "render_slices"]
