"""ctypes view of the C ABI in include/mgauss.h (argument marshalling only).

Loading fails loudly when the built library is missing: there is no fallback
path of any kind.
"""
from __future__ import annotations

import ctypes
import os

from .build import LIB

c_i32, c_i64, c_f32, c_p, c_sz = ctypes.c_int32, ctypes.c_int64, ctypes.c_float, ctypes.c_void_p, ctypes.c_size_t


class MgGaussians(ctypes.Structure):
    _fields_ = [("n", c_i64), ("mean", c_p), ("quat", c_p), ("scale", c_p), ("alpha", c_p)]


class MgStack(ctypes.Structure):
    _fields_ = [("n_slices", c_i32), ("H", c_i32), ("W", c_i32), ("dx", c_f32), ("dy", c_f32),
                ("thickness", c_f32), ("xform", c_p), ("psf_u", c_f32), ("psf_v", c_f32)]


class MgOpts(ctypes.Structure):
    _fields_ = [("cutoff_k", c_f32), ("f64_ratio", c_f32), ("cap_records", c_i64), ("cap_entries", c_i64),
                ("local_set", c_i32), ("grid_res", c_i32), ("block_radius", c_i32), ("grid_centre", c_f32 * 3),
                ("grid_half", c_f32)]


MG_LOCAL_KSIGMA, MG_LOCAL_CELLS = 0, 1


class MgRenderStats(ctypes.Structure):
    _fields_ = [("records", c_i64), ("entries", c_i64), ("tiles", c_i64), ("cap_records", c_i64),
                ("cap_entries", c_i64), ("status", c_i32), ("reserved", c_i32)]


class MgWsLayout(ctypes.Structure):
    _fields_ = [("rec_gid", ctypes.c_uint64), ("rec_slice", ctypes.c_uint64), ("rec_rect", ctypes.c_uint64),
                ("rec_inset", ctypes.c_uint64), ("tile_off", ctypes.c_uint64), ("entries", ctypes.c_uint64),
                ("total_bytes", ctypes.c_uint64)]


class MgNrf(ctypes.Structure):
    _fields_ = [("encoding", c_i32), ("precision", c_i32), ("params", c_p), ("table", c_p), ("log2_table", c_i32),
                ("n_min", c_i32), ("n_max", c_i32), ("out_scale", c_f32), ("enc", c_p), ("enc_mode", c_i32)]


MG_NRF_ENC_NONE, MG_NRF_ENC_STORE, MG_NRF_ENC_LOAD = 0, 1, 2


class MgAdamGroup(ctypes.Structure):
    _fields_ = [("param", c_p), ("grad", c_p), ("m", c_p), ("v", c_p), ("n", c_i64), ("lr", c_f32),
                ("clamp_lo", c_f32), ("clamp_hi", c_f32)]


MG_WS_FAIL_BITS = 0x0F
MG_TILE_EDGE = 8  # edge of the evaluation tiles in pixels
MG_ADAM_MAX_GROUPS = 8

MG_NRF_FOURIER, MG_NRF_GRID = 0, 1
MG_NRF_BF16, MG_NRF_FP32 = 0, 1

MG_OK, MG_ERR_INVALID_ARG, MG_ERR_CUDA, MG_ERR_CAPACITY, MG_ERR_DEVICE_TIMEOUT, MG_ERR_NOT_FINITE, \
    MG_ERR_STALE_WORKSPACE = range(7)

# every symbol include/mgauss.h declares, with (restype, argtypes)
SIGNATURES = {
    "mg_default_opts": (MgOpts, []),
    "mg_render_workspace_size": (c_sz, [ctypes.POINTER(MgGaussians), ctypes.POINTER(MgStack), ctypes.c_int,
                                        ctypes.POINTER(MgOpts)]),
    "mg_render_fwd": (ctypes.c_int, [ctypes.POINTER(MgGaussians), ctypes.POINTER(MgStack), ctypes.c_int,
                                     ctypes.POINTER(MgOpts), c_p, c_p, c_sz, c_p]),
    "mg_render_fwd_l1l2": (ctypes.c_int, [ctypes.POINTER(MgGaussians), ctypes.POINTER(MgStack), ctypes.c_int,
                                          ctypes.POINTER(MgOpts), c_p, c_p, c_p, c_p, c_p, c_sz, c_p]),
    "mg_render_bwd": (ctypes.c_int, [ctypes.POINTER(MgGaussians), ctypes.POINTER(MgStack), ctypes.c_int,
                                     ctypes.POINTER(MgOpts), c_p, c_p, c_p, c_p, c_p, c_p, c_sz, c_p]),
    "mg_render_pose_grad": (ctypes.c_int, [ctypes.POINTER(MgGaussians), ctypes.POINTER(MgStack), ctypes.c_int,
                                           ctypes.POINTER(MgOpts), c_p, c_p, c_sz, c_p]),
    "mg_render_ws_layout": (ctypes.c_int, [ctypes.POINTER(MgGaussians), ctypes.POINTER(MgStack), ctypes.c_int,
                                           ctypes.POINTER(MgOpts), ctypes.POINTER(MgWsLayout)]),
    "mg_sample_ws_layout": (ctypes.c_int, [c_i64, c_i32, ctypes.POINTER(MgOpts), ctypes.POINTER(MgWsLayout)]),
    "mg_render_stats_get": (ctypes.c_int, [c_p, c_sz, ctypes.POINTER(MgRenderStats), c_p]),
    "mg_sample_workspace_size": (c_sz, [c_i64, c_i32, ctypes.POINTER(MgOpts)]),
    "mg_sample_volume": (ctypes.c_int, [ctypes.POINTER(MgGaussians), ctypes.POINTER(c_f32), c_f32, c_i32,
                                        ctypes.POINTER(MgOpts), c_p, c_p, c_sz, c_p]),
    "mg_reduce_workspace_size": (c_sz, [c_i64]),
    "mg_loss_l1l2": (ctypes.c_int, [c_p, c_p, c_i64, c_p, c_p, c_p, c_sz, c_p]),
    "mg_loss_l1l2_noalloc": (ctypes.c_int, [c_p, c_p, c_i64, c_p, c_p, c_p]),
    "mg_sq_diff_sum": (ctypes.c_int, [c_p, c_p, c_i64, c_p, c_p, c_sz, c_p]),
    "mg_loss_recon_workspace_size": (c_sz, [ctypes.POINTER(MgStack), ctypes.c_int]),
    "mg_loss_recon": (ctypes.c_int, [c_p, c_p, ctypes.POINTER(MgStack), ctypes.c_int, c_f32, c_p, c_p, c_p, c_sz,
                                     c_p]),
    "mg_render_pair_count": (ctypes.c_int, [ctypes.POINTER(MgGaussians), ctypes.POINTER(MgStack), ctypes.c_int,
                                            ctypes.POINTER(MgOpts), c_p, c_sz, ctypes.POINTER(c_i64), c_p]),
    "mg_nrf_param_count": (c_i64, [c_i32]),
    "mg_nrf_enc_bytes": (ctypes.c_size_t, [c_p, c_i64]),
    "mg_nrf_fwd": (ctypes.c_int, [ctypes.POINTER(MgNrf), c_p, c_i64, c_p, c_p]),
    "mg_nrf_bwd": (ctypes.c_int, [ctypes.POINTER(MgNrf), c_p, c_i64, c_p, c_p, c_p, c_p]),
    "mg_nrf_fwd_at": (ctypes.c_int, [ctypes.POINTER(MgNrf), c_p, c_i64, c_p, c_i64, c_p, c_p]),
    "mg_nrf_bwd_at": (ctypes.c_int, [ctypes.POINTER(MgNrf), c_p, c_i64, c_p, c_i64, c_p, c_p, c_p, c_p]),
    "mg_adam_step": (ctypes.c_int, [ctypes.POINTER(MgAdamGroup), ctypes.c_int, c_f32, c_f32, c_f32, c_p, c_p,
                                    ctypes.c_uint32, c_p]),
    "mg_params_workspace_size": (c_sz, [c_i64]),
    "mg_params_fwd": (ctypes.c_int, [c_i64, c_p, c_p, c_p, ctypes.POINTER(c_f32), c_f32, c_f32, c_p, c_p, c_p, c_p,
                                     c_p, c_sz, c_p]),
    "mg_params_bwd": (ctypes.c_int, [c_i64, c_p, c_p, c_f32, c_f32, c_f32, c_p, c_p, c_p, c_p, c_p, c_p, c_p]),
    "mg_profile_enable": (ctypes.c_int, [ctypes.c_int]),
    "mg_profile_stages": (ctypes.c_int, [ctypes.c_uint32]),
    "mg_profile_stage_count": (ctypes.c_int, []),
    "mg_profile_stage_name": (ctypes.c_char_p, [ctypes.c_int]),
    "mg_profile_read": (ctypes.c_int, [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(c_i64), ctypes.c_int]),
    "mg_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "mg_last_error": (ctypes.c_char_p, []),
    "mg_version": (ctypes.c_char_p, []),
}

_lib = None


def lib():
    """The loaded library (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise ImportError(f"mgauss CUDA library not built: {LIB} is missing "
                              "(run `python -m paper_2603_00145_b300.build`)")
        L = ctypes.CDLL(LIB)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class MgError(RuntimeError):
    def __init__(self, status: int, where: str):
        L = lib()
        msg = L.mg_last_error().decode(errors="replace")
        super().__init__(f"{where}: {L.mg_status_string(status).decode()} ({status}): {msg}")
        self.status = status


def check(status: int, where: str):
    if status != MG_OK:
        raise MgError(status, where)
