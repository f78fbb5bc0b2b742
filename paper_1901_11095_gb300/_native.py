"""ctypes binding of libsal.so: the C ABI of include/sal.h, call for call.

Argument marshalling only.  Tensors are torch CUDA tensors (device memory owned by the
caller); every computation happens in the library's CUDA kernels.  There is no CPU
fallback: if libsal.so is missing or fails to load, every call raises.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsal.so")

SAL_OK, SAL_ERR_INVALID_ARG, SAL_ERR_UNSUPPORTED, SAL_ERR_WORKSPACE, SAL_ERR_CUDA, SAL_ERR_TIMEOUT, \
    SAL_ERR_INTERNAL = range(7)
SAL_PREC_FP32, SAL_PREC_TF32, SAL_PREC_BF16 = 0, 1, 2
SAL_BND_REFLECT, SAL_BND_PERIODIC = 0, 1
SAL_STENCIL_26, SAL_STENCIL_LINE, SAL_STENCIL_DIAG_TX = 0, 1, 2
SAL_STENCIL_MAX_OFFSETS, SAL_STENCIL_MAX_RADIUS = 64, 7
SAL_STATS_LEN = 9
SAL_DCS_STATIC_MAX_TILES = 131072
SAL_BATCH_MAX = 128
SAL_SURR_LAYERS, SAL_SURR_WIDTH = 5, 24
SAL_PROBE_CHAINS = 8


class SalDims(ctypes.Structure):
    _fields_ = [("T", ctypes.c_int64), ("X", ctypes.c_int64), ("Y", ctypes.c_int64)]


class SalParams(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int32), ("precision", ctypes.c_int32), ("boundary", ctypes.c_int32),
                ("stencil", ctypes.c_int32), ("sigma", ctypes.c_float), ("stride", ctypes.c_int32),
                ("a", ctypes.c_double), ("b", ctypes.c_double), ("c", ctypes.c_double), ("eps", ctypes.c_double)]


class SalUserStencil(ctypes.Structure):
    _fields_ = [("count", ctypes.c_int32 * 3),
                ("offset", ((ctypes.c_int32 * 3) * SAL_STENCIL_MAX_OFFSETS) * 3),
                ("weight", (ctypes.c_float * SAL_STENCIL_MAX_OFFSETS) * 3)]


class SalVolume(ctypes.Structure):
    _fields_ = [("V", ctypes.c_void_p), ("S", ctypes.c_void_p), ("T", ctypes.c_int64), ("X", ctypes.c_int64),
                ("Y", ctypes.c_int64)]


class SalTileChoice(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int32), ("precision", ctypes.c_int32), ("size_class", ctypes.c_int32),
                ("shape", ctypes.c_int32), ("bt", ctypes.c_int32), ("bx", ctypes.c_int32), ("by", ctypes.c_int32),
                ("mode", ctypes.c_int32), ("ms", ctypes.c_float)]


class SalError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} [status {status}]")
        self.status = status


_lib = None


def lib():
    """The loaded libsal.so (raises if it is not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libsal.so is not built ({LIB_PATH}); run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, sz, i64p = ctypes.c_void_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_int64)
        pp = ctypes.POINTER(SalParams)
        sig = {
            "sal_params_default": [pp],
            "sal_workspace_size": [SalDims, pp, ctypes.POINTER(sz)],
            "sal_dcs_workspace_size": [SalDims, pp, ctypes.POINTER(sz)],
            "sal_local_spectra": [vp, SalDims, pp, i64p, i64p, vp, vp],
            "sal_project": [vp, ctypes.c_int64, ctypes.c_int32, vp, vp],
            "sal_spectral_energy": [vp, SalDims, pp, vp, vp],
            "sal_directional_compare": [vp, SalDims, pp, vp, vp, vp, sz, vp],
            "sal_directional_compare_static": [vp, SalDims, pp, vp, vp, vp],
            "sal_directional_compare_user": [vp, SalDims, pp, ctypes.POINTER(SalUserStencil), vp, vp, vp, sz, vp],
            "sal_lattice_dims": [SalDims, pp, ctypes.POINTER(SalDims)],
            "sal_lattice_energy": [vp, SalDims, pp, vp, vp],
            "sal_interpolate_lattice": [vp, SalDims, pp, vp, vp],
            "sal_slab_halo": [pp, i64p],
            "sal_slab_workspace_size": [ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, pp, ctypes.POINTER(sz)],
            "sal_slab_maps": [vp, SalDims, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, pp, vp, vp,
                              vp, sz, vp],
            "sal_stats_merge": [vp, ctypes.c_int32, vp, vp],
            "sal_combine": [vp, vp, SalDims, pp, vp, vp],
            "sal_saliency": [vp, SalDims, pp, vp, vp, vp, sz, vp],
            "sal_host_workspace_size": [SalDims, pp, ctypes.POINTER(sz)],
            "sal_saliency_host": [vp, SalDims, pp, vp, vp, vp, sz, vp, vp],
            "sal_host_release": [vp],
            "sal_batch_workspace_size": [ctypes.POINTER(SalVolume), ctypes.c_int32, pp, ctypes.POINTER(sz)],
            "sal_saliency_batched": [ctypes.POINTER(SalVolume), ctypes.c_int32, pp, vp, vp, sz, vp],
            "sal_graph_create_batched": [ctypes.POINTER(SalVolume), ctypes.c_int32, pp, vp, vp, sz, vp,
                                         ctypes.POINTER(vp)],
            "sal_graph_launch": [vp, vp],
            "sal_graph_destroy": [vp],
            "sal_autotune": [vp, SalDims, pp, vp, vp, ctypes.POINTER(SalTileChoice)],
            "sal_autotune_batched": [ctypes.POINTER(SalVolume), ctypes.c_int32, pp, vp, sz, vp,
                                     ctypes.POINTER(SalTileChoice)],
            "sal_autotune_query": [ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, ctypes.POINTER(SalTileChoice)],
            "sal_autotune_save": [ctypes.c_char_p],
            "sal_autotune_load": [ctypes.c_char_p],
            "sal_autotune_clear": [],
            "sal_device_status": [vp],
            "sal_surrogate_param_count": [ctypes.POINTER(ctypes.c_int64)],
            "sal_surrogate_workspace_size": [SalDims, ctypes.c_int32, ctypes.POINTER(sz)],
            "sal_surrogate_forward": [vp, SalDims, pp, vp, vp, ctypes.c_int32, vp, sz, vp],
            "sal_surrogate_backward": [vp, SalDims, pp, vp, vp, ctypes.c_int32, vp, vp, vp, sz, vp],
            "sal_surrogate_adam_step": [vp, vp, vp, vp, ctypes.c_int32, ctypes.c_float, ctypes.c_float,
                                        ctypes.c_float, ctypes.c_float, vp],
            "sal_surrogate_infer_workspace_size": [SalDims, pp, ctypes.POINTER(sz)],
            "sal_surrogate_infer": [vp, SalDims, pp, vp, vp, ctypes.c_float, vp, vp, sz, vp],
            "sal_test_stall_tensor_cores": [ctypes.c_int32],
            "sal_probe_fma_rate": [vp, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, vp],
        }
        for name, args in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        L.sal_status_string.argtypes = [ctypes.c_int]
        L.sal_status_string.restype = ctypes.c_char_p
        L.sal_last_error.argtypes = []
        L.sal_last_error.restype = ctypes.c_char_p
        _lib = L
    return _lib


def check(status: int) -> None:
    if status != SAL_OK:
        l = lib()
        raise SalError(status, f"{l.sal_status_string(status).decode()}: {l.sal_last_error().decode()}")


def exported_symbols() -> list[str]:
    return ["sal_params_default", "sal_workspace_size", "sal_dcs_workspace_size", "sal_local_spectra",
            "sal_project", "sal_spectral_energy", "sal_directional_compare", "sal_directional_compare_static",
            "sal_directional_compare_user", "sal_lattice_dims", "sal_lattice_energy", "sal_interpolate_lattice",
            "sal_slab_halo", "sal_slab_workspace_size", "sal_slab_maps",
            "sal_stats_merge", "sal_combine", "sal_saliency", "sal_host_workspace_size", "sal_saliency_host", "sal_host_release",
            "sal_batch_workspace_size", "sal_saliency_batched",
            "sal_graph_create_batched", "sal_graph_launch", "sal_graph_destroy", "sal_autotune",
            "sal_autotune_batched", "sal_autotune_query", "sal_autotune_save", "sal_autotune_load",
            "sal_autotune_clear", "sal_device_status", "sal_test_stall_tensor_cores", "sal_surrogate_param_count",
            "sal_surrogate_workspace_size", "sal_surrogate_forward", "sal_surrogate_backward",
            "sal_surrogate_adam_step", "sal_surrogate_infer_workspace_size", "sal_surrogate_infer",
            "sal_probe_fma_rate", "sal_status_string", "sal_last_error"]
