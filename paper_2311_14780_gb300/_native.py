"""ctypes declarations of the C ABI in ``include/ptycho.h``.

Loading never falls back to anything: if the CUDA library has not been built, every
entry point raises.  Build it with ``__graft_entry__.build()`` or
``python paper_2311_14780_gb300/build.py``.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

c_int32_p = ctypes.POINTER(ctypes.c_int32)
c_double_p = ctypes.POINTER(ctypes.c_double)


class Geom(ctypes.Structure):
    _fields_ = [
        ("L", ctypes.c_int32), ("M", ctypes.c_int32), ("F", ctypes.c_int32), ("J", ctypes.c_int32),
        ("obj_h", c_int32_p), ("obj_w", c_int32_p), ("pos", c_int32_p), ("lam", c_double_p),
        ("z", ctypes.c_double), ("det_pixel", ctypes.c_double), ("tilt_rad", ctypes.c_double),
        ("remap", ctypes.c_int32), ("loss", ctypes.c_int32), ("eps", ctypes.c_float),
        ("scratch_bytes", ctypes.c_int64), ("overlap", ctypes.c_int32), ("flags", ctypes.c_int32),
        ("col_groups", ctypes.c_int32),
        ("read_noise_var", ctypes.c_float),
        ("zoom", ctypes.POINTER(ctypes.c_double)),
    ]


class Adam(ctypes.Structure):
    _fields_ = [
        ("lr_O", ctypes.c_float), ("lr_P", ctypes.c_float), ("beta1", ctypes.c_float),
        ("beta2", ctypes.c_float), ("eps", ctypes.c_float), ("t", ctypes.c_int32),
        ("mO", ctypes.c_void_p), ("vO", ctypes.c_void_p), ("mP", ctypes.c_void_p), ("vP", ctypes.c_void_p),
        ("t_dev", ctypes.c_void_p),
        ("lr_sigma", ctypes.c_float), ("lr_bg", ctypes.c_float),
        ("m_sigma", ctypes.c_void_p), ("v_sigma", ctypes.c_void_p), ("m_bg", ctypes.c_void_p),
        ("v_bg", ctypes.c_void_p),
        ("lr_delta", ctypes.c_float), ("m_delta", ctypes.c_void_p), ("v_delta", ctypes.c_void_p),
        ("g_z", ctypes.c_void_p),
        ("reg_l1", ctypes.c_float), ("reg_tv", ctypes.c_float), ("reg_eta", ctypes.c_float),
    ]


class Site(ctypes.Structure):
    _fields_ = [
        ("O", ctypes.c_void_p), ("P", ctypes.c_void_p), ("I_meas", ctypes.c_void_p), ("mask", ctypes.c_void_p),
        ("mask_per_frame", ctypes.c_int32), ("sigma", ctypes.c_void_p), ("bg", ctypes.c_void_p),
        ("lr_O", ctypes.c_float), ("lr_P", ctypes.c_float), ("beta1", ctypes.c_float), ("beta2", ctypes.c_float),
        ("eps", ctypes.c_float), ("iterations", ctypes.c_int32),
    ]


# (name, restype, argtypes) of every exported entry point
_VP = ctypes.c_void_p
_I = ctypes.c_int
SIGNATURES = [
    ("ptycho_plan_create", _I, [ctypes.POINTER(Geom), ctypes.POINTER(_VP)]),
    ("ptycho_plan_destroy", _I, [_VP]),
    ("ptycho_plan_workspace_bytes", ctypes.c_int64, [_VP]),
    ("ptycho_plan_numel_O", ctypes.c_int64, [_VP]),
    ("ptycho_plan_numel_P", ctypes.c_int64, [_VP]),
    ("ptycho_plan_last_launches", ctypes.c_int64, [_VP]),
    ("ptycho_forward", _I, [_VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    ("ptycho_loss", _I, [_VP, _VP, _VP, _VP, _VP, _VP, _VP, _I, _VP, _I, _VP, _VP]),
    ("ptycho_adjoint", _I, [_VP, _VP, _VP, _VP, _VP, _VP, _VP, _I, _VP, _I, _VP, _VP, _VP, _VP]),
    ("ptycho_adjoint_ex", _I, [_VP, _VP, _VP, _VP, _VP, _VP, _VP, _I, _VP, _I, _VP, _VP, _VP, _VP, _VP, _VP, _VP,
                               _VP]),
    ("ptycho_plan_set_distance", _I, [_VP, ctypes.c_double]),
    ("ptycho_plan_set_offsets", _I, [_VP, _VP]),
    ("ptycho_step", _I, [_VP, ctypes.POINTER(Adam), _VP, _VP, _VP, _VP, _VP, _VP, _I, _VP, _I, _VP, _VP]),
    ("ptycho_step_host", _I, [_VP, ctypes.POINTER(Adam), _VP, _VP, _VP, _VP, _VP, _VP, _VP, _I, _VP, _I, _VP, _VP,
                              _VP]),
    ("ptycho_plan_status", _I, [_VP, c_int32_p]),
    ("ptycho_plan_profile", _I, [_VP, _I]),
    ("ptycho_plan_profile_read", _I, [_VP, c_double_p, ctypes.POINTER(ctypes.c_int64)]),
    ("ptycho_kernel_name", ctypes.c_char_p, [_I]),
    ("ptycho_forward_noalloc", _I, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, c_int32_p,
                                    c_int32_p, c_int32_p, _VP, _VP, _VP, _VP, _VP, _VP]),
    ("ptycho_plain_step", _I, [_VP, ctypes.POINTER(Adam), _VP, _VP, _VP, _VP, _VP, _VP, _I, _VP, _VP]),
    ("ptycho_server_create", _I, [ctypes.c_int64, ctypes.c_int32, ctypes.POINTER(_VP)]),
    ("ptycho_server_set_mode", _I, [_VP, ctypes.c_int32]),
    ("ptycho_server_destroy", _I, [_VP]),
    ("ptycho_server_admit", _I, [_VP, ctypes.POINTER(Geom), ctypes.POINTER(Site), c_int32_p]),
    ("ptycho_server_tick", _I, [_VP, _VP, c_int32_p]),
    ("ptycho_server_site_status", _I, [_VP, ctypes.c_int32, c_int32_p, c_double_p]),
    ("ptycho_server_release", _I, [_VP, ctypes.c_int32]),
    ("ptycho_server_used_bytes", ctypes.c_int64, [_VP]),
    ("ptycho_tilt_correct", _I, [ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                 _VP, ctypes.c_float, ctypes.c_float, _VP, _VP, _VP]),
    ("ptycho_regularise", _I, [_VP, _VP, ctypes.c_float, ctypes.c_float, ctypes.c_float, _VP, _VP, _VP]),
    ("ptycho_tilt_table_bytes", ctypes.c_int64, [ctypes.c_int32]),
    ("ptycho_tilt_table", _I, [ctypes.c_int32, ctypes.c_double, ctypes.c_double, ctypes.c_double, _VP, _VP]),
    ("ptycho_tilt_apply", _I, [ctypes.c_int32, ctypes.c_int64, _VP, _VP, ctypes.c_float, ctypes.c_float, _VP, _VP,
                               _VP]),
    ("ptycho_strerror", ctypes.c_char_p, [_I]),
]

NUM_KERNELS = 13
_LIB = None


def lib_path() -> str:
    return _build.lib_path()


def lib() -> ctypes.CDLL:
    """The loaded CUDA library (raises if it has not been built)."""
    global _LIB
    if _LIB is None:
        path = lib_path()
        if not os.path.exists(path):
            raise RuntimeError(
                f"CUDA library {path} is missing: build it with __graft_entry__.build(); "
                "there is no CPU fallback")
        h = ctypes.CDLL(path)
        for name, res, args in SIGNATURES:
            fn = getattr(h, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = h
    return _LIB
