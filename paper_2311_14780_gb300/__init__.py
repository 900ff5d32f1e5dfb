"""GB300-native multi-wavelength, multi-mode ptychography hot path (arXiv 2311.14780).

The compute path is the CUDA library ``_lib/libptycho_gb300.so`` (C ABI in
``include/ptycho.h``); Python only marshals arguments.  Importing this package does not
load the library; the first compute call does, and raises if it has not been built.
"""
from .api import (AdamState, Plan, PtychoError, pack_objects, plan_for, tilt_apply, tilt_correct,  # noqa: F401
                  tilt_table, unpack_objects)

__all__ = ["Plan", "AdamState", "PtychoError", "pack_objects", "unpack_objects", "plan_for", "tilt_correct",
           "tilt_table", "tilt_apply"]
