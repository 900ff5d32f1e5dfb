"""Seeded synthetic inputs shaped like the paper's EUV reflection-ptychography workloads.

This package builds *inputs only*: objects, probe modes, scan positions, geometry,
masks and the Poisson noise draw applied to a caller-supplied clean intensity.  It
holds none of the forward model, loss, gradient or optimiser arithmetic, so the CPU
oracle (``oracle/``) and the CUDA path (``paper_2311_14780_gb300``) can both consume
it without sharing any of the method's code.
"""
from .workloads import *  # noqa: F401,F403
