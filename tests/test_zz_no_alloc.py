"""The allocation-free forward entry point against the plan-based one and the oracle.

``ptycho_forward_noalloc`` serves callers that cannot allocate device memory while they
run (all memory handed to their own pool at start-up, latency-critical loops, rules that
ban allocation after initialisation).  It keeps its intermediates in one fixed device
array, so these checks call it through the C ABI several times in a row with different
problems (each call reuses the array the previous one left behind) and compare each
result with ``ptycho_forward`` on a plan and with the FP64 oracle, within the intensity
bars of the parity tests.  The problems cover several position batches (more than 32
positions) and the path that splits a position's fields into chunks because they do not
all fit the array (512^2 frames, 16 fields).  The rejection of problems that do not fit
is checked on the host (tests/test_capi_cpu.py).  This file is collected last so that a
run stopping at its first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

from oracle import ptycho_oracle as orc
from synthetic import workloads as syn

pytestmark = pytest.mark.gpu

TOL_I = 1e-5          # relative L2 over all frames
TOL_I_MAX = 1e-5      # per frame: max |error| / max |oracle frame|


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def _max_rel_frames(a, b):
    a = a.reshape(len(a), -1)
    b = b.reshape(len(b), -1)
    return float((np.abs(a - b).max(1) / np.abs(b).max(1)).max())


def _problem(F, L, M, n_side, seed, dev):
    w = syn.tiny_workload(F=F, L=L, M=M, n_side=n_side, step=F // 8, seed=seed, with_sigma=True, with_bg=True)
    from paper_2311_14780_gb300 import pack_objects
    O = pack_objects(w.O0, dev)
    P = torch.as_tensor(w.P0, dtype=torch.complex64, device=dev).contiguous()
    sig = torch.as_tensor(w.sigma, dtype=torch.float32, device=dev).contiguous()
    bg = torch.as_tensor(w.bg, dtype=torch.float32, device=dev).contiguous()
    return w, O, P, sig, bg


def _noalloc(lib, w, O, P, sig, bg, out):
    assert out.numel() == w.J * w.F * w.F           # the output always holds every frame
    h = np.ascontiguousarray([s[0] for s in w.obj_shapes], np.int32)
    wd = np.ascontiguousarray([s[1] for s in w.obj_shapes], np.int32)
    pos = np.ascontiguousarray(w.pos, np.int32)
    ip = ctypes.POINTER(ctypes.c_int32)
    vp = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
    return lib.ptycho_forward_noalloc(w.L, w.M, w.F, w.J, h.ctypes.data_as(ip), wd.ctypes.data_as(ip),
                                      pos.ctypes.data_as(ip), vp(torch.view_as_real(O)),
                                      vp(torch.view_as_real(P)), vp(sig), vp(bg), vp(out),
                                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_noalloc_forward_matches_plan_forward_and_oracle_in_a_row():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2311_14780_gb300 import _native, plan_for
    lib = _native.lib()
    dev = torch.device("cuda", 0)
    # problems back to back; each reuses the array the previous one filled.  (64, 1, 2, 6): 36
    # positions, more than one batch of the array; (512, 4, 4, 2): 16 fields of 2 MB do not fit
    # next to the tables, so each position's fields run in two chunks.
    for (F, L, M, n_side, seed) in ((128, 2, 3, 3, 31), (64, 3, 2, 3, 32), (64, 1, 2, 6, 34), (512, 4, 4, 2, 35)):
        w, O, P, sig, bg = _problem(F, L, M, n_side, seed, dev)
        out = torch.full((w.J, F, F), float("nan"), dtype=torch.float32, device=dev)
        assert _noalloc(lib, w, O, P, sig, bg, out) == 0
        plan = plan_for(w, remap=False)
        ref = plan.forward(O, P, sig, bg)
        torch.cuda.synchronize()
        got, exp = out.cpu().numpy(), ref.cpu().numpy()
        plan.close()
        assert np.isfinite(got).all()
        assert _rel(got, exp) < TOL_I, (F, L, M, n_side)
        O64 = [np.asarray(o).astype(np.complex64).astype(np.complex128) for o in w.O0]
        P64 = np.asarray(w.P0).astype(np.complex64).astype(np.complex128)
        Ir = orc.predict(O64, P64, w.pos, np.asarray(w.sigma, np.float32).astype(np.float64),
                         np.asarray(w.bg, np.float32).astype(np.float64), None)
        assert _rel(got, Ir) < TOL_I, (F, L, M, n_side, _rel(got, Ir))
        assert _max_rel_frames(got, Ir) < TOL_I_MAX, (F, L, M, n_side, _max_rel_frames(got, Ir))
