"""The allocation-free forward entry point against the plan-based one.

``ptycho_forward_noalloc`` serves callers that cannot allocate device memory while they
run (all memory handed to their own pool at start-up, latency-critical loops, rules that
ban allocation after initialisation).  It keeps its intermediates in one fixed device
array, so these checks call it through the C ABI twice in a row with different problems
(the second call reuses the array the first one left behind) and compare each result
with ``ptycho_forward`` on a plan, within the intensity tolerance of the parity tests.
This file is collected last so that a run stopping at its first failure has already run
every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

from synthetic import workloads as syn

pytestmark = pytest.mark.gpu

TOL_I = 1e-5


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def _problem(F, L, M, seed, dev):
    w = syn.tiny_workload(F=F, L=L, M=M, n_side=3, step=F // 8, seed=seed, with_sigma=True, with_bg=True)
    from paper_2311_14780_gb300 import pack_objects
    O = pack_objects(w.O0, dev)
    P = torch.as_tensor(w.P0, dtype=torch.complex64, device=dev).contiguous()
    sig = torch.as_tensor(w.sigma, dtype=torch.float32, device=dev).contiguous()
    bg = torch.as_tensor(w.bg, dtype=torch.float32, device=dev).contiguous()
    return w, O, P, sig, bg


def _noalloc(lib, w, O, P, sig, bg, out):
    h = np.ascontiguousarray([s[0] for s in w.obj_shapes], np.int32)
    wd = np.ascontiguousarray([s[1] for s in w.obj_shapes], np.int32)
    pos = np.ascontiguousarray(w.pos, np.int32)
    ip = ctypes.POINTER(ctypes.c_int32)
    vp = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
    return lib.ptycho_forward_noalloc(w.L, w.M, w.F, w.J, h.ctypes.data_as(ip), wd.ctypes.data_as(ip),
                                      pos.ctypes.data_as(ip), vp(torch.view_as_real(O)),
                                      vp(torch.view_as_real(P)), vp(sig), vp(bg), vp(out),
                                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_noalloc_forward_matches_plan_forward_twice_in_a_row():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2311_14780_gb300 import _native, plan_for
    lib = _native.lib()
    dev = torch.device("cuda", 0)
    # two different problems back to back; the second reuses the array the first filled
    for (F, L, M, seed) in ((128, 2, 3, 31), (64, 3, 2, 32)):
        w, O, P, sig, bg = _problem(F, L, M, seed, dev)
        out = torch.full((w.J, F, F), float("nan"), dtype=torch.float32, device=dev)
        assert _noalloc(lib, w, O, P, sig, bg, out) == 0
        plan = plan_for(w, remap=False)
        ref = plan.forward(O, P, sig, bg)
        torch.cuda.synchronize()
        got, exp = out.cpu().numpy(), ref.cpu().numpy()
        assert np.isfinite(got).all()
        assert _rel(got, exp) < TOL_I
        plan.close()


def test_noalloc_rejects_bad_sizes_with_clear_errors():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2311_14780_gb300 import _native
    lib = _native.lib()
    dev = torch.device("cuda", 0)
    w, O, P, sig, bg = _problem(64, 1, 1, 33, dev)
    out = torch.empty((w.J, 64, 64), dtype=torch.float32, device=dev)
    w.F = 100
    assert _noalloc(lib, w, O, P, sig, bg, out) == -6
    w.F = 64
    w.J = 3_000_000            # position tables alone exceed the fixed array
    w.pos = np.zeros((w.L, w.J, 2), np.int32)
    assert _noalloc(lib, w, O, P, sig, bg, out) == -7
    assert b"fixed array" in lib.ptycho_strerror(-7)
