"""Data-side tilt correction on the GPU (ptycho_tilt_correct) vs the FP64 oracle.

The camera index is evaluated in FP64 on both sides with the same sequence of separately
rounded operations, so the masks (floor, range and threshold decisions) must agree bit for
bit.  The interpolated values are FP32 sums of four FP32 taps with FP32 weights on the GPU
and FP64 in the oracle: they agree to a few FP32 roundings of the pattern's scale.
"""
import math

import numpy as np
import pytest
import torch

from oracle import ptycho_oracle as orc
from synthetic import workloads as syn

pytestmark = pytest.mark.gpu

Z, P = syn.PAPER_Z, syn.PAPER_DET_PIXEL


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2311_14780_gb300 import _native
    _native.lib()
    return torch.device("cuda", 0)


def run_gpu(I_cam, dev, z, tilt, lo=-math.inf, hi=math.inf):
    from paper_2311_14780_gb300 import tilt_correct
    out, mask = tilt_correct(torch.as_tensor(I_cam, device=dev), z, P, tilt, lo, hi)
    torch.cuda.synchronize()
    return out.cpu().numpy(), mask.cpu().numpy()


def check(I_cam, out, mask, z, tilt, lo=-math.inf, hi=math.inf):
    ref, mref = orc.tilt_correct(I_cam, z, P, tilt, lo, hi)
    assert (mask.astype(bool) == mref).all(), f"{int((mask.astype(bool) != mref).sum())} mask pixels differ"
    scale = max(float(np.abs(ref).max()), 1e-30)
    err = np.abs(out.astype(np.float64) - ref)
    assert err.max() <= 4e-7 * scale + 1e-30, err.max() / scale
    assert (out[~mref] == 0).all()
    return ref, mref


@pytest.mark.parametrize("F,J,z,tilt_deg", [(64, 1, 0.02, 70.0), (64, 37, 0.02, 70.0), (100, 7, 0.03, 70.0),
                                            (256, 13, Z, 70.0), (128, 5, 0.05, -35.0), (96, 3, Z, 0.0),
                                            (2, 2, 1e-3, 10.0)])
def test_tilt_correct_matches_the_oracle(dev, F, J, z, tilt_deg):
    """Several pixel blocks with a ragged last one (F^2 not a multiple of 64), ragged frame
    chunks, no tilt, negative tilt, and the smallest grid."""
    I_cam = syn.camera_frames(J, F, seed=F + J)
    out, mask = run_gpu(I_cam, dev, z, math.radians(tilt_deg))
    ref, mref = check(I_cam, out, mask, z, math.radians(tilt_deg))
    if F > 2:
        assert mref.any() and (tilt_deg == 0.0 or not mref.all())


@pytest.mark.parametrize("F,J", [(64, 9), (256, 6)])
def test_tilt_correct_thresholds_match_the_oracle(dev, F, J):
    """The paper's thresholds (4 <= v < 65535): saturated specular pixels and the dark halo
    remove the model pixels whose taps touch them; exact values at the thresholds included."""
    I_cam = syn.camera_frames(J, F, seed=5 * F + J)
    I_cam[0, F // 2 + 3, F // 2 - 5] = 4.0
    I_cam[1, F // 3, F // 4] = 65535.0
    out, mask = run_gpu(I_cam, dev, Z, syn.PAPER_TILT, 4.0, 65535.0)
    ref, mref = check(I_cam, out, mask, Z, syn.PAPER_TILT, 4.0, 65535.0)
    fov = orc.tilt_correct(I_cam[:1], Z, P, syn.PAPER_TILT)[1][0]
    assert (mref.sum(axis=(1, 2)) < fov.sum()).all()


def test_tilt_correct_full_size_camera_stack_sampled_frames(dev):
    """400 camera frames of 256^2 (the configuration-2 scan), one launch; sampled frames
    (first, last, and three in between) against the oracle."""
    J, F = 400, 256
    I_cam = syn.camera_frames(J, F, seed=2)
    out, mask = run_gpu(I_cam, dev, Z, syn.PAPER_TILT, 4.0, 65535.0)
    for j in (0, 1, 137, 398, 399):
        check(I_cam[j:j + 1], out[j:j + 1], mask[j:j + 1], Z, syn.PAPER_TILT, 4.0, 65535.0)


def test_tilt_table_and_apply_match_the_one_shot_correction(dev):
    """A table built once serves several stacks (different J, ragged chunks) and gives the
    one-shot call's result bit for bit."""
    from paper_2311_14780_gb300 import tilt_apply, tilt_correct, tilt_table
    F, z, t = 128, 0.05, syn.PAPER_TILT
    table = tilt_table(F, z, P, t, device=dev)
    for J, seed in ((1, 1), (17, 2), (40, 3)):
        I_cam = torch.as_tensor(syn.camera_frames(J, F, seed=seed), device=dev)
        a_out, a_mask = tilt_apply(table, I_cam, 4.0, 65535.0)
        c_out, c_mask = tilt_correct(I_cam, z, P, t, 4.0, 65535.0)
        torch.cuda.synchronize()
        assert torch.equal(a_out, c_out) and torch.equal(a_mask, c_mask)
    ref, mref = orc.tilt_correct(I_cam.cpu().numpy()[-3:], z, P, t, 4.0, 65535.0)
    assert (a_mask.cpu().numpy()[-3:].astype(bool) == mref).all()


def test_tilt_correct_without_mask_and_empty_stack(dev):
    from paper_2311_14780_gb300 import tilt_correct
    I_cam = syn.camera_frames(3, 64, seed=9)
    out, m = tilt_correct(torch.as_tensor(I_cam, device=dev), 0.02, P, 1.2, with_mask=False)
    assert m is None
    ref, _ = orc.tilt_correct(I_cam, 0.02, P, 1.2)
    assert np.abs(out.cpu().numpy() - ref).max() <= 4e-7 * np.abs(ref).max()
    e_out, e_m = tilt_correct(torch.empty((0, 64, 64), device=dev), 0.02, P, 1.2)
    assert e_out.shape == (0, 64, 64) and e_m.shape == (0, 64, 64)
    with pytest.raises(Exception):
        tilt_correct(torch.as_tensor(I_cam, device=dev), 0.02, P, 1.2, lo=5.0, hi=5.0)


def test_reconstruction_on_tilt_corrected_data_matches_the_oracle(dev):
    """The paper's preprocessing flow: correct the camera data once (GPU), then evaluate the
    loss and gradients with a plan without the in-model remap and the per-frame mask; the
    oracle does the same with its own correction."""
    from paper_2311_14780_gb300 import pack_objects, plan_for
    w = syn.tiny_workload(F=64, L=2, M=2, n_side=3, step=12, seed=3, remap=True, loss="poisson")
    taps = orc.remap_taps(w.F, w.geom.z, w.geom.det_pixel, w.geom.tilt_rad)
    Ih = syn.poisson_measure(orc.predict(w.O_true, w.P_true, w.pos, taps=taps), 11)
    I_mod, m_mod = orc.tilt_correct(Ih, w.geom.z, w.geom.det_pixel, w.geom.tilt_rad)
    eps = syn.default_eps(Ih)
    from paper_2311_14780_gb300 import tilt_correct
    Ig, mg = tilt_correct(torch.as_tensor(Ih, dtype=torch.float32, device=dev), w.geom.z, w.geom.det_pixel,
                          w.geom.tilt_rad)
    assert (mg.cpu().numpy().astype(bool) == m_mod).all()
    plan = plan_for(w, eps=eps, remap=False)
    O0 = [np.asarray(o).astype(np.complex64).astype(np.complex128) for o in w.O0]
    P0 = np.asarray(w.P0).astype(np.complex64).astype(np.complex128)
    O = pack_objects(O0, dev)
    Pt = torch.as_tensor(P0, dtype=torch.complex64, device=dev).contiguous()
    loss, gO, gP = plan.adjoint(O, Pt, Ig, mask=mg)
    I_ref = I_mod.astype(np.float32).astype(np.float64)      # the oracle's own correction, stored as FP32
    Lr, gOr, gPr = orc.gradient(O0, P0, w.pos, I_ref, "poisson", eps, None, None, m_mod.astype(np.uint8), None)
    gOr_flat = np.concatenate([g.reshape(-1) for g in gOr])
    assert abs(float(loss.item()) - Lr) <= 1e-5 * abs(Lr)
    assert np.linalg.norm(gO.cpu().numpy() - gOr_flat) <= 1e-4 * np.linalg.norm(gOr_flat)
    assert np.linalg.norm(gP.cpu().numpy() - gPr) <= 1e-4 * np.linalg.norm(gPr)
    plan.close()
