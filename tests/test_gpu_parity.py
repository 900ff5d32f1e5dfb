"""GPU path vs the FP64 oracle on the same seeded inputs.

Bars (from the stated accuracy targets): relative L2 <= 1e-5 on predicted intensities
and on the loss, <= 1e-4 on the gradients.  Beside every L2 bar sits an element-wise
bar with the same number in the max norm: no pixel of a predicted frame may differ from
the oracle by more than 1e-5 of that frame's largest value, and no element of a gradient
array by more than 1e-4 of the array's largest magnitude.  Evaluating the oracle's own
steps in complex64 (numpy keeps complex64 FFTs in single precision) departs from FP64 by
at most 2.1e-7 (intensities, per frame) and 5.3e-6 (gradients) in that norm on configs
1, 2 and the 128^2 x 8 modes x 5 wavelengths sweep point, so both element-wise bars sit
20-50x above the precision floor.  Inputs are complex64 on the GPU and the same values
in FP64 for the oracle.
"""
import math

import numpy as np
import pytest
import torch

from oracle import ptycho_oracle as orc
from synthetic import workloads as syn

pytestmark = pytest.mark.gpu

TOL_I = 1e-5
TOL_L = 1e-5
TOL_G = 1e-4
TOL_I_MAX = 1e-5      # per frame: max |GPU - oracle| / max |oracle frame|
TOL_G_MAX = 1e-4      # per array: max |GPU - oracle| / max |oracle|


def rel(a, b):
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def max_rel(a, b):
    """Largest element-wise deviation relative to the largest reference magnitude."""
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def max_rel_frames(a, b):
    """max_rel taken frame by frame ([J, F, F] stacks); the worst frame."""
    a = np.asarray(a).reshape(len(a), -1)
    b = np.asarray(b).reshape(len(b), -1)
    return float((np.abs(a - b).max(1) / np.maximum(np.abs(b).max(1), 1e-300)).max())


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2311_14780_gb300 import _native
    _native.lib()
    return torch.device("cuda", 0)


def c64(x, dev):
    return torch.as_tensor(np.asarray(x), dtype=torch.complex64, device=dev).contiguous()


def f32(x, dev):
    return None if x is None else torch.as_tensor(np.asarray(x), dtype=torch.float32, device=dev).contiguous()


def as_c64_roundtrip(x):
    """The values the GPU actually sees (complex64), back in FP64 for the oracle."""
    return np.asarray(x).astype(np.complex64).astype(np.complex128)


class Case:
    """A workload with its remap geometry, measured data and GPU tensors."""

    def __init__(self, w, dev, z=None, loss=None, mask_kind=None, seed=0):
        from paper_2311_14780_gb300 import pack_objects
        self.w = w
        self.loss = loss or w.loss
        self.z = z if z is not None else w.geom.z
        self.taps = orc.remap_taps(w.F, self.z, w.geom.det_pixel, w.geom.tilt_rad) if w.geom.remap else None
        self.O0 = [as_c64_roundtrip(o) for o in w.O0]
        self.P0 = as_c64_roundtrip(w.P0)
        self.sigma = None if w.sigma is None else np.asarray(w.sigma, np.float32).astype(np.float64)
        self.bg = None if w.bg is None else np.asarray(w.bg, np.float32).astype(np.float64)
        clean = orc.predict(w.O_true, w.P_true, w.pos, w.sigma, w.bg, self.taps)
        self.Ih = syn.poisson_measure(clean, 100 + seed)
        self.eps = syn.default_eps(self.Ih)
        rng = np.random.default_rng(seed)
        self.mask = None
        if mask_kind == "shared":
            self.mask = (rng.uniform(size=(w.F, w.F)) > 0.1).astype(np.uint8)
        elif mask_kind == "frame":
            self.mask = (rng.uniform(size=(w.J, w.F, w.F)) > 0.1).astype(np.uint8)
        self.O = pack_objects(self.O0, dev)
        self.P = c64(self.P0, dev)
        self.sig_t = f32(self.sigma, dev)
        self.bg_t = f32(self.bg, dev)
        self.Im = torch.as_tensor(self.Ih, device=dev).contiguous()
        self.mask_t = None if self.mask is None else torch.as_tensor(self.mask, device=dev).contiguous()
        self.dev = dev

    def plan(self, **kw):
        from paper_2311_14780_gb300 import plan_for
        return plan_for(self.w, loss=self.loss, eps=self.eps, z=self.z, **kw)

    def oracle_grad(self, frames=None):
        return orc.gradient(self.O0, self.P0, self.w.pos, self.Ih, self.loss, self.eps, self.sigma, self.bg,
                            self.mask, self.taps, frames)


def check_all(case, plan, frames=None):
    w = case.w
    batch = None if frames is None else torch.as_tensor(np.asarray(frames, np.int32), device=case.dev)
    # forward
    Ip = plan.forward(case.O, case.P, case.sig_t, case.bg_t).cpu().numpy()
    Ir = orc.predict(case.O0, case.P0, w.pos, case.sigma, case.bg, case.taps)
    e_I = rel(Ip, Ir)
    # loss
    Lg = float(plan.loss(case.O, case.P, case.Im, case.sig_t, case.bg_t, case.mask_t, batch).item())
    # adjoint
    La, gO, gP = plan.adjoint(case.O, case.P, case.Im, case.sig_t, case.bg_t, case.mask_t, batch)
    Lr, gOr, gPr = case.oracle_grad(frames)
    gOr = np.concatenate([g.reshape(-1) for g in gOr])
    gO, gP = gO.cpu().numpy(), gP.cpu().numpy()
    out = dict(I=e_I, L=abs(Lg - Lr) / abs(Lr), La=abs(float(La.item()) - Lr) / abs(Lr),
               gO=rel(gO, gOr), gP=rel(gP, gPr), I_max=max_rel_frames(Ip, Ir), gO_max=max_rel(gO, gOr),
               gP_max=max_rel(gP, gPr), status=plan.status())
    return out


def assert_ok(err):
    assert err.get("status", 0) == 0, err          # no bad index, no timed-out bulk copy
    assert err["I"] < TOL_I, err
    assert err["L"] < TOL_L and err["La"] < TOL_L, err
    assert err["gO"] < TOL_G and err["gP"] < TOL_G, err
    assert err["I_max"] < TOL_I_MAX, err
    assert err["gO_max"] < TOL_G_MAX and err["gP_max"] < TOL_G_MAX, err


# z chosen so that the remap visibly distorts small frames (F p / z ~ 0.5)
def strong_z(F):
    return F * 15e-6 / 0.5


@pytest.mark.parametrize("flags", [0, 32, 2048, 4096, 8192, 16384, 32768, 65536])
def test_fused_row_adjoint_at_512_with_eight_modes(dev, flags):
    """F = 512 with 8 modes takes the fused row passes (all modes of a wavelength per block:
    forward rows with the probe row in registers, 16 threads per row; adjoint rows with one warp
    per row, the object-gradient rows summed over the modes in shared memory and the probe rows
    through L1/L2); flag 32 forces the per-mode row adjoint, 2048 the 16-thread adjoint rows with
    the probe rows through L1/L2, 4096 the 16-thread adjoint rows that hold the probe rows in
    shared memory, 8192 the per-position forward row pass, 16384 16 threads per row in both fused
    passes, 32768 one warp per row in the forward too, 65536 the one-block TMA column passes (full
    exchange area, staged dL/dI factors).  Several position batches and splits."""
    w = syn.tiny_workload(F=512, L=1, M=8, n_side=3, step=64, seed=77, remap=True, loss="poisson",
                          with_sigma=True, with_bg=True)
    case = Case(w, dev, z=strong_z(512), mask_kind="frame", seed=12)
    plan = case.plan(flags=flags, scratch_bytes=3 * 8 * 512 * 512 * 8)
    assert_ok(check_all(case, plan))
    assert_ok(check_all(case, plan, frames=[7, 0, 4]))
    plan.close()


def test_row_adjoint_one_warp_per_row_ten_modes_two_wavelengths(dev):
    """The one-warp-per-row adjoint at 512^2 with the full block of 10 modes (320 threads), two
    wavelengths, a ragged last batch, against the oracle and against the 16-thread row adjoint
    (same arithmetic in another order: equal to rounding)."""
    w = syn.tiny_workload(F=512, L=2, M=10, n_side=3, step=64, seed=78, remap=True, loss="poisson",
                          with_sigma=True, with_bg=True)
    case = Case(w, dev, z=strong_z(512), mask_kind="frame", seed=15)
    sb = 4 * 20 * 512 * 512 * 8                           # 4 positions per batch: 4 + 4 + 1
    plan_w = case.plan(scratch_bytes=sb)
    assert_ok(check_all(case, plan_w))
    plan_d = case.plan(flags=2048, scratch_bytes=sb)
    La, gO, gP = plan_w.adjoint(case.O, case.P, case.Im, case.sig_t, case.bg_t, case.mask_t)
    Lb, gOb, gPb = plan_d.adjoint(case.O, case.P, case.Im, case.sig_t, case.bg_t, case.mask_t)
    assert max_rel(gO.cpu().numpy(), gOb.cpu().numpy()) < TOL_G_MAX
    assert max_rel(gP.cpu().numpy(), gPb.cpu().numpy()) < TOL_G_MAX
    assert plan_w.status() == 0
    plan_w.close()
    plan_d.close()


@pytest.mark.parametrize("M", [4, 5])
@pytest.mark.parametrize("flags", [0, 32768])
def test_fused_forward_rows_at_512_with_four_and_five_modes(dev, M, flags):
    """From 4 modes at 512^2 the forward row pass takes all modes of a wavelength per block, 16
    threads per row, or with 32768 one warp per row (two rows of 4 modes per block: 256 threads;
    one row of 5 modes: 160).  Two wavelengths, several position batches."""
    w = syn.tiny_workload(F=512, L=2, M=M, n_side=3, step=64, seed=90 + M, remap=True, loss="poisson",
                          with_sigma=True, with_bg=True)
    case = Case(w, dev, z=strong_z(512), mask_kind="frame", seed=M + flags)
    plan = case.plan(flags=flags, scratch_bytes=4 * 2 * M * 512 * 512 * 8)
    assert_ok(check_all(case, plan))
    plan.close()


def test_row_adjoint_one_warp_per_row_with_offsets(dev):
    """The one-warp-per-row adjoint reads the shifted object patches when offsets are registered."""
    w = syn.tiny_workload(F=512, L=1, M=8, n_side=3, step=64, seed=79, remap=True, loss="poisson",
                          with_sigma=True, with_bg=True)
    case = Case(w, dev, z=strong_z(512), mask_kind="shared", seed=16)
    plan = case.plan()
    _assert_offsets_ok(_offset_errors(case, plan, _offsets(w, 512)))
    plan.close()


@pytest.mark.parametrize("F", [64, 128, 256, 512])
@pytest.mark.parametrize("loss", ["amplitude", "poisson"])
def test_tiny_all_frame_sizes(dev, F, loss):
    w = syn.tiny_workload(F=F, L=2, M=2, n_side=3, step=F // 8, seed=F + (loss == "poisson"), remap=True,
                          loss=loss, with_sigma=True, with_bg=True)
    case = Case(w, dev, z=strong_z(F), mask_kind="shared", seed=F)
    plan = case.plan()
    assert_ok(check_all(case, plan))
    plan.close()


@pytest.mark.parametrize("remap", [False, True])
@pytest.mark.parametrize("mask_kind", [None, "frame"])
def test_options_remap_mask(dev, remap, mask_kind):
    w = syn.tiny_workload(F=64, L=3, M=2, n_side=3, step=10, seed=5, remap=remap, loss="poisson")
    case = Case(w, dev, z=strong_z(64), mask_kind=mask_kind, seed=3)
    plan = case.plan()
    assert_ok(check_all(case, plan))
    plan.close()


@pytest.mark.parametrize("F", [64, 256, 512])
def test_recompute_mode_and_ragged_batches(dev, F):
    """Tiny scratch budgets force mode chunks (fields recomputed) and ragged position batches."""
    w = syn.tiny_workload(F=F, L=2, M=3, n_side=3, step=F // 8, seed=9, remap=True, loss="amplitude",
                          with_sigma=True)
    case = Case(w, dev, z=strong_z(F), seed=4)
    frame = F * F * 8
    for budget in (frame, 2 * frame, 4 * 6 * frame):   # 1 mode per chunk, 2 per chunk, 4 positions x all
        plan = case.plan(scratch_bytes=budget)
        assert_ok(check_all(case, plan))
        plan.close()


def test_position_subset_in_any_order(dev):
    w = syn.tiny_workload(F=64, L=2, M=2, n_side=4, step=9, seed=12, remap=True, loss="poisson", with_bg=True)
    case = Case(w, dev, z=strong_z(64), mask_kind="frame", seed=6)
    plan = case.plan(scratch_bytes=3 * 4 * 64 * 64 * 8)
    assert_ok(check_all(case, plan, frames=[13, 2, 7, 0, 9]))
    plan.close()


def test_single_mode_single_wavelength_config1(dev):
    """Config 1: plain ptychography, 64 frames of 64x64, amplitude loss, one Adam step."""
    from paper_2311_14780_gb300 import AdamState
    w = syn.config1()
    case = Case(w, dev)
    plan = case.plan()
    assert_ok(check_all(case, plan))
    # one Adam step against the oracle's
    st = AdamState(plan, lr_O=1e-2, lr_P=1e-1)
    O, P = case.O.clone(), case.P.clone()
    plan.step(st, O, P, case.Im)
    ost = orc.AdamState([o.shape for o in case.O0], case.P0.shape)
    _, On, Pn = orc.step(case.O0, case.P0, w.pos, case.Ih, case.loss, case.eps, ost, 1e-2, 1e-1)
    assert st.t == 1
    dO = O.cpu().numpy() - np.concatenate([o.reshape(-1) for o in case.O0])
    dOr = np.concatenate([(a - b).reshape(-1) for a, b in zip(On, case.O0)])
    dP = P.cpu().numpy() - case.P0
    # the first Adam step is lr * sign(g) where |g| >> eps: compare the updates
    assert rel(dO, dOr) < 1e-4 and rel(dP, Pn - case.P0) < 1e-4
    plan.close()


def _config2_sampled(dev, O_eval, P_eval, sample, seed=7):
    """GPU vs oracle on full-size config 2 (all 400 positions planned): the predicted frames of
    a sample, and loss + gradient of that sample as a position subset."""
    from paper_2311_14780_gb300 import pack_objects, plan_for
    w = syn.config2()
    taps = orc.remap_taps(w.F, w.geom.z, w.geom.det_pixel, w.geom.tilt_rad)
    O0 = [as_c64_roundtrip(o) for o in O_eval]
    P0 = as_c64_roundtrip(P_eval)
    clean = np.zeros((w.J, w.F, w.F))
    clean[sample] = orc.predict(w.O_true, w.P_true, w.pos, None, None, taps, frames=sample)
    Ih = syn.poisson_measure(clean, seed)
    eps = 1e-9 * float(Ih[sample].mean())
    plan = plan_for(w, eps=eps)
    O = pack_objects(O0, dev)
    P = c64(P0, dev)
    Ip = plan.forward(O, P).cpu().numpy()
    Ir = orc.predict(O0, P0, w.pos, None, None, taps, frames=sample)
    Im = torch.as_tensor(Ih, device=dev).contiguous()
    bt = torch.as_tensor(np.asarray(sample, np.int32), device=dev)
    La, gO, gP = plan.adjoint(O, P, Im, batch=bt)
    Lr, gOr, gPr = orc.gradient(O0, P0, w.pos, Ih, "poisson", eps, None, None, None, taps, frames=sample)
    gOr = np.concatenate([g.reshape(-1) for g in gOr])
    gO, gP = gO.cpu().numpy(), gP.cpu().numpy()
    err = dict(I=rel(Ip[sample], Ir), L=abs(float(La.item()) - Lr) / abs(Lr), La=0.0,
               gO=rel(gO, gOr), gP=rel(gP, gPr), I_max=max_rel_frames(Ip[sample], Ir), gO_max=max_rel(gO, gOr),
               gP_max=max_rel(gP, gPr))
    plan.close()
    return err, (w, O0, P0, Ih, eps, taps, gOr, gPr)


@pytest.mark.slow
def test_config2_full_size_near_truth(dev):
    """Config 2 at full size (3 wavelengths x 4 modes, 256^2 frames, 400 positions, remap,
    Poisson) at an evaluation point near the truth: the stated bars."""
    w = syn.config2()
    O_e, P_e = syn.near_truth(w, seed=1)
    sample = sorted(np.random.default_rng(0).choice(w.J, size=6, replace=False).tolist())
    err, _ = _config2_sampled(dev, O_e, P_e, sample)
    assert_ok(err)


@pytest.mark.slow
def test_config2_full_size_flat_object_start(dev):
    """At the flat-object start (Section "Experimental setup") Poisson data put photons where
    the model predicts ~1e-7, so dL/dI reaches ~1e6 and complex64 arithmetic itself departs
    from FP64 by ~2e-4 in the gradient.  The bar there is the complex64 floor, measured by
    running the oracle's own steps on complex64 inputs (its FFTs stay in complex64)."""
    w = syn.config2()
    sample = sorted(np.random.default_rng(0).choice(w.J, size=6, replace=False).tolist())
    err, (w, O0, P0, Ih, eps, taps, gOr, gPr) = _config2_sampled(dev, w.O0, w.P0, sample)
    assert err["I"] < TOL_I and err["L"] < TOL_L and err["I_max"] < TOL_I_MAX, err
    _, gO32, gP32 = orc.gradient([o.astype(np.complex64) for o in O0], P0.astype(np.complex64), w.pos, Ih,
                                 "poisson", eps, None, None, None, taps, frames=sample)
    gO32 = np.concatenate([g.reshape(-1) for g in gO32])
    floor_O, floor_P = rel(gO32, gOr), rel(gP32, gPr)
    assert err["gO"] < max(TOL_G, 1.5 * floor_O), (err, floor_O)
    assert err["gP"] < max(TOL_G, 1.5 * floor_P), (err, floor_P)
    # element-wise: the same reading, with the complex64 floor taken in the max norm
    mfloor_O, mfloor_P = max_rel(gO32, gOr), max_rel(gP32, gPr)
    assert err["gO_max"] < max(TOL_G_MAX, 1.5 * mfloor_O), (err, mfloor_O)
    assert err["gP_max"] < max(TOL_G_MAX, 1.5 * mfloor_P), (err, mfloor_P)


def test_autograd_function_directional_derivative(dev):
    """torch.autograd path: dL along a random direction vs central differences (complex64)."""
    from paper_2311_14780_gb300.autograd import ptycho_loss
    w = syn.tiny_workload(F=64, L=2, M=2, n_side=3, step=10, seed=21, remap=True, loss="poisson", with_bg=True)
    case = Case(w, dev, z=strong_z(64), seed=8)
    plan = case.plan()
    O = case.O.clone().requires_grad_(True)
    P = case.P.clone().requires_grad_(True)
    L = ptycho_loss(O, P, plan, case.Im, None, case.bg_t)
    L.backward()
    g = torch.Generator(device="cpu").manual_seed(0)
    dO = torch.randn(O.shape, dtype=torch.complex64, generator=g).to(dev)
    dP = torch.randn(P.shape, dtype=torch.complex64, generator=g).to(dev)
    an = float((torch.real(torch.vdot(O.grad, dO)) + torch.real(torch.vdot(P.grad.reshape(-1), dP.reshape(-1)))).item())
    with torch.no_grad():
        h = 1e-3 * float(O.abs().mean().item())
        Lp = float(ptycho_loss(O + h * dO, P + h * dP, plan, case.Im, None, case.bg_t).item())
        Lm = float(ptycho_loss(O - h * dO, P - h * dP, plan, case.Im, None, case.bg_t).item())
    fd = (Lp - Lm) / (2 * h)
    assert abs(fd - an) < 2e-3 * abs(an), (fd, an)
    plan.close()


def test_deterministic_repeat(dev):
    """Fixed-order reductions: two identical calls give bit-identical gradients and loss."""
    w = syn.tiny_workload(F=128, L=2, M=3, n_side=3, step=14, seed=2, remap=True, loss="poisson")
    case = Case(w, dev, z=strong_z(128), seed=1)
    plan = case.plan()
    a = plan.adjoint(case.O, case.P, case.Im)
    b = plan.adjoint(case.O, case.P, case.Im)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1]) and torch.equal(a[2], b[2])
    plan.close()


@pytest.mark.parametrize("flags", [0, 2])
def test_overlapped_batches_match_one_stream(dev, flags):
    """Batches in flight on four streams add into the gradients in batch order: bit-identical
    to the same batches on one stream (a missing cross-stream ordering shows up here)."""
    w = syn.tiny_workload(F=64, L=2, M=3, n_side=6, step=8, seed=7, remap=True, loss="poisson", with_sigma=True)
    case = Case(w, dev, z=strong_z(64), seed=7)
    scratch = 2 * 6 * 64 * 64 * 8                                 # two positions per batch: 18 batches
    res = []
    for overlap in (1, 4):
        plan = case.plan(scratch_bytes=scratch, overlap=overlap, flags=flags)
        res.append([plan.adjoint(case.O, case.P, case.Im, case.sig_t) for _ in range(3)])
        plan.close()
    ref = res[0][0]
    for run in res[0][1:] + res[1]:
        assert torch.equal(run[0], ref[0])
        assert torch.equal(run[2], ref[2])                      # grad P: register sums in batch order
        if flags == 0:                                          # grad O: tile-owned, in batch order
            assert torch.equal(run[1], ref[1])


def _sampled_full_size(dev, w, n_frames, n_grad, seed):
    """Full-size plan; predicted frames of a sample and the gradient of a smaller subset
    checked against the oracle, at a near-truth evaluation point."""
    from paper_2311_14780_gb300 import pack_objects, plan_for
    taps = orc.remap_taps(w.F, w.geom.z, w.geom.det_pixel, w.geom.tilt_rad) if w.geom.remap else None
    rng = np.random.default_rng(seed)
    frames = sorted(rng.choice(w.J, size=n_frames, replace=False).tolist())
    gframes = frames[:n_grad]
    O_e, P_e = syn.near_truth(w, seed=seed)
    O0 = [as_c64_roundtrip(o) for o in O_e]
    P0 = as_c64_roundtrip(P_e)
    clean = np.zeros((w.J, w.F, w.F))
    clean[gframes] = orc.predict(w.O_true, w.P_true, w.pos, None, None, taps, frames=gframes)
    Ih = syn.poisson_measure(clean, seed)
    eps = 1e-9 * float(Ih[gframes].mean())
    plan = plan_for(w, eps=eps)
    O = pack_objects(O0, dev)
    P = c64(P0, dev)
    Ip = plan.forward(O, P).cpu().numpy()
    Ir = orc.predict(O0, P0, w.pos, None, None, taps, frames=frames)
    bt = torch.as_tensor(np.asarray(gframes, np.int32), device=dev)
    La, gO, gP = plan.adjoint(O, P, torch.as_tensor(Ih, device=dev).contiguous(), batch=bt)
    Lr, gOr, gPr = orc.gradient(O0, P0, w.pos, Ih, w.loss, eps, None, None, None, taps, frames=gframes)
    gOr = np.concatenate([g.reshape(-1) for g in gOr])
    gO, gP = gO.cpu().numpy(), gP.cpu().numpy()
    err = dict(I=rel(Ip[frames], Ir), L=abs(float(La.item()) - Lr) / abs(Lr), La=0.0,
               gO=rel(gO, gOr), gP=rel(gP, gPr), I_max=max_rel_frames(Ip[frames], Ir), gO_max=max_rel(gO, gOr),
               gP_max=max_rel(gP, gPr))
    plan.close()
    return err


@pytest.mark.slow
@pytest.mark.parametrize("F,M,L", [(128, 1, 1), (128, 8, 5), (256, 4, 3), (256, 1, 5), (512, 4, 3), (512, 8, 1)])
def test_config3_points_full_size_sampled(dev, F, M, L):
    """Throughput-sweep points (400 positions, 70 % overlap, rectangle objects, remap,
    Poisson) at full size: sampled frames and a position subset's gradient."""
    w = syn.config3(F, M, L)
    assert_ok(_sampled_full_size(dev, w, n_frames=3, n_grad=2, seed=F + M + L))


@pytest.mark.slow
def test_config4_full_size_sampled(dev):
    """~200M-parameter case (6 wavelengths x 10 modes of 512^2, 6 objects of 3584^2, 900
    positions): sampled frames and the gradient of one position against the oracle."""
    w = syn.config4()
    assert_ok(_sampled_full_size(dev, w, n_frames=2, n_grad=1, seed=4))


def _full_size_all_positions(dev, w, seed):
    """Every position of a full-size workload under the plan's default batching (several
    position batches of about 1200 evaluations, three in flight on their own streams, the
    object gradient tiled over 32 x 32 tiles that gather many overlapping patches), at a
    near-truth evaluation point: all predicted frames, the loss and the whole gradient
    against the oracle."""
    from paper_2311_14780_gb300 import pack_objects, plan_for
    taps = orc.remap_taps(w.F, w.geom.z, w.geom.det_pixel, w.geom.tilt_rad) if w.geom.remap else None
    O_e, P_e = syn.near_truth(w, seed=seed)
    O0 = [as_c64_roundtrip(o) for o in O_e]
    P0 = as_c64_roundtrip(P_e)
    Ih = syn.poisson_measure(orc.predict(w.O_true, w.P_true, w.pos, None, None, taps), seed)
    eps = syn.default_eps(Ih)
    plan = plan_for(w, eps=eps)
    O = pack_objects(O0, dev)
    P = c64(P0, dev)
    Im = torch.as_tensor(Ih, device=dev).contiguous()
    Ip = plan.forward(O, P).cpu().numpy()
    launches_fwd = plan.last_launches
    La, gO, gP = plan.adjoint(O, P, Im)
    Lg = float(plan.loss(O, P, Im).item())
    status = plan.status()
    plan.close()
    Ir = orc.predict(O0, P0, w.pos, None, None, taps)
    Lr, gOr, gPr = orc.gradient(O0, P0, w.pos, Ih, w.loss, eps, None, None, None, taps)
    gOr = np.concatenate([g.reshape(-1) for g in gOr])
    gO, gP = gO.cpu().numpy(), gP.cpu().numpy()
    return dict(I=rel(Ip, Ir), I_max=max_rel_frames(Ip, Ir), L=abs(Lg - Lr) / abs(Lr),
                La=abs(float(La.item()) - Lr) / abs(Lr), gO=rel(gO, gOr), gP=rel(gP, gPr), gO_max=max_rel(gO, gOr),
                gP_max=max_rel(gP, gPr), status=status, launches_fwd=launches_fwd)


@pytest.mark.slow
def test_config2_all_positions_default_batching(dev):
    """Config 2 at full size with all 400 positions in one call (four position batches, three
    in flight), not a position subset: every frame, the loss and the whole gradient."""
    err = _full_size_all_positions(dev, syn.config2(), seed=12)
    assert err["launches_fwd"] >= 3 * 3, err        # row pass, column pass, loss per batch: several batches
    assert_ok(err)


@pytest.mark.slow
@pytest.mark.parametrize("F,M,L", [(512, 1, 1), (128, 8, 5)])
def test_config3_points_all_positions_default_batching(dev, F, M, L):
    """Sweep points with the largest frames (512^2, one field per position: many positions per
    batch) and the most fields (128^2 x 8 modes x 5 wavelengths: forty fields per position),
    all 400 positions under the default batching."""
    err = _full_size_all_positions(dev, syn.config3(F, M, L), seed=F + 10 * M + L)
    assert_ok(err)


RESIDENT_FRAMES = 1024


@pytest.mark.parametrize("flags", [0, 1, 2, 3, 4, 8, 16, 17, 20, 32, 64, 68, 192, 256, 288, 512, 1024, 2048])
@pytest.mark.parametrize("F", [64, 128, 256])
def test_pipeline_variants(dev, flags, F):
    """Recompute-the-columns, atomic object-gradient, keep-Psi, TMA-staged columns (and plain
    loads where TMA is the default), per-mode row adjoint, cp.async-staged columns (8 and 4
    wide), fused forward row pass, launches without programmatic dependent launch and the
    frame-resident passes (F <= 128) all meet the same bars."""
    w = syn.tiny_workload(F=F, L=2, M=3, n_side=4, step=F // 8, seed=60 + flags, remap=True, loss="poisson",
                          with_sigma=True, with_bg=True)
    case = Case(w, dev, z=strong_z(F), mask_kind="frame", seed=flags)
    plan = case.plan(flags=flags, scratch_bytes=5 * 6 * F * F * 8)    # several batches in flight
    assert_ok(check_all(case, plan))
    plan.close()


@pytest.mark.parametrize("F", [64, 128])
@pytest.mark.parametrize("remap,loss,mask_kind", [(True, "poisson", "frame"), (False, "amplitude", "shared")])
def test_frame_resident_passes(dev, F, remap, loss, mask_kind):
    """The frame-resident forward and adjoint (F <= 128, RESIDENT_FRAMES: fields never leave the
    SM) with several position batches in flight, mode groups, position splits of the probe
    gradient, power coefficients and background: against the oracle, on a position subset in
    any order, bit-identical on repeat, and within the bars of the scratch passes."""
    w = syn.tiny_workload(F=F, L=2, M=3, n_side=5, step=F // 8, seed=80 + F, remap=remap, loss=loss,
                          with_sigma=True, with_bg=True)
    case = Case(w, dev, z=strong_z(F), mask_kind=mask_kind, seed=F)
    plan = case.plan(scratch_bytes=4 * 6 * F * F * 8, flags=RESIDENT_FRAMES)   # 4 positions per batch: 7 batches
    plan.profile(True)
    assert_ok(check_all(case, plan))
    assert_ok(check_all(case, plan, frames=[17, 3, 24, 0, 9, 12]))
    prof = plan.profile_read()
    plan.profile(False)
    assert prof["res_fwd"][1] > 0 and prof["res_adj"][1] > 0, prof
    assert prof["row_fwd"][1] == 0 and prof["col_fwd"][1] == 0 and prof["col_adj"][1] == 0, prof
    a = plan.adjoint(case.O, case.P, case.Im, case.sig_t, case.bg_t, case.mask_t)
    b = plan.adjoint(case.O, case.P, case.Im, case.sig_t, case.bg_t, case.mask_t)
    assert all(torch.equal(x, y) for x, y in zip(a, b))
    ref = case.plan(scratch_bytes=4 * 6 * F * F * 8)
    c = ref.adjoint(case.O, case.P, case.Im, case.sig_t, case.bg_t, case.mask_t)
    Ia = plan.forward(case.O, case.P, case.sig_t, case.bg_t).cpu().numpy()
    Ic = ref.forward(case.O, case.P, case.sig_t, case.bg_t).cpu().numpy()
    assert rel(Ia, Ic) < TOL_I and max_rel_frames(Ia, Ic) < TOL_I_MAX
    assert abs(float(a[0].item()) - float(c[0].item())) < TOL_L * abs(float(c[0].item()))
    for x, y in zip(a[1:], c[1:]):
        assert rel(x.cpu().numpy(), y.cpu().numpy()) < TOL_G and max_rel(x.cpu().numpy(), y.cpu().numpy()) < TOL_G_MAX
    ref.close()
    plan.close()


# ---------------------------------------------------------------------------------------
# gradients of the power coefficients sigma_j and the background N (Eq. 1; the paper lists
# both among the optimised variables)
# ---------------------------------------------------------------------------------------

def _sigma_bg_errors(case, plan, frames=None):
    batch = None if frames is None else torch.as_tensor(np.asarray(frames, np.int32), device=case.dev)
    La, gO, gP, gs, gb, _, _ = plan.adjoint_ex(case.O, case.P, case.Im, case.sig_t, case.bg_t, case.mask_t, batch)
    Lr, gsr, gbr = orc.gradient_sigma_bg(case.O0, case.P0, case.w.pos, case.Ih, case.loss, case.eps, case.sigma,
                                         case.bg, case.mask, case.taps, frames)
    _, gOr, gPr = case.oracle_grad(frames)
    gOr = np.concatenate([g.reshape(-1) for g in gOr])
    got = dict(gO=gO.cpu().numpy(), gP=gP.cpu().numpy(), gs=gs.cpu().numpy(), gb=gb.cpu().numpy())
    ref = dict(gO=gOr, gP=gPr, gs=gsr, gb=gbr)
    e = dict(L=abs(float(La.item()) - Lr) / abs(Lr), gs_gpu=got["gs"], status=plan.status())
    for k in got:
        e[k] = rel(got[k], ref[k])
        e[k + "_max"] = max_rel(got[k], ref[k])
    return e


@pytest.mark.parametrize("remap,loss,mask_kind", [(True, "poisson", "frame"), (False, "amplitude", None),
                                                   (True, "amplitude", "shared"), (False, "poisson", "frame")])
def test_sigma_background_gradients(dev, remap, loss, mask_kind):
    w = syn.tiny_workload(F=64, L=2, M=3, n_side=3, step=10, seed=31, remap=remap, loss=loss, with_sigma=True,
                          with_bg=True)
    case = Case(w, dev, z=strong_z(64), mask_kind=mask_kind, seed=5)
    plan = case.plan()
    e = _sigma_bg_errors(case, plan)
    assert e["status"] == 0 and e["L"] < TOL_L, e
    for k in ("gO", "gP", "gs", "gb"):
        assert e[k] < TOL_G and e[k + "_max"] < TOL_G_MAX, (k, e)
    plan.close()


@pytest.mark.parametrize("F", [64, 256])
def test_sigma_background_gradients_batches_and_subset(dev, F):
    """Several position batches on overlapping streams, recompute mode and a position subset in
    any order: sigma's gradient is 0 outside the subset and the background's sums the subset."""
    w = syn.tiny_workload(F=F, L=2, M=2, n_side=4, step=F // 8, seed=33, remap=True, loss="poisson",
                          with_sigma=True, with_bg=True)
    case = Case(w, dev, z=strong_z(F), mask_kind="frame", seed=9)
    frames = [11, 3, 0, 14, 7]
    for kw in (dict(scratch_bytes=2 * 4 * F * F * 8, overlap=3), dict(scratch_bytes=F * F * 8)):
        plan = case.plan(**kw)
        for fr in (None, frames):
            e = _sigma_bg_errors(case, plan, fr)
            assert e["status"] == 0 and e["L"] < TOL_L, (kw, fr, e)
            for k in ("gO", "gP", "gs", "gb"):
                assert e[k] < TOL_G and e[k + "_max"] < TOL_G_MAX, (kw, fr, k, e)
            if fr is not None:
                outside = np.setdiff1d(np.arange(w.J), fr)
                assert np.all(e["gs_gpu"][outside] == 0.0)
        plan.close()


def test_sigma_gradient_without_sigma_and_at_zero(dev):
    """sigma NULL means all ones; a zero sigma_j has a zero derivative (I is quadratic in it)."""
    w = syn.tiny_workload(F=64, L=1, M=2, n_side=3, step=10, seed=35, remap=False, loss="amplitude", with_bg=True)
    case = Case(w, dev, seed=2)
    plan = case.plan()
    _, _, _, gs, _, _, _ = plan.adjoint_ex(case.O, case.P, case.Im, None, case.bg_t)
    _, gsr, _ = orc.gradient_sigma_bg(case.O0, case.P0, w.pos, case.Ih, case.loss, case.eps, None, case.bg)
    assert rel(gs.cpu().numpy(), gsr) < TOL_G
    sig = torch.ones(w.J, dtype=torch.float32, device=dev)
    sig[4] = 0.0
    _, _, _, gs0, _, _, _ = plan.adjoint_ex(case.O, case.P, case.Im, sig, case.bg_t)
    assert float(gs0[4].item()) == 0.0
    _, gsr0, _ = orc.gradient_sigma_bg(case.O0, case.P0, w.pos, case.Ih, case.loss, case.eps,
                                       sig.cpu().numpy().astype(np.float64), case.bg)
    assert rel(gs0.cpu().numpy(), gsr0) < TOL_G
    plan.close()


@pytest.mark.parametrize("device_counter", [False, True])
def test_step_updates_sigma_and_background(dev, device_counter):
    """ptycho_step with lr_sigma, lr_bg > 0: two steps, each checked against the oracle's Adam
    (real and imaginary parts as separate real parameters) applied to the same state and to the
    gradients ptycho_adjoint_ex gives there (the call is deterministic, so ptycho_step uses the
    same ones).  Those gradients are checked against the oracle's at the first step; Adam's
    per-component normalisation would otherwise turn the FP32 rounding of near-zero gradient
    components (object pixels far from the probe) into differences of order lr."""
    from paper_2311_14780_gb300 import AdamState
    w = syn.tiny_workload(F=64, L=2, M=2, n_side=3, step=10, seed=37, remap=True, loss="poisson", with_sigma=True,
                          with_bg=True)
    case = Case(w, dev, z=strong_z(64), seed=6)
    plan = case.plan()
    lr = dict(lr_O=1e-2, lr_P=1e-1, lr_sigma=1e-2, lr_bg=1e-1)
    st = AdamState(plan, lr["lr_O"], lr["lr_P"], device_counter=device_counter, lr_sigma=lr["lr_sigma"],
                   lr_bg=lr["lr_bg"])
    O, P = case.O.clone(), case.P.clone()
    sig, bg = case.sig_t.clone(), case.bg_t.clone()
    frames = [0, 5, 8, 2]
    bt = torch.as_tensor(np.asarray(frames, np.int32), device=dev)

    def c128(t):
        return t.detach().cpu().numpy().astype(np.complex128).reshape(-1)

    def f64(t):
        return t.detach().cpu().numpy().astype(np.float64).reshape(-1)

    for it in range(2):
        x0 = dict(O=c128(O), P=c128(P), s=f64(sig), b=f64(bg))
        mom = {k: f64(getattr(st, k)) for k in ("mO", "vO", "mP", "vP", "m_sigma", "v_sigma", "m_bg", "v_bg")}
        La, gO, gP, gs, gb, _, _ = plan.adjoint_ex(O, P, case.Im, sig, bg, batch=bt)
        if it == 0:
            Lr, gsr, gbr = orc.gradient_sigma_bg(case.O0, case.P0, w.pos, case.Ih, case.loss, case.eps, case.sigma,
                                                 case.bg, None, case.taps, frames)
            _, gOr, gPr = case.oracle_grad(frames)
            assert abs(float(La.item()) - Lr) < TOL_L * abs(Lr)
            assert rel(c128(gO), np.concatenate([g.reshape(-1) for g in gOr])) < TOL_G
            assert rel(c128(gP), gPr) < TOL_G and rel(f64(gs), gsr) < TOL_G and rel(f64(gb), gbr.reshape(-1)) < TOL_G
        L = float(plan.step(st, O, P, case.Im, sig, bg, batch=bt).item())
        assert L == float(La.item())                           # the step took the same (deterministic) pass
        t = it + 1
        mO, vO = mom["mO"].reshape(-1, 2), mom["vO"].reshape(-1, 2)
        mP, vP = mom["mP"].reshape(-1, 2), mom["vP"].reshape(-1, 2)
        hp = dict(b1=float(np.float32(0.9)), b2=float(np.float32(0.999)), eps=float(np.float32(1e-8)))  # as the ABI takes them
        On = orc.adam_update(x0["O"], c128(gO), mO, vO, t, lr["lr_O"], **hp)
        Pn = orc.adam_update(x0["P"], c128(gP), mP, vP, t, lr["lr_P"], **hp)
        sn = orc.adam_update_real(x0["s"], f64(gs), mom["m_sigma"], mom["v_sigma"], t, lr["lr_sigma"], **hp)
        bn = orc.adam_update_real(x0["b"], f64(gb), mom["m_bg"], mom["v_bg"], t, lr["lr_bg"], **hp)
        for name, new, ref, old in (("O", c128(O), On, x0["O"]), ("P", c128(P), Pn, x0["P"]),
                                    ("sigma", f64(sig), sn, x0["s"]), ("bg", f64(bg), bn, x0["b"])):
            assert rel(new - old, ref - old) < 1e-5, (it, name, rel(new - old, ref - old))
        for name in ("m_sigma", "v_sigma", "m_bg", "v_bg"):                # FP32 moments (tiny ones subnormal)
            ref = mom[name]
            assert np.allclose(f64(getattr(st, name)), ref, rtol=1e-5, atol=1e-6 * np.abs(ref).max()), (it, name)
        if it == 0:                                              # zero gradient outside the batch: sigma unchanged
            outside = np.setdiff1d(np.arange(w.J), frames)
            assert np.all(f64(sig)[outside] == x0["s"][outside])
    plan.close()


def test_step_host_matches_step(dev):
    """ptycho_step_host (measured patterns in pinned host memory, copied on the stream; the loss
    copied back to the host) takes exactly the step ptycho_step takes on device data."""
    from paper_2311_14780_gb300 import AdamState
    w = syn.tiny_workload(F=64, L=2, M=2, n_side=3, step=10, seed=38, remap=True, loss="poisson")
    case = Case(w, dev, z=strong_z(64), seed=3)
    plan = case.plan()
    s1, s2 = AdamState(plan, 1e-2, 1e-1), AdamState(plan, 1e-2, 1e-1)
    O1, P1 = case.O.clone(), case.P.clone()
    O2, P2 = case.O.clone(), case.P.clone()
    host = torch.as_tensor(case.Ih).contiguous().pin_memory()
    staging = torch.full_like(case.Im, float("nan"))
    l1 = torch.zeros(1, dtype=torch.float64, device=dev)
    l2 = torch.zeros(1, dtype=torch.float64, device=dev)
    lh = torch.zeros(1, dtype=torch.float64).pin_memory()
    for _ in range(2):
        plan.step(s1, O1, P1, case.Im, loss_out=l1)
        plan.step_host(s2, O2, P2, host, staging, l2, lh)
        torch.cuda.synchronize()
        assert float(lh.item()) == float(l1.item()) == float(l2.item())
    assert torch.equal(staging, case.Im) and s2.t == s1.t == 2
    assert torch.equal(O1, O2) and torch.equal(P1, P2)
    plan.close()


def test_autograd_sigma_background(dev):
    """torch.autograd through sigma and bg: a directional derivative vs central differences."""
    from paper_2311_14780_gb300.autograd import ptycho_loss
    w = syn.tiny_workload(F=64, L=2, M=2, n_side=3, step=10, seed=39, remap=True, loss="amplitude", with_sigma=True,
                          with_bg=True)
    case = Case(w, dev, z=strong_z(64), seed=4)
    plan = case.plan()
    sig = case.sig_t.clone().requires_grad_(True)
    bg = case.bg_t.clone().requires_grad_(True)
    L = ptycho_loss(case.O, case.P, plan, case.Im, sig, bg)
    L.backward()
    g = torch.Generator(device="cpu").manual_seed(1)
    ds = torch.randn(sig.shape, generator=g).to(dev)
    db = torch.randn(bg.shape, generator=g).to(dev)
    an = float((torch.dot(sig.grad, ds) + torch.dot(bg.grad.reshape(-1), db.reshape(-1))).item())
    with torch.no_grad():
        h = 1e-3
        Lp = float(ptycho_loss(case.O, case.P, plan, case.Im, sig + h * ds, bg + h * db).item())
        Lm = float(ptycho_loss(case.O, case.P, plan, case.Im, sig - h * ds, bg - h * db).item())
    fd = (Lp - Lm) / (2 * h)
    assert abs(fd - an) < 2e-3 * abs(an), (fd, an)
    plan.close()


# ---------------------------------------------------------------------------------------
# fractional scan offsets (f2 by the Fourier shift theorem) and the position gradient
# ---------------------------------------------------------------------------------------

def _offsets(w, seed, amp=0.5):
    return np.random.default_rng(seed).uniform(-amp, amp, size=(w.L, w.J, 2))


def _offset_errors(case, plan, delta, frames=None):
    """GPU forward, loss and every gradient with offsets registered, against the oracle."""
    w = case.w
    d32 = np.asarray(delta, np.float32).astype(np.float64)          # the values the GPU sees
    dt = torch.as_tensor(np.asarray(delta, np.float32), device=case.dev).contiguous()
    plan.set_offsets(dt)
    batch = None if frames is None else torch.as_tensor(np.asarray(frames, np.int32), device=case.dev)
    Ip = plan.forward(case.O, case.P, case.sig_t, case.bg_t).cpu().numpy()
    Ir = orc.predict(case.O0, case.P0, w.pos, case.sigma, case.bg, case.taps, delta=d32)
    La, gO, gP, gs, gb, gd, _ = plan.adjoint_ex(case.O, case.P, case.Im, case.sig_t, case.bg_t, case.mask_t, batch)
    args = (case.O0, case.P0, w.pos, case.Ih, case.loss, case.eps)
    Lr, gOr, gPr = orc.gradient(*args, case.sigma, case.bg, case.mask, case.taps, frames, delta=d32)
    _, gdr = orc.gradient_delta(*args, d32, case.sigma, case.bg, case.mask, case.taps, frames)
    _, gsr, gbr = orc.gradient_sigma_bg(*args, case.sigma, case.bg, case.mask, case.taps, frames, delta=d32)
    gOr = np.concatenate([g.reshape(-1) for g in gOr])
    got = dict(gO=gO.cpu().numpy(), gP=gP.cpu().numpy(), gd=gd.cpu().numpy(), gs=gs.cpu().numpy(),
               gb=gb.cpu().numpy())
    ref = dict(gO=gOr, gP=gPr, gd=gdr, gs=gsr, gb=gbr)
    e = dict(I=rel(Ip, Ir), I_max=max_rel_frames(Ip, Ir), L=abs(float(La.item()) - Lr) / abs(Lr),
             gd_gpu=got["gd"], status=plan.status())
    for k in got:
        e[k] = rel(got[k], ref[k])
        e[k + "_max"] = max_rel(got[k], ref[k])
    return e


def _assert_offsets_ok(e):
    assert e["status"] == 0, e
    assert e["I"] < TOL_I and e["L"] < TOL_L and e["I_max"] < TOL_I_MAX, e
    for k in ("gO", "gP", "gd", "gs", "gb"):
        assert e[k] < TOL_G and e[k + "_max"] < TOL_G_MAX, (k, e)


@pytest.mark.parametrize("F", [64, 128, 256, 512])
def test_offsets_all_frame_sizes(dev, F):
    w = syn.tiny_workload(F=F, L=2, M=2, n_side=3, step=F // 8, seed=70 + F, remap=True, loss="poisson",
                          with_sigma=True, with_bg=True)
    case = Case(w, dev, z=strong_z(F), mask_kind="shared", seed=F + 1)
    plan = case.plan()
    _assert_offsets_ok(_offset_errors(case, plan, _offsets(w, F)))
    plan.close()


@pytest.mark.parametrize("loss,remap", [("amplitude", False), ("poisson", False), ("amplitude", True)])
def test_offsets_losses_and_geometry(dev, loss, remap):
    w = syn.tiny_workload(F=64, L=3, M=2, n_side=3, step=10, seed=81, remap=remap, loss=loss, with_sigma=True,
                          with_bg=True)
    case = Case(w, dev, z=strong_z(64), mask_kind="frame", seed=12)
    plan = case.plan()
    _assert_offsets_ok(_offset_errors(case, plan, _offsets(w, 3, amp=0.9)))
    plan.close()


@pytest.mark.parametrize("F", [64, 256])
def test_offsets_batches_overlap_and_subset(dev, F):
    """Several position batches on overlapping streams and a position subset in any order: the
    position gradient is 0 outside the subset."""
    w = syn.tiny_workload(F=F, L=2, M=3, n_side=4, step=F // 8, seed=83, remap=True, loss="poisson",
                          with_sigma=True, with_bg=True)
    case = Case(w, dev, z=strong_z(F), mask_kind="frame", seed=13)
    plan = case.plan(scratch_bytes=2 * 6 * F * F * 8, overlap=3)
    delta = _offsets(w, 5)
    _assert_offsets_ok(_offset_errors(case, plan, delta))
    frames = [12, 1, 7, 4, 15]
    e = _offset_errors(case, plan, delta, frames)
    _assert_offsets_ok(e)
    outside = np.setdiff1d(np.arange(w.J), frames)
    assert np.all(e["gd_gpu"][:, outside, :] == 0.0)
    plan.close()


def test_zero_offsets_match_integer_positions_and_clearing_restores_them(dev):
    w = syn.tiny_workload(F=128, L=2, M=2, n_side=3, step=14, seed=85, remap=True, loss="poisson", with_bg=True)
    case = Case(w, dev, z=strong_z(128), seed=14)
    plan = case.plan()
    L0, gO0, gP0 = plan.adjoint(case.O, case.P, case.Im, None, case.bg_t)
    plan.set_offsets(torch.zeros(w.L, w.J, 2, dtype=torch.float32, device=dev))
    L1, gO1, gP1, _, _, gd1, _ = plan.adjoint_ex(case.O, case.P, case.Im, None, case.bg_t)
    assert abs(float(L1.item()) - float(L0.item())) < 1e-6 * abs(float(L0.item()))
    assert rel(gO1.cpu().numpy(), gO0.cpu().numpy()) < 1e-5 and rel(gP1.cpu().numpy(), gP0.cpu().numpy()) < 1e-5
    _, gdr = orc.gradient_delta(case.O0, case.P0, w.pos, case.Ih, case.loss, case.eps, np.zeros((w.L, w.J, 2)),
                                None, case.bg, None, case.taps)
    assert rel(gd1.cpu().numpy(), gdr) < TOL_G
    plan.set_offsets(None)
    L2, gO2, _ = plan.adjoint(case.O, case.P, case.Im, None, case.bg_t)
    assert torch.equal(L2, L0) and torch.equal(gO2, gO0)          # the integer path again, bit for bit
    plan.close()


def test_offsets_reject_what_they_cannot_do(dev):
    from paper_2311_14780_gb300 import AdamState, PtychoError, _native
    from paper_2311_14780_gb300.api import _ptr
    w = syn.tiny_workload(F=64, L=1, M=2, n_side=3, step=10, seed=87, remap=False, loss="amplitude")
    case = Case(w, dev, seed=15)
    plan = case.plan()
    gd = torch.empty(w.L, w.J, 2, dtype=torch.float32, device=dev)
    gO = torch.empty(plan.numel_O, dtype=torch.complex64, device=dev)
    gP = torch.empty_like(case.P)
    rc = _native.lib().ptycho_adjoint_ex(plan.handle, _ptr(torch.view_as_real(case.O)), _ptr(torch.view_as_real(case.P)),
                                         None, None, _ptr(case.Im), None, 0, None, 0, _ptr(torch.view_as_real(gO)),
                                         _ptr(torch.view_as_real(gP)), None, None, _ptr(gd), None, None, None)
    assert rc == -1                                               # a position gradient needs offsets
    plan.set_offsets(torch.zeros(w.L, w.J, 2, dtype=torch.float32, device=dev))
    with pytest.raises(PtychoError):
        plan.plain_step(AdamState(plan, 1e-2, 1e-2), case.O.clone(), case.P.clone(), case.Im)
    plan.close()


def test_step_updates_offsets(dev):
    """ptycho_step with lr_delta > 0 moves the registered offsets by Adam on the position
    gradient (checked against the oracle's Adam on the same gradient and state); the object,
    probe and offsets updates all come from one deterministic pass."""
    from paper_2311_14780_gb300 import AdamState
    w = syn.tiny_workload(F=64, L=2, M=2, n_side=3, step=10, seed=89, remap=True, loss="poisson", with_sigma=True)
    case = Case(w, dev, z=strong_z(64), seed=16)
    plan = case.plan()
    delta = torch.as_tensor(_offsets(w, 9).astype(np.float32), device=dev).contiguous()
    plan.set_offsets(delta)
    st = AdamState(plan, 1e-2, 1e-1, lr_delta=5e-2)
    O, P = case.O.clone(), case.P.clone()
    hp = dict(b1=float(np.float32(0.9)), b2=float(np.float32(0.999)), eps=float(np.float32(1e-8)))
    for it in range(2):
        d0 = delta.detach().cpu().numpy().astype(np.float64).reshape(-1)
        m0 = st.m_delta.cpu().numpy().astype(np.float64)
        v0 = st.v_delta.cpu().numpy().astype(np.float64)
        La, _, _, _, _, gd, _ = plan.adjoint_ex(O, P, case.Im, case.sig_t)
        if it == 0:
            _, gdr = orc.gradient_delta(case.O0, case.P0, w.pos, case.Ih, case.loss, case.eps,
                                        d0.reshape(w.L, w.J, 2), case.sigma, None, None, case.taps)
            assert rel(gd.cpu().numpy(), gdr) < TOL_G
        L = float(plan.step(st, O, P, case.Im, case.sig_t).item())
        assert L == float(La.item())
        ref = orc.adam_update_real(d0, gd.cpu().numpy().astype(np.float64).reshape(-1), m0, v0, it + 1, 5e-2, **hp)
        new = delta.detach().cpu().numpy().astype(np.float64).reshape(-1)
        assert rel(new - d0, ref - d0) < 1e-5, it
    plan.close()


# ---------------------------------------------------------------------------------------
# propagation distance z (through the tilted-plane remap)
# ---------------------------------------------------------------------------------------

def _z_errors(case, plan, frames=None, delta=None):
    w = case.w
    batch = None if frames is None else torch.as_tensor(np.asarray(frames, np.int32), device=case.dev)
    La, _, _, _, _, _, gz = plan.adjoint_ex(case.O, case.P, case.Im, case.sig_t, case.bg_t, case.mask_t, batch)
    rates = orc.remap_index_rates(w.F, case.z, w.geom.det_pixel, w.geom.tilt_rad)
    Lr, gzr = orc.gradient_z(case.O0, case.P0, w.pos, case.Ih, case.loss, case.eps, case.taps, rates, case.sigma,
                             case.bg, case.mask, frames, delta)
    return abs(float(La.item()) - Lr) / abs(Lr), abs(float(gz.item()) - gzr) / abs(gzr)


@pytest.mark.parametrize("F,loss,mask_kind", [(64, "poisson", "frame"), (64, "amplitude", None),
                                              (256, "poisson", "shared"), (512, "amplitude", None)])
def test_z_gradient(dev, F, loss, mask_kind):
    w = syn.tiny_workload(F=F, L=2, M=2, n_side=3, step=F // 8, seed=91 + F, remap=True, loss=loss, with_sigma=True,
                          with_bg=True)
    case = Case(w, dev, z=strong_z(F), mask_kind=mask_kind, seed=17)
    plan = case.plan(scratch_bytes=2 * 4 * F * F * 8)                      # several batches
    eL, ez = _z_errors(case, plan)
    assert eL < TOL_L and ez < TOL_G, (eL, ez)
    eL, ez = _z_errors(case, plan, frames=[5, 0, 7])
    assert eL < TOL_L and ez < TOL_G, (eL, ez)
    plan.close()


def test_z_gradient_with_offsets(dev):
    w = syn.tiny_workload(F=64, L=2, M=2, n_side=3, step=8, seed=95, remap=True, loss="poisson", with_bg=True)
    case = Case(w, dev, z=strong_z(64), seed=18)
    plan = case.plan()
    delta = np.random.default_rng(3).uniform(-0.5, 0.5, size=(w.L, w.J, 2)).astype(np.float32)
    plan.set_offsets(torch.as_tensor(delta, device=dev))
    eL, ez = _z_errors(case, plan, delta=delta.astype(np.float64))
    assert eL < TOL_L and ez < TOL_G, (eL, ez)
    plan.close()


def test_set_distance_rebuilds_the_remap(dev):
    """After ptycho_plan_set_distance(z2) the model is the oracle's at z2; going back to z gives
    the first results bit for bit; the remap-free plan refuses both z calls."""
    from paper_2311_14780_gb300 import PtychoError
    w = syn.tiny_workload(F=128, L=2, M=2, n_side=3, step=14, seed=97, remap=True, loss="poisson", with_bg=True)
    z1 = strong_z(128)
    case = Case(w, dev, z=z1, seed=19)
    plan = case.plan()
    I1 = plan.forward(case.O, case.P, None, case.bg_t).clone()
    g1 = plan.adjoint_ex(case.O, case.P, case.Im, None, case.bg_t)
    z2 = 1.3 * z1
    plan.set_distance(z2)
    taps2 = orc.remap_taps(w.F, z2, w.geom.det_pixel, w.geom.tilt_rad)
    I2 = plan.forward(case.O, case.P, None, case.bg_t).cpu().numpy()
    assert rel(I2, orc.predict(case.O0, case.P0, w.pos, None, case.bg, taps2)) < TOL_I
    _, _, _, _, _, _, gz2 = plan.adjoint_ex(case.O, case.P, case.Im, None, case.bg_t)
    _, gzr = orc.gradient_z(case.O0, case.P0, w.pos, case.Ih, case.loss, case.eps, taps2,
                            orc.remap_index_rates(w.F, z2, w.geom.det_pixel, w.geom.tilt_rad), None, case.bg)
    assert abs(float(gz2.item()) - gzr) < TOL_G * abs(gzr)
    plan.set_distance(z1)
    assert torch.equal(plan.forward(case.O, case.P, None, case.bg_t), I1)
    g1b = plan.adjoint_ex(case.O, case.P, case.Im, None, case.bg_t)
    assert torch.equal(g1b[0], g1[0]) and torch.equal(g1b[1], g1[1]) and torch.equal(g1b[6], g1[6])
    with pytest.raises(PtychoError):
        plan.set_distance(-1.0)
    plan.close()
    w0 = syn.tiny_workload(F=64, L=1, M=1, n_side=2, step=8, seed=98, remap=False)
    c0 = Case(w0, dev, seed=20)
    p0 = c0.plan()
    with pytest.raises(PtychoError):
        p0.set_distance(0.1)
    assert p0.adjoint_ex(c0.O, c0.P, c0.Im)[6] is None
    p0.close()


def test_step_writes_the_z_gradient_of_its_pass(dev):
    from paper_2311_14780_gb300 import AdamState
    w = syn.tiny_workload(F=64, L=2, M=2, n_side=3, step=8, seed=99, remap=True, loss="poisson", with_bg=True)
    case = Case(w, dev, z=strong_z(64), seed=21)
    plan = case.plan()
    _, _, _, _, _, _, gz = plan.adjoint_ex(case.O, case.P, case.Im, None, case.bg_t)
    st = AdamState(plan, 1e-3, 1e-3, with_z_gradient=True)
    plan.step(st, case.O.clone(), case.P.clone(), case.Im, None, case.bg_t)
    assert torch.equal(st.g_z, gz)                                  # same deterministic pass
    plan.close()


# ---------------------------------------------------------------------------------------
# mixed Poisson-Gaussian loss (shifted-Poisson reading)
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("F,remap", [(64, True), (256, True), (128, False)])
def test_mixed_poisson_gaussian_loss(dev, F, remap):
    from paper_2311_14780_gb300 import pack_objects, plan_for
    w = syn.tiny_workload(F=F, L=2, M=2, n_side=3, step=F // 8, seed=101 + F, remap=remap, loss="poisson",
                          with_sigma=True, with_bg=True)
    z = strong_z(F)
    taps = orc.remap_taps(w.F, z, w.geom.det_pixel, w.geom.tilt_rad) if remap else None
    s2 = 2.25
    rng = np.random.default_rng(F)
    clean = orc.predict(w.O_true, w.P_true, w.pos, w.sigma, w.bg, taps)
    Ih = (syn.poisson_measure(clean, 30) + rng.normal(0.0, 1.5, size=clean.shape)).astype(np.float32)
    eps = syn.default_eps(np.maximum(Ih, 0))
    kind = ("poisson_gaussian", float(np.float32(s2)))
    plan = plan_for(w, loss="poisson_gaussian", read_noise_var=s2, eps=eps, z=z)
    O0 = [as_c64_roundtrip(o) for o in w.O0]
    P0 = as_c64_roundtrip(w.P0)
    sig = np.asarray(w.sigma, np.float32).astype(np.float64)
    bg = np.asarray(w.bg, np.float32).astype(np.float64)
    Ihd = Ih.astype(np.float64)
    La, gO, gP = plan.adjoint(pack_objects(O0, dev), c64(P0, dev), torch.as_tensor(Ih, device=dev).contiguous(),
                              f32(sig, dev), f32(bg, dev))
    Lr, gOr, gPr = orc.gradient(O0, P0, w.pos, Ihd, kind, float(np.float32(eps)), sig, bg, None, taps)
    gOr = np.concatenate([g.reshape(-1) for g in gOr])
    assert abs(float(La.item()) - Lr) < TOL_L * abs(Lr)
    assert rel(gO.cpu().numpy(), gOr) < TOL_G and rel(gP.cpu().numpy(), gPr) < TOL_G
    plan.close()


# ---------------------------------------------------------------------------------------
# chirp-z (zoom DFT) propagator
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("F,loss,remap", [(64, "poisson", True), (128, "amplitude", False), (256, "poisson", True),
                                         (512, "amplitude", True)])
def test_czt_propagator_against_the_oracle(dev, F, loss, remap):
    from paper_2311_14780_gb300 import pack_objects, plan_for
    w = syn.tiny_workload(F=F, L=3, M=2, n_side=3, step=F // 8, seed=111 + F, remap=remap, loss=loss,
                          with_sigma=True, with_bg=True)
    zeta = [1.0, 1.0 / 1.1, 1.0 / 1.2]                        # lambda_1 / lambda_l
    case = Case(w, dev, z=strong_z(F), mask_kind="shared", seed=22)
    clean = orc.predict(w.O_true, w.P_true, w.pos, w.sigma, w.bg, case.taps, zeta=zeta)
    Ih = syn.poisson_measure(clean, 40 + F)
    eps = syn.default_eps(Ih)
    plan = plan_for(w, loss=loss, eps=eps, z=case.z, zoom=zeta, scratch_bytes=2 * 6 * F * F * 8)
    Im = torch.as_tensor(Ih, device=dev).contiguous()
    Ip = plan.forward(case.O, case.P, case.sig_t, case.bg_t).cpu().numpy()
    Ir = orc.predict(case.O0, case.P0, w.pos, case.sigma, case.bg, case.taps, zeta=zeta)
    assert rel(Ip, Ir) < TOL_I and max_rel_frames(Ip, Ir) < TOL_I_MAX
    La, gO, gP, gs, gb, _, _ = plan.adjoint_ex(case.O, case.P, Im, case.sig_t, case.bg_t, case.mask_t)
    Lr, gOr, gPr = orc.gradient(case.O0, case.P0, w.pos, Ih, loss, eps, case.sigma, case.bg, case.mask, case.taps,
                                zeta=zeta)
    gOr = np.concatenate([g.reshape(-1) for g in gOr])
    gO, gP = gO.cpu().numpy(), gP.cpu().numpy()
    assert abs(float(La.item()) - Lr) < TOL_L * abs(Lr)
    assert rel(gO, gOr) < TOL_G and rel(gP, gPr) < TOL_G
    assert max_rel(gO, gOr) < TOL_G_MAX and max_rel(gP, gPr) < TOL_G_MAX
    assert plan.status() == 0
    plan.close()


@pytest.mark.parametrize("F", [128, 512])
def test_czt_at_unit_zoom_gives_the_dft_intensities_and_rejects_what_it_cannot_do(dev, F):
    from paper_2311_14780_gb300 import PtychoError
    w = syn.tiny_workload(F=F, L=2, M=2, n_side=3, step=F // 8, seed=113 + F, remap=True, loss="poisson",
                          with_bg=True)
    case = Case(w, dev, z=strong_z(F), seed=23)
    p_dft = case.plan()
    p_czt = case.plan(zoom=[1.0, 1.0])
    I1 = p_dft.forward(case.O, case.P, None, case.bg_t).cpu().numpy()
    I2 = p_czt.forward(case.O, case.P, None, case.bg_t).cpu().numpy()
    assert rel(I2, I1) < TOL_I and max_rel_frames(I2, I1) < TOL_I_MAX
    with pytest.raises(PtychoError):
        p_czt.set_offsets(torch.zeros(w.L, w.J, 2, dtype=torch.float32, device=dev))
    p_dft.close()
    p_czt.close()
