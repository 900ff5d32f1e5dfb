"""Object regulariser on the GPU (ptycho_regularise, and inside ptycho_step) vs the FP64 oracle."""
import numpy as np
import pytest
import torch

from oracle import ptycho_oracle as orc
from synthetic import workloads as syn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2311_14780_gb300 import _native
    _native.lib()
    return torch.device("cuda", 0)


def rel(a, b):
    a, b = np.asarray(a).ravel(), np.asarray(b).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def c64(x):
    return np.asarray(x).astype(np.complex64).astype(np.complex128)


@pytest.mark.parametrize("H,mu1,mutv,eta", [(81, 0.3, 0.7, 0.05), (96, 0.0, 1.0, 1e-3), (125, 0.5, 0.0, 0.01)])
def test_regularise_matches_the_oracle(dev, H, mu1, mutv, eta):
    """Objects of H x (H + 2) pixels per wavelength (tiles of 32 x 32 with ragged edges), L = 3;
    gradient and value added onto non-zero buffers."""
    from paper_2311_14780_gb300 import pack_objects, plan_for
    w = syn.tiny_workload(F=64, L=3, M=1, n_side=2, step=8, seed=H, H=H)
    plan = plan_for(w)
    O0 = [c64(o) for o in w.O0]
    O = pack_objects(O0, dev)
    rng = np.random.default_rng(H)
    g0 = (rng.standard_normal(O.numel()) + 1j * rng.standard_normal(O.numel())).astype(np.complex64)
    gO = torch.as_tensor(g0, device=dev)
    loss = torch.full((1,), 1.5, dtype=torch.float64, device=dev)
    plan.regularise(O, mu1, mutv, eta, gO=gO, loss_out=loss)
    torch.cuda.synchronize()
    R, gr = orc.regulariser(O0, mu1, mutv, eta)
    gr = np.concatenate([g.reshape(-1) for g in gr])
    assert abs(float(loss.item()) - 1.5 - R) <= 1e-6 * abs(R)
    got = gO.cpu().numpy().astype(np.complex128) - g0.astype(np.complex128)
    # FP32 amplitudes carry ~1 ulp of rounding, which the quotients dx/t amplify by up to a/eta
    # where the object is flat; the same formulas evaluated in FP32 by NumPy depart from FP64
    # by up to 4.6e-6 (L2) and 2.8e-5 (largest element) on these cases
    assert rel(got, gr) < 2e-5
    assert np.abs(got - gr).max() <= 1e-4 * np.abs(gr).max()
    plan.close()


def test_regularise_with_zero_weights_launches_nothing(dev):
    from paper_2311_14780_gb300 import pack_objects, plan_for
    w = syn.tiny_workload(F=64, L=2, M=1, n_side=2, step=8, seed=3)
    plan = plan_for(w)
    O = pack_objects(w.O0, dev)
    loss, gO = plan.regularise(O, 0.0, 0.0, 1e-3)
    torch.cuda.synchronize()
    assert plan.last_launches == 0 and float(loss.item()) == 0.0 and not gO.abs().max().item()
    with pytest.raises(Exception):
        plan.regularise(O, 0.1, 0.1, 0.0)
    plan.close()


def test_step_with_regularisation(dev):
    """ptycho_step with reg_l1 / reg_tv: its loss is the data loss plus R, and O moves by Adam
    on the data gradient plus the regulariser's (checked against the oracle's Adam on the same
    state and the GPU's gradients, which are checked against the oracle's first)."""
    from paper_2311_14780_gb300 import AdamState, pack_objects, plan_for
    w = syn.tiny_workload(F=64, L=2, M=2, n_side=3, step=10, seed=37, remap=True, loss="poisson")
    taps = orc.remap_taps(w.F, w.geom.z, w.geom.det_pixel, w.geom.tilt_rad)
    Ih = syn.poisson_measure(orc.predict(w.O_true, w.P_true, w.pos, taps=taps), 5)
    eps = syn.default_eps(Ih)
    plan = plan_for(w, eps=eps)
    O0 = [c64(o) for o in w.O0]
    P0 = c64(w.P0)
    O = pack_objects(O0, dev)
    P = torch.as_tensor(P0, dtype=torch.complex64, device=dev).contiguous()
    Im = torch.as_tensor(Ih, device=dev).contiguous()
    mu1, mutv, eta = 20.0, 50.0, 1e-2
    La, gO, gP = plan.adjoint(O, P, Im)
    Lreg, gR = plan.regularise(O, mu1, mutv, eta)
    torch.cuda.synchronize()
    Lr, gOr, _ = orc.gradient(O0, P0, w.pos, Ih, "poisson", eps, taps=taps)
    Rr, gRr = orc.regulariser(O0, mu1, mutv, eta)
    gsum = gO.cpu().numpy().astype(np.complex128) + gR.cpu().numpy().astype(np.complex128)
    gref = np.concatenate([g.reshape(-1) for g in gOr]) + np.concatenate([g.reshape(-1) for g in gRr])
    assert rel(gsum, gref) < 1e-4
    st = AdamState(plan, 1e-2, 1e-1, reg_l1=mu1, reg_tv=mutv, reg_eta=eta)
    O1, P1 = O.clone(), P.clone()
    L = float(plan.step(st, O1, P1, Im).item())
    assert L == pytest.approx(float(La.item()) + Rr, rel=1e-5)
    hp = dict(b1=float(np.float32(0.9)), b2=float(np.float32(0.999)), eps=float(np.float32(1e-8)))
    theta = O.cpu().numpy().astype(np.complex128)
    m = np.zeros(theta.shape + (2,))
    v = np.zeros(theta.shape + (2,))
    ref = orc.adam_update(theta, gsum, m, v, 1, 1e-2, **hp)
    assert rel(O1.cpu().numpy() - theta, ref - theta) < 1e-5
    plan.close()


def test_plain_step_rejects_regularisation(dev):
    from paper_2311_14780_gb300 import AdamState, PtychoError, pack_objects, plan_for
    w = syn.tiny_workload(F=64, L=2, M=1, n_side=2, step=8, seed=3)
    plan = plan_for(w)
    O = pack_objects(w.O0, dev)
    P = torch.as_tensor(w.P0, dtype=torch.complex64, device=dev).contiguous()
    Im = torch.ones(w.J, 64, 64, device=dev)
    st = AdamState(plan, 1e-2, 1e-2, reg_tv=1.0)
    with pytest.raises(PtychoError):
        plan.plain_step(st, O, P, Im)
    plan.close()
