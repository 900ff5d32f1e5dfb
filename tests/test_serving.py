"""Multi-site serving (continuous batching) and the plain unfused baseline."""
import ctypes

import numpy as np
import pytest
import torch

from synthetic import workloads as syn

REL = 1e-5


def rel(a, b):
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def test_server_create_rejects_bad_arguments():
    from paper_2311_14780_gb300 import _native, build
    import os
    if not os.path.exists(build.lib_path()):
        build.build()
    lib = _native.lib()
    h = ctypes.c_void_p()
    assert lib.ptycho_server_create(0, 4, ctypes.byref(h)) == -1
    assert lib.ptycho_server_create(1 << 30, 0, ctypes.byref(h)) == -1
    assert lib.ptycho_server_destroy(None) == 0
    assert b"budget" in lib.ptycho_strerror(-8)


def _request(F, L, M, n_side, seed, dev, iterations=4, name=None, arrival=0.0):
    """A small serving request with measured data from the GPU forward model on the truth
    (input synthesis only; these tests compare GPU paths with each other)."""
    from paper_2311_14780_gb300 import pack_objects, plan_for
    from paper_2311_14780_gb300.serve import Request
    w = syn.tiny_workload(F=F, L=L, M=M, n_side=n_side, step=F // 8, seed=seed, remap=True, loss="poisson")
    z = F * 15e-6 / 0.5
    pt = plan_for(w, z=z)
    I = pt.forward(pack_objects(w.O_true, dev), torch.as_tensor(w.P_true, dtype=torch.complex64, device=dev))
    pt.close()
    Ih = torch.as_tensor(syn.poisson_measure(I.cpu().numpy(), seed), device=dev).contiguous()
    return Request(name or f"F{F}L{L}M{M}", arrival, F, L, M, w.J, w.obj_shapes, w.pos,
                   pack_objects(w.O0, dev), torch.as_tensor(w.P0, dtype=torch.complex64, device=dev).contiguous(),
                   Ih, iterations=iterations, loss="poisson", eps=syn.default_eps(Ih.cpu().numpy()), z=z,
                   lr_O=1e-2, lr_P=1e-2)


@pytest.mark.gpu
def test_site_result_is_the_same_alone_and_in_the_mix():
    from paper_2311_14780_gb300.serve import Server
    dev = torch.device("cuda", 0)
    a_alone = _request(64, 1, 2, 3, 40, dev, iterations=5)
    sv = Server(8 << 30)
    slot = sv.admit(a_alone)
    while sv.tick():
        pass
    torch.cuda.synchronize()
    _, loss_alone = sv.status(slot)
    sv.release(slot)
    sv.close()

    # the same request, admitted while two other sites are already running
    a_mix = _request(64, 1, 2, 3, 40, dev, iterations=5)
    b = _request(128, 2, 1, 3, 41, dev, iterations=7)
    c = _request(64, 2, 3, 4, 42, dev, iterations=3)
    sv = Server(8 << 30)
    sb, sc = sv.admit(b), sv.admit(c)
    assert sv.tick() == 2
    sa = sv.admit(a_mix)
    counts = []
    while True:
        n = sv.tick()
        if n == 0:
            break
        counts.append(n)
    torch.cuda.synchronize()
    assert max(counts) == 3                       # all three overlapped in one launch
    it, loss_mix = sv.status(sa)
    assert it == 5
    assert sv.status(sb)[0] == 7 and sv.status(sc)[0] == 3
    for s in (sa, sb, sc):
        sv.release(s)
    assert sv.used_bytes == 0
    sv.close()
    assert torch.equal(a_mix.O, a_alone.O) and torch.equal(a_mix.P, a_alone.P)
    assert loss_mix == loss_alone


@pytest.mark.gpu
def test_served_iterations_match_ptycho_step():
    from paper_2311_14780_gb300 import AdamState
    from paper_2311_14780_gb300.api import plan_geometry_plan
    from paper_2311_14780_gb300.serve import Server
    dev = torch.device("cuda", 0)
    r = _request(128, 2, 2, 3, 43, dev, iterations=3)
    O0, P0 = r.O.clone(), r.P.clone()
    sv = Server(8 << 30)
    slot = sv.admit(r)
    while sv.tick():
        pass
    torch.cuda.synchronize()
    sv.release(slot)
    sv.close()
    plan = plan_geometry_plan(r)
    st = AdamState(plan, r.lr_O, r.lr_P)
    for _ in range(3):
        plan.step(st, O0, P0, r.I_meas)
    torch.cuda.synchronize()
    assert rel(r.O.cpu().numpy(), O0.cpu().numpy()) < REL
    assert rel(r.P.cpu().numpy(), P0.cpu().numpy()) < REL
    plan.close()


@pytest.mark.gpu
def test_admission_is_refused_over_budget_and_frees_everything():
    from paper_2311_14780_gb300.serve import Server
    dev = torch.device("cuda", 0)
    r = _request(128, 2, 2, 3, 44, dev)
    sv = Server(1 << 20)                         # 1 MiB: far too small
    assert sv.admit(r) is None
    assert sv.used_bytes == 0
    sv.close()
    sv = Server(8 << 30, max_sites=1)
    s0 = sv.admit(r)
    assert s0 is not None and sv.used_bytes > 0
    assert sv.admit(_request(64, 1, 1, 3, 45, dev)) is None    # no free slot
    sv.release(s0)
    assert sv.used_bytes == 0
    sv.close()


@pytest.mark.gpu
@pytest.mark.parametrize("F", [64, 256])
def test_plain_step_matches_fused_step(F):
    from paper_2311_14780_gb300 import AdamState
    from paper_2311_14780_gb300.api import plan_geometry_plan
    dev = torch.device("cuda", 0)
    r = _request(F, 2, 2, 3, 46, dev)
    plan = plan_geometry_plan(r)
    O1, P1 = r.O.clone(), r.P.clone()
    O2, P2 = r.O.clone(), r.P.clone()
    s1, s2 = AdamState(plan, 1e-2, 1e-2), AdamState(plan, 1e-2, 1e-2)
    l1 = torch.zeros(1, dtype=torch.float64, device=dev)
    l2 = torch.zeros(1, dtype=torch.float64, device=dev)
    for it in range(3):
        plan.step(s1, O1, P1, r.I_meas, loss_out=l1)
        plan.plain_step(s2, O2, P2, r.I_meas, loss_out=l2)
        torch.cuda.synchronize()
        # the first loss is taken at identical parameters; later ones after Adam steps that
        # differ on near-zero gradient components (see below), which moves the loss by ~1e-5
        bar = REL if it == 0 else 10 * REL
        assert abs(float(l1.item()) - float(l2.item())) <= bar * abs(float(l1.item())), it
    # parameters: Adam's early steps are +-lr per component whatever the gradient size, so
    # components whose gradient is at the level of FP32 rounding (object pixels under the
    # probe's far tails) take the sign of that rounding, which the plain form's atomic
    # summation order changes; a few hundred such components give ~2e-3 here.  The equal-loss
    # check above is the stated bar.
    assert rel(O2.cpu().numpy(), O1.cpu().numpy()) < 1e-2
    assert rel(P2.cpu().numpy(), P1.cpu().numpy()) < 1e-2
    plan.close()


@pytest.mark.gpu
def test_reused_slot_runs_the_new_site():
    """A released slot re-filled by another site, with the active slot set unchanged
    ({0, 1} before and after): the tick must run the new site's graph."""
    from paper_2311_14780_gb300.serve import Server
    dev = torch.device("cuda", 0)
    b_alone = _request(128, 1, 2, 3, 48, dev, iterations=3)
    sv = Server(8 << 30)
    s = sv.admit(b_alone)
    while sv.tick():
        pass
    torch.cuda.synchronize()
    sv.release(s)
    sv.close()

    a = _request(64, 1, 1, 3, 47, dev, iterations=2)
    c = _request(64, 2, 2, 3, 49, dev, iterations=6)
    b = _request(128, 1, 2, 3, 48, dev, iterations=3)
    sv = Server(8 << 30)
    sa, sc = sv.admit(a), sv.admit(c)
    assert (sa, sc) == (0, 1)
    assert sv.tick() == 2 and sv.tick() == 2     # a is done after two ticks
    sv.release(sa)
    sb = sv.admit(b)
    assert sb == 0                              # same slot, same active set {0, 1}
    while sv.tick():
        pass
    torch.cuda.synchronize()
    assert sv.status(sb)[0] == 3
    sv.release(sb)
    sv.release(sc)
    sv.close()
    assert torch.equal(b.O, b_alone.O) and torch.equal(b.P, b_alone.P)


@pytest.mark.gpu
def test_graph_replayed_steps_match_eager_steps():
    """ptycho_step with a device step counter, captured once as a CUDA graph and replayed,
    gives the same parameters as eager steps with the host counter."""
    from paper_2311_14780_gb300 import AdamState
    from paper_2311_14780_gb300.api import plan_geometry_plan
    dev = torch.device("cuda", 0)
    r = _request(128, 2, 2, 4, 50, dev)
    plan = plan_geometry_plan(r)
    O1, P1 = r.O.clone(), r.P.clone()
    O2, P2 = r.O.clone(), r.P.clone()
    s1 = AdamState(plan, 1e-2, 1e-2)
    s2 = AdamState(plan, 1e-2, 1e-2, device_counter=True)
    l2 = torch.zeros(1, dtype=torch.float64, device=dev)
    for _ in range(3):
        plan.step(s1, O1, P1, r.I_meas)
    plan.step(s2, O2, P2, r.I_meas, loss_out=l2)          # first step eagerly (warms up)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        plan.step(s2, O2, P2, r.I_meas, loss_out=l2)
    g.replay()                                              # step 2 (capturing ran nothing)
    g.replay()                                              # step 3
    torch.cuda.synchronize()
    assert int(s2.t_dev.item()) == 3
    assert rel(O2.cpu().numpy(), O1.cpu().numpy()) < REL
    assert rel(P2.cpu().numpy(), P1.cpu().numpy()) < REL
    plan.close()
