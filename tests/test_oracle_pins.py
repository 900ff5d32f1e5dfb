"""Pins of the FP64 oracle against facts fixed by mathematics and by the paper.

None of these re-types the oracle's formula: each checks it against an independent
statement (a brute-force sum, a closed form, an invariance of Eq. 1, a finite
difference, an adjoint identity, or a number printed in the paper).
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import ptycho_oracle as orc
from synthetic import workloads as syn

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(np.asarray(b).ravel()), 1e-300))


def crandn(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


# ----------------------------------------------------------------------------
# f4: propagation
# ----------------------------------------------------------------------------

def brute_dft2_centred(x):
    """O(F^4) DFT with exp(-2 pi i k n / F), 1/F scaling, zero frequency stored at F/2."""
    F = x.shape[0]
    out = np.zeros((F, F), np.complex128)
    for k1 in range(F):
        for k2 in range(F):
            acc = 0j
            for n1 in range(F):
                for n2 in range(F):
                    acc += x[n1, n2] * complex(math.cos(-2 * math.pi * (k1 * n1 + k2 * n2) / F),
                                               math.sin(-2 * math.pi * (k1 * n1 + k2 * n2) / F))
            out[(k1 + F // 2) % F, (k2 + F // 2) % F] = acc / F
    return out


def test_propagate_matches_bruteforce_dft_8x8():
    rng = np.random.default_rng(0)
    x = crandn(rng, 8, 8)
    assert rel(orc.f4_propagate(x), brute_dft2_centred(x)) < 1e-12


def test_propagate_adjoint_is_inverse_and_adjoint():
    rng = np.random.default_rng(1)
    x, y = crandn(rng, 16, 16), crandn(rng, 16, 16)
    assert rel(orc.f4_adjoint(orc.f4_propagate(x)), x) < 1e-12
    # <A x, y> = <x, A^H y>
    lhs = np.vdot(y, orc.f4_propagate(x))
    rhs = np.vdot(orc.f4_adjoint(y), x)
    assert abs(lhs - rhs) < 1e-10 * abs(lhs)


def test_parseval():
    rng = np.random.default_rng(2)
    for F in (8, 64, 256):
        x = crandn(rng, F, F)
        assert abs((np.abs(orc.f4_propagate(x)) ** 2).sum() / (np.abs(x) ** 2).sum() - 1) < 1e-12


def test_plane_wave_diffracts_to_one_pixel():
    """A flat probe on an object e^{2 pi i (u r + v c)/F} puts all power at (F/2+u, F/2+v)."""
    F, u, v = 32, 3, -5
    H = 48
    rr, cc = np.mgrid[0:H, 0:H]
    O = np.exp(2j * math.pi * (u * rr + v * cc) / F)
    P = np.full((1, 1, F, F), 0.7 + 0.2j)
    pos = np.array([[[4, 9]]], np.int32)
    I = orc.predict([O], P, pos)[0]
    expect = np.zeros((F, F))
    expect[F // 2 + u, F // 2 + v] = F * F * abs(0.7 + 0.2j) ** 2
    assert np.abs(I - expect).max() < 1e-9 * expect.max()


def test_point_probe_gives_flat_pattern_of_the_right_object_pixel():
    """A probe that is a delta at (r0, c0) diffracts to |P O(y+r0, x+c0)|^2 / F^2 everywhere."""
    rng = np.random.default_rng(3)
    F, H, W = 16, 30, 34
    O = crandn(rng, H, W)
    P = np.zeros((1, 1, F, F), np.complex128)
    r0, c0 = 3, 11
    P[0, 0, r0, c0] = 2.0 - 1.0j
    y, x = 7, 2
    I = orc.predict([O], P, np.array([[[y, x]]], np.int32))[0]
    flat = abs((2.0 - 1.0j) * O[y + r0, x + c0]) ** 2 / F ** 2
    assert np.abs(I - flat).max() < 1e-12 * flat


def test_single_mode_frame_equals_textbook_bruteforce():
    """L = M = 1 reduces to |DFT(P . O_patch)|^2 with the patch read pixel by pixel."""
    rng = np.random.default_rng(4)
    F, H, W = 8, 13, 15
    O = crandn(rng, H, W)
    P = crandn(rng, 1, 1, F, F)
    y, x = 4, 6
    ex = np.zeros((F, F), np.complex128)
    for r in range(F):
        for c in range(F):
            ex[r, c] = P[0, 0, r, c] * O[y + r, x + c]
    expect = np.abs(brute_dft2_centred(ex)) ** 2
    got = orc.predict([O], P, np.array([[[y, x]]], np.int32))[0]
    assert rel(got, expect) < 1e-12


# ----------------------------------------------------------------------------
# Eq. 1 structure: incoherent sums and invariances
# ----------------------------------------------------------------------------

def test_incoherent_sum_is_sum_of_single_mode_patterns():
    w = syn.tiny_workload(F=16, L=2, M=3, seed=11)
    full = orc.predict(w.O_true, w.P_true, w.pos)
    acc = np.zeros_like(full)
    for l in range(w.L):
        for m in range(w.M):
            acc += orc.predict([w.O_true[l]], w.P_true[l:l + 1, m:m + 1], w.pos[l:l + 1])
    assert rel(full, acc) < 1e-12


def test_unitary_mode_mixing_and_global_phase_invariance():
    w = syn.tiny_workload(F=16, L=2, M=3, seed=12)
    rng = np.random.default_rng(5)
    base = orc.predict(w.O_true, w.P_true, w.pos)
    P2 = np.empty_like(w.P_true)
    for l in range(w.L):
        q, _ = np.linalg.qr(crandn(rng, w.M, w.M))
        P2[l] = np.einsum("ab,bij->aij", q, w.P_true[l])
    assert rel(orc.predict(w.O_true, P2, w.pos), base) < 1e-12
    assert rel(orc.predict(w.O_true, w.P_true * np.exp(1.234j), w.pos), base) < 1e-12
    # and O -> c O, P -> P / c
    c = 1.7 * np.exp(0.3j)
    assert rel(orc.predict([o * c for o in w.O_true], w.P_true / c, w.pos), base) < 1e-12


def test_power_coefficient_scales_the_pattern_quadratically():
    w = syn.tiny_workload(F=16, L=2, M=2, seed=13)
    sigma = np.linspace(0.5, 1.5, w.J)
    a = orc.predict(w.O_true, w.P_true, w.pos, sigma=sigma)
    b = orc.predict(w.O_true, w.P_true, w.pos)
    assert rel(a, b * (sigma ** 2)[:, None, None]) < 1e-12


def test_patch_outside_object_is_an_error():
    w = syn.tiny_workload(F=16, L=1, M=1, seed=14)
    pos = w.pos.copy()
    pos[0, 0] = (w.obj_shapes[0][0] - 15, 0)
    with pytest.raises(ValueError):
        orc.predict(w.O_true, w.P_true, pos)
    pos[0, 0] = (-1, 0)
    with pytest.raises(ValueError):
        orc.predict(w.O_true, w.P_true, pos)


# ----------------------------------------------------------------------------
# losses
# ----------------------------------------------------------------------------

def test_loss_derivative_matches_finite_difference_per_pixel():
    rng = np.random.default_rng(6)
    I = rng.uniform(0.5, 20, size=200)
    Ih = np.floor(rng.uniform(0, 25, size=200))
    for kind in orc.LOSS_KINDS:
        h = 1e-6
        fd = (orc.loss_terms(I + h, Ih, kind, 1e-3) - orc.loss_terms(I - h, Ih, kind, 1e-3)) / (2 * h)
        assert rel(orc.loss_derivative(I, Ih, kind, 1e-3), fd) < 1e-7


def test_poisson_deviance_differs_from_plain_nll_by_a_constant():
    rng = np.random.default_rng(7)
    Ih = np.floor(rng.uniform(0, 25, size=100))
    I1, I2 = rng.uniform(0.5, 20, size=100), rng.uniform(0.5, 20, size=100)
    nll = lambda I: I - Ih * np.log(I)  # noqa: E731
    d1 = orc.loss_terms(I1, Ih, "poisson", 0.0) - nll(I1)
    d2 = orc.loss_terms(I2, Ih, "poisson", 0.0) - nll(I2)
    assert np.abs(d1 - d2).max() < 1e-10
    # and the deviance vanishes at I = Ihat (0 log 0 := 0 at empty pixels)
    assert np.abs(orc.loss_terms(Ih, Ih, "poisson", 0.0)).max() < 1e-12


def test_amplitude_loss_is_squared_modulus_difference():
    I = np.array([4.0, 9.0, 0.25])
    Ih = np.array([1.0, 16.0, 0.0])
    assert np.allclose(orc.loss_terms(I, Ih, "amplitude", 0.0), [1.0, 1.0, 0.25], atol=1e-15)


@pytest.mark.parametrize("kind", orc.LOSS_KINDS)
@pytest.mark.parametrize("remap", [False, True])
def test_zero_loss_and_zero_gradient_at_noiseless_truth(kind, remap):
    w = syn.tiny_workload(F=16, L=2, M=2, seed=15, remap=remap, with_bg=True, with_sigma=True)
    taps = orc.remap_taps(w.F, 2e-3, 15e-6, math.radians(70)) if remap else None
    Ih = orc.predict(w.O_true, w.P_true, w.pos, w.sigma, w.bg, taps)
    L, gO, gP = orc.gradient(w.O_true, w.P_true, w.pos, Ih, kind, 0.0, w.sigma, w.bg, None, taps)
    assert abs(L) < 1e-18 * max(1.0, float(Ih.sum()))
    assert max(np.abs(g).max() for g in gO) < 1e-12
    assert np.abs(gP).max() < 1e-12


# ----------------------------------------------------------------------------
# gradient: central finite differences
# ----------------------------------------------------------------------------

def _fd_case(kind, remap, with_mask):
    w = syn.tiny_workload(F=16, L=2, M=2, seed=21, remap=remap, loss=kind, with_sigma=True,
                          with_bg=True)
    taps = orc.remap_taps(w.F, 2e-3, 15e-6, math.radians(70)) if remap else None
    Ih = syn.poisson_measure(orc.predict(w.O_true, w.P_true, w.pos, w.sigma, w.bg, taps), 3)
    mask = None
    if with_mask:
        mask = (np.random.default_rng(9).uniform(size=(w.J, w.F, w.F)) > 0.2).astype(np.uint8)
    return w, taps, Ih, mask


@pytest.mark.parametrize("kind", orc.LOSS_KINDS)
@pytest.mark.parametrize("remap,with_mask", [(False, False), (True, True)])
def test_gradient_matches_central_finite_differences(kind, remap, with_mask):
    w, taps, Ih, mask = _fd_case(kind, remap, with_mask)
    eps = 1e-3
    args = (w.pos, Ih, kind, eps, w.sigma, w.bg, mask, taps)
    _, gO, gP = orc.gradient(w.O0, w.P0, *args)
    rng = np.random.default_rng(10)
    h = 1e-5
    L0 = abs(orc.loss(w.O0, w.P0, *args))
    noise = 50 * 2.2e-16 * L0 / h        # rounding floor of a central difference
    checks = 0
    for _ in range(6):
        l = int(rng.integers(w.L))
        # an object pixel inside the scanned area
        y, x = w.pos[l][int(rng.integers(w.J))] + rng.integers(0, w.F, size=2)
        for comp in (1.0, 1.0j):
            Op = [o.copy() for o in w.O0]
            Om = [o.copy() for o in w.O0]
            Op[l][y, x] += h * comp
            Om[l][y, x] -= h * comp
            fd = (orc.loss(Op, w.P0, *args) - orc.loss(Om, w.P0, *args)) / (2 * h)
            an = gO[l][y, x].real if comp == 1.0 else gO[l][y, x].imag
            assert abs(fd - an) <= 1e-6 * abs(an) + noise, (fd, an, noise)
            checks += 1
        m = int(rng.integers(w.M))
        r, c = rng.integers(0, w.F, size=2)
        for comp in (1.0, 1.0j):
            Pp, Pm = w.P0.copy(), w.P0.copy()
            Pp[l, m, r, c] += h * comp
            Pm[l, m, r, c] -= h * comp
            fd = (orc.loss(w.O0, Pp, *args) - orc.loss(w.O0, Pm, *args)) / (2 * h)
            an = gP[l, m, r, c].real if comp == 1.0 else gP[l, m, r, c].imag
            assert abs(fd - an) <= 1e-6 * abs(an) + noise, (fd, an, noise)
            checks += 1
    assert checks == 24


def test_gradient_directional_derivative():
    """dL along a random complex direction d equals Re<g, d> summed over all parameters."""
    w, taps, Ih, mask = _fd_case("poisson", True, True)
    args = (w.pos, Ih, "poisson", 1e-3, w.sigma, w.bg, mask, taps)
    _, gO, gP = orc.gradient(w.O0, w.P0, *args)
    rng = np.random.default_rng(11)
    dO = [crandn(rng, *o.shape) for o in w.O0]
    dP = crandn(rng, *w.P0.shape)
    h = 1e-6
    Lp = orc.loss([o + h * d for o, d in zip(w.O0, dO)], w.P0 + h * dP, *args)
    Lm = orc.loss([o - h * d for o, d in zip(w.O0, dO)], w.P0 - h * dP, *args)
    fd = (Lp - Lm) / (2 * h)
    an = sum(np.real(np.vdot(g, d)) for g, d in zip(gO, dO)) + np.real(np.vdot(gP, dP))
    assert abs(fd - an) < 1e-6 * abs(an)


def test_gradient_vanishes_outside_the_scanned_area():
    w, taps, Ih, mask = _fd_case("amplitude", False, False)
    _, gO, _ = orc.gradient(w.O0, w.P0, w.pos, Ih, "amplitude", 1e-3, w.sigma, w.bg, None, None)
    for l in range(w.L):
        cov = np.zeros(w.obj_shapes[l], bool)
        for j in range(w.J):
            y, x = w.pos[l][j]
            cov[y:y + w.F, x:x + w.F] = True
        assert np.abs(gO[l][~cov]).max() == 0.0


def test_masked_pixels_do_not_enter_the_loss():
    w, taps, Ih, mask = _fd_case("amplitude", False, True)
    a = orc.loss(w.O0, w.P0, w.pos, Ih, "amplitude", 1e-3, w.sigma, w.bg, mask, None)
    Ih2 = Ih.copy()
    Ih2[mask == 0] += 1000.0
    b = orc.loss(w.O0, w.P0, w.pos, Ih2, "amplitude", 1e-3, w.sigma, w.bg, mask, None)
    assert a == b


# ----------------------------------------------------------------------------
# power coefficients sigma_j and background N
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("kind", orc.LOSS_KINDS)
@pytest.mark.parametrize("remap,with_mask", [(False, False), (True, True)])
def test_sigma_bg_gradient_matches_central_finite_differences(kind, remap, with_mask):
    w, taps, Ih, mask = _fd_case(kind, remap, with_mask)
    eps = 1e-3
    _, g_s, g_bg = orc.gradient_sigma_bg(w.O0, w.P0, w.pos, Ih, kind, eps, w.sigma, w.bg, mask, taps)

    def L(sig, bg):
        return orc.loss(w.O0, w.P0, w.pos, Ih, kind, eps, sig, bg, mask, taps)

    h = 1e-5
    L0 = abs(L(w.sigma, w.bg))
    noise = 50 * 2.2e-16 * L0 / h
    rng = np.random.default_rng(12)
    for j in rng.choice(w.J, size=3, replace=False):
        sp, sm = w.sigma.astype(np.float64).copy(), w.sigma.astype(np.float64).copy()
        sp[j] += h
        sm[j] -= h
        fd = (L(sp, w.bg) - L(sm, w.bg)) / (2 * h)
        assert abs(fd - g_s[j]) <= 1e-6 * abs(g_s[j]) + noise, (fd, g_s[j])
    for _ in range(4):
        r, c = rng.integers(w.F // 4, 3 * w.F // 4, size=2)
        bp, bm = w.bg.astype(np.float64).copy(), w.bg.astype(np.float64).copy()
        bp[r, c] += h
        bm[r, c] -= h
        fd = (L(w.sigma, bp) - L(w.sigma, bm)) / (2 * h)
        assert abs(fd - g_bg[r, c]) <= 1e-6 * abs(g_bg[r, c]) + noise, (fd, g_bg[r, c])


def test_sigma_gradient_equals_its_intensity_form():
    """Parseval: sum_r conj(psi) chi = 2 sum_k G_k |Psi_k|^2, so
    sigma_j dL/dsigma_j = 2 sum_u G_ju (I_ju - N_u) on the model grid."""
    w, taps, Ih, mask = _fd_case("poisson", True, True)
    eps = 1e-3
    _, g_s, _ = orc.gradient_sigma_bg(w.O0, w.P0, w.pos, Ih, "poisson", eps, w.sigma, w.bg, mask, taps)
    for j in range(w.J):
        _, Psi = orc.frame_fields(w.O0, w.P0, w.pos, j, w.sigma)
        I_sum = (np.abs(Psi) ** 2).sum(axis=(0, 1))
        Ic = orc.f5_measure(I_sum, w.bg, taps)
        mk = orc.frame_mask(mask, j, w.F, taps)
        D = np.where(mk, orc.loss_derivative(Ic, Ih[j], "poisson", eps), 0.0)
        G = orc.remap_adjoint(D, taps)
        exp = 2.0 * float((G * I_sum).sum()) / float(w.sigma[j])
        assert abs(g_s[j] - exp) < 1e-9 * max(abs(exp), 1e-30), (j, g_s[j], exp)


def test_sigma_gradient_matches_probe_gradient_along_scaling():
    """sigma_j multiplies P, so scaling every sigma by c equals scaling P by c:
    sum_j sigma_j dL/dsigma_j = Re <P, grad P> (sum over all modes)."""
    w, taps, Ih, mask = _fd_case("amplitude", True, True)
    args = (w.pos, Ih, "amplitude", 1e-3, w.sigma, w.bg, mask, taps)
    _, _, gP = orc.gradient(w.O0, w.P0, *args)
    _, g_s, _ = orc.gradient_sigma_bg(w.O0, w.P0, *args)
    lhs = float((w.sigma * g_s).sum())
    rhs = float(np.real(np.vdot(w.P0, gP)))
    assert abs(lhs - rhs) < 1e-10 * abs(rhs)


@pytest.mark.parametrize("remap", [False, True])
def test_sigma_bg_gradients_vanish_at_noiseless_truth(remap):
    w = syn.tiny_workload(F=16, L=2, M=2, seed=15, remap=remap, with_bg=True, with_sigma=True)
    taps = orc.remap_taps(w.F, 2e-3, 15e-6, math.radians(70)) if remap else None
    Ih = orc.predict(w.O_true, w.P_true, w.pos, w.sigma, w.bg, taps)
    _, g_s, g_bg = orc.gradient_sigma_bg(w.O_true, w.P_true, w.pos, Ih, "poisson", 0.0, w.sigma, w.bg, None, taps)
    assert np.abs(g_s).max() < 1e-12 and np.abs(g_bg).max() < 1e-12


def test_sigma_gradient_is_zero_for_frames_not_requested():
    w, taps, Ih, mask = _fd_case("poisson", False, False)
    _, g_s, g_bg = orc.gradient_sigma_bg(w.O0, w.P0, w.pos, Ih, "poisson", 1e-3, w.sigma, w.bg, None, None,
                                         frames=[1, 3])
    _, g1, b1 = orc.gradient_sigma_bg(w.O0, w.P0, w.pos, Ih, "poisson", 1e-3, w.sigma, w.bg, None, None, frames=[1])
    _, g3, b3 = orc.gradient_sigma_bg(w.O0, w.P0, w.pos, Ih, "poisson", 1e-3, w.sigma, w.bg, None, None, frames=[3])
    assert np.count_nonzero(g_s) == 2 and g_s[1] == g1[1] and g_s[3] == g3[3]
    assert np.abs(g_bg - (b1 + b3)).max() < 1e-12 * np.abs(g_bg).max()


def test_adam_real_first_step_closed_form():
    rng = np.random.default_rng(16)
    th, g = rng.normal(size=9), rng.normal(size=9)
    m, v = np.zeros(9), np.zeros(9)
    out = orc.adam_update_real(th, g, m, v, 1, 0.05)
    assert np.abs(out - (th - 0.05 * g / (np.abs(g) + 1e-8))).max() < 1e-15


# ----------------------------------------------------------------------------
# tilted-plane remap
# ----------------------------------------------------------------------------

def test_remap_dot_product_identity():
    taps = orc.remap_taps(64, 0.02, 15e-6, math.radians(70))
    rng = np.random.default_rng(12)
    x, y = rng.standard_normal((64, 64)), rng.standard_normal((64, 64))
    lhs = float((orc.remap_apply(x, taps) * y).sum())
    rhs = float((x * orc.remap_adjoint(y, taps)).sum())
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_remap_is_near_identity_without_tilt():
    taps = orc.remap_taps(64, 88e-3, 15e-6, 0.0)
    assert taps.valid.all()
    yy, xx = np.mgrid[0:64, 0:64]
    assert np.abs(taps.yhat - yy).max() < 1e-3
    assert np.abs(taps.xhat - xx).max() < 1e-3
    rng = np.random.default_rng(13)
    I = rng.uniform(size=(64, 64))
    assert np.abs(orc.remap_apply(I, taps) - I).max() < 2e-3


def test_remap_keeps_a_constant_inside_the_field_of_view():
    taps = orc.remap_taps(64, 0.02, 15e-6, math.radians(70))
    out = orc.remap_apply(np.full((64, 64), 3.25), taps)
    assert not taps.valid.all() and taps.valid.any()
    assert np.abs(out[taps.valid] - 3.25).max() < 1e-12
    assert (out[~taps.valid] == 0).all()
    # the specular pixel maps onto itself
    assert taps.yhat[32, 32] == pytest.approx(32.0, abs=1e-9)
    assert taps.xhat[32, 32] == pytest.approx(32.0, abs=1e-12)


def test_remap_geometry_against_the_paper_numbers():
    """NA, tilt-corrected pixel ratio and resolution printed in the paper."""
    g = json.load(open(os.path.join(GOLDEN, "paper_geometry.json")))
    F = g["camera_pixels"]["value"]
    z, p = g["z_m"]["value"], g["det_pixel_m"]["value"]
    alpha = math.radians(g["tilt_deg"]["value"])
    taps = orc.remap_taps(F, z, p, alpha)
    # direction cosine along the untilted axis at the camera edge = detection NA
    na_x = abs(taps.xhat[F // 2, 0] - F / 2) * (p / z)
    assert na_x == pytest.approx(g["na"]["value"][0], rel=0.02)
    # the tilt-corrected grid is 15 um x 5 um: model spacing along the tilt / across it
    px = g["tilt_corrected_pixel_um"]["value"]
    assert taps.db / taps.da == pytest.approx(px[1] / px[0], rel=0.04)
    # the specular pixel maps to the grid centre and rows near it map one to one
    assert taps.yhat[F // 2, F // 2] == pytest.approx(F / 2, abs=1e-6)
    assert taps.yhat[F // 2 + 1, F // 2] - taps.yhat[F // 2, F // 2] == pytest.approx(1.0, abs=1e-3)
    # diffraction-limited resolution lambda / (2 NA)
    assert g["lambda_m"]["value"] / (2 * na_x) == pytest.approx(g["resolution_m"]["value"], rel=0.10)


# ----------------------------------------------------------------------------
# data-side tilt correction
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("F,z,alpha_deg", [(64, 0.02, 70.0), (256, 0.088, 70.0), (2048, 0.088, 70.0),
                                           (128, 0.05, 35.0)])
def test_tilt_inverse_map_undoes_the_remap_geometry(F, z, alpha_deg):
    """Camera pixel -> fractional model index (remap_taps) -> camera position
    (tilt_camera_index) returns the pixel: the two maps are each other's inverse."""
    p, alpha = 15e-6, math.radians(alpha_deg)
    taps = orc.remap_taps(F, z, p, alpha)
    y, x, ok = orc.tilt_camera_index(F, z, p, alpha, taps.yhat, taps.xhat)
    yy, xx = np.mgrid[0:F, 0:F]
    assert ok.all()
    assert np.abs(y - yy).max() < 1e-9 * F and np.abs(x - xx).max() < 1e-9 * F
    # the specular direction sits at the centre of both grids
    yc, xc, okc = orc.tilt_camera_index(F, z, p, alpha, F / 2, F / 2)
    assert okc and abs(yc - F / 2) < 1e-9 and abs(xc - F / 2) < 1e-9


def test_tilt_correction_reproduces_affine_camera_patterns_exactly():
    """Bilinear interpolation is exact for patterns affine in the camera indices, so the
    corrected pattern is the affine function at the mapped camera positions; a swapped
    axis, weight or tap would break it (different slopes along y and x)."""
    F, z, p, alpha = 64, 0.02, 15e-6, math.radians(70)
    yy, xx = np.mgrid[0:F, 0:F].astype(np.float64)
    coef = [(2.0, 0.3, -0.7), (5.0, -1.25, 0.5)]
    I_cam = np.stack([c0 + c1 * yy + c2 * xx for c0, c1, c2 in coef])
    out, mask = orc.tilt_correct(I_cam, z, p, alpha)
    y, x, _ = orc.tilt_camera_index(F, z, p, alpha, yy, xx)
    assert mask.any() and not mask.all()
    for j, (c0, c1, c2) in enumerate(coef):
        m = mask[j]
        assert np.abs(out[j][m] - (c0 + c1 * y[m] + c2 * x[m])).max() < 1e-12
        assert (out[j][~m] == 0).all()
    # the mask is the set of model pixels whose taps lie inside the crop
    inside = (y >= 0) & (y < F - 1) & (x >= 0) & (x < F - 1)
    assert (mask[0] == inside).all() and (mask[1] == inside).all()


def test_tilt_correction_without_tilt_is_near_identity():
    F = 64
    yy, xx = np.mgrid[0:F, 0:F].astype(np.float64)
    y, x, ok = orc.tilt_camera_index(F, 88e-3, 15e-6, 0.0, yy, xx)
    assert ok.all()
    assert np.abs(y - yy).max() < 1e-3 and np.abs(x - xx).max() < 1e-3
    I = np.exp(-((yy - 30) ** 2 + (xx - 34) ** 2) / 200.0)[None]
    out, mask = orc.tilt_correct(I, 88e-3, 15e-6, 0.0)
    inner = np.zeros((F, F), bool)
    inner[1:F - 1, 1:F - 1] = True
    assert mask[0][inner].all()
    assert np.abs(out[0] - I[0])[inner].max() < 1e-4


def test_tilt_correction_masks_the_model_pixels_that_touch_a_rejected_camera_pixel():
    """A camera pixel outside [lo, hi) removes exactly the model pixels whose bilinear
    footprint (floor(y)..floor(y)+1, floor(x)..floor(x)+1) contains it."""
    F, z, p, alpha = 64, 0.02, 15e-6, math.radians(70)
    I_cam = np.full((2, F, F), 10.0)
    I_cam[0, 30, 41] = 65535.0          # saturated (the upper threshold itself is rejected)
    I_cam[1, 12, 7] = 1.0               # below the noise threshold (< lo)
    I_cam[1, 40, 20] = 4.0              # the lower threshold itself is kept
    out, mask = orc.tilt_correct(I_cam, z, p, alpha, lo=4.0, hi=65535.0)
    yy, xx = np.mgrid[0:F, 0:F].astype(np.float64)
    y, x, _ = orc.tilt_camera_index(F, z, p, alpha, yy, xx)
    inside = (y >= 0) & (y < F - 1) & (x >= 0) & (x < F - 1)
    fy, fx = np.floor(np.where(inside, y, -9)), np.floor(np.where(inside, x, -9))
    for j, (cy, cx) in enumerate([(30, 41), (12, 7)]):
        touches = inside & ((fy == cy) | (fy == cy - 1)) & ((fx == cx) | (fx == cx - 1))
        assert touches.any()
        assert (mask[j] == (inside & ~touches)).all()
        if j == 0:
            assert np.abs(out[j][mask[j]] - 10.0).max() < 1e-12


def test_tilt_correction_undoes_the_in_model_remap_of_smooth_patterns():
    """Remap a smooth model-grid pattern to the camera (remap_apply) and correct it back:
    the result is the pattern again, to the error of two bilinear interpolations."""
    F, z, p, alpha = 64, 0.02, 15e-6, math.radians(70)
    taps = orc.remap_taps(F, z, p, alpha)
    yy, xx = np.mgrid[0:F, 0:F].astype(np.float64)
    I = 1.0 + np.exp(-((yy - 33) ** 2 / 300.0 + (xx - 29) ** 2 / 150.0))
    cam = orc.remap_apply(I, taps)
    out, mask = orc.tilt_correct(cam[None], z, p, alpha)
    y, x, _ = orc.tilt_camera_index(F, z, p, alpha, yy, xx)
    # model pixels whose four camera taps all received a value from the remap
    y0 = np.clip(np.floor(y), 0, F - 2).astype(int)
    x0 = np.clip(np.floor(x), 0, F - 2).astype(int)
    v = taps.valid
    full = mask[0] & v[y0, x0] & v[y0 + 1, x0] & v[y0, x0 + 1] & v[y0 + 1, x0 + 1]
    assert full.sum() > F * F // 2
    assert np.abs(out[0] - I)[full].max() < 5e-3


# ----------------------------------------------------------------------------
# object regularisation (L1 and TV of the smoothed amplitude)
# ----------------------------------------------------------------------------

def test_regulariser_gradient_matches_central_finite_differences():
    rng = np.random.default_rng(41)
    O = [crandn(rng, 5, 7), crandn(rng, 4, 3)]
    mu1, mutv, eta = 0.3, 0.7, 0.05
    _, g = orc.regulariser(O, mu1, mutv, eta)
    h = 1e-6
    for l, (r, c) in [(0, (0, 0)), (0, (2, 3)), (0, (4, 6)), (0, (4, 0)), (1, (1, 2)), (1, (3, 2))]:
        for part, unit in (("re", 1.0), ("im", 1j)):
            Op = [o.copy() for o in O]
            Om = [o.copy() for o in O]
            Op[l][r, c] += h * unit
            Om[l][r, c] -= h * unit
            fd = (orc.regulariser(Op, mu1, mutv, eta)[0] - orc.regulariser(Om, mu1, mutv, eta)[0]) / (2 * h)
            an = g[l][r, c].real if part == "re" else g[l][r, c].imag
            assert fd == pytest.approx(an, rel=1e-6, abs=1e-9), (l, r, c, part)


def test_regulariser_of_a_constant_amplitude_object():
    """|O| constant: every difference is 0, so TV = N eta and its gradient vanishes; the L1
    part is N a with gradient mu_l1 O / a."""
    rng = np.random.default_rng(42)
    ph = rng.uniform(-np.pi, np.pi, size=(6, 9))
    O = [0.8 * np.exp(1j * ph)]
    mu1, mutv, eta = 0.4, 1.3, 0.02
    R, g = orc.regulariser(O, mu1, mutv, eta)
    a = math.sqrt(0.64 + eta * eta)
    assert R == pytest.approx(54 * (mu1 * a + mutv * eta), rel=1e-13)
    assert np.abs(g[0] - mu1 * O[0] / a).max() < 1e-13
    R0, g0 = orc.regulariser(O, 0.0, mutv, eta)
    assert np.abs(g0[0]).max() < 1e-13


def test_regulariser_of_a_linear_amplitude_ramp():
    """One row with amplitudes 0, s, 2s, ...: W-1 differences of s and one 0 at the end."""
    W, s, eta = 8, 0.25, 1e-3
    amp = s * np.arange(W, dtype=np.float64)
    a = np.sqrt(amp ** 2 + eta ** 2)
    O = [(amp * np.exp(0.3j))[None, :]]
    R, _ = orc.regulariser(O, 0.0, 1.0, eta)
    exp = float(np.sqrt(np.diff(a) ** 2 + eta ** 2).sum()) + eta
    assert R == pytest.approx(exp, rel=1e-14)
    assert R == pytest.approx((W - 1) * s, rel=1e-3)


def test_regulariser_is_invariant_under_a_global_phase():
    rng = np.random.default_rng(43)
    O = [crandn(rng, 6, 5)]
    R, g = orc.regulariser(O, 0.2, 0.9, 0.03)
    Rr, gr = orc.regulariser([O[0] * np.exp(0.7j)], 0.2, 0.9, 0.03)
    assert Rr == pytest.approx(R, rel=1e-13)
    assert np.abs(gr[0] - g[0] * np.exp(0.7j)).max() < 1e-13


# ----------------------------------------------------------------------------
# Adam
# ----------------------------------------------------------------------------

def test_adam_first_step_closed_form():
    rng = np.random.default_rng(14)
    th = crandn(rng, 5, 7)
    g = crandn(rng, 5, 7)
    m = np.zeros((5, 7, 2))
    v = np.zeros((5, 7, 2))
    lr, eps = 0.01, 1e-8
    out = orc.adam_update(th, g, m, v, 1, lr, 0.9, 0.999, eps)
    exp = th - lr * (g.real / (np.abs(g.real) + eps) + 1j * g.imag / (np.abs(g.imag) + eps))
    assert np.abs(out - exp).max() < 1e-15
    assert np.allclose(m[..., 0], 0.1 * g.real) and np.allclose(v[..., 1], 0.001 * g.imag ** 2)


def test_adam_second_step_against_hand_expansion():
    g1, g2 = 0.3, -0.7
    th = np.array([1.0 + 0j])
    m, v = np.zeros((1, 2)), np.zeros((1, 2))
    th = orc.adam_update(th, np.array([g1 + 0j]), m, v, 1, 0.1)
    th = orc.adam_update(th, np.array([g2 + 0j]), m, v, 2, 0.1)
    m2 = 0.9 * 0.1 * g1 + 0.1 * g2
    v2 = 0.999 * 0.001 * g1 ** 2 + 0.001 * g2 ** 2
    step2 = 0.1 * (m2 / (1 - 0.81)) / (math.sqrt(v2 / (1 - 0.999 ** 2)) + 1e-8)
    exp = 1.0 - 0.1 * g1 / (abs(g1) + 1e-8) - step2
    assert abs(th[0].real - exp) < 1e-14 and th[0].imag == 0.0


# ----------------------------------------------------------------------------
# f2 with fractional scan offsets (Fourier shift theorem) and the position gradient
# ----------------------------------------------------------------------------

def _subpixel_case(kind="poisson", remap=True, seed=41):
    w = syn.tiny_workload(F=16, L=2, M=2, seed=seed, remap=remap, loss=kind, with_sigma=True, with_bg=True)
    taps = orc.remap_taps(w.F, 2e-3, 15e-6, math.radians(70)) if remap else None
    rng = np.random.default_rng(seed + 1)
    delta = rng.uniform(-0.5, 0.5, size=(w.L, w.J, 2))
    return w, taps, delta


def test_subpixel_shift_zero_and_whole_pixels():
    """delta = 0 leaves the patch alone; a whole-pixel delta is a cyclic roll of the patch
    (sampling at r + delta), in either axis and sign."""
    rng = np.random.default_rng(50)
    p = crandn(rng, 16, 16)
    assert rel(orc.f2_subpixel(p, (0.0, 0.0)), p) < 1e-14
    assert rel(orc.f2_subpixel(p, (1.0, 0.0)), np.roll(p, -1, axis=0)) < 1e-12
    assert rel(orc.f2_subpixel(p, (0.0, -1.0)), np.roll(p, 1, axis=1)) < 1e-12
    assert rel(orc.f2_subpixel(p, (-2.0, 3.0)), np.roll(np.roll(p, 2, axis=0), -3, axis=1)) < 1e-12


def test_subpixel_shift_of_band_limited_plane_waves():
    """A sum of in-band plane waves sampled on the grid, shifted by a fraction, equals the same
    function sampled at the shifted points (the shift theorem is exact for it)."""
    F = 16
    n = np.arange(F)
    rng = np.random.default_rng(51)
    terms = [(int(a), int(b), complex(c)) for a, b, c in zip(rng.integers(-7, 8, 5), rng.integers(-7, 8, 5),
                                                               crandn(rng, 5))]

    def sample(dy, dx):
        y = (n + dy)[:, None]
        x = (n + dx)[None, :]
        return sum(c * np.exp(2j * np.pi * (a * y + b * x) / F) for a, b, c in terms)

    d = (0.37, -0.81)
    assert rel(orc.f2_subpixel(sample(0.0, 0.0), d), sample(*d)) < 1e-12


def test_subpixel_shift_is_unitary_composes_and_has_the_stated_adjoint():
    rng = np.random.default_rng(52)
    p, q = crandn(rng, 16, 16), crandn(rng, 16, 16)
    d1, d2 = (0.3, -0.45), (-0.2, 0.7)
    assert abs(np.linalg.norm(orc.f2_subpixel(p, d1)) - np.linalg.norm(p)) < 1e-12 * np.linalg.norm(p)
    two = orc.f2_subpixel(orc.f2_subpixel(p, d1), d2)
    assert rel(two, orc.f2_subpixel(p, (d1[0] + d2[0], d1[1] + d2[1]))) < 1e-12
    lhs = np.vdot(q, orc.f2_subpixel(p, d1))
    rhs = np.vdot(orc.f2_subpixel_adjoint(q, d1), p)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_subpixel_derivative_matches_finite_difference_of_the_shift():
    rng = np.random.default_rng(53)
    p = crandn(rng, 16, 16)
    d = (0.21, -0.34)
    h = 1e-6
    for a in range(2):
        dp = np.array(d)
        dm = np.array(d)
        dp[a] += h
        dm[a] -= h
        fd = (orc.f2_subpixel(p, dp) - orc.f2_subpixel(p, dm)) / (2 * h)
        assert rel(orc.f2_subpixel_derivative(p, d, a), fd) < 1e-8


def test_zero_offsets_reduce_to_the_integer_model():
    w, taps, _ = _subpixel_case()
    Ih = syn.poisson_measure(orc.predict(w.O_true, w.P_true, w.pos, w.sigma, w.bg, taps), 5)
    zero = np.zeros((w.L, w.J, 2))
    a = orc.gradient(w.O0, w.P0, w.pos, Ih, "poisson", 1e-3, w.sigma, w.bg, None, taps)
    b = orc.gradient(w.O0, w.P0, w.pos, Ih, "poisson", 1e-3, w.sigma, w.bg, None, taps, delta=zero)
    assert abs(a[0] - b[0]) <= 1e-13 * abs(a[0])
    assert max(rel(x, y) for x, y in zip(a[1], b[1])) < 1e-12 and rel(a[2], b[2]) < 1e-12


@pytest.mark.parametrize("kind", orc.LOSS_KINDS)
@pytest.mark.parametrize("remap", [False, True])
def test_position_gradient_matches_central_finite_differences(kind, remap):
    w, taps, delta = _subpixel_case(kind, remap)
    Ih = syn.poisson_measure(orc.predict(w.O_true, w.P_true, w.pos, w.sigma, w.bg, taps), 6)
    args = (w.pos, Ih, kind, 1e-3)
    kw = dict(sigma=w.sigma, bg=w.bg, taps=taps)
    L0, gd = orc.gradient_delta(w.O0, w.P0, *args, delta, **kw)
    assert abs(L0 - orc.loss(w.O0, w.P0, *args, delta=delta, **kw)) <= 1e-13 * abs(L0)
    h = 1e-6
    noise = 50 * 2.2e-16 * abs(L0) / h
    rng = np.random.default_rng(54)
    for _ in range(6):
        l, j, a = int(rng.integers(w.L)), int(rng.integers(w.J)), int(rng.integers(2))
        dp, dm = delta.copy(), delta.copy()
        dp[l, j, a] += h
        dm[l, j, a] -= h
        fd = (orc.loss(w.O0, w.P0, *args, delta=dp, **kw) - orc.loss(w.O0, w.P0, *args, delta=dm, **kw)) / (2 * h)
        assert abs(fd - gd[l, j, a]) <= 1e-6 * abs(gd[l, j, a]) + noise, (l, j, a, fd, gd[l, j, a])


def test_object_and_probe_gradients_with_offsets_match_finite_differences():
    w, taps, delta = _subpixel_case("amplitude", True)
    Ih = syn.poisson_measure(orc.predict(w.O_true, w.P_true, w.pos, w.sigma, w.bg, taps), 7)
    args = (w.pos, Ih, "amplitude", 1e-3, w.sigma, w.bg, None, taps)
    _, gO, gP = orc.gradient(w.O0, w.P0, *args, delta=delta)
    rng = np.random.default_rng(55)
    dO = [crandn(rng, *o.shape) for o in w.O0]
    dP = crandn(rng, *w.P0.shape)
    h = 1e-6
    Lp = orc.loss([o + h * d for o, d in zip(w.O0, dO)], w.P0 + h * dP, *args, delta=delta)
    Lm = orc.loss([o - h * d for o, d in zip(w.O0, dO)], w.P0 - h * dP, *args, delta=delta)
    fd = (Lp - Lm) / (2 * h)
    an = sum(np.real(np.vdot(g, d)) for g, d in zip(gO, dO)) + np.real(np.vdot(gP, dP))
    assert abs(fd - an) < 1e-6 * abs(an)


def test_position_gradient_vanishes_at_noiseless_truth_and_for_frames_not_requested():
    w, taps, delta = _subpixel_case()
    Ih = orc.predict(w.O_true, w.P_true, w.pos, w.sigma, w.bg, taps, delta=delta)
    L, gd = orc.gradient_delta(w.O_true, w.P_true, w.pos, Ih, "poisson", 0.0, delta, w.sigma, w.bg, None, taps)
    assert abs(L) < 1e-18 * float(Ih.sum()) and np.abs(gd).max() < 1e-10
    Ih2 = syn.poisson_measure(Ih, 8)
    _, gd2 = orc.gradient_delta(w.O0, w.P0, w.pos, Ih2, "poisson", 1e-3, delta, w.sigma, w.bg, None, taps,
                                frames=[1, 4])
    assert np.all(gd2[:, [0, 2, 3, 5, 6, 7, 8], :] == 0.0) and np.abs(gd2[:, [1, 4], :]).max() > 0


# ----------------------------------------------------------------------------
# propagation distance z (through the tilted-plane remap)
# ----------------------------------------------------------------------------

def test_remap_index_rates_match_finite_differences_and_vanish_at_the_specular_pixel():
    F, z, p, al = 32, 4e-3, 15e-6, math.radians(70)
    dy, dx = orc.remap_index_rates(F, z, p, al)
    h = 1e-7 * z
    tp, tm = orc.remap_taps(F, z + h, p, al), orc.remap_taps(F, z - h, p, al)
    assert rel(dy, (tp.yhat - tm.yhat) / (2 * h)) < 1e-6 and rel(dx, (tp.xhat - tm.xhat) / (2 * h)) < 1e-6
    assert abs(dy[F // 2, F // 2]) < 1e-12 * np.abs(dy).max() and dx[F // 2, F // 2] == 0.0


def test_remap_rate_is_exact_for_an_intensity_linear_on_the_model_grid():
    """Bilinear interpolation reproduces a linear function, so R I = al*yhat + be*xhat + c on
    valid pixels and d(R I)/dz = al*dyhat/dz + be*dxhat/dz there."""
    F, z, p, al = 32, 4e-3, 15e-6, math.radians(70)
    taps = orc.remap_taps(F, z, p, al)
    rates = orc.remap_index_rates(F, z, p, al)
    r, c = np.mgrid[0:F, 0:F].astype(np.float64)
    I = 0.7 * r - 0.3 * c + 5.0
    got = orc.remap_apply_rate(I, taps, rates)
    want = np.where(taps.valid, 0.7 * rates[0] - 0.3 * rates[1], 0.0)
    assert rel(got, want) < 1e-12


@pytest.mark.parametrize("kind", orc.LOSS_KINDS)
def test_z_gradient_matches_central_finite_differences(kind):
    w = syn.tiny_workload(F=16, L=2, M=2, seed=61, remap=True, loss=kind, with_sigma=True, with_bg=True)
    p, al = 15e-6, math.radians(70)
    z = 2e-3
    taps = orc.remap_taps(w.F, z, p, al)
    Ih = syn.poisson_measure(orc.predict(w.O_true, w.P_true, w.pos, w.sigma, w.bg, taps), 9)
    L0, gz = orc.gradient_z(w.O0, w.P0, w.pos, Ih, kind, 1e-3, taps, orc.remap_index_rates(w.F, z, p, al), w.sigma,
                            w.bg)
    assert abs(L0 - orc.loss(w.O0, w.P0, w.pos, Ih, kind, 1e-3, w.sigma, w.bg, None, taps)) <= 1e-13 * abs(L0)
    h = 1e-9 * z
    tp, tm = orc.remap_taps(w.F, z + h, p, al), orc.remap_taps(w.F, z - h, p, al)
    assert np.array_equal(tp.valid, tm.valid) and np.array_equal(tp.i0, tm.i0) and np.array_equal(tp.j0, tm.j0)
    fd = (orc.loss(w.O0, w.P0, w.pos, Ih, kind, 1e-3, w.sigma, w.bg, None, tp) -
          orc.loss(w.O0, w.P0, w.pos, Ih, kind, 1e-3, w.sigma, w.bg, None, tm)) / (2 * h)
    assert abs(fd - gz) <= 1e-5 * abs(gz) + 50 * 2.2e-16 * abs(L0) / h, (fd, gz)


# ----------------------------------------------------------------------------
# mixed Poisson-Gaussian loss (shifted-Poisson reading)
# ----------------------------------------------------------------------------

def test_mixed_loss_reduces_to_poisson_and_vanishes_at_its_minimum():
    rng = np.random.default_rng(70)
    I = rng.uniform(0.0, 50.0, size=200)
    Ih = rng.poisson(I).astype(np.float64)
    eps = 1e-3
    assert np.array_equal(orc.loss_terms(I, Ih, ("poisson_gaussian", 0.0), eps), orc.loss_terms(I, Ih, "poisson", eps))
    s2 = 4.0
    # each term is >= 0 and vanishes, with its derivative, where I + eps equals Ihat
    t = orc.loss_terms(I, Ih, ("poisson_gaussian", s2), eps)
    assert np.all(t >= -1e-12)
    at = orc.loss_terms(Ih - eps, Ih, ("poisson_gaussian", s2), eps)
    dt = orc.loss_derivative(Ih - eps, Ih, ("poisson_gaussian", s2), eps)
    assert np.abs(at).max() < 1e-10 and np.abs(dt).max() < 1e-12


def test_mixed_loss_derivative_and_gaussian_limit():
    rng = np.random.default_rng(71)
    I = rng.uniform(1.0, 30.0, size=100)
    Ih = I + rng.normal(0.0, 2.0, size=100)
    kind = ("poisson_gaussian", 9.0)
    h = 1e-6
    fd = (orc.loss_terms(I + h, Ih, kind, 0.0) - orc.loss_terms(I - h, Ih, kind, 0.0)) / (2 * h)
    assert rel(orc.loss_derivative(I, Ih, kind, 0.0), fd) < 1e-7
    # read noise much larger than the misfit: the deviance becomes the Gaussian
    # (I - Ihat)^2 / (2 (Ihat + s2)) with the measured-plus-read-noise variance
    big = ("poisson_gaussian", 1e6)
    gauss = (I - Ih) ** 2 / (2 * (Ih + 1e6))
    assert rel(orc.loss_terms(I, Ih, big, 0.0), gauss) < 1e-4


def test_mixed_loss_gradient_matches_finite_differences():
    w = syn.tiny_workload(F=16, L=2, M=2, seed=72, remap=True, loss="poisson", with_bg=True)
    taps = orc.remap_taps(w.F, 2e-3, 15e-6, math.radians(70))
    rng = np.random.default_rng(73)
    clean = orc.predict(w.O_true, w.P_true, w.pos, None, w.bg, taps)
    Ih = syn.poisson_measure(clean, 10) + rng.normal(0.0, 1.5, size=clean.shape)
    kind = ("poisson_gaussian", 2.25)
    args = (w.pos, Ih, kind, 1e-3, None, w.bg, None, taps)
    _, gO, gP = orc.gradient(w.O0, w.P0, *args)
    dO = [crandn(rng, *o.shape) for o in w.O0]
    dP = crandn(rng, *w.P0.shape)
    h = 1e-6
    Lp = orc.loss([o + h * d for o, d in zip(w.O0, dO)], w.P0 + h * dP, *args)
    Lm = orc.loss([o - h * d for o, d in zip(w.O0, dO)], w.P0 - h * dP, *args)
    an = sum(np.real(np.vdot(g, d)) for g, d in zip(gO, dO)) + np.real(np.vdot(gP, dP))
    assert abs((Lp - Lm) / (2 * h) - an) < 1e-6 * abs(an)


# ----------------------------------------------------------------------------
# chirp-z (zoom DFT) propagator
# ----------------------------------------------------------------------------

def test_czt_at_unit_zoom_is_the_dft_up_to_a_checkerboard_phase():
    """With zeta = 1 the zoom DFT of the centred window equals numpy's DFT moved to the centre,
    times (-1)^(k_row + k_col) (the input index is centred too): same intensities."""
    rng = np.random.default_rng(80)
    F = 16
    x = crandn(rng, F, F)
    c = np.arange(F) - F // 2
    sign = (-1.0) ** (c[:, None] + c[None, :])
    assert rel(orc.f4_propagate_czt(x, 1.0), orc.f4_propagate(x) * sign) < 1e-12
    assert rel(orc.f4_adjoint_czt(orc.f4_propagate_czt(x, 1.0), 1.0), x) < 1e-12


def test_czt_of_a_plane_wave_is_the_closed_form_dirichlet_kernel():
    """A plane wave of a cycles per window (constant along columns) gives, at output (k, kc),
    (1/F) D(2 pi (a - zeta k)/F) D(-2 pi zeta kc / F) / F with D the geometric series
    sum_{n=-F/2}^{F/2-1} exp(i theta n); its peak F^2 / F^2 = 1 sits at k = a / zeta."""
    F = 32
    n = np.arange(F) - F // 2

    def D(theta):
        theta = np.asarray(theta, dtype=np.float64)
        out = np.empty(theta.shape, np.complex128)
        small = np.abs(np.exp(1j * theta) - 1.0) < 1e-14
        out[small] = F
        th = theta[~small]
        out[~small] = np.exp(-1j * th * F / 2) * (1 - np.exp(1j * th * F)) / (1 - np.exp(1j * th))
        return out

    for a, zeta in ((6, 0.75), (-9, 1.5), (4, 0.5), (3, 0.9)):
        x = np.exp(2j * np.pi * a * n / F)[:, None] * np.ones(F)[None, :] / F
        Psi = orc.f4_propagate_czt(x, zeta)
        want = D(2 * np.pi * (a - zeta * n) / F)[:, None] * D(-2 * np.pi * zeta * n / F)[None, :] / F / F
        assert rel(Psi, want) < 1e-11
        if float(a / zeta).is_integer():
            assert abs(abs(Psi[int(a / zeta) + F // 2, F // 2]) - 1.0) < 1e-12


def test_czt_adjoint_identity_and_zoom_two_subsamples_the_dft():
    rng = np.random.default_rng(81)
    F = 16
    x, y = crandn(rng, F, F), crandn(rng, F, F)
    for zeta in (0.83, 1.17):
        lhs = np.vdot(y, orc.f4_propagate_czt(x, zeta))
        rhs = np.vdot(orc.f4_adjoint_czt(y, zeta), x)
        assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    # zeta = 2: output k' is the centred DFT at frequency 2 k' (mod F)
    Zd = orc.czt_matrix(F, 1.0)
    Z2 = orc.czt_matrix(F, 2.0)
    c = np.arange(F) - F // 2
    assert rel(Z2, Zd[(2 * c + F // 2) % F]) < 1e-12


@pytest.mark.parametrize("kind", orc.LOSS_KINDS)
def test_czt_model_gradient_matches_finite_differences(kind):
    w = syn.tiny_workload(F=16, L=2, M=2, seed=82, remap=True, loss=kind, with_sigma=True, with_bg=True)
    taps = orc.remap_taps(w.F, 2e-3, 15e-6, math.radians(70))
    zeta = [1.0, 1.0 / 1.1]
    Ih = syn.poisson_measure(orc.predict(w.O_true, w.P_true, w.pos, w.sigma, w.bg, taps, zeta=zeta), 11)
    args = (w.pos, Ih, kind, 1e-3, w.sigma, w.bg, None, taps)
    _, gO, gP = orc.gradient(w.O0, w.P0, *args, zeta=zeta)
    rng = np.random.default_rng(83)
    dO = [crandn(rng, *o.shape) for o in w.O0]
    dP = crandn(rng, *w.P0.shape)
    h = 1e-6
    Lp = orc.loss([o + h * d for o, d in zip(w.O0, dO)], w.P0 + h * dP, *args, zeta=zeta)
    Lm = orc.loss([o - h * d for o, d in zip(w.O0, dO)], w.P0 - h * dP, *args, zeta=zeta)
    an = sum(np.real(np.vdot(g, d)) for g, d in zip(gO, dO)) + np.real(np.vdot(gP, dP))
    assert abs((Lp - Lm) / (2 * h) - an) < 1e-6 * abs(an)
    Lt, gOt, gPt = orc.gradient(w.O_true, w.P_true, w.pos, orc.predict(w.O_true, w.P_true, w.pos, w.sigma, w.bg, taps,
                                                                       zeta=zeta), kind, 0.0, w.sigma, w.bg, None,
                                taps, zeta=zeta)
    assert abs(Lt) < 1e-18 * float(Ih.sum()) and np.abs(gPt).max() < 1e-10
