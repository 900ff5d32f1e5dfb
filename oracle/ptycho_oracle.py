"""FP64 CPU oracle of the multi-wavelength, multi-mode ptychography model.

TEST INFRASTRUCTURE ONLY.  This module is the plain, slow, obviously-correct
statement of what the GPU library computes.  Only ``tests/``, ``__graft_entry__.smoke``
and the CPU-baseline / reference legs of ``bench.py`` may import it; the library
never calls it and shares no code with it.

It follows the paper's universal model (Eq. 1) written as the composite of sub-models
f1..f5 (Eq. 2): f1 scales the probe power by sigma_j, f2 shifts the object by the scan
position s_j, f3 forms the exit wave P*O, f4 propagates to the detector, f5 applies the
measurement effects (background, tilted-plane remap, mask).  The loss (amplitude MSE
or Poisson, Section "Universal Ptychography Algorithm") is summed over frames and
pixels; its gradient is the analytic adjoint of the same steps (the reverse pass that
Fig. 1B describes).  Every frame is handled in an explicit loop.

Readings of points where the paper is silent (each also recorded in the design notes):

* propagation D_{lambda,z}: orthonormal 2D DFT with the zero frequency moved to
  (F/2, F/2); each wavelength is sampled at its own object pixel size so all
  wavelengths share one detector grid; optionally the chirp-z (zoom DFT) propagator
  (1/F) Z psi Z^T with centred indices and zoom zeta_l = lambda_ref / lambda_l, which puts
  every wavelength on one object grid;
* integer scan shift: the patch is O_l[y:y+F, x:x+F]; a patch outside the object is
  an error (no wrap-around, no clamping);
* fractional scan offsets (optional): the integer patch is resampled at r + delta by the
  Fourier shift theorem, taking the patch as one period of a band-limited function (so
  the edge rows and columns wrap; the probe is negligible there);
* tilted-plane remap: a fixed bilinear operator R from the model grid (uniform in
  sample-plane spatial frequency) to the camera grid, derived from the camera being
  perpendicular to the specular beam (Section "Experimental setup"); taps outside the
  model grid remove the camera pixel from the mask;
* the same geometry applied once to the data (the paper's preprocessing form): each camera
  pattern is interpolated at the camera position of every model-grid pixel (the inverse
  map, with the reflected ray leaving the sample surface) and a mask keeps the pixels whose
  four taps lie inside the camera crop and inside the value thresholds;
* background N(rho) lives on the model grid and is added before the remap;
* losses: amplitude  sum (sqrt(I+eps) - sqrt(Ihat))^2, Poisson deviance
  sum (I+eps) - Ihat - Ihat*log((I+eps)/Ihat) with 0*log(.) := 0; no normalisation;
  mixed Poisson-Gaussian with read-noise variance s2: the Poisson deviance of
  (I+eps+s2, max(Ihat+s2, 0)) (the shifted-Poisson approximation);
* object regularisation (optional): L1 and total variation of the smoothed amplitude
  sqrt(|O|^2 + eta^2), forward differences with none across the last row and column;
* gradient convention g = dL/dRe + i dL/dIm (complex parameters);
* Adam acts on real and imaginary parts as separate real parameters.

Parity pins: see ``tests/test_oracle_pins.py`` (brute-force DFT, Parseval, unitary
mode-mixing and global-phase invariance, closed-form diffraction of plane waves,
zero loss and zero gradient at noiseless truth, central finite differences, remap
dot-product / identity / constant tests, the Adam first-step closed form and the
paper's geometry numbers; for the sigma and background gradients: finite differences,
the intensity-level form of the sigma gradient that Parseval's theorem gives, and the
identity between the sigma gradient and the probe gradient along P -> cP; for the
fractional offsets: whole-pixel offsets as cyclic rolls, band-limited plane waves sampled
at the shifted points, unitarity, composition, the adjoint identity, reduction to the
integer model, and finite differences of the loss in the offsets, O and P; for z: finite
differences of the fractional model indices and of the loss with the remap rebuilt at z +- h,
exactness for an intensity linear on the model grid, and zero rate at the specular pixel; for
the data-side tilt correction: the inverse map undoes the forward map at every camera pixel,
exactness for patterns affine on the camera, near-identity without tilt, the mask of a
saturated pixel, and undoing the in-model remap of smooth patterns; for the object regulariser:
finite differences, the closed form of an object of constant amplitude and of a linear
amplitude ramp, and invariance under a global phase).  The tilted-plane remap formula itself is a reading of the
cited geometry and is only partially pinned (identity limit, constants, adjointness,
the paper's NA and pixel-ratio figures).
"""
from __future__ import annotations

import math
from typing import List, Optional, Sequence

import numpy as np

LOSS_KINDS = ("amplitude", "poisson")


# ----------------------------------------------------------------------------
# f1, f2, f3: probe power, object shift, exit wave  (Eq. 2)
# ----------------------------------------------------------------------------

def f1_power(P_lm: np.ndarray, sigma_j: float) -> np.ndarray:
    """f1: scale the probe mode by the power coefficient sigma_j (Eq. 1)."""
    return sigma_j * P_lm


def f2_shift(O_l: np.ndarray, s_j: Sequence[int], F: int) -> np.ndarray:
    """f2: the object seen through an F x F window whose corner sits at s_j = (row, col)."""
    y, x = int(s_j[0]), int(s_j[1])
    H, W = O_l.shape
    if y < 0 or x < 0 or y + F > H or x + F > W:
        raise ValueError(f"patch at ({y},{x}) of size {F} leaves the {H}x{W} object")
    return O_l[y:y + F, x:x + F]


def _shift_ramp(F: int, delta: Sequence[float]) -> np.ndarray:
    """exp(2 pi i (f_y d_y + f_x d_x)) on the DFT grid, f = k / F in numpy's fftfreq order."""
    fy = np.fft.fftfreq(F)[:, None]
    fx = np.fft.fftfreq(F)[None, :]
    return np.exp(2j * np.pi * (fy * float(delta[0]) + fx * float(delta[1])))


def f2_subpixel(patch: np.ndarray, delta: Sequence[float]) -> np.ndarray:
    """f2 for a fractional part of the scan position: the patch resampled at r + delta by the
    Fourier shift theorem (the paper shifts with it, Section "Benchmarking ..."), the patch
    taken as one period of a band-limited function.  delta = (rows, cols) in pixels."""
    F = patch.shape[0]
    return np.fft.ifft2(np.fft.fft2(patch) * _shift_ramp(F, delta))


def f2_subpixel_adjoint(g: np.ndarray, delta: Sequence[float]) -> np.ndarray:
    """Adjoint (= inverse) of f2_subpixel: the conjugate phase ramp."""
    F = g.shape[0]
    return np.fft.ifft2(np.fft.fft2(g) * np.conj(_shift_ramp(F, delta)))


def f2_subpixel_derivative(patch: np.ndarray, delta: Sequence[float], axis: int) -> np.ndarray:
    """d f2_subpixel / d delta[axis]: the shift theorem's factor 2 pi i f along that axis."""
    F = patch.shape[0]
    f = np.fft.fftfreq(F)
    fac = 2j * np.pi * (f[:, None] if axis == 0 else f[None, :])
    return np.fft.ifft2(np.fft.fft2(patch) * _shift_ramp(F, delta) * fac)


def f3_interaction(P_scaled: np.ndarray, patch: np.ndarray) -> np.ndarray:
    """f3: multiplicative exit wave psi = (sigma P) * O(r - s)."""
    return P_scaled * patch


# ----------------------------------------------------------------------------
# f4: propagation to the detector
# ----------------------------------------------------------------------------

def f4_propagate(psi: np.ndarray) -> np.ndarray:
    """f4: orthonormal 2D DFT, zero frequency moved to (F/2, F/2)."""
    return np.fft.fftshift(np.fft.fft2(psi, norm="ortho"))


def f4_adjoint(Psi: np.ndarray) -> np.ndarray:
    """Adjoint (= inverse) of f4: undo the centring, orthonormal inverse 2D DFT."""
    return np.fft.ifft2(np.fft.ifftshift(Psi), norm="ortho")


def czt_matrix(F: int, zeta: float) -> np.ndarray:
    """The zoom DFT along one axis: Z[k', n'] = exp(-2 pi i zeta n' k' / F) with both indices
    centred, n', k' in [-F/2, F/2) (array index = index + F/2).  zeta = 1 is the centred DFT;
    zeta = lambda_ref / lambda_l samples wavelength l's far field on the detector pixels of a
    common object grid (the chirp-z propagator the paper uses, Section "Benchmarking ...")."""
    c = np.arange(F) - F // 2
    return np.exp(-2j * np.pi * float(zeta) * np.outer(c, c) / F)


def f4_propagate_czt(psi: np.ndarray, zeta: float) -> np.ndarray:
    """f4 with the chirp-z propagator: (1/F) Z psi Z^T (rows, then columns), output centred."""
    Z = czt_matrix(psi.shape[0], zeta)
    return Z @ psi @ Z.T / psi.shape[0]


def f4_adjoint_czt(Psi: np.ndarray, zeta: float) -> np.ndarray:
    """Adjoint of f4_propagate_czt: (1/F) Z^H Psi conj(Z)."""
    Z = czt_matrix(Psi.shape[0], zeta)
    return Z.conj().T @ Psi @ Z.conj() / Psi.shape[0]


def _prop(psi, zeta, l):
    return f4_propagate(psi) if zeta is None else f4_propagate_czt(psi, zeta[l])


def _prop_adj(Psi, zeta, l):
    return f4_adjoint(Psi) if zeta is None else f4_adjoint_czt(Psi, zeta[l])


# ----------------------------------------------------------------------------
# tilted-plane remap (part of the measurement f5 in the in-model form)
# ----------------------------------------------------------------------------

class RemapTaps:
    """Bilinear taps of the model-grid -> camera-grid remap for one geometry."""

    def __init__(self, valid, i0, j0, wy, wx, yhat, xhat, db, da):
        self.valid, self.i0, self.j0, self.wy, self.wx = valid, i0, j0, wy, wx
        self.yhat, self.xhat = yhat, xhat
        self.db, self.da = db, da      # model-grid spacings in direction cosines

    @property
    def F(self) -> int:
        return self.valid.shape[0]


def remap_taps(F: int, z: float, det_pixel: float, tilt_rad: float) -> RemapTaps:
    """Where each camera pixel samples the model grid.

    The camera is perpendicular to the specular beam at distance z.  Camera pixel
    (y, x) sees the direction (X, Y, z) with X = (x - F/2) p, Y = (y - F/2) p.  In the
    sample frame, tilted by alpha from the normal, its in-plane direction cosines are
    a = X / R and b = (Y cos(alpha) + z sin(alpha)) / R - sin(alpha), R = |(X, Y, z)|.
    The model grid is uniform in (b, a) with spacings (p/z) cos(alpha) and p/z, centred
    on the specular direction, which reproduces the 3:1 pixel anisotropy reported for
    the 70 degree geometry.  The fractional model index is
    (b / db + F/2, a / da + F/2); the pixel is valid when all four bilinear taps fall
    inside the grid.
    """
    c, s = math.cos(tilt_rad), math.sin(tilt_rad)
    da = det_pixel / z
    db = da * c
    y, x = np.mgrid[0:F, 0:F].astype(np.float64)
    X = (x - F / 2) * det_pixel
    Y = (y - F / 2) * det_pixel
    R = np.sqrt(X * X + Y * Y + z * z)
    a = X / R
    b = (Y * c + z * s) / R - s
    yhat = b / db + F / 2
    xhat = a / da + F / 2
    valid = (yhat >= 0.0) & (yhat < F - 1) & (xhat >= 0.0) & (xhat < F - 1)
    i0 = np.where(valid, np.floor(yhat), 0).astype(np.int64)
    j0 = np.where(valid, np.floor(xhat), 0).astype(np.int64)
    wy = np.where(valid, yhat - i0, 0.0)
    wx = np.where(valid, xhat - j0, 0.0)
    return RemapTaps(valid, i0, j0, wy, wx, yhat, xhat, db, da)


def remap_index_rates(F: int, z: float, det_pixel: float, tilt_rad: float):
    """d yhat / dz and d xhat / dz of every camera pixel's fractional model index (the
    propagation distance z is among the variables the paper optimises).  With
    yhat = z b / (p cos(alpha)) + F/2 and xhat = z a / p + F/2 (see remap_taps):
    d yhat/dz = (b + z db/dz) / (p cos(alpha)), db/dz = sin(alpha)/R - (Y cos(alpha) + z sin(alpha)) z / R^3,
    d xhat/dz = (X / p) (1/R - z^2 / R^3)."""
    c, s = math.cos(tilt_rad), math.sin(tilt_rad)
    y, x = np.mgrid[0:F, 0:F].astype(np.float64)
    X = (x - F / 2) * det_pixel
    Y = (y - F / 2) * det_pixel
    R = np.sqrt(X * X + Y * Y + z * z)
    b = (Y * c + z * s) / R - s
    dbdz = s / R - (Y * c + z * s) * z / R ** 3
    dy = (b + z * dbdz) / (det_pixel * c)
    dx = (X / det_pixel) * (1.0 / R - z * z / R ** 3)
    return dy, dx


def remap_apply_rate(I_model: np.ndarray, taps: RemapTaps, rates) -> np.ndarray:
    """d(R I)/dz at fixed model-grid I: the bilinear interpolant's slopes along the row and
    column fractions times the index rates (0 where the pixel is invalid)."""
    i, j, u, v, ok = taps.i0, taps.j0, taps.wy, taps.wx, taps.valid
    I00, I01 = I_model[i, j], I_model[i, j + 1]
    I10, I11 = I_model[i + 1, j], I_model[i + 1, j + 1]
    d_row = ((1 - v) * I10 + v * I11) - ((1 - v) * I00 + v * I01)
    d_col = (1 - u) * (I01 - I00) + u * (I11 - I10)
    return np.where(ok, d_row * rates[0] + d_col * rates[1], 0.0)


def _tap_weights(taps: RemapTaps):
    """The four (row, col, weight) taps of every camera pixel; weight 0 where invalid."""
    i, j, u, v, ok = taps.i0, taps.j0, taps.wy, taps.wx, taps.valid
    return [(i, j, np.where(ok, (1 - u) * (1 - v), 0.0)),
            (i, j + 1, np.where(ok, (1 - u) * v, 0.0)),
            (i + 1, j, np.where(ok, u * (1 - v), 0.0)),
            (i + 1, j + 1, np.where(ok, u * v, 0.0))]


def remap_apply(I_model: np.ndarray, taps: RemapTaps) -> np.ndarray:
    """R: bilinear interpolation of the model-grid pattern at each camera pixel (0 if invalid)."""
    out = np.zeros(taps.valid.shape)
    for (ii, jj, w) in _tap_weights(taps):
        out += w * I_model[ii, jj]
    return out


def remap_adjoint(D_cam: np.ndarray, taps: RemapTaps) -> np.ndarray:
    """R^T: scatter each camera-pixel value back onto its four model-grid taps."""
    out = np.zeros(taps.valid.shape)
    for (ii, jj, w) in _tap_weights(taps):
        np.add.at(out, (ii, jj), w * D_cam)
    return out


# ----------------------------------------------------------------------------
# data-side tilt correction (the remap applied once to the measurements)
# ----------------------------------------------------------------------------

def tilt_camera_index(F: int, z: float, det_pixel: float, tilt_rad: float, yhat, xhat):
    """Where the model-grid point (yhat, xhat) (fractional indices of the grid of
    remap_taps) lies on the camera: the inverse of the map in remap_taps.

    The model index fixes the reflected ray's in-plane direction cosines
    b = (yhat - F/2) db and a = (xhat - F/2) da.  Rotated by alpha about the camera's x
    axis, the ray is (a, b + sin(alpha), w) with w = sqrt(1 - a^2 - (b + sin(alpha))^2),
    taken >= 0 (the reflected ray leaves the sample surface).  In the camera frame its
    components are d_y = (b + sin) cos - w sin and d_z = (b + sin) sin + w cos, and it
    meets the camera plane at X = z a / d_z, Y = z d_y / d_z.  Returns (y, x, ok): the
    fractional camera indices Y/p + F/2 and X/p + F/2, and whether the ray exists and
    reaches the camera (1 - a^2 - (b + sin)^2 > 0 and d_z > 0)."""
    c, s = math.cos(tilt_rad), math.sin(tilt_rad)
    da = det_pixel / z
    db = da * c
    b = (np.asarray(yhat, np.float64) - F / 2) * db
    a = (np.asarray(xhat, np.float64) - F / 2) * da
    u = b + s
    w2 = 1.0 - a * a - u * u
    w = np.sqrt(np.where(w2 > 0, w2, 0.0))
    dy = u * c - w * s
    dz = u * s + w * c
    ok = (w2 > 0) & (dz > 0)
    dzs = np.where(ok, dz, 1.0)
    X = z * a / dzs
    Y = z * dy / dzs
    return Y / det_pixel + F / 2, X / det_pixel + F / 2, ok


def tilt_correct(I_cam: np.ndarray, z: float, det_pixel: float, tilt_rad: float,
                 lo: float = -math.inf, hi: float = math.inf):
    """The tilt correction of Section "Experimental setup and ptychography reconstruction",
    applied once to the data: every camera pattern I_cam[j] (F x F, zero frequency at
    (F/2, F/2)) is interpolated (bilinear) at the camera position of each model-grid pixel
    (tilt_camera_index), which puts it on the grid uniform in sample-plane spatial
    frequency.  It also makes the mask the paper describes: a model pixel is kept when its
    ray reaches the camera, its four camera taps lie inside the F x F crop
    (0 <= y < F-1, 0 <= x < F-1), and every tap's value lies in [lo, hi) (the paper's
    thresholds against noise-corrupted and saturated pixels).  Returns (I_model, mask), both
    [J][F][F]; I_model is 0 where the mask is 0."""
    I_cam = np.asarray(I_cam)
    J, F, _ = I_cam.shape
    ii, kk = np.mgrid[0:F, 0:F].astype(np.float64)
    y, x, ok = tilt_camera_index(F, z, det_pixel, tilt_rad, ii, kk)
    inside = ok & (y >= 0.0) & (y < F - 1) & (x >= 0.0) & (x < F - 1)
    y0 = np.where(inside, np.floor(np.where(inside, y, 0.0)), 0).astype(np.int64)
    x0 = np.where(inside, np.floor(np.where(inside, x, 0.0)), 0).astype(np.int64)
    u = np.where(inside, y - y0, 0.0)
    v = np.where(inside, x - x0, 0.0)
    out = np.zeros((J, F, F))
    mask = np.zeros((J, F, F), bool)
    for j in range(J):
        cam = I_cam[j].astype(np.float64)
        taps = [(cam[y0, x0], (1 - u) * (1 - v)), (cam[y0, x0 + 1], (1 - u) * v),
                (cam[y0 + 1, x0], u * (1 - v)), (cam[y0 + 1, x0 + 1], u * v)]
        keep = inside.copy()
        val = np.zeros((F, F))
        for t, wt in taps:
            keep &= (t >= lo) & (t < hi)
            val += wt * t
        out[j] = np.where(keep, val, 0.0)
        mask[j] = keep
    return out, mask


# ----------------------------------------------------------------------------
# f5: measurement (background, remap) and the mask
# ----------------------------------------------------------------------------

def f5_measure(I_sum: np.ndarray, bg: Optional[np.ndarray], taps: Optional[RemapTaps]) -> np.ndarray:
    """f5: add the common background on the model grid, then remap to the camera grid."""
    I = I_sum if bg is None else I_sum + bg
    return I if taps is None else remap_apply(I, taps)


def frame_mask(mask: Optional[np.ndarray], j: int, F: int, taps: Optional[RemapTaps]) -> np.ndarray:
    """Pixels that enter the loss for frame j: user mask AND remap validity."""
    if mask is None:
        mk = np.ones((F, F), bool)
    elif mask.ndim == 3:
        mk = mask[j] != 0
    else:
        mk = mask != 0
    if taps is not None:
        mk = mk & taps.valid
    return mk


# ----------------------------------------------------------------------------
# losses (Section "Universal Ptychography Algorithm")
# ----------------------------------------------------------------------------

def _shifted(I, Ihat, kind, eps):
    """Mixed Poisson-Gaussian noise (MLE with mixed statistics, Section "Universal
    Ptychography Algorithm"), kind = ("poisson_gaussian", s2): the shifted-Poisson reading,
    Ihat + s2 taken as Poisson with mean I + eps + s2 (Ihat + s2 clipped at 0)."""
    if isinstance(kind, tuple) and kind[0] == "poisson_gaussian":
        s2 = float(kind[1])
        return I + eps + s2, np.maximum(Ihat.astype(np.float64) + s2, 0.0), "poisson"
    return I + eps, Ihat.astype(np.float64), kind


def loss_terms(I: np.ndarray, Ihat: np.ndarray, kind, eps: float) -> np.ndarray:
    """Per-pixel loss.  amplitude: (sqrt(I+eps) - sqrt(Ihat))^2; Poisson: deviance; mixed
    Poisson-Gaussian: the Poisson deviance of the shifted arguments (see _shifted)."""
    Ie, Ihat, kind = _shifted(I, Ihat, kind, eps)
    if kind == "amplitude":
        return (np.sqrt(Ie) - np.sqrt(Ihat)) ** 2
    if kind == "poisson":
        with np.errstate(divide="ignore", invalid="ignore"):
            lg = np.where(Ihat > 0, Ihat * np.log(Ie / np.where(Ihat > 0, Ihat, 1.0)), 0.0)
        return Ie - Ihat - lg
    raise ValueError(kind)


def loss_derivative(I: np.ndarray, Ihat: np.ndarray, kind, eps: float) -> np.ndarray:
    """dL/dI per pixel.  amplitude: 1 - sqrt(Ihat)/sqrt(I+eps); Poisson: 1 - Ihat/(I+eps);
    mixed Poisson-Gaussian: 1 - (Ihat+s2)/(I+eps+s2)."""
    Ie, Ihat, kind = _shifted(I, Ihat, kind, eps)
    if kind == "amplitude":
        return 1.0 - np.sqrt(Ihat) / np.sqrt(Ie)
    if kind == "poisson":
        return 1.0 - Ihat / Ie
    raise ValueError(kind)


# ----------------------------------------------------------------------------
# the model (Eq. 1) and its adjoint
# ----------------------------------------------------------------------------

def _sigma(sigma, j):
    return 1.0 if sigma is None else float(sigma[j])


def frame_patch(O_l, pos, l, j, F, delta=None):
    """f2: the object patch of frame j at wavelength l; with delta [L][J][2] the integer
    window is shifted further by the fractional offset delta[l][j]."""
    p = f2_shift(O_l, pos[l][j], F)
    return p if delta is None else f2_subpixel(p, delta[l][j])


def frame_fields(O, P, pos, j, sigma=None, delta=None, zeta=None):
    """Exit waves and propagated fields Psi_{j,l,m} for one frame (f1..f4); zeta [L] selects the
    chirp-z propagator with zoom zeta[l] instead of the DFT."""
    L, M, F = P.shape[0], P.shape[1], P.shape[2]
    s = _sigma(sigma, j)
    patches, Psi = [], np.empty((L, M, F, F), np.complex128)
    for l in range(L):
        p = frame_patch(O[l], pos, l, j, F, delta)
        patches.append(p)
        for m in range(M):
            Psi[l, m] = _prop(f3_interaction(f1_power(P[l, m], s), p), zeta, l)
    return patches, Psi


def predict_frame(O, P, pos, j, sigma=None, bg=None, taps=None, delta=None, zeta=None) -> np.ndarray:
    """Eq. 1 for frame j: remap( sum_l sum_m |D[sigma_j P_lm O_l(r - s_j)]|^2 + N )."""
    _, Psi = frame_fields(O, P, pos, j, sigma, delta, zeta)
    I_sum = (np.abs(Psi) ** 2).sum(axis=(0, 1))
    return f5_measure(I_sum, bg, taps)


def predict(O, P, pos, sigma=None, bg=None, taps=None, frames=None, delta=None, zeta=None) -> np.ndarray:
    """Predicted camera-grid patterns for the requested frames (default: all)."""
    J = pos.shape[1]
    frames = range(J) if frames is None else frames
    return np.stack([predict_frame(O, P, pos, j, sigma, bg, taps, delta, zeta) for j in frames])


def loss(O, P, pos, Imeas, kind, eps, sigma=None, bg=None, mask=None, taps=None, frames=None, delta=None,
         zeta=None) -> float:
    """Total loss over the requested frames and their masked pixels."""
    F = P.shape[2]
    J = pos.shape[1]
    frames = range(J) if frames is None else frames
    total = 0.0
    for j in frames:
        Ic = predict_frame(O, P, pos, j, sigma, bg, taps, delta, zeta)
        mk = frame_mask(mask, j, F, taps)
        total += float(loss_terms(Ic, Imeas[j], kind, eps)[mk].sum())
    return total


def gradient(O, P, pos, Imeas, kind, eps, sigma=None, bg=None, mask=None, taps=None, frames=None, delta=None,
             zeta=None):
    """Loss and its gradient (dL/dRe + i dL/dIm) with respect to every O_l and P_lm.

    For each frame: forward fields Psi_{lm}; I = sum |Psi|^2 (+bg); camera pattern R I;
    D = mask * dL/dI_cam; G = R^T D; chi_{lm} = f4^-1(2 G Psi_{lm}) is the gradient
    with respect to the exit wave; then grad P_lm += conj(sigma p_l) chi_lm and
    grad O_l[patch] += conj(sigma P_lm) chi_lm (with sub-pixel offsets, the patch
    gradient goes through the adjoint of the Fourier shift before it is added).
    """
    L, M, F = P.shape[0], P.shape[1], P.shape[2]
    J = pos.shape[1]
    frames = range(J) if frames is None else frames
    gO = [np.zeros_like(o, dtype=np.complex128) for o in O]
    gP = np.zeros_like(P, dtype=np.complex128)
    total = 0.0
    for j in frames:
        s = _sigma(sigma, j)
        patches, Psi = frame_fields(O, P, pos, j, sigma, delta, zeta)
        I_sum = (np.abs(Psi) ** 2).sum(axis=(0, 1))
        Ic = f5_measure(I_sum, bg, taps)
        mk = frame_mask(mask, j, F, taps)
        total += float(loss_terms(Ic, Imeas[j], kind, eps)[mk].sum())
        with np.errstate(divide="ignore", invalid="ignore"):
            D = np.where(mk, loss_derivative(Ic, Imeas[j], kind, eps), 0.0)
        G = D if taps is None else remap_adjoint(D, taps)
        for l in range(L):
            y, x = int(pos[l][j][0]), int(pos[l][j][1])
            g_patch = np.zeros((F, F), np.complex128)
            for m in range(M):
                chi = _prop_adj(2.0 * G * Psi[l, m], zeta, l)
                gP[l, m] += np.conj(s * patches[l]) * chi
                g_patch += np.conj(s * P[l, m]) * chi
            if delta is not None:
                g_patch = f2_subpixel_adjoint(g_patch, delta[l][j])
            gO[l][y:y + F, x:x + F] += g_patch
    return total, gO, gP


def gradient_delta(O, P, pos, Imeas, kind, eps, delta, sigma=None, bg=None, mask=None, taps=None, frames=None):
    """Loss and its gradient with respect to the fractional scan offsets delta [L][J][2]
    (the scan positions s_k are among the variables the paper optimises, Section
    "Universal Ptychography Algorithm"; its position correction differentiates the
    Fourier shift).  By the chain rule through the exit waves,
    dL/d delta[l][j][a] = Re sum_r conj(g_p(r)) d p(r) / d delta_a with
    g_p = sum_m conj(sigma P_lm) chi_jlm the gradient with respect to the shifted patch.
    Returns (loss, g_delta [L][J][2], 0 for frames not requested)."""
    L, M, F = P.shape[0], P.shape[1], P.shape[2]
    J = pos.shape[1]
    frames = range(J) if frames is None else frames
    g_delta = np.zeros((L, J, 2))
    total = 0.0
    for j in frames:
        s = _sigma(sigma, j)
        patches, Psi = frame_fields(O, P, pos, j, sigma, delta)
        I_sum = (np.abs(Psi) ** 2).sum(axis=(0, 1))
        Ic = f5_measure(I_sum, bg, taps)
        mk = frame_mask(mask, j, F, taps)
        total += float(loss_terms(Ic, Imeas[j], kind, eps)[mk].sum())
        with np.errstate(divide="ignore", invalid="ignore"):
            D = np.where(mk, loss_derivative(Ic, Imeas[j], kind, eps), 0.0)
        G = D if taps is None else remap_adjoint(D, taps)
        for l in range(L):
            g_patch = np.zeros((F, F), np.complex128)
            for m in range(M):
                chi = f4_adjoint(2.0 * G * Psi[l, m])
                g_patch += np.conj(s * P[l, m]) * chi
            window = f2_shift(O[l], pos[l][j], F)
            for a in range(2):
                dp = f2_subpixel_derivative(window, delta[l][j], a)
                g_delta[l, j, a] = float(np.real(np.vdot(g_patch, dp)))
    return total, g_delta


def gradient_sigma_bg(O, P, pos, Imeas, kind, eps, sigma=None, bg=None, mask=None, taps=None, frames=None,
                      delta=None):
    """Loss and its gradient with respect to the power coefficients sigma_j and the
    background N (two of the model variables the paper lists as optimisable, Section
    "Universal Ptychography Algorithm", the paragraph after Eq. 2).

    sigma_j is a real factor of every probe mode of frame j (f1), so by the chain rule
    through the exit wave dL/dsigma_j = sum_{l,m} sum_r Re(conj(P_lm p_jl) chi_jlm), with
    chi the exit-wave gradient of ``gradient``.  N is added to the incoherent sum on the
    model grid before the remap (Eq. 1), so dL/dN = sum_j G_j with G_j = R^T(mask dL/dI_cam).
    Returns (loss, g_sigma [J] (0 for frames not requested), g_bg [F, F]).
    """
    L, M, F = P.shape[0], P.shape[1], P.shape[2]
    J = pos.shape[1]
    frames = range(J) if frames is None else frames
    g_sigma = np.zeros(J)
    g_bg = np.zeros((F, F))
    total = 0.0
    for j in frames:
        patches, Psi = frame_fields(O, P, pos, j, sigma, delta)
        I_sum = (np.abs(Psi) ** 2).sum(axis=(0, 1))
        Ic = f5_measure(I_sum, bg, taps)
        mk = frame_mask(mask, j, F, taps)
        total += float(loss_terms(Ic, Imeas[j], kind, eps)[mk].sum())
        with np.errstate(divide="ignore", invalid="ignore"):
            D = np.where(mk, loss_derivative(Ic, Imeas[j], kind, eps), 0.0)
        G = D if taps is None else remap_adjoint(D, taps)
        g_bg += G
        for l in range(L):
            for m in range(M):
                chi = f4_adjoint(2.0 * G * Psi[l, m])
                g_sigma[j] += float(np.real(np.conj(P[l, m] * patches[l]) * chi).sum())
    return total, g_sigma, g_bg


def gradient_z(O, P, pos, Imeas, kind, eps, taps, rates, sigma=None, bg=None, mask=None, frames=None, delta=None):
    """Loss and dL/dz through the tilted-plane remap (the propagator itself is the
    orthonormal DFT, with no z in it; a caller holding physical scan positions adds the
    chain through the object pixel size, sum_j g_delta . d pos / dz).  For each frame,
    dL/dz = sum over the camera grid of (mask dL/dI) * d(R (sum |Psi|^2 + N))/dz; the mask
    boundary (pixels whose taps leave the grid) has measure zero and is held fixed."""
    F = P.shape[2]
    J = pos.shape[1]
    frames = range(J) if frames is None else frames
    total, gz = 0.0, 0.0
    for j in frames:
        _, Psi = frame_fields(O, P, pos, j, sigma, delta)
        I_model = (np.abs(Psi) ** 2).sum(axis=(0, 1))
        if bg is not None:
            I_model = I_model + bg
        Ic = remap_apply(I_model, taps)
        mk = frame_mask(mask, j, F, taps)
        total += float(loss_terms(Ic, Imeas[j], kind, eps)[mk].sum())
        with np.errstate(divide="ignore", invalid="ignore"):
            D = np.where(mk, loss_derivative(Ic, Imeas[j], kind, eps), 0.0)
        gz += float((D * remap_apply_rate(I_model, taps, rates)).sum())
    return total, gz


# ----------------------------------------------------------------------------
# Adam (Kingma & Ba), real and imaginary parts as separate real parameters
# ----------------------------------------------------------------------------

def regulariser(O, mu_l1: float, mu_tv: float, eta: float):
    """Object regularisation (the loss adapted by regularisers, Section "Universal Ptychography
    Algorithm"; the paper names L1 and total-variation regularisation of the object amplitude in
    Section "3D structure information characterisation"; the exact forms are in the missing
    Supplementary Information).  Reading: with the smoothed amplitude a = sqrt(|O|^2 + eta^2) of
    every pixel of every object O_l,
        R = mu_l1 * sum a + mu_tv * sum sqrt(dx^2 + dy^2 + eta^2),
    dx = a[r][c+1] - a[r][c] (0 in the last column), dy = a[r+1][c] - a[r][c] (0 in the last row).
    Returns (R, [dR/dRe O_l + i dR/dIm O_l]); the gradient of a with respect to the real and
    imaginary parts is O/a, so g = (dR/da) O / a."""
    R = 0.0
    grads = []
    for O_l in O:
        O_l = np.asarray(O_l, np.complex128)
        a = np.sqrt(np.abs(O_l) ** 2 + eta * eta)
        dx = np.zeros_like(a)
        dy = np.zeros_like(a)
        dx[:, :-1] = a[:, 1:] - a[:, :-1]
        dy[:-1, :] = a[1:, :] - a[:-1, :]
        t = np.sqrt(dx * dx + dy * dy + eta * eta)
        R += mu_l1 * float(a.sum()) + mu_tv * float(t.sum())
        px, py = dx / t, dy / t
        dRda = np.full(a.shape, float(mu_l1)) - mu_tv * (px + py)   # through dx, dy of the pixel itself
        dRda[:, 1:] += mu_tv * px[:, :-1]                           # through dx of the left neighbour
        dRda[1:, :] += mu_tv * py[:-1, :]                           # through dy of the upper neighbour
        grads.append(dRda * O_l / a)
    return R, grads


class AdamState:
    def __init__(self, shapes_O: List[tuple], shape_P: tuple):
        self.mO = [np.zeros(s + (2,)) for s in shapes_O]
        self.vO = [np.zeros(s + (2,)) for s in shapes_O]
        self.mP = np.zeros(shape_P + (2,))
        self.vP = np.zeros(shape_P + (2,))
        self.t = 0


def _as_real(z: np.ndarray) -> np.ndarray:
    return np.stack([z.real, z.imag], axis=-1)


def adam_update(theta: np.ndarray, g: np.ndarray, m: np.ndarray, v: np.ndarray, t: int,
                lr: float, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
    """One Adam step on a complex array; m and v are [..., 2] real arrays updated in place."""
    gr = _as_real(g)
    m *= b1
    m += (1.0 - b1) * gr
    v *= b2
    v += (1.0 - b2) * gr * gr
    mhat = m / (1.0 - b1 ** t)
    vhat = v / (1.0 - b2 ** t)
    upd = lr * mhat / (np.sqrt(vhat) + eps)
    return theta - (upd[..., 0] + 1j * upd[..., 1])


def adam_update_real(theta: np.ndarray, g: np.ndarray, m: np.ndarray, v: np.ndarray, t: int,
                     lr: float, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
    """One Adam step on a real array; m and v (same shape) are updated in place."""
    m *= b1
    m += (1.0 - b1) * g
    v *= b2
    v += (1.0 - b2) * g * g
    mhat = m / (1.0 - b1 ** t)
    vhat = v / (1.0 - b2 ** t)
    return theta - lr * mhat / (np.sqrt(vhat) + eps)


def step_sigma_bg(O, P, sigma, bg, pos, Imeas, kind, eps, state: AdamState, m_sigma, v_sigma, m_bg, v_bg,
                  lr_O: float, lr_P: float, lr_sigma: float, lr_bg: float, b1=0.9, b2=0.999, adam_eps=1e-8,
                  mask=None, taps=None, frames=None):
    """One step that also optimises sigma ([J]) and the background ([F, F]) with Adam; every
    component of sigma takes the update (its gradient is 0 for frames outside ``frames``).
    Returns (loss, O, P, sigma, bg)."""
    total, gO, gP = gradient(O, P, pos, Imeas, kind, eps, sigma, bg, mask, taps, frames)
    _, g_sigma, g_bg = gradient_sigma_bg(O, P, pos, Imeas, kind, eps, sigma, bg, mask, taps, frames)
    state.t += 1
    O_new = [adam_update(O[l], gO[l], state.mO[l], state.vO[l], state.t, lr_O, b1, b2, adam_eps)
             for l in range(len(O))]
    P_new = adam_update(P, gP, state.mP, state.vP, state.t, lr_P, b1, b2, adam_eps)
    s_new = adam_update_real(np.asarray(sigma, np.float64), g_sigma, m_sigma, v_sigma, state.t, lr_sigma, b1, b2,
                             adam_eps)
    bg_new = adam_update_real(np.asarray(bg, np.float64), g_bg, m_bg, v_bg, state.t, lr_bg, b1, b2, adam_eps)
    return total, O_new, P_new, s_new, bg_new


def step(O, P, pos, Imeas, kind, eps, state: AdamState, lr_O: float, lr_P: float,
         b1=0.9, b2=0.999, adam_eps=1e-8, sigma=None, bg=None, mask=None, taps=None, frames=None):
    """One optimisation step: loss and gradient over ``frames``, then Adam on O and P."""
    total, gO, gP = gradient(O, P, pos, Imeas, kind, eps, sigma, bg, mask, taps, frames)
    state.t += 1
    O_new = [adam_update(O[l], gO[l], state.mO[l], state.vO[l], state.t, lr_O, b1, b2, adam_eps)
             for l in range(len(O))]
    P_new = adam_update(P, gP, state.mP, state.vP, state.t, lr_P, b1, b2, adam_eps)
    return total, O_new, P_new
