"""Seeded synthetic workloads shaped like the paper's experiment (inputs only).

The paper's dataset (Au/Ti structures on a Si wafer imaged with two HHG harmonics
on a 2048x2048 EUV camera, Section "Experimental setup") is not available.  These
generators produce stand-ins with the same structure: complex objects per
wavelength, mutually incoherent probe modes per wavelength, a jittered raster scan,
reflection geometry (88 mm, 15 um pixels, 70 degrees from the normal) and Poisson
photon noise.

Nothing here evaluates the forward model, a loss, a gradient or an optimiser step.
The measured patterns are made by the *caller*: it evaluates its own forward model
on ``truth`` parameters and passes the clean intensity to :func:`poisson_measure`.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Tuple

import numpy as np

try:  # scipy is normally present; the FFT fallback below covers its absence
    from scipy.ndimage import gaussian_filter as _gaussian_filter
except Exception:  # pragma: no cover
    _gaussian_filter = None

__all__ = [
    "Geometry", "Workload", "smooth_noise", "zernike_noll", "zernike_phase",
    "gaussian_amplitude", "probe_modes", "elliptical_aperture_modes",
    "object_smooth", "object_rectangles", "raster_positions", "scale_positions", "camera_frames",
    "round_half_away", "poisson_measure", "default_eps", "config1", "config2", "near_truth",
    "serving_workload", "serving_request_inputs", "TextureBank",
    "config3", "config4", "config5_requests", "tiny_workload", "CONFIG3_GRID",
]

PAPER_Z = 88e-3            # sample-to-camera distance (Section "Experimental setup")
PAPER_DET_PIXEL = 15e-6    # camera pixel pitch (same section)
PAPER_TILT = math.radians(70.0)  # angle of incidence from the surface normal
PAPER_LAMBDAS = (17.30e-9, 17.93e-9)  # the two harmonics of Fig. 3


@dataclasses.dataclass
class Geometry:
    lambdas: np.ndarray                 # [L] metres
    z: float = PAPER_Z
    det_pixel: float = PAPER_DET_PIXEL
    tilt_rad: float = PAPER_TILT
    remap: bool = False                 # tilted-plane remap inside the model


@dataclasses.dataclass
class Workload:
    """All inputs of one reconstruction problem (no measured data yet)."""
    name: str
    F: int
    L: int
    M: int
    J: int
    obj_shapes: List[Tuple[int, int]]
    O_true: List[np.ndarray]            # L x [H_l, W_l] complex128
    P_true: np.ndarray                  # [L, M, F, F] complex128
    O0: List[np.ndarray]                # evaluation point (initial guess)
    P0: np.ndarray
    pos: np.ndarray                     # [L, J, 2] int32, (row, col) of patch corner
    geom: Geometry
    loss: str = "amplitude"             # "amplitude" | "poisson"
    photons: float = 1e4
    sigma: Optional[np.ndarray] = None  # [J] power coefficients (None = 1)
    bg: Optional[np.ndarray] = None     # [F, F] background on the model grid
    mask: Optional[np.ndarray] = None   # [F, F] or [J, F, F] uint8 (None = all 1)
    seed: int = 0

    @property
    def n_evals(self) -> int:
        return self.J * self.L * self.M


# ----------------------------------------------------------------------------
# basic random fields
# ----------------------------------------------------------------------------

def smooth_noise(rng: np.random.Generator, shape, sigma: float) -> np.ndarray:
    """Uniform noise smoothed by a Gaussian of width ``sigma`` px, min-max scaled to [0, 1]."""
    u = rng.uniform(size=shape)
    if _gaussian_filter is not None:
        s = _gaussian_filter(u, sigma, mode="wrap")
    else:  # pragma: no cover - periodic Gaussian blur through the FFT
        ky = np.fft.fftfreq(shape[0])[:, None]
        kx = np.fft.fftfreq(shape[1])[None, :]
        g = np.exp(-2 * (math.pi * sigma) ** 2 * (ky ** 2 + kx ** 2))
        s = np.real(np.fft.ifft2(np.fft.fft2(u) * g))
    lo, hi = s.min(), s.max()
    return (s - lo) / (hi - lo)


def zernike_noll(j: int, rho: np.ndarray, theta: np.ndarray) -> np.ndarray:
    """Zernike polynomial with Noll index j = 1..10 (Noll 1976 normalisation)."""
    r2 = rho * rho
    if j == 1:
        return np.ones_like(rho)
    if j == 2:
        return 2 * rho * np.cos(theta)
    if j == 3:
        return 2 * rho * np.sin(theta)
    if j == 4:
        return math.sqrt(3) * (2 * r2 - 1)
    if j == 5:
        return math.sqrt(6) * r2 * np.sin(2 * theta)
    if j == 6:
        return math.sqrt(6) * r2 * np.cos(2 * theta)
    if j == 7:
        return math.sqrt(8) * (3 * r2 * rho - 2 * rho) * np.sin(theta)
    if j == 8:
        return math.sqrt(8) * (3 * r2 * rho - 2 * rho) * np.cos(theta)
    if j == 9:
        return math.sqrt(8) * r2 * rho * np.sin(3 * theta)
    if j == 10:
        return math.sqrt(8) * r2 * rho * np.cos(3 * theta)
    raise ValueError("Noll index must be in 1..10")


def _polar(F: int, radius: float):
    yy, xx = np.mgrid[0:F, 0:F].astype(np.float64)
    yy -= F / 2
    xx -= F / 2
    rho = np.sqrt(yy ** 2 + xx ** 2) / radius
    theta = np.arctan2(yy, xx)
    return rho, theta


def zernike_phase(F: int, coeffs: np.ndarray, radius: float) -> np.ndarray:
    """sum_j c_j Z_j on a disk of ``radius`` px centred at (F/2, F/2); zero outside."""
    rho, theta = _polar(F, radius)
    ph = np.zeros((F, F))
    for j, c in enumerate(coeffs, start=1):
        ph += c * zernike_noll(j, rho, theta)
    ph[rho > 1] = 0.0
    return ph


def gaussian_amplitude(F: int, fwhm: float) -> np.ndarray:
    """Gaussian amplitude of full width at half maximum ``fwhm`` px (of the amplitude)."""
    s = fwhm / (2 * math.sqrt(2 * math.log(2)))
    yy, xx = np.mgrid[0:F, 0:F].astype(np.float64)
    return np.exp(-((yy - F / 2) ** 2 + (xx - F / 2) ** 2) / (2 * s * s))


def probe_modes(rng: np.random.Generator, F: int, M: int, fwhm: float,
                powers, photons: float, zernike_sigma: float = 0.5) -> np.ndarray:
    """M mutually orthogonal Zernike-aberrated Gaussian probe modes.

    Each candidate mode is a Gaussian with a random Zernike phase (Noll 1..10,
    coefficients ~ N(0, zernike_sigma) rad).  The M candidates are orthogonalised
    through the SVD of the [M, F*F] matrix and scaled so mode m carries
    ``powers[m] * photons`` (sum over pixels of |P|^2).
    """
    amp = gaussian_amplitude(F, fwhm)
    cand = []
    for _ in range(M):
        c = rng.normal(0.0, zernike_sigma, size=10)
        cand.append(amp * np.exp(1j * zernike_phase(F, c, F / 2)))
    A = np.stack([c.reshape(-1) for c in cand])
    if M > 1:
        _, _, vh = np.linalg.svd(A, full_matrices=False)
        base = vh
    else:
        base = A / np.linalg.norm(A)
    powers = np.asarray(powers, dtype=np.float64)
    powers = powers / powers.sum()
    modes = base * np.sqrt(powers * photons)[:, None]
    return modes.reshape(M, F, F)


def elliptical_aperture_modes(F: int, M: int, centre=(0.0, 0.0), axes=None,
                              angle: float = 0.0, photons: float = 1e4) -> np.ndarray:
    """Initial probe guess: a uniform elliptical aperture (Section "Experimental setup").

    Mode 0 is the aperture; further modes are the aperture times low-order Zernike
    patterns, at decreasing power, so that the modes start distinct.
    """
    if axes is None:
        axes = (F / 6, F / 4)
    yy, xx = np.mgrid[0:F, 0:F].astype(np.float64)
    yy -= F / 2 + centre[0]
    xx -= F / 2 + centre[1]
    ca, sa = math.cos(angle), math.sin(angle)
    u = (ca * xx + sa * yy) / axes[1]
    v = (-sa * xx + ca * yy) / axes[0]
    ap = (u * u + v * v <= 1.0).astype(np.float64)
    rho, theta = _polar(F, max(axes))
    out = np.zeros((M, F, F), dtype=np.complex128)
    for m in range(M):
        shape = ap if m == 0 else ap * zernike_noll(2 + (m - 1) % 9, rho, theta)
        p = 1.0 / (2 ** m)
        out[m] = shape * math.sqrt(p * photons / max((np.abs(shape) ** 2).sum(), 1e-30))
    return out


# ----------------------------------------------------------------------------
# objects
# ----------------------------------------------------------------------------

def object_smooth(rng: np.random.Generator, H: int, W: int, sigma: float = 3.0) -> np.ndarray:
    """Amplitude 0.6 + 0.3*s1, phase pi*s2 with s1, s2 smoothed uniform noise."""
    s1 = smooth_noise(rng, (H, W), sigma)
    s2 = smooth_noise(rng, (H, W), sigma)
    return (0.6 + 0.3 * s1) * np.exp(1j * math.pi * s2)


def _rectangles(rng: np.random.Generator, H: int, W: int, lo: int, hi: int, cover: float):
    rects = []
    occ = np.zeros((H, W), bool)
    covered, target = 0, cover * H * W
    while covered < target:
        h = int(rng.integers(lo, hi + 1))
        w = int(rng.integers(lo, hi + 1))
        y = int(rng.integers(0, H - h + 1))
        x = int(rng.integers(0, W - w + 1))
        rects.append((y, x, h, w))
        covered += int(h * w - np.count_nonzero(occ[y:y + h, x:x + w]))
        occ[y:y + h, x:x + w] = True
    return rects


def object_rectangles(rng: np.random.Generator, H: int, W: int, lambdas,
                      feature=(8, 40), cover: float = 0.30,
                      phase_step: float = 0.4) -> List[np.ndarray]:
    """One object per wavelength: binary random rectangles on a smooth background.

    Rectangles (sides 8-40 px in wavelength-1 pixels, ~30 % coverage) have amplitude
    0.9 and phase step ``phase_step * lambda_1 / lambda_l``; the background has
    amplitude 0.5 and phase 0.2*s (smooth noise).  The same physical pattern is drawn
    for every wavelength at that wavelength's pixel size (proportional to lambda).
    """
    rects = _rectangles(rng, H, W, feature[0], feature[1], cover)
    s = smooth_noise(rng, (H, W), 3.0)
    out = []
    lam1 = float(lambdas[0])
    for lam in lambdas:
        r = lam1 / float(lam)          # lambda-1 pixels -> lambda-l pixels
        occ = np.zeros((H, W), bool)
        for (y, x, h, w) in rects:
            y0, x0 = int(round(y * r)), int(round(x * r))
            y1, x1 = int(round((y + h) * r)), int(round((x + w) * r))
            occ[y0:max(y1, y0 + 1), x0:max(x1, x0 + 1)] = True
        bgc = 0.5 * np.exp(1j * 0.2 * s)
        obj = np.where(occ, 0.9 * np.exp(1j * phase_step * r), bgc)
        out.append(obj.astype(np.complex128))
    return out


# ----------------------------------------------------------------------------
# scan positions
# ----------------------------------------------------------------------------

def round_half_away(x) -> np.ndarray:
    x = np.asarray(x, dtype=np.float64)
    return (np.sign(x) * np.floor(np.abs(x) + 0.5)).astype(np.int64)


def raster_positions(rng: np.random.Generator, ny: int, nx: int, step: int,
                     jitter: int, offset: int) -> np.ndarray:
    """Jittered raster: (row, col) patch corners, uniform integer jitter in [-jitter, jitter]."""
    iy, ix = np.mgrid[0:ny, 0:nx]
    base = np.stack([iy.reshape(-1), ix.reshape(-1)], axis=1) * step + offset
    jit = rng.integers(-jitter, jitter + 1, size=base.shape)
    return (base + jit).astype(np.int64)


def scale_positions(pos1: np.ndarray, lambdas) -> np.ndarray:
    """Positions in wavelength-l pixels: round_half_away(pos_1 * lambda_1 / lambda_l)."""
    lam1 = float(lambdas[0])
    return np.stack([round_half_away(pos1 * (lam1 / float(lam))) for lam in lambdas]).astype(np.int32)


# ----------------------------------------------------------------------------
# measurement noise (applied to a caller-computed clean intensity)
# ----------------------------------------------------------------------------

def poisson_measure(I_clean: np.ndarray, seed: int) -> np.ndarray:
    """Poisson photon counts for a clean intensity, as float32."""
    rng = np.random.default_rng(seed)
    lam = np.clip(np.asarray(I_clean, dtype=np.float64), 0.0, None)
    return rng.poisson(lam).astype(np.float32)


def camera_frames(J: int, F: int, seed: int, photons: float = 1e6, full_well: float = 65535.0) -> np.ndarray:
    """Raw camera patterns [J][F][F] float32 shaped like the experiment's (zero frequency at
    (F/2, F/2), a bright specular peak over a smooth speckle halo, Poisson photon noise) and
    clipped at a 16-bit full well, so that the brightest pixels saturate and the dark halo
    has pixels below a noise threshold of a few counts.  Inputs for the data-side tilt
    correction; no part of the measurement model is evaluated here."""
    rng = np.random.default_rng(seed)
    yy, xx = np.mgrid[0:F, 0:F].astype(np.float64) - F / 2
    out = np.empty((J, F, F), np.float32)
    for j in range(J):
        peak = np.exp(-(yy ** 2 + xx ** 2) / 2.0)
        halo = smooth_noise(rng, (F, F), max(1.0, F / 32)) * np.exp(-np.hypot(yy, xx) / (0.25 * F))
        I = photons * (0.7 * peak / peak.sum() + 0.3 * halo / max(halo.sum(), 1e-300))
        out[j] = np.minimum(rng.poisson(I), full_well).astype(np.float32)
    return out


def default_eps(I_meas: np.ndarray) -> float:
    """Intensity floor used by both losses: 1e-9 times the mean measured count."""
    return float(1e-9 * max(float(np.mean(I_meas, dtype=np.float64)), 1e-30))


# ----------------------------------------------------------------------------
# the five workloads
# ----------------------------------------------------------------------------

def _redraw_phase(rng, P_true: np.ndarray, F: int, fwhm_l, photons_l) -> np.ndarray:
    L, M = P_true.shape[:2]
    P0 = np.empty_like(P_true)
    for l in range(L):
        pw = (np.abs(P_true[l]) ** 2).reshape(M, -1).sum(1)
        P0[l] = probe_modes(rng, F, M, fwhm_l[l], pw, photons_l[l])
    return P0


def config1(seed: int = 0) -> Workload:
    """Plain single-wavelength single-mode ptychography (64x64 frames, 8x8 raster)."""
    rng = np.random.default_rng(seed)
    F, H = 64, 192
    lambdas = np.array([PAPER_LAMBDAS[0]])
    O = [object_smooth(rng, H, H, 3.0)]
    P = probe_modes(rng, F, 1, 24.0, [1.0], 1e4)[None]
    pos1 = raster_positions(rng, 8, 8, 16, 2, (H - (7 * 16 + F)) // 2)
    pos = scale_positions(pos1, lambdas)
    rng1 = np.random.default_rng(seed + 1)
    P0 = probe_modes(rng1, F, 1, 24.0, [1.0], 1e4)[None]
    return Workload("config1", F, 1, 1, pos.shape[1], [(H, H)], O, P,
                    [np.ones((H, H), np.complex128)], P0, pos,
                    Geometry(lambdas, remap=False), loss="amplitude", photons=1e4, seed=seed)


def _multi(name: str, seed: int, F: int, L: int, M: int, n_side: int, step: int,
           H: int, lam_ratio, photons: float, loss: str, remap: bool,
           powers=None, jitter: int = 2) -> Workload:
    rng = np.random.default_rng(seed)
    lambdas = PAPER_LAMBDAS[0] * np.asarray(lam_ratio, dtype=np.float64)[:L]
    O = object_rectangles(rng, H, H, lambdas)
    if powers is None:
        powers = [0.6, 0.25, 0.1, 0.05] if M == 4 else list(0.5 ** np.arange(M))
    fwhm1 = 3.0 * F / 8.0
    fwhm_l = [fwhm1 * lambdas[0] / lam for lam in lambdas]
    ph_l = [photons / L] * L
    P = np.stack([probe_modes(rng, F, M, fwhm_l[l], powers, ph_l[l]) for l in range(L)])
    offset = (H - ((n_side - 1) * step + F)) // 2
    assert offset >= jitter, "object too small for the scan"
    pos1 = raster_positions(rng, n_side, n_side, step, jitter, offset)
    pos = scale_positions(pos1, lambdas)
    rng1 = np.random.default_rng(seed + 1)
    P0 = _redraw_phase(rng1, P, F, fwhm_l, ph_l)
    O0 = [np.ones((H, H), np.complex128) for _ in range(L)]
    return Workload(name, F, L, M, pos.shape[1], [(H, H)] * L, O, P, O0, P0, pos,
                    Geometry(lambdas, remap=remap), loss=loss, photons=photons, seed=seed)


def config2(seed: int = 2) -> Workload:
    """3 wavelengths (1:1.1:1.2) x 4 modes, 256x256 frames, 20x20 raster, tilt remap, Poisson."""
    return _multi("config2", seed, 256, 3, 4, 20, 24, 768, [1.0, 1.1, 1.2], 1e5,
                  "poisson", True, powers=[0.6, 0.25, 0.1, 0.05])


CONFIG3_GRID = [(F, M, L) for F in (128, 256, 512) for M in (1, 4, 8) for L in (1, 3, 5)]


def config3(F: int, M: int, L: int, seed: int = 3, n_side: int = 20) -> Workload:
    """Throughput sweep point: 20x20 raster, 70 % overlap, rectangle objects."""
    step = int(round(0.1125 * F))
    side = (n_side - 1) * step + F + 8
    side = ((side + 15) // 16) * 16
    ratios = [1.0 + 0.05 * i for i in range(L)]
    return _multi(f"config3_F{F}_M{M}_L{L}", seed, F, L, M, n_side, step, side, ratios,
                  1e5, "poisson", True)


def config4(seed: int = 4) -> Workload:
    """~200M-parameter case: 6 wavelengths x 10 modes of 512^2, 6 x 3584^2 objects, 900 frames."""
    ratios = [1.0 + 0.0364 * i for i in range(6)]
    return _multi("config4", seed, 512, 6, 10, 30, 96, 3584, ratios, 1e5, "poisson", True)


def config5_requests(n: int = 64, seed: int = 5, mean_interval_s: float = 0.05,
                     frame_sizes=(128, 256, 512), j_range=(100, 900), l_max: int = 5,
                     m_max: int = 8):
    """Serving stream: request descriptors with Poisson arrivals.

    Returns a list of dicts with ``arrival_s``, ``F``, ``J``, ``L``, ``M`` and ``seed``.
    Workloads are built lazily with :func:`serving_workload` from these descriptors.
    """
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(n):
        t += float(rng.exponential(mean_interval_s))
        r = np.random.default_rng(1000 + i)
        out.append(dict(index=i, arrival_s=t, F=int(r.choice(frame_sizes)),
                        J=int(r.integers(j_range[0], j_range[1] + 1)),
                        L=int(r.integers(1, l_max + 1)), M=int(r.integers(1, m_max + 1)),
                        seed=1000 + i))
    return out


class TextureBank:
    """One large complex texture (rectangles on a smooth background) that serving requests
    crop their objects from, so that a stream of many requests is generated quickly."""

    def __init__(self, side: int = 2304, seed: int = 99):
        rng = np.random.default_rng(seed)
        self.tex = object_rectangles(rng, side, side, [PAPER_LAMBDAS[0]])[0]
        self.side = side

    def crop(self, rng: np.random.Generator, H: int, W: int) -> np.ndarray:
        y = int(rng.integers(0, self.side - H + 1))
        x = int(rng.integers(0, self.side - W + 1))
        return self.tex[y:y + H, x:x + W].copy()


def serving_request_inputs(desc: dict, bank: TextureBank) -> Workload:
    """Inputs of one serving request: config-3 scan rules, objects cropped from a texture
    bank, Zernike probe modes (truth) and elliptical-aperture modes with a flat object as
    the starting point (Section "Experimental setup")."""
    F, J, L, M, seed = desc["F"], desc["J"], desc["L"], desc["M"], desc["seed"]
    rng = np.random.default_rng(seed)
    n_side = int(math.ceil(math.sqrt(J)))
    step = int(round(0.1125 * F))
    side = (n_side - 1) * step + F + 8
    side = ((side + 15) // 16) * 16
    lambdas = PAPER_LAMBDAS[0] * (1.0 + 0.05 * np.arange(L))
    O = [bank.crop(rng, side, side) for _ in range(L)]
    fwhm1 = 3.0 * F / 8.0
    powers = list(0.5 ** np.arange(M))
    P = np.stack([probe_modes(rng, F, M, fwhm1 * lambdas[0] / lambdas[l], powers, 1e5 / L) for l in range(L)])
    offset = (side - ((n_side - 1) * step + F)) // 2
    pos1 = raster_positions(rng, n_side, n_side, step, 2, offset)[:J]
    pos = scale_positions(pos1, lambdas)
    P0 = np.stack([elliptical_aperture_modes(F, M, photons=1e5 / L) for _ in range(L)])
    O0 = [np.ones((side, side), np.complex128) for _ in range(L)]
    return Workload(f"request{desc['index']}_F{F}_J{J}_L{L}_M{M}", F, L, M, J, [(side, side)] * L, O, P, O0, P0,
                    pos, Geometry(lambdas, remap=True), loss="poisson", photons=1e5, seed=seed)


def serving_workload(desc: dict) -> Workload:
    """A request of the serving stream: config-3 rules, elliptical-aperture start."""
    F, J, L, M, seed = desc["F"], desc["J"], desc["L"], desc["M"], desc["seed"]
    n_side = int(math.ceil(math.sqrt(J)))
    w = config3(F, M, L, seed=seed, n_side=n_side)
    w.pos = w.pos[:, :J].copy()
    w.J = J
    P0 = np.stack([elliptical_aperture_modes(F, M, photons=w.photons / L) for _ in range(L)])
    w.P0 = P0
    w.name = f"request{desc['index']}_F{F}_J{J}_L{L}_M{M}"
    return w


def near_truth(w: Workload, seed: int = 0, amp: float = 0.05):
    """An evaluation point close to the ground truth: small smooth amplitude and phase
    perturbations of every object and a small extra Zernike phase on every probe mode."""
    rng = np.random.default_rng(seed)
    O = []
    for o in w.O_true:
        s1 = smooth_noise(rng, o.shape, 4.0) - 0.5
        s2 = smooth_noise(rng, o.shape, 4.0) - 0.5
        O.append(o * (1.0 + amp * s1) * np.exp(1j * amp * s2))
    P = np.empty_like(w.P_true)
    for l in range(w.L):
        for m in range(w.M):
            c = rng.normal(0.0, amp, size=10)
            P[l, m] = w.P_true[l, m] * np.exp(1j * zernike_phase(w.F, c, w.F / 2))
    return O, P


def tiny_workload(F: int = 16, L: int = 2, M: int = 2, n_side: int = 3, step: int = 4,
                  seed: int = 7, remap: bool = False, loss: str = "amplitude",
                  with_sigma: bool = False, with_bg: bool = False, H: Optional[int] = None,
                  photons: float = 1e3) -> Workload:
    """A small multi-wavelength, multi-mode case for exhaustive checks."""
    rng = np.random.default_rng(seed)
    if H is None:
        H = (n_side - 1) * step + F + 6
    lambdas = PAPER_LAMBDAS[0] * (1.0 + 0.1 * np.arange(L))
    O = [object_smooth(rng, H, H + 2, 1.5) for _ in range(L)]
    P = np.stack([probe_modes(rng, F, M, F / 3.0, 0.5 ** np.arange(M), photons / L)
                  for _ in range(L)])
    pos1 = raster_positions(rng, n_side, n_side, step, 1, 2)
    pos = scale_positions(pos1, lambdas)
    O0 = [o * np.exp(0.1j) * 0.9 + 0.05 for o in O]
    P0 = P * 1.1 * np.exp(-0.2j)
    sigma = (1.0 + 0.1 * rng.standard_normal(pos.shape[1])) if with_sigma else None
    bg = (0.5 + rng.uniform(size=(F, F))) if with_bg else None
    return Workload(f"tiny_F{F}", F, L, M, pos.shape[1], [(H, H + 2)] * L, O, P, O0, P0, pos,
                    Geometry(lambdas, remap=remap), loss=loss, photons=photons,
                    sigma=sigma, bg=bg, seed=seed)
