"""Seeded synthetic inputs shared by the tests, the bench and the oracle checks.

This module only draws inputs: baseline coordinates (u, v, w) in wavelengths,
sky images of point sources, visibility noise and index subsamples.  It holds
none of the measurement operator's arithmetic (no taper, kernel, chirp,
gridding or FFT), so the oracle and the CUDA path can both take their inputs
from here without sharing any of the method.

The shapes follow the paper's workload (an MWA observation of Fornax A,
Sec. 4): a wide field (20-25 deg) imaged at 2048^2 and larger, hundreds of
thousands to 10^8 visibilities, and |w| of hundreds to thousands of
wavelengths.  The real data set is not available, so Earth-rotation tracks of
a random 128-antenna array stand in for it.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, asdict

import numpy as np


# ----------------------------------------------------------------------------
# Workload descriptions (operator parameters + input recipe)
# ----------------------------------------------------------------------------

@dataclass
class Workload:
    name: str
    image_n: int              # N: image side in pixels
    oversample: float         # os: padded grid side = os * N
    fov_deg: float            # full field of view (direction-cosine width)
    support: int              # J: Kaiser-Bessel support in grid pixels
    n_stacks: int             # K: number of k-means w-stacks
    conj_fold: bool           # fold every visibility onto w >= 0 (Sec. 3.3)
    n_vis: int                # visibilities before dropping out-of-grid ones
    uvw: dict = field(default_factory=dict)   # recipe for the baselines
    n_sources: int = 20
    noise_frac: float = 0.0   # complex noise sigma relative to the rms signal
    seed: int = 0

    def as_dict(self):
        return asdict(self)


def tiny(seed: int = 0, n_vis: int = 5000) -> Workload:
    """128^2 image, 256^2 grid, FOV 20 deg, J=4, one stack, 5000 visibilities
    with (u, v) uniform in a 60-wavelength disk and w uniform in [-40, 40]."""
    return Workload("tiny-128-fp64", 128, 2.0, 20.0, 4, 1, False, n_vis,
                    dict(kind="disk", radius=60.0, wmax=40.0),
                    n_sources=20, seed=seed)


def mwa_snapshot(seed: int = 0) -> Workload:
    """2048^2 image, 4096^2 grid, FOV 25 deg, 150 MHz, 128 antennas in a 3 km
    disk, 2 min at 0.5 s cadence (240 x 8128 = 1,950,720 visibilities),
    |w| rescaled to 500 wavelengths, 8 stacks, fold on."""
    return Workload("mwa-2048-8stack", 2048, 2.0, 25.0, 4, 8, True, 240 * 8128,
                    dict(kind="earth", n_ant=128, radius_m=3000.0, freq_hz=150e6,
                         lat_deg=-26.7, dec_deg=-37.2, ha_min=-1.0, ha_max=1.0,
                         n_times=240, wmax=500.0),
                    n_sources=200, noise_frac=0.01, seed=seed)


def precision_study(seed: int = 0) -> Workload:
    """4096^2 image, 8192^2 grid, same array over 2 h (2153 samples,
    17.5M visibilities), |w| up to 1500, 32 stacks, fold on."""
    return Workload("precision-4096-32stack", 4096, 2.0, 25.0, 4, 32, True, 2153 * 8128,
                    dict(kind="earth", n_ant=128, radius_m=3000.0, freq_hz=150e6,
                         lat_deg=-26.7, dec_deg=-37.2, ha_min=-60.0, ha_max=60.0,
                         n_times=2153, wmax=1500.0),
                    n_sources=200, seed=seed)


def differentiable(seed: int = 0) -> Workload:
    """4096^2 image, 10M visibilities (1231 samples), 16 stacks, fold on."""
    return Workload("diff-4096-16stack", 4096, 2.0, 25.0, 4, 16, True, 1231 * 8128,
                    dict(kind="earth", n_ant=128, radius_m=3000.0, freq_hz=150e6,
                         lat_deg=-26.7, dec_deg=-37.2, ha_min=-60.0, ha_max=60.0,
                         n_times=1231, wmax=1000.0),
                    n_sources=200, seed=seed)


# ----------------------------------------------------------------------------
# Baselines
# ----------------------------------------------------------------------------

def uvw_disk(n_vis: int, radius: float, wmax: float, seed: int = 0) -> np.ndarray:
    """(u, v) area-uniform in a disk of the given radius, w uniform in
    [-wmax, wmax]; float64 (n_vis, 3) in wavelengths."""
    rng = np.random.default_rng(seed)
    r = radius * np.sqrt(rng.random(n_vis))
    t = 2.0 * np.pi * rng.random(n_vis)
    w = rng.uniform(-wmax, wmax, n_vis)
    return np.ascontiguousarray(np.stack([r * np.cos(t), r * np.sin(t), w], axis=1))


def antennas_in_disk(n_ant: int, radius_m: float, seed: int = 0) -> np.ndarray:
    """East/north antenna positions (metres), area-uniform in a disk."""
    rng = np.random.default_rng(seed + 1000)
    r = radius_m * np.sqrt(rng.random(n_ant))
    t = 2.0 * np.pi * rng.random(n_ant)
    return np.stack([r * np.cos(t), r * np.sin(t)], axis=1)


def uvw_earth_rotation(n_ant: int, radius_m: float, freq_hz: float, lat_deg: float,
                       dec_deg: float, ha_min: float, ha_max: float, n_times: int,
                       wmax: float | None = None, seed: int = 0) -> np.ndarray:
    """Earth-rotation synthesis tracks of a planar array.

    Baselines (east, north, up=0) are turned into equatorial (X, Y, Z) at the
    array latitude and then projected on the phase centre at hour angle H and
    declination dec with the standard textbook rotation (Thompson, Moran &
    Swenson, Eq. 4.1).  Hour angles are in minutes of time.  When wmax is
    given, w is rescaled linearly so that max|w| == wmax (u and v untouched).
    Result: float64 (n_times * n_baselines, 3), time-major.
    """
    lam = 299792458.0 / freq_hz
    pos = antennas_in_disk(n_ant, radius_m, seed)
    i, j = np.triu_indices(n_ant, k=1)
    e = (pos[j, 0] - pos[i, 0]) / lam
    n = (pos[j, 1] - pos[i, 1]) / lam
    lat = math.radians(lat_deg)
    dec = math.radians(dec_deg)
    X = -math.sin(lat) * n
    Y = e
    Z = math.cos(lat) * n
    ha = np.linspace(ha_min, ha_max, n_times) * (2.0 * np.pi / (24.0 * 60.0))
    sh = np.sin(ha)[:, None]
    ch = np.cos(ha)[:, None]
    u = sh * X + ch * Y
    v = -math.sin(dec) * ch * X + math.sin(dec) * sh * Y + math.cos(dec) * Z
    w = math.cos(dec) * ch * X - math.cos(dec) * sh * Y + math.sin(dec) * Z
    if wmax is not None:
        w = w * (wmax / np.max(np.abs(w)))
    return np.ascontiguousarray(np.stack([u.ravel(), v.ravel(), w.ravel()], axis=1))


def uvw_for(wl: Workload) -> np.ndarray:
    spec = dict(wl.uvw)
    kind = spec.pop("kind")
    if kind == "disk":
        return uvw_disk(wl.n_vis, spec["radius"], spec["wmax"], wl.seed)
    if kind == "earth":
        return uvw_earth_rotation(seed=wl.seed, **spec)
    raise ValueError(kind)


# ----------------------------------------------------------------------------
# Images, noise, subsamples
# ----------------------------------------------------------------------------

def point_sources(n: int, n_src: int, seed: int = 0, inner: float = 0.9,
                  flux=(0.1, 1.0)) -> np.ndarray:
    """Real n x n image (float64, row = m, column = l) with n_src point
    sources at distinct pixel centres inside the central `inner` fraction of
    the image, fluxes uniform in `flux`."""
    rng = np.random.default_rng(seed + 2000)
    lo = int(round(n * (1.0 - inner) / 2.0))
    hi = n - lo
    img = np.zeros((n, n))
    placed = 0
    while placed < n_src:
        r, c = rng.integers(lo, hi, 2)
        if img[r, c] == 0.0:
            img[r, c] = rng.uniform(*flux)
            placed += 1
    return img


def random_image(n: int, seed: int = 0) -> np.ndarray:
    """Dense real image with standard normal pixels (for adjoint tests)."""
    return np.random.default_rng(seed + 3000).standard_normal((n, n))


def random_vis(m: int, seed: int = 0) -> np.ndarray:
    """Complex standard normal visibilities (complex128)."""
    rng = np.random.default_rng(seed + 4000)
    return rng.standard_normal(m) + 1j * rng.standard_normal(m)


def complex_noise(m: int, sigma: float, seed: int = 0) -> np.ndarray:
    rng = np.random.default_rng(seed + 5000)
    return sigma * (rng.standard_normal(m) + 1j * rng.standard_normal(m)) / math.sqrt(2.0)


def subsample(m: int, k: int, seed: int = 0) -> np.ndarray:
    """Sorted distinct indices of k out of m items."""
    rng = np.random.default_rng(seed + 6000)
    k = min(k, m)
    return np.sort(rng.choice(m, size=k, replace=False))


def dde_kernels(m: int, taps: int, seed: int = 0):
    """Synthetic separable direction-dependent-effect kernels on the grid,
    one pair per visibility: a[i] (u offsets -h..h) and b[i] (v offsets),
    taps = 2 h + 1.  Each is a sampled Gaussian of width U[0.4, 1.2] pixels
    centred U[-0.5, 0.5] pixels off, times a phase ramp of U[-0.5, 0.5] rad per
    pixel (a smooth aperture-plane blur and shift, as a primary-beam or
    ionospheric model would give), normalised to unit sum of magnitudes.
    complex128 (m, taps) each."""
    rng = np.random.default_rng(seed + 7000)
    h = (taps - 1) // 2
    s = np.arange(-h, h + 1, dtype=np.float64)

    def one():
        sig = rng.uniform(0.4, 1.2, (m, 1))
        off = rng.uniform(-0.5, 0.5, (m, 1))
        ramp = rng.uniform(-0.5, 0.5, (m, 1))
        k = np.exp(-0.5 * ((s[None, :] - off) / sig) ** 2) * np.exp(1j * ramp * s[None, :])
        return k / np.sum(np.abs(k), axis=1, keepdims=True)
    return one(), one()
