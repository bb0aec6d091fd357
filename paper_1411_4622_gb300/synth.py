"""Seeded synthetic inputs shaped like the paper's experiments.

This module holds no step of the reconstruction method.  It makes the things
a tomography experiment starts from: a phantom image (random ellipses,
standing in for the paper's Phantoms 1-3, whose images are not available), a
reconstruction-space mask (the "uniform solid circle" of Sec. III), an
initial estimate, and measurement noise applied to a clean sinogram that the
caller computes.  Both the CUDA path and the CPU reference draw their inputs
from here, with numpy's PCG64 generator seeded per slice.

Geometry convention (shared by every part of the project): pixel (i, j) of an
n x n image has its centre at x = j - (n-1)/2, y = (n-1)/2 - i.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


def bins_for(n: int) -> int:
    """Detector bins covering the image diagonal: 2*floor(n/sqrt(2)) + 1."""
    return 2 * int(math.floor(n / math.sqrt(2.0))) + 1


def angles_for(n_angles: int) -> np.ndarray:
    """Evenly spaced parallel-beam angles over [0, pi)."""
    return np.pi * np.arange(n_angles, dtype=np.float64) / n_angles


@dataclass(frozen=True)
class Ellipses:
    cx: np.ndarray
    cy: np.ndarray
    ax: np.ndarray
    ay: np.ndarray
    angle: np.ndarray
    density: np.ndarray


def random_ellipses(n: int, count: int, seed: int) -> Ellipses:
    """Ellipse parameters: centres uniform in a disk of radius 0.6*n/2,
    semi-axes uniform in [0.05, 0.35]*n/2 (shrunk so that every ellipse stays
    inside radius 0.9*n/2), orientation uniform in [0, pi), density uniform
    in [0, 1]."""
    rng = np.random.default_rng(seed)
    R = 0.5 * n
    rad = 0.6 * R * np.sqrt(rng.random(count))
    phi = 2.0 * np.pi * rng.random(count)
    cx, cy = rad * np.cos(phi), rad * np.sin(phi)
    ax = rng.uniform(0.05, 0.35, count) * R
    ay = rng.uniform(0.05, 0.35, count) * R
    room = np.maximum(0.9 * R - rad, 0.5)
    shrink = np.minimum(1.0, room / np.maximum(ax, ay))
    ax, ay = ax * shrink, ay * shrink
    angle = rng.uniform(0.0, np.pi, count)
    density = rng.uniform(0.0, 1.0, count)
    return Ellipses(cx, cy, ax, ay, angle, density)


def rasterize(e: Ellipses, n: int) -> np.ndarray:
    """Point-sample the ellipses at pixel centres; later ellipses overwrite
    earlier ones (painter's order).  Returns float64 [n, n]."""
    j = np.arange(n, dtype=np.float64)
    x = (j - 0.5 * (n - 1))[None, :]
    y = (0.5 * (n - 1) - j)[:, None]
    img = np.zeros((n, n), dtype=np.float64)
    for q in range(len(e.cx)):
        c, s = math.cos(e.angle[q]), math.sin(e.angle[q])
        dx, dy = x - e.cx[q], y - e.cy[q]
        xr = dx * c + dy * s
        yr = -dx * s + dy * c
        inside = (xr / e.ax[q]) ** 2 + (yr / e.ay[q]) ** 2 <= 1.0
        img[inside] = e.density[q]
    return img


def phantom(n: int, count: int, seed: int) -> np.ndarray:
    return rasterize(random_ellipses(n, count, seed), n)


def disk_mask(n: int, radius: float | None = None) -> np.ndarray:
    """Pixels whose centre lies within `radius` (default n/2) of the centre."""
    r = 0.5 * n if radius is None else radius
    j = np.arange(n, dtype=np.float64) - 0.5 * (n - 1)
    return ((j[None, :] ** 2 + j[:, None] ** 2) <= r * r).astype(np.uint8)


def initial_image(n: int, value: float = 0.5, mask: np.ndarray | None = None) -> np.ndarray:
    """Uniform grey image, or a uniform solid circle when a mask is given."""
    img = np.full((n, n), value, dtype=np.float64)
    if mask is not None:
        img *= mask.astype(np.float64)
    return img


def gaussian_noise(sino: np.ndarray, sigma_frac: float, seed: int) -> np.ndarray:
    """Additive white Gaussian noise with sigma = sigma_frac * max(sino)."""
    rng = np.random.default_rng(seed)
    s = np.asarray(sino, dtype=np.float64)
    return s + rng.normal(0.0, sigma_frac * float(np.max(s)), size=s.shape)


def poisson_noise(sino: np.ndarray, i0: float, seed: int, peak_attenuation: float = 2.0) -> np.ndarray:
    """Transmission noise: scale a so that max(a*sino) = peak_attenuation,
    draw counts ~ Poisson(i0 * exp(-a*sino)), return -ln(max(c, 1)/i0) / a."""
    rng = np.random.default_rng(seed)
    s = np.asarray(sino, dtype=np.float64)
    peak = float(np.max(s))
    a = peak_attenuation / peak if peak > 0 else 1.0
    counts = rng.poisson(i0 * np.exp(-a * s))
    return -np.log(np.maximum(counts, 1) / i0) / a


def rmse(img: np.ndarray, ref: np.ndarray, mask: np.ndarray | None = None) -> float:
    d = np.asarray(img, np.float64) - np.asarray(ref, np.float64)
    if mask is not None:
        d = d[mask.astype(bool)]
    return float(np.sqrt(np.mean(d * d)))


def nrmse(img: np.ndarray, ref: np.ndarray) -> float:
    """RMS difference divided by the phantom's mean (Sec. III-B)."""
    return rmse(img, ref) / float(np.mean(ref))


# Workloads shaped like the paper's experiments (sizes, angles, bins, noise,
# estimates per move, sweeps).
WORKLOADS = {
    "plain64": dict(n=64, ellipses=10, n_angles=90, n_bins=91, noise=None, bome_k=1, n_sweeps=20,
                    t0=1e-2, tn=0.0, mask=False, beta=1.0),
    "sat256": dict(n=256, ellipses=20, n_angles=180, n_bins=363, noise=("gauss", 0.01), bome_k=8,
                   n_sweeps=100, t0=-1.0, tn=-1.0, mask=True, beta=1.0, sirt_iters=200),
    "batch128x512": dict(n=128, ellipses=20, n_angles=120, n_bins=181, noise=None, bome_k=4,
                         n_sweeps=50, t0=-1.0, tn=-1.0, mask=True, beta=1.0, slices=512),
    "precision512": dict(n=512, ellipses=40, n_angles=360, n_bins=725, noise=("poisson", 1e5),
                         bome_k=8, n_sweeps=200, t0=-1.0, tn=-1.0, mask=True, beta=1.0),
}


def slice_seeds(index: int) -> tuple[int, int, int]:
    """(phantom seed, noise seed, annealing seed) of slice `index`."""
    return 1000 + index, 2000 + index, 3000 + index
