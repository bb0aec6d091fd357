"""Reference oracle: filtered back-projection.  TEST INFRASTRUCTURE ONLY:
imported by the tests, __graft_entry__.smoke() and bench.py's CPU legs, never
by the library.

The paper uses FBP for the start image, for beta and for the spatial
constraint (Step 1, Step 2, Fig. 9) without giving its filter.  Reading used:
the standard parallel-beam FBP with the discrete Ram-Lak (ramp) filter for
unit bin spacing (Kak & Slaney, Principles of Computerized Tomographic
Imaging, ch. 3):

    h(0) = 1/4,  h(k) = -1/(pi^2 k^2) for odd k,  h(k) = 0 for even k != 0,
    q_u(k) = sum_k' p_u(k') h(k - k')            (linear, zero-padded)
    f(x, y) = (pi / U) sum_u q_u(s),  s = x cos(theta_u) + y sin(theta_u),

with q_u(s) linearly interpolated between bin centres s_k = k - (B - 1)/2
(zero outside the detector) and pixel (i, j) at (j - (n-1)/2, (n-1)/2 - i).
FP64, plain numpy.
"""
from __future__ import annotations

import numpy as np


def ramlak(B: int) -> np.ndarray:
    """Filter taps h(k) for k = -(B-1) .. B-1 (index k + B - 1)."""
    k = np.arange(-(B - 1), B, dtype=np.float64)
    h = np.zeros_like(k)
    h[k == 0] = 0.25
    odd = (np.abs(k) % 2) == 1
    h[odd] = -1.0 / (np.pi ** 2 * k[odd] ** 2)
    return h


def angles_of(U: int, angles=None) -> np.ndarray:
    return np.asarray(angles, np.float64) if angles is not None else np.pi * np.arange(U) / U


def filter_sino(sino: np.ndarray) -> np.ndarray:
    """q_u = p_u convolved with the Ram-Lak taps, same length B."""
    p = np.asarray(sino, np.float64)
    U, B = p.shape
    h = ramlak(B)
    q = np.empty_like(p)
    for u in range(U):
        full = np.convolve(p[u], h)  # length 3B - 2; output k sits at index k + B - 1
        q[u] = full[B - 1:2 * B - 1]
    return q


def backproject(q: np.ndarray, n: int, angles=None) -> np.ndarray:
    U, B = q.shape
    th = angles_of(U, angles)
    c = np.cos(th)
    s = np.sin(th)
    c[np.abs(c) < 1e-12] = 0.0
    s[np.abs(s) < 1e-12] = 0.0
    j = np.arange(n, dtype=np.float64) - 0.5 * (n - 1)
    x = np.broadcast_to(j[None, :], (n, n))
    y = np.broadcast_to(-j[:, None], (n, n))
    f = np.zeros((n, n))
    for u in range(U):
        pos = x * c[u] + y * s[u] + 0.5 * (B - 1)  # fractional bin index
        k0 = np.floor(pos).astype(np.int64)
        a = pos - k0
        v0 = np.where((k0 >= 0) & (k0 < B), q[u][np.clip(k0, 0, B - 1)], 0.0)
        v1 = np.where((k0 + 1 >= 0) & (k0 + 1 < B), q[u][np.clip(k0 + 1, 0, B - 1)], 0.0)
        f += (1.0 - a) * v0 + a * v1
    return f * (np.pi / U)


def fbp(sino: np.ndarray, n: int, angles=None) -> np.ndarray:
    """FBP image [n, n] of a parallel-beam sinogram [U, B]."""
    return backproject(filter_sino(sino), n, angles)
