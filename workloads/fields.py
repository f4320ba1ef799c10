"""Analytic electromagnetic fields and seeded random positions.

These are exact solutions of the loss-free Maxwell system eps E' = curl H,
mu H' = -curl E (or plain initial data), evaluated pointwise.  They are
inputs: the discretisations project them onto their own spaces.
"""

import numpy as np


def te110_fields(x, t):
    """(1,1,0) mode of the PEC unit-cube cavity with E parallel to z, eps = mu = 1.

    E = z sin(pi x) sin(pi y) cos(w t)
    H = (pi/w)(-sin(pi x) cos(pi y), cos(pi x) sin(pi y), 0) sin(w t),  w = pi sqrt(2).
    x: (..., 3). Returns E, H of shape (..., 3).
    """
    w = np.pi * np.sqrt(2.0)
    sx, cx = np.sin(np.pi * x[..., 0]), np.cos(np.pi * x[..., 0])
    sy, cy = np.sin(np.pi * x[..., 1]), np.cos(np.pi * x[..., 1])
    E = np.zeros(x.shape)
    H = np.zeros(x.shape)
    E[..., 2] = sx * sy * np.cos(w * t)
    H[..., 0] = -(np.pi / w) * sx * cy * np.sin(w * t)
    H[..., 1] = (np.pi / w) * cx * sy * np.sin(w * t)
    return E, H


def te110_omega():
    return np.pi * np.sqrt(2.0)


def gaussian_pulse_fields(x, centre, width=0.1):
    """E = z exp(-|x - c|^2 / width^2), H = 0."""
    r2 = np.sum((x - np.asarray(centre)) ** 2, axis=-1)
    E = np.zeros(x.shape)
    E[..., 2] = np.exp(-r2 / width ** 2)
    return E, np.zeros(x.shape)


PLANE_WAVE_K = 2.0 * np.pi * np.array([1.0, 2.0, 3.0])
PLANE_WAVE_E0 = np.array([2.0, -1.0, 0.0]) / np.sqrt(5.0)


def plane_wave_fields(x, t, k=PLANE_WAVE_K, e0=PLANE_WAVE_E0):
    """E = e0 cos(k.x - w t), H = (k x e0)/w cos(k.x - w t), w = |k| (eps = mu = 1)."""
    k = np.asarray(k, dtype=float)
    e0 = np.asarray(e0, dtype=float)
    w = np.linalg.norm(k)
    ph = np.cos(x @ k - w * t)
    E = ph[..., None] * e0
    H = ph[..., None] * (np.cross(k, e0) / w)
    return E, H


def dipole_waveform(t, t0, tau, amp=1.0):
    """Zero-mean Gaussian-derivative pulse f(t) = -amp ((t-t0)/tau) exp(-((t-t0)/tau)^2)."""
    s = (np.asarray(t) - t0) / tau
    return -amp * s * np.exp(-s * s)


def random_points(seed, count, lo, hi):
    """count points uniform in [lo, hi]^3 (PCG64, seeded)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(lo, hi, size=(count, 3))
