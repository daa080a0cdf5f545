"""Seeded synthetic direction sets, density fields, generators and materials.

These produce the inputs of the transport sweep: a discrete-ordinates direction
set with weights, lognormal density fields, Voronoi generators, and per-cell
absorption, scattering and emissivity. They hold none of the method's
arithmetic.
"""
from __future__ import annotations

import math

import numpy as np


# ----------------------------------------------------------------------------------------------
# Directions
# ----------------------------------------------------------------------------------------------
def random_rotation(rng: np.random.Generator) -> np.ndarray:
    """Uniform random rotation matrix from a random unit quaternion."""
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


def fibonacci_directions(n: int, seed: int | None = 0):
    """n unit vectors on a Fibonacci sphere, rotated by a seeded random rotation.

    Returns (omega[n,3], weight[n]) with equal weights 4*pi/n (the solid angle of one
    direction bin is 4*pi/N_dir, paper Sec. 2.6). seed=None skips the rotation.
    """
    i = np.arange(n, dtype=np.float64)
    z = 1.0 - (2.0 * i + 1.0) / n
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    phi = i * math.pi * (3.0 - math.sqrt(5.0))
    om = np.stack([r * np.cos(phi), r * np.sin(phi), z], 1)
    if seed is not None:
        om = om @ random_rotation(np.random.default_rng(seed)).T
    om /= np.linalg.norm(om, axis=1)[:, None]
    return np.ascontiguousarray(om), np.full(n, 4.0 * math.pi / n)


# ----------------------------------------------------------------------------------------------
# Density fields
# ----------------------------------------------------------------------------------------------
def lognormal_field(ngrid: int, slope: float, sigma_ln: float, seed: int) -> np.ndarray:
    """Lognormal density rho = exp(delta - sigma^2/2) on a periodic ngrid^3 grid.

    delta is a Gaussian random field with power spectrum P(k) ~ k^slope, scaled to
    standard deviation sigma_ln. Returned array is indexed [ix, iy, iz], mean ~ 1.
    """
    rng = np.random.default_rng(seed)
    white = rng.normal(size=(ngrid, ngrid, ngrid))
    wk = np.fft.rfftn(white)
    kx = np.fft.fftfreq(ngrid) * ngrid
    kz = np.fft.rfftfreq(ngrid) * ngrid
    k2 = kx[:, None, None] ** 2 + kx[None, :, None] ** 2 + kz[None, None, :] ** 2
    k2[0, 0, 0] = 1.0
    amp = k2 ** (slope / 4.0)
    amp[0, 0, 0] = 0.0
    delta = np.fft.irfftn(wk * amp, s=(ngrid, ngrid, ngrid), axes=(0, 1, 2))
    delta *= sigma_ln / delta.std()
    return np.exp(delta - 0.5 * sigma_ln ** 2)


def sample_field(field: np.ndarray, pts: np.ndarray) -> np.ndarray:
    """Nearest-grid-point value of a periodic grid field at points in the unit box."""
    ng = field.shape[0]
    idx = np.floor(pts * ng).astype(np.int64) % ng
    return field[idx[:, 0], idx[:, 1], idx[:, 2]]


def generators_poisson(n: int, seed: int) -> np.ndarray:
    return np.random.default_rng(seed).random((n, 3))


def generators_from_density(field: np.ndarray, n: int, seed: int) -> np.ndarray:
    """n points with probability density proportional to the grid field (uniform inside a grid cell)."""
    rng = np.random.default_rng(seed)
    ng = field.shape[0]
    p = field.ravel() / field.sum()
    cells = rng.choice(p.size, size=n, p=p)
    ix, iy, iz = np.unravel_index(cells, field.shape)
    pts = (np.stack([ix, iy, iz], 1) + rng.random((n, 3))) / ng
    return np.clip(pts, 0.0, np.nextafter(1.0, 0.0))


def hilbert_order(pts: np.ndarray, bits: int = 10) -> np.ndarray:
    """Permutation sorting points along a 3-D Hilbert curve (a Peano-Hilbert cell ordering)."""
    n = pts.shape[0]
    x = np.minimum((pts * (1 << bits)).astype(np.int64), (1 << bits) - 1)
    X = [x[:, 0].copy(), x[:, 1].copy(), x[:, 2].copy()]
    # Skilling's transpose algorithm: axes -> transposed Hilbert index
    M = 1 << (bits - 1)
    Q = M
    while Q > 1:
        P = Q - 1
        for i in range(3):
            hi = (X[i] & Q) != 0
            X[0] = np.where(hi, X[0] ^ P, X[0])
            t = np.where(hi, 0, (X[0] ^ X[i]) & P)
            X[0] ^= t
            X[i] ^= t
        Q >>= 1
    for i in range(1, 3):
        X[i] ^= X[i - 1]
    t = np.zeros(n, np.int64)
    Q = M
    while Q > 1:
        t = np.where((X[2] & Q) != 0, t ^ (Q - 1), t)
        Q >>= 1
    for i in range(3):
        X[i] ^= t
    key = np.zeros(n, np.int64)
    for b in range(bits - 1, -1, -1):
        for i in range(3):
            key = (key << 1) | ((X[i] >> b) & 1)
    return np.argsort(key, kind="stable")


# ----------------------------------------------------------------------------------------------
# Materials
# ----------------------------------------------------------------------------------------------
GROUP_FACTORS = (1.0, 0.3, 0.1, 0.03)


def kappa_from_density(rho: np.ndarray, volume: np.ndarray, n_groups: int, tau_lo: float = 0.01,
                       tau_hi: float = 10.0) -> np.ndarray:
    """Absorption kappa[c,g] = k0 * f_g * rho_c with per-cell optical depth kappa*V^(1/3) in [tau_lo, tau_hi].

    k0 puts the median per-cell optical depth of group 0 at sqrt(tau_lo*tau_hi).
    """
    h = np.cbrt(volume)
    tau = rho * h
    k0 = math.sqrt(tau_lo * tau_hi) / np.median(tau)
    tau0 = np.clip(k0 * tau, tau_lo, tau_hi)
    kap0 = tau0 / h
    f = np.array(GROUP_FACTORS[:n_groups])
    return np.ascontiguousarray(kap0[:, None] * f[None, :])


def point_sources(weight: np.ndarray, n_src: int, seed: int, log_range: float | None = None) -> tuple:
    """Pick n_src distinct cells with probability proportional to weight (e.g. mass rho*V).

    Returns (cells, emissivity): unit emissivity, or log-uniform over log_range decades.
    """
    rng = np.random.default_rng(seed)
    p = weight / weight.sum()
    n_src = min(n_src, int(np.count_nonzero(p)))
    cells = np.sort(rng.choice(p.size, size=n_src, replace=False, p=p))
    if log_range is None:
        em = np.ones(n_src)
    else:
        em = 10.0 ** (rng.random(n_src) * log_range)
    return cells, em


def emissivity_array(n_cells: int, n_groups: int, cells: np.ndarray, em: np.ndarray) -> np.ndarray:
    eps = np.zeros((n_cells, n_groups))
    eps[cells, :] = em[:, None]
    return eps
