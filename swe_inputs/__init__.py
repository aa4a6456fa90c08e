"""Seeded synthetic inputs for the rotating shallow-water SDC workloads.

This module is shared by the CUDA path (bench, tests) and by the CPU oracle
(tests only).  It holds workload descriptions, the spectral-coefficient
packing convention, seeded random draws and the analytic height bump; it
holds none of the time integrator's or the spectral transform's arithmetic.

The paper benchmarks on the Galewsky barotropic-instability case (Sec. 5.1);
its analytic state is not reproduced here.  These seeded synthetic states
stand in for it: random vorticity/divergence spectra with amplitude
proportional to n^-1.5, scaled to a prescribed area-weighted rms wind, plus
Gaussian height bumps.

Spectral packing ("m-major triangular"): for orders m = 0..T and degrees
n = m..T the coefficient (n, m) sits at index off(m) + (n - m) with
off(m) = m (2T + 3 - m) / 2, so ncoef = (T + 1)(T + 2) / 2.  Fields are
complex; the m = 0 coefficients of a real field have zero imaginary part.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

# Physical constants of the workloads (Earth values).
RADIUS = 6.371e6          # m
OMEGA = 7.292e-5          # s^-1
GRAVITY = 9.80616         # m s^-2
MEAN_DEPTH = 1.0e4        # m

SEED_BASE = 240320135     # digits of the paper's arXiv identifier

# seed "purpose" slots
PURPOSE_ZETA, PURPOSE_DIV, PURPOSE_BUMPS, PURPOSE_TARGET, PURPOSE_DIRECTIONS = range(5)


@dataclass(frozen=True)
class Workload:
    """One seeded workload: truncation, Gauss grid, SDC nodes/sweeps, step size."""
    key: str
    index: int            # seed index
    T: int                # triangular truncation
    nlat: int             # Gauss latitudes J
    nlon: int             # longitudes L
    nodes: int            # M collocation nodes (Radau-right)
    sweeps: int           # K sweeps
    dt: float             # s
    nsteps: int
    nbumps: int
    bump_amp: tuple       # (low, high) amplitude in m
    rms_wind: float = 20.0
    div_scale: float = 0.1
    bump_radius: float = 500.0e3

    @property
    def ncoef(self) -> int:
        return ncoef(self.T)

    def describe(self) -> str:
        return (f"T{self.T} {self.nlat}x{self.nlon} Gauss grid, M={self.nodes} Radau-right, "
                f"K={self.sweeps}, dt={self.dt:g}s, {self.nsteps} steps")


WORKLOADS = {
    "t31": Workload("t31", 0, 31, 48, 96, 3, 3, 600.0, 20, 1, (100.0, 100.0)),
    "t127": Workload("t127", 1, 127, 192, 384, 4, 4, 300.0, 200, 3, (50.0, 150.0)),
    "t255": Workload("t255", 2, 255, 384, 768, 4, 5, 150.0, 500, 1, (100.0, 100.0)),
    "t127adj": Workload("t127adj", 3, 127, 192, 384, 4, 4, 300.0, 96, 1, (100.0, 100.0)),
    "t511": Workload("t511", 4, 511, 768, 1536, 4, 5, 75.0, 400, 1, (100.0, 100.0)),
}


def ncoef(T: int) -> int:
    return (T + 1) * (T + 2) // 2


def order_offset(T: int, m: int) -> int:
    return m * (2 * T + 3 - m) // 2


def degree_order_arrays(T: int):
    """(n, m) of every packed coefficient, as int arrays of length ncoef."""
    n_list, m_list = [], []
    for m in range(T + 1):
        for n in range(m, T + 1):
            n_list.append(n)
            m_list.append(m)
    return np.array(n_list, dtype=np.int64), np.array(m_list, dtype=np.int64)


def rng(index: int, purpose: int) -> np.random.Generator:
    return np.random.default_rng([SEED_BASE, index, purpose])


def _random_spectrum(T: int, g: np.random.Generator) -> np.ndarray:
    n, m = degree_order_arrays(T)
    re = g.standard_normal(n.size)
    im = g.standard_normal(n.size)
    c = (re + 1j * im)
    c[m == 0] = re[m == 0]
    amp = np.zeros(n.size)
    amp[n >= 1] = n[n >= 1].astype(np.float64) ** -1.5
    return c * amp


def rms_wind_of(T: int, zeta: np.ndarray, div: np.ndarray, radius: float = RADIUS) -> float:
    """Area-weighted rms of |V| implied by a vorticity/divergence spectrum.

    By Parseval on the sphere, with psi = -a^2 zeta_n / (n(n+1)) and the same for
    chi, the mean of |V|^2 over the sphere is (a^2/2) sum_{n>=1} w_m
    (|zeta_n^m|^2 + |div_n^m|^2) / (n(n+1)), where w_m = 1 for m = 0 and 2 for
    m > 0 (the negative orders).  This is the input recipe's scaling rule.
    """
    n, m = degree_order_arrays(T)
    w = np.where(m == 0, 1.0, 2.0)
    sel = n >= 1
    nn1 = (n * (n + 1)).astype(np.float64)
    s = np.sum(w[sel] * (np.abs(zeta[sel]) ** 2 + np.abs(div[sel]) ** 2) / nn1[sel])
    return float(np.sqrt(0.5 * radius ** 2 * s))


def vorticity_divergence(wl: Workload):
    """Seeded (zeta, div) spectra, complex128 of length ncoef, rms wind = wl.rms_wind."""
    zeta = _random_spectrum(wl.T, rng(wl.index, PURPOSE_ZETA))
    div = wl.div_scale * _random_spectrum(wl.T, rng(wl.index, PURPOSE_DIV))
    scale = wl.rms_wind / rms_wind_of(wl.T, zeta, div)
    return zeta * scale, div * scale


def bump_parameters(wl: Workload):
    """Bump centres (mu0 = sin latitude, lambda0) uniform on the sphere, amplitudes in m."""
    g = rng(wl.index, PURPOSE_BUMPS)
    mu0 = g.uniform(-1.0, 1.0, wl.nbumps)
    lam0 = g.uniform(0.0, 2.0 * np.pi, wl.nbumps)
    lo, hi = wl.bump_amp
    amp = g.uniform(lo, hi, wl.nbumps) if hi > lo else np.full(wl.nbumps, lo)
    return mu0, lam0, amp


def bump_height(wl: Workload, mu: np.ndarray, lam: np.ndarray, radius: float = RADIUS) -> np.ndarray:
    """h - H on the points (mu[j], lam[k]) -> array (len(mu), len(lam)), in m.

    Sum of A_b exp(-(d_b / R)^2), d_b the great-circle distance to centre b.
    """
    mu = np.asarray(mu, dtype=np.float64)[:, None]
    lam = np.asarray(lam, dtype=np.float64)[None, :]
    out = np.zeros((mu.shape[0], lam.shape[1]))
    for mu0, lam0, a in zip(*bump_parameters(wl)):
        cosd = mu * mu0 + np.sqrt(1.0 - mu * mu) * np.sqrt(1.0 - mu0 * mu0) * np.cos(lam - lam0)
        d = radius * np.arccos(np.clip(cosd, -1.0, 1.0))
        out += a * np.exp(-(d / wl.bump_radius) ** 2)
    return out


def direction(wl: Workload, which: int, purpose: int = PURPOSE_DIRECTIONS):
    """A seeded perturbation (zeta, div, h-bump-free) with the same spectral law.

    Returns (dphi, dzeta, ddiv) spectra; dphi follows the same n^-1.5 law
    scaled so that its rms matches a 100 m height perturbation's order of
    magnitude in geopotential.  Used for finite-difference directions and for
    target perturbations.
    """
    g = rng(wl.index, purpose * 1000 + which)
    dz = _random_spectrum(wl.T, g)
    dd = wl.div_scale * _random_spectrum(wl.T, g)
    dp = _random_spectrum(wl.T, g)
    s = wl.rms_wind / rms_wind_of(wl.T, dz, dd)
    n, m = degree_order_arrays(wl.T)
    w = np.where(m == 0, 1.0, 2.0)
    rms_p = np.sqrt(0.5 * np.sum(w * np.abs(dp) ** 2))
    dp = dp * (GRAVITY * 100.0 / rms_p)
    return dp, dz * s, dd * s
