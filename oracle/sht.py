"""Spherical-harmonic transform on a Gauss grid, as plain definitions (FP64).

Test infrastructure only (see the package docstring).

The paper's SWEET variant evaluates its explicit tendencies by transforming
the spectral state to the grid and back, a longitude FFT plus a Legendre
transform on Gauss latitudes (Sec. 3.2).  The paper defers the conventions to
SHTns and to Hack & Jakob (1992); this oracle fixes them as follows (the CUDA
path uses the same discrete operators, so parity is rounding only):

* Grid: mu_j = sin(latitude_j) are the roots of the Legendre polynomial P_J,
  ordered north to south (mu descending); w_j the Gauss weights (sum 2);
  longitudes lambda_k = 2 pi k / L.
* Basis: normalised associated Legendre functions with
  int_{-1}^{1} Pbar_n^m(mu)^2 dmu = 1 and no Condon-Shortley phase, and
  H_n^m = (1 - mu^2) dPbar_n^m / dmu.
* Fourier: f(lambda) = sum_{m=-T}^{T} f_m e^{i m lambda} with
  f_{-m} = conj(f_m), i.e. f_0 + 2 Re sum_{m>=1} f_m e^{i m lambda}, and
  f_m = (1/L) sum_k f(lambda_k) e^{-i m lambda_k}.
* Synthesis f_m(mu_j) = sum_{n=m}^{T} f_n^m Pbar_n^m(mu_j);
  analysis f_n^m = sum_j w_j f_m(mu_j) Pbar_n^m(mu_j).
"""
from __future__ import annotations

import numpy as np

from swe_inputs import ncoef, order_offset


def _legendre_pair(J: int, x: np.ndarray):
    """(P_J(x), P_{J-1}(x)) by the three-term recurrence k P_k = (2k-1) x P_{k-1} - (k-1) P_{k-2}."""
    p0 = np.ones_like(x)
    p1 = x.copy()
    if J == 0:
        return p0, np.zeros_like(x)
    for k in range(2, J + 1):
        p0, p1 = p1, ((2 * k - 1) * x * p1 - (k - 1) * p0) / k
    return p1, p0


def gauss_grid(J: int):
    """Gauss-Legendre nodes mu (descending, north to south) and weights w.

    The nodes are the roots of P_J, found by Newton's method in the colatitude
    theta (mu = cos theta) from the classical first guess
    theta = pi (j - 1/4) / (J + 1/2); the weights are
    w = 2 / ((1 - mu^2) P_J'(mu)^2) = 2 (1 - mu^2) / (J P_{J-1}(mu))^2 at a root,
    with 1 - mu^2 = sin^2 theta taken from theta so that polar weights keep
    full relative precision.  Nodes are computed for the northern half and
    mirrored (the roots are symmetric).
    """
    h = (J + 1) // 2
    theta = np.pi * (np.arange(1, h + 1) - 0.25) / (J + 0.5)
    for _ in range(30):
        x = np.cos(theta)
        pj, pj1 = _legendre_pair(J, x)
        # dP_J/dtheta = -sin(theta) P_J'(x) = -J (P_{J-1} - x P_J) / sin(theta)
        dp = -J * (pj1 - x * pj) / np.sin(theta)
        step = pj / dp
        theta = theta - step
        if np.max(np.abs(step)) < 1e-16:
            break
    x = np.cos(theta)
    pj, pj1 = _legendre_pair(J, x)
    s2 = np.sin(theta) ** 2
    # (1 - x^2) P_J'(x) = J (P_{J-1} - x P_J); keeping the x P_J term (zero at an
    # exact root) makes the weight insensitive to the last bits of the root,
    # whereas P_{J-1} alone is small and steep near the poles.
    w = 2.0 * s2 / (J * (pj1 - x * pj)) ** 2
    if J % 2 == 1:
        x[-1] = 0.0
    mu = np.concatenate([x, -x[: J // 2][::-1]])
    wt = np.concatenate([w, w[: J // 2][::-1]])
    return mu, wt


def epsilon(n, m):
    """eps_n^m = sqrt((n^2 - m^2) / (4 n^2 - 1)), the recurrence coefficient."""
    n = np.asarray(n, dtype=np.float64)
    return np.sqrt((n * n - m * m) / (4.0 * n * n - 1.0))


def legendre_pbar(T: int, mu: np.ndarray, nmax_extra: int = 1, orders=None):
    """Pbar[m] = array (len(mu), T + 1 + nmax_extra - m) of Pbar_n^m(mu), n = m..T+nmax_extra.

    Pbar_0^0 = 1/sqrt(2); Pbar_m^m = sqrt((2m+1)/(2m)) sqrt(1-mu^2) Pbar_{m-1}^{m-1};
    Pbar_n^m = (mu Pbar_{n-1}^m - eps_{n-1}^m Pbar_{n-2}^m) / eps_n^m.
    With ``orders`` given, only those orders' columns are formed (the others
    are None); the sectoral start still runs through every m.
    """
    mu = np.asarray(mu, dtype=np.float64)
    s = np.sqrt((1.0 - mu) * (1.0 + mu))          # sqrt(1 - mu^2) without cancellation near the poles
    nmax = T + nmax_extra
    out = []
    pmm = np.full(mu.shape, 1.0 / np.sqrt(2.0))
    for m in range(T + 1):
        if m > 0:
            pmm = np.sqrt((2.0 * m + 1.0) / (2.0 * m)) * s * pmm
        if orders is not None and m not in orders:
            out.append(None)
            continue
        col = np.zeros(mu.shape + (nmax + 1 - m,))
        col[..., 0] = pmm
        for n in range(m + 1, nmax + 1):
            prev2 = col[..., n - m - 2] if n - 2 >= m else 0.0
            col[..., n - m] = (mu * col[..., n - m - 1] - epsilon(n - 1, m) * prev2) / epsilon(n, m)
        out.append(col)
    return out


def legendre_h(T: int, pbar):
    """H[m] = array (J, T + 1 - m) of H_n^m = (1-mu^2) dPbar_n^m/dmu, n = m..T.

    Uses the identity H_n^m = -n eps_{n+1}^m Pbar_{n+1}^m + (n+1) eps_n^m Pbar_{n-1}^m,
    so pbar must reach degree T + 1.
    """
    out = []
    for m in range(T + 1):
        P = pbar[m]
        J = P.shape[0]
        H = np.zeros((J, T + 1 - m))
        for n in range(m, T + 1):
            h = -n * epsilon(n + 1, m) * P[:, n + 1 - m]
            if n - 1 >= m:
                h = h + (n + 1) * epsilon(n, m) * P[:, n - 1 - m]
            H[:, n - m] = h
        out.append(H)
    return out


class Grid:
    """Gauss grid + Legendre tables for truncation T on J x L points."""

    def __init__(self, T: int, J: int, L: int):
        self.T, self.J, self.L = T, J, L
        self.ncoef = ncoef(T)
        self.mu, self.w = gauss_grid(J)
        self.lam = 2.0 * np.pi * np.arange(L) / L
        self.pbar = legendre_pbar(T, self.mu)
        self.h = legendre_h(T, self.pbar)
        # naive DFT tables, angles reduced modulo L before cos/sin
        k = np.arange(L)
        m = np.arange(T + 1)
        ang = 2.0 * np.pi * ((m[:, None] * k[None, :]) % L) / L
        self.cos = np.cos(ang)      # (T+1, L)
        self.sin = np.sin(ang)

    # ---- packing -------------------------------------------------------
    def block(self, m: int) -> slice:
        o = order_offset(self.T, m)
        return slice(o, o + self.T + 1 - m)

    # ---- longitude (naive DFT) -----------------------------------------
    def fourier_to_grid(self, F: np.ndarray) -> np.ndarray:
        """F (..., T+1) complex Fourier coefficients m = 0..T -> real values (..., L)."""
        F = np.asarray(F)
        wts = np.full(self.T + 1, 2.0)
        wts[0] = 1.0
        re = (F.real * wts) @ self.cos
        im = (F.imag * wts) @ self.sin
        return re - im

    def grid_to_fourier(self, f: np.ndarray) -> np.ndarray:
        """Real values (..., L) -> Fourier coefficients (..., T+1), f_m = (1/L) sum_k f_k e^{-i m lambda_k}."""
        f = np.asarray(f, dtype=np.float64)
        return (f @ self.cos.T - 1j * (f @ self.sin.T)) / self.L

    # ---- Legendre (direct sums) ----------------------------------------
    def synth(self, coef: np.ndarray, table: str = "p") -> np.ndarray:
        """Spectral coef (ncoef,) -> Fourier coefficients on latitudes (J, T+1).

        table "p": sum_n c_n Pbar_n^m(mu_j);  table "h": sum_n c_n H_n^m(mu_j).
        """
        out = np.zeros((self.J, self.T + 1), dtype=np.complex128)
        for m in range(self.T + 1):
            tab = self.pbar[m][:, : self.T + 1 - m] if table == "p" else self.h[m]
            out[:, m] = tab @ coef[self.block(m)]
        return out

    def analyse(self, F: np.ndarray, weights: np.ndarray, table: str = "p") -> np.ndarray:
        """Fourier (J, T+1) -> spectral (ncoef,): c_n^m = sum_j weights_j F_m(mu_j) T_n^m(mu_j)."""
        out = np.zeros(self.ncoef, dtype=np.complex128)
        for m in range(self.T + 1):
            tab = self.pbar[m][:, : self.T + 1 - m] if table == "p" else self.h[m]
            out[self.block(m)] = tab.T @ (weights * F[:, m])
        return out

    # ---- full scalar transforms ----------------------------------------
    def spec_to_grid(self, coef: np.ndarray) -> np.ndarray:
        return self.fourier_to_grid(self.synth(coef))

    def grid_to_spec(self, f: np.ndarray) -> np.ndarray:
        return self.analyse(self.grid_to_fourier(f), self.w)
