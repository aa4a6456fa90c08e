"""Rotating shallow-water operators in vorticity-divergence form (FP64 oracle).

Test infrastructure only (see the package docstring).

State u = (Phi', zeta, div): spherical-harmonic coefficients (the paper's
U-hat, Sec. 3.2, with the divergence written div instead of rho), array of
shape (3, ncoef) complex.  Eq. (4) splits the right-hand side into

* L_g(u) = (-Phibar div, -grad Phi): in spectral space, with
  lap Y_n^m = -n(n+1)/a^2 Y_n^m, L_g(Phi') = -Phibar div,
  L_g(zeta) = 0, L_g(div) = +lambda_n Phi', lambda_n = n(n+1)/a^2;
* T_E = L_c + N_a + N_r, evaluated on the grid.  Reading of the garbled N_r
  row: N_a + N_r in the Phi equation is taken as -div(Phi' V) (flux form,
  which conserves mass), i.e. N_r = -Phi' div V.  In vorticity-divergence
  form, with eta = zeta + f and f = 2 Omega mu:
      d zeta/dt = -div(eta V),  d div/dt = curl(eta V) - lap E,
      d Phi'/dt = -div(Phi' V),  E = |V|^2 / 2.

The spectral forms below are the Galerkin projections with Gauss quadrature,
the divergence and curl moved onto the basis by integration by parts
(H_n^m = (1 - mu^2) dPbar_n^m/dmu), following Hack & Jakob (1992) cited in
Sec. 3.2.  U = u cos(lat), V = v cos(lat).
"""
from __future__ import annotations

import numpy as np

from swe_inputs import degree_order_arrays

PHI, ZETA, DIV = 0, 1, 2


class Physics:
    def __init__(self, radius: float, omega: float, gravity: float, mean_depth: float):
        self.a = radius
        self.omega = omega
        self.g = gravity
        self.H = mean_depth
        self.phibar = gravity * mean_depth


class SWE:
    """The SWEET shallow-water problem on a Gauss grid (oracle)."""

    def __init__(self, grid, phys: Physics):
        self.grid = grid
        self.phys = phys
        n, m = degree_order_arrays(grid.T)
        self.n = n
        self.m = m
        self.lam = n * (n + 1) / phys.a ** 2          # -eigenvalue of the Laplacian
        inv = np.zeros(n.size)
        inv[n >= 1] = 1.0 / (n[n >= 1] * (n[n >= 1] + 1.0))
        self.inv_nn1 = inv
        # i m factor per packed coefficient
        self.im = 1j * m.astype(np.float64)
        # per-latitude weights
        mu = grid.mu
        self.w = grid.w
        self.wt = grid.w / ((1.0 - mu) * (1.0 + mu))  # w_j / (1 - mu_j^2)
        self.n_explicit = 0                           # counters (Table 1)
        self.n_solve = 0

    # ---- spectral helpers -----------------------------------------------
    def streamfunction(self, zeta):
        """psi_n^m = -a^2 zeta_n^m / (n(n+1)) (0 at n = 0); the same maps div -> chi."""
        return -self.phys.a ** 2 * self.inv_nn1 * zeta

    def wind_fourier(self, zeta, div):
        """(U_m, V_m) on latitudes, (J, T+1) each:
        U_m = (1/a) sum_n [i m chi_n Pbar - psi_n H],  V_m = (1/a) sum_n [i m psi_n Pbar + chi_n H]."""
        g, a = self.grid, self.phys.a
        psi = self.streamfunction(zeta)
        chi = self.streamfunction(div)
        U = (g.synth(self.im * chi, "p") - g.synth(psi, "h")) / a
        V = (g.synth(self.im * psi, "p") + g.synth(chi, "h")) / a
        return U, V

    # ---- L_g and its solve (Eq. (4), Eq. (8)) --------------------------
    def linear(self, u):
        out = np.zeros_like(u)
        out[PHI] = -self.phys.phibar * u[DIV]
        out[ZETA] = 0.0
        out[DIV] = self.lam * u[PHI]
        return out

    def solve(self, alpha: float, beta):
        """u with u - alpha L_g(u) = beta, per mode by dense 3x3 Gaussian elimination."""
        self.n_solve += 1
        nc = beta.shape[1]
        A = np.zeros((nc, 3, 3))
        A[:, 0, 0] = 1.0
        A[:, 1, 1] = 1.0
        A[:, 2, 2] = 1.0
        A[:, PHI, DIV] += alpha * self.phys.phibar     # -alpha * (-Phibar)
        A[:, DIV, PHI] += -alpha * self.lam            # -alpha * (+lambda_n)
        rhs = np.stack([beta.real.T, beta.imag.T], axis=-1)   # (nc, 3, 2)
        x = np.linalg.solve(A, rhs)
        return (x[..., 0] + 1j * x[..., 1]).T.copy()

    # ---- T_E = L_c + N_a + N_r ------------------------------------------
    def grid_fields(self, u):
        """Grid values (J, L) of Phi', zeta, U, V for state u."""
        g = self.grid
        U, V = self.wind_fourier(u[ZETA], u[DIV])
        return (g.fourier_to_grid(g.synth(u[PHI])), g.fourier_to_grid(g.synth(u[ZETA])),
                g.fourier_to_grid(U), g.fourier_to_grid(V))

    def explicit(self, u):
        """T_E(u) (Eq. (4): L_c + N_a + N_r), returned in spectral space."""
        self.n_explicit += 1
        g, a, om = self.grid, self.phys.a, self.phys.omega
        phi, zeta, U, V = self.grid_fields(u)
        mu = g.mu[:, None]
        eta = zeta + 2.0 * om * mu
        A = eta * U
        B = eta * V
        C = phi * U
        D = phi * V
        E = (U * U + V * V) / (2.0 * (1.0 - mu) * (1.0 + mu))
        Am, Bm, Cm, Dm, Em = (g.grid_to_fourier(x) for x in (A, B, C, D, E))
        out = np.zeros_like(u)
        # zeta: -div(eta V)_n^m = -(1/a) sum_j wt_j [i m A_m Pbar - B_m H]
        out[ZETA] = -(self.im * g.analyse(Am, self.wt, "p") - g.analyse(Bm, self.wt, "h")) / a
        # div: curl(eta V)_n^m - (lap E)_n^m
        out[DIV] = ((self.im * g.analyse(Bm, self.wt, "p") + g.analyse(Am, self.wt, "h")) / a
                    + self.lam * g.analyse(Em, self.w, "p"))
        # Phi': -div(Phi' V)
        out[PHI] = -(self.im * g.analyse(Cm, self.wt, "p") - g.analyse(Dm, self.wt, "h")) / a
        return out

    def rhs(self, u):
        return self.linear(u) + self.explicit(u)

    # ---- diagnostics ------------------------------------------------------
    def mode_weights(self):
        """Parseval weights: 1 for m = 0, 2 for m > 0 (the negative orders)."""
        return np.where(self.m == 0, 1.0, 2.0)

    def field_norms(self, r):
        """Per-field Parseval-weighted L2 norm sqrt(sum_modes w |r|^2), shape (3,)."""
        w = self.mode_weights()
        return np.sqrt(np.sum(w[None, :] * np.abs(r) ** 2, axis=1))

    def height_grid(self, u):
        """h on the grid: H + Phi' / g."""
        g = self.grid
        return self.phys.H + g.fourier_to_grid(g.synth(u[PHI])) / self.phys.g


def initial_state(wl, swe: SWE):
    """Seeded initial state of a workload: (Phi', zeta, div) spectra.

    zeta and div come from the seeded spectrum law; Phi' = g (h - H) with the
    seeded Gaussian bumps evaluated on this grid and analysed onto degree <= T.
    """
    import swe_inputs
    zeta, div = swe_inputs.vorticity_divergence(wl)
    g = swe.grid
    hb = swe_inputs.bump_height(wl, g.mu, g.lam, radius=swe.phys.a)
    u = np.zeros((3, g.ncoef), dtype=np.complex128)
    u[PHI] = g.grid_to_spec(swe.phys.g * hb)
    u[ZETA] = zeta
    u[DIV] = div
    return u


def default_physics():
    import swe_inputs
    return Physics(swe_inputs.RADIUS, swe_inputs.OMEGA, swe_inputs.GRAVITY, swe_inputs.MEAN_DEPTH)
