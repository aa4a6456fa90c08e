"""Discrete adjoint of the dSDC shallow-water step (FP64 oracle).

Test infrastructure only (see the package docstring).

The adjoint is the exact transpose of the discrete forward map with respect
to the real degrees of freedom of the stored arrays (real and imaginary parts
of every complex coefficient, the Euclidean inner product
<a, b> = Re sum conj(a) b).  Gradients are returned in the same complex
layout: real part = dL/dRe, imaginary part = dL/dIm.

Transposes of the building blocks (each follows from writing the complex map
as a real 2x2-block map):
* multiplication by a complex constant z  ->  multiplication by conj(z)
  (so the i m factor of a longitude derivative becomes -i m);
* a real Legendre matrix applied to complex coefficients -> its transpose;
* f = F_0 + 2 Re sum_{m>0} F_m e^{i m lambda}  ->  Fbar_m = w_m sum_k f_k e^{-i m lambda_k}
  with w_0 = 1, w_m = 2;
* F_m = (1/L) sum_k f_k e^{-i m lambda_k}  ->  fbar_k = (1/L) sum_m Re(Fbar_m e^{i m lambda_k});
* the grid products A = eta U, ..., E = (U^2 + V^2) / (2 (1 - mu^2)) -> their
  Jacobians transposed pointwise (they need the base state's grid fields).

The step adjoint reverses Algorithm 2 with the node update Eq. (7): it first
re-runs the forward step to record every node iterate ("retape"), then walks
the sweeps backwards.  The loss of the differentiation workload is
0.5 sum over the grid of (h(T) - h_target)^2 with h = H + Phi'/g.
"""
from __future__ import annotations

import numpy as np

from .sdc import Collocation, qdelta
from .swe import DIV, PHI, ZETA


# ---------------------------------------------------------------------------
# transposes of the transform building blocks
# ---------------------------------------------------------------------------
def fourier_to_grid_T(g, r):
    """Transpose of Grid.fourier_to_grid: real grid (..., L) -> Fourier adjoint (..., T+1)."""
    w = np.full(g.T + 1, 2.0)
    w[0] = 1.0
    return w * (r @ g.cos.T - 1j * (r @ g.sin.T))


def grid_to_fourier_T(g, Fbar):
    """Transpose of Grid.grid_to_fourier: Fourier adjoint (..., T+1) -> real grid (..., L)."""
    return (Fbar.real @ g.cos - Fbar.imag @ g.sin) / g.L


def synth_T(g, Xbar, table="p"):
    """Transpose of Grid.synth: Fourier adjoint on latitudes (J, T+1) -> spectral (ncoef,)."""
    out = np.zeros(g.ncoef, dtype=np.complex128)
    for m in range(g.T + 1):
        tab = g.pbar[m][:, : g.T + 1 - m] if table == "p" else g.h[m]
        out[g.block(m)] = tab.T @ Xbar[:, m]
    return out


def analyse_T(g, cbar, weights, table="p"):
    """Transpose of Grid.analyse: spectral adjoint (ncoef,) -> Fourier adjoint (J, T+1)."""
    out = np.zeros((g.J, g.T + 1), dtype=np.complex128)
    for m in range(g.T + 1):
        tab = g.pbar[m][:, : g.T + 1 - m] if table == "p" else g.h[m]
        out[:, m] = weights * (tab @ cbar[g.block(m)])
    return out


# ---------------------------------------------------------------------------
# adjoint of T_E
# ---------------------------------------------------------------------------
def explicit_vjp(swe, u, abar):
    """J_E(u)^T abar: the transpose of the Jacobian of T_E (SWE.explicit) at base u."""
    g, a, om = swe.grid, swe.phys.a, swe.phys.omega
    im = swe.im
    cim = np.conj(im)
    mu = g.mu[:, None]
    c2 = (1.0 - mu) * (1.0 + mu)
    # base grid fields
    phi, zeta, U, V = swe.grid_fields(u)
    eta = zeta + 2.0 * om * mu
    # analysis transposes
    Abar_m = (analyse_T(g, -cim * abar[ZETA] / a, swe.wt, "p")
              + analyse_T(g, abar[DIV] / a, swe.wt, "h"))
    Bbar_m = (analyse_T(g, abar[ZETA] / a, swe.wt, "h")
              + analyse_T(g, cim * abar[DIV] / a, swe.wt, "p"))
    Cbar_m = analyse_T(g, -cim * abar[PHI] / a, swe.wt, "p")
    Dbar_m = analyse_T(g, abar[PHI] / a, swe.wt, "h")
    Ebar_m = analyse_T(g, swe.lam * abar[DIV], swe.w, "p")
    Ab, Bb, Cb, Db, Eb = (grid_to_fourier_T(g, x) for x in (Abar_m, Bbar_m, Cbar_m, Dbar_m, Ebar_m))
    # pointwise product transposes
    zeta_b = Ab * U + Bb * V
    phi_b = Cb * U + Db * V
    U_b = Ab * eta + Cb * phi + Eb * U / c2
    V_b = Bb * eta + Db * phi + Eb * V / c2
    # synthesis transposes
    out = np.zeros_like(u)
    out[PHI] = synth_T(g, fourier_to_grid_T(g, phi_b), "p")
    out[ZETA] = synth_T(g, fourier_to_grid_T(g, zeta_b), "p")
    Um_b = fourier_to_grid_T(g, U_b) / a
    Vm_b = fourier_to_grid_T(g, V_b) / a
    # U = (1/a)[synth(i m chi, P) - synth(psi, H)],  V = (1/a)[synth(i m psi, P) + synth(chi, H)]
    chi_b = cim * synth_T(g, Um_b, "p") + synth_T(g, Vm_b, "h")
    psi_b = -synth_T(g, Um_b, "h") + cim * synth_T(g, Vm_b, "p")
    s = -a ** 2 * swe.inv_nn1
    out[ZETA] += s * psi_b
    out[DIV] += s * chi_b
    return out


def linear_T(swe, x):
    """L_g^T: (L^T x)_Phi = lambda_n x_div, (L^T x)_div = -Phibar x_Phi, (L^T x)_zeta = 0."""
    out = np.zeros_like(x)
    out[PHI] = swe.lam * x[DIV]
    out[DIV] = -swe.phys.phibar * x[PHI]
    return out


def solve_T(swe, alpha, b):
    """(I - alpha L_g)^{-T} b per mode, dense 3x3 elimination of the transposed matrix."""
    nc = b.shape[1]
    A = np.zeros((nc, 3, 3))
    A[:, 0, 0] = A[:, 1, 1] = A[:, 2, 2] = 1.0
    A[:, PHI, DIV] += alpha * swe.phys.phibar
    A[:, DIV, PHI] += -alpha * swe.lam
    At = np.transpose(A, (0, 2, 1))
    rhs = np.stack([b.real.T, b.imag.T], axis=-1)
    x = np.linalg.solve(At, rhs)
    return (x[..., 0] + 1j * x[..., 1]).T.copy()


# ---------------------------------------------------------------------------
# adjoint of one dSDC step (Algorithm 2, Eq. (7))
# ---------------------------------------------------------------------------
def dsdc_step_vjp(u_n, ubar_next, f_E, f_E_vjp, f_I, f_I_T, solve, solve_T_, coll: Collocation, K: int,
                  dt: float):
    """ubar_n = (d u_{n+1} / d u_n)^T ubar_next for one dSDC step, generic problem."""
    M, Q = coll.M, coll.Q

    def alpha(k, m):                    # sweep k (1-based)
        return dt * qdelta(coll.tau, k, coll.rule)[m]

    # retape: node iterates u[k][j], k = 0..K-1
    E0 = f_E(u_n)
    u = [[u_n] * M]
    E = [[E0] * M]
    for k in range(K - 1):
        new = []
        for m in range(M):
            quad = sum(Q[m, j] * (f_I(u[k][j]) + E[k][j]) for j in range(M))
            beta = u_n + dt * quad - alpha(k + 1, m) * f_I(u[k][m])
            new.append(solve(alpha(k + 1, m), beta))
        u.append(new)
        E.append([f_E(x) for x in new])

    zero = np.zeros_like(u_n)
    ubar_n = zero.copy()
    # last sweep K: node M only
    s = solve_T_(alpha(K, M - 1), ubar_next)
    ubar_n += s
    ubar_u = [zero.copy() for _ in range(M)]
    Ebar = [zero.copy() for _ in range(M)]
    for j in range(M):
        ubar_u[j] += dt * Q[M - 1, j] * f_I_T(s)
        Ebar[j] += dt * Q[M - 1, j] * s
    ubar_u[M - 1] += -alpha(K, M - 1) * f_I_T(s)
    # sweeps K-1 .. 1 (k + 1 = sweep index), from iterate k + 1 back to k
    for k in range(K - 2, -1, -1):
        for j in range(M):
            ubar_u[j] = ubar_u[j] + f_E_vjp(u[k + 1][j], Ebar[j])
        nub = [zero.copy() for _ in range(M)]
        nEb = [zero.copy() for _ in range(M)]
        for m in range(M):
            s = solve_T_(alpha(k + 1, m), ubar_u[m])
            ubar_n += s
            for j in range(M):
                nub[j] += dt * Q[m, j] * f_I_T(s)
                nEb[j] += dt * Q[m, j] * s
            nub[m] += -alpha(k + 1, m) * f_I_T(s)
        ubar_u, Ebar = nub, nEb
    # iterate 0: every u_j^0 is u_n and every E_j^0 is T_E(u_n)
    ubar_n += sum(ubar_u)
    ubar_n += f_E_vjp(u_n, sum(Ebar))
    return ubar_n


def swe_step_vjp(swe, u_n, ubar_next, coll: Collocation, K: int, dt: float):
    return dsdc_step_vjp(u_n, ubar_next, swe.explicit, lambda x, a: explicit_vjp(swe, x, a), swe.linear,
                         lambda x: linear_T(swe, x), swe.solve, lambda al, b: solve_T(swe, al, b), coll, K, dt)


# ---------------------------------------------------------------------------
# loss of the differentiation workload and its gradient
# ---------------------------------------------------------------------------
def height_loss(swe, u, h_target):
    """0.5 sum over the grid of (h - h_target)^2, h = H + Phi'/g."""
    r = swe.height_grid(u) - h_target
    return 0.5 * float(np.sum(r * r))


def height_loss_seed(swe, u, h_target):
    """dL/du for the height loss (only the Phi' field is non-zero)."""
    g = swe.grid
    r = swe.height_grid(u) - h_target
    out = np.zeros_like(u)
    out[PHI] = synth_T(g, fourier_to_grid_T(g, r / swe.phys.g), "p")
    return out


def loss_and_gradient(swe, u0, coll: Collocation, K: int, dt: float, nsteps: int, h_target):
    """Loss after nsteps dSDC steps and its gradient w.r.t. u0 (all states stored)."""
    from .sdc import swe_step
    states = [u0]
    for _ in range(nsteps):
        states.append(swe_step(swe, states[-1], coll, K, dt))
    loss = height_loss(swe, states[-1], h_target)
    ubar = height_loss_seed(swe, states[-1], h_target)
    for n in range(nsteps - 1, -1, -1):
        ubar = swe_step_vjp(swe, states[n], ubar, coll, K, dt)
    return loss, ubar
