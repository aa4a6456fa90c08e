"""The paper's two reference integrators for the same problem (FP64 oracle).

Test infrastructure only (see the package docstring).

* Serial IMEX SDC, Algorithm 1 with the node update Eq. (6): sweep k and node
  m (sequential over m)
    u_m^{k+1} = u_n + dt sum_j Q[m,j] (f_I(u_j^k) + f_E(u_j^k))
              + dt sum_{j<m} dtau_{j+1} (f_E(u_j^{k+1}) - f_E(u_j^k))
              + dt sum_{j<=m} dtau_j (f_I(u_j^{k+1}) - f_I(u_j^k)),
  dtau_1 = tau_1, dtau_j = tau_j - tau_{j-1} (1-based), u_m^0 = u_n.  The j = m
  implicit term makes each node update a solve u - dt dtau_m f_I(u) = beta
  (Eq. (8)).  All K sweeps update all M nodes; u_{n+1} = u_M^K.  Option
  implicit="lu": the implicit weights dtau_j (j <= m) are replaced by the
  lower-triangular U^T of the factorisation Q^T = L U with L unit lower
  triangular (the lower-triangular q^Delta Sec. 4.2 mentions first); the
  explicit weights stay dtau_{j+1}.
* IMEX-o2 (Sec. 3.2): second-order Strang splitting with Crank-Nicolson for
  L_g and Heun's method for L_c + N_a + N_r = T_E.  The paper does not say
  which part takes the half steps; here the implicit part does (one explicit
  full step in the middle, two evaluations of T_E per step):
    a = CN(dt/2) u_n,   b = a + dt f_E(a),
    c = a + dt/2 (f_E(a) + f_E(b)),   u_{n+1} = CN(dt/2) c,
  with CN(h) u = (I - h/2 f_I)^{-1} (I + h/2 f_I) u.
"""
from __future__ import annotations

import numpy as np

from .sdc import Collocation


def lu_weights(Q):
    """U^T of Q^T = L U, L unit lower triangular (Doolittle, no pivoting)."""
    A = np.array(Q, dtype=float).T
    M = A.shape[0]
    L, U = np.eye(M), np.zeros((M, M))
    for i in range(M):
        for k in range(i, M):
            U[i, k] = A[i, k] - L[i, :i] @ U[:i, k]
        for k in range(i + 1, M):
            L[k, i] = (A[k, i] - L[k, :i] @ U[:i, i]) / U[i, i]
    return U.T


def imex_sdc_step(u_n, f_E, f_I, solve, coll: Collocation, K: int, dt: float, implicit: str = "euler"):
    """One serial IMEX SDC step t_n -> t_n + dt (Algorithm 1, Eq. (6))."""
    M, Q, tau = coll.M, coll.Q, coll.tau
    dtau = [tau[0]] + [tau[j] - tau[j - 1] for j in range(1, M)]
    if implicit == "euler":
        QI = np.array([[dtau[j] if j <= m else 0.0 for j in range(M)] for m in range(M)])
    elif implicit == "lu":
        QI = lu_weights(Q)
    else:
        raise ValueError(f"unknown implicit weights {implicit!r}")
    E0, I0 = f_E(u_n), f_I(u_n)
    u, E, I = [u_n] * M, [E0] * M, [I0] * M
    for _ in range(K):
        un, En, In = [], [], []
        for m in range(M):
            beta = u_n + dt * sum(Q[m, j] * (I[j] + E[j]) for j in range(M))
            for j in range(m):
                beta = beta + dt * dtau[j + 1] * (En[j] - E[j])
                beta = beta + dt * QI[m, j] * (In[j] - I[j])
            beta = beta - dt * QI[m, m] * I[m]         # the j = m term moves to the solve
            x = solve(dt * QI[m, m], beta)
            un.append(x)
            En.append(f_E(x))
            In.append(f_I(x))
        u, E, I = un, En, In
    return u[M - 1]


def imex2_step(u, f_E, f_I, solve, dt: float):
    """One IMEX-o2 step: CN half step on f_I, Heun full step on f_E, CN half step."""
    h = 0.5 * dt

    def cn(x):
        return solve(0.5 * h, x + 0.5 * h * f_I(x))

    a = cn(u)
    ea = f_E(a)
    b = a + dt * ea
    c = a + 0.5 * dt * (ea + f_E(b))
    return cn(c)


def swe_imex_sdc_run(swe, u0, coll: Collocation, K: int, dt: float, nsteps: int, implicit: str = "euler"):
    u = u0
    for _ in range(nsteps):
        u = imex_sdc_step(u, swe.explicit, swe.linear, swe.solve, coll, K, dt, implicit)
    return u


def swe_imex2_run(swe, u0, dt: float, nsteps: int):
    u = u0
    for _ in range(nsteps):
        u = imex2_step(u, swe.explicit, swe.linear, swe.solve, dt)
    return u
