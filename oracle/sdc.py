"""Diagonal IMEX SDC (dSDC) with MIN-SR-FLEX coefficients (FP64 oracle).

Test infrastructure only (see the package docstring).

* Collocation (Sec. 4.1, Sec. 4.2): Radau-right nodes 0 < tau_1 < ... < tau_M = 1,
  the roots of P_M(2 tau - 1) - P_{M-1}(2 tau - 1); Q[m, j] = int_0^{tau_m} l_j(s) ds
  with l_j the Lagrange basis on the nodes.
* MIN-SR-FLEX (Sec. 4.2): q^Delta_{m,m} = tau_m / k at sweep k (k = 1..K).  The
  paper always runs K = M; for sweeps k > M this oracle offers two readings,
  "clamped" q(k) = min(k, M) (default) and "literal" q(k) = k.  Two further
  diagonals from the family the paper points to for other coefficient
  choices (Sec. 4.2, Sec. 6): "min-sr-ns" q^Delta_{m,m} = tau_m / M in every
  sweep, "ie" q^Delta_{m,m} = tau_m in every sweep (each node one implicit
  Euler step from t_n), and "min-sr-s": the positive diagonal D, increasing
  in m, for which I - D^{-1} Q is nilpotent (all eigenvalues of D^{-1} Q
  equal to 1), found as the root of "characteristic polynomial of D^{-1} Q
  = (x - 1)^M" by a general nonlinear solver from D = 2 tau / M.
* Node update, Eq. (7): u_m^{k+1} = u_n + dt sum_j Q[m,j] (f_I(u_j^k) + f_E(u_j^k))
  + dt q^Delta_{m,m} (f_I(u_m^{k+1}) - f_I(u_m^k)), solved as
  u_m^{k+1} - alpha f_I(u_m^{k+1}) = beta (Eq. (8)) with alpha = dt q^Delta_{m,m}.
  (The SWEET form Eq. (10) drops the Q f_I and -q^Delta f_I(u_m^k) terms; its
  fixed point would not be the collocation solution, so the general form
  Eq. (7) is used with f_I = L_g, f_E = T_E.)
* Step, Algorithm 2: u_m^0 = u_n for all m; sweeps k = 0..K-2 update all M
  nodes (the parallel loop) and re-evaluate the tendencies; the last sweep
  updates node M only; u_{n+1} = u_M^K, with no tendency evaluation at the end.
* Residual (not in the paper, which fixes K): before sweep k+1 the collocation
  residual R_m^k = u_n + dt sum_j Q[m,j] F(u_j^k) - u_m^k of every node the
  sweep updates; its norm per field, maximum over those nodes.
"""
from __future__ import annotations

import numpy as np
from numpy.polynomial import legendre as npleg
from numpy.polynomial import polynomial as nppoly


def radau_right_nodes(M: int) -> np.ndarray:
    """Radau IIA abscissae on [0, 1] (ascending, last = 1)."""
    if M == 1:
        return np.array([1.0])
    c = np.zeros(M + 1)
    c[M] = 1.0
    c[M - 1] = -1.0                       # P_M - P_{M-1} as a Legendre series
    x = np.sort(np.real(npleg.legroots(c)))
    x[-1] = 1.0
    return (x + 1.0) / 2.0


def collocation_matrix(tau: np.ndarray) -> np.ndarray:
    """Q[m, j] = int_0^{tau_m} l_j(s) ds, l_j the Lagrange basis polynomial on tau."""
    M = tau.size
    Q = np.zeros((M, M))
    for j in range(M):
        others = np.delete(tau, j)
        lj = nppoly.polyfromroots(others) / np.prod(tau[j] - others)
        Lj = nppoly.polyint(lj)           # antiderivative with Lj(0) = 0
        Q[:, j] = nppoly.polyval(tau, Lj)
    return Q


QDELTA_RULES = ("clamped", "literal", "min-sr-ns", "ie", "min-sr-s")


_MIN_SR_S_CACHE: dict = {}


def min_sr_s(tau: np.ndarray) -> np.ndarray:
    """MIN-SR-S diagonal: eigenvalues of D^{-1} Q all 1 (see the module notes)."""
    key = tuple(np.asarray(tau, dtype=float).tolist())
    if key not in _MIN_SR_S_CACHE:
        _MIN_SR_S_CACHE[key] = _min_sr_s_solve(np.asarray(tau, dtype=float))
    return _MIN_SR_S_CACHE[key].copy()


def _min_sr_s_solve(tau: np.ndarray) -> np.ndarray:
    from scipy.optimize import root
    M = tau.size
    if M == 1:                                        # D^{-1} Q = q_11 / d_1 = 1 / d_1
        return np.ones(1)
    Q = collocation_matrix(tau)
    target = np.poly(np.ones(M))                      # coefficients of (x - 1)^M
    sol = root(lambda d: np.poly(Q / d[:, None])[1:] - target[1:], 2.0 * tau / M, method="hybr",
               options={"xtol": 1e-14})
    d = sol.x
    if not (np.all(d > 0) and np.all(np.diff(d) > 0)):
        raise ValueError("MIN-SR-S: the increasing positive root was not reached")
    return d


def qdelta(tau: np.ndarray, k: int, rule: str = "clamped") -> np.ndarray:
    """Diagonal q^Delta_{m,m} at sweep k (1-based) under the named rule."""
    M = tau.size
    if rule == "clamped":
        return tau / float(min(k, M))
    if rule == "literal":
        return tau / float(k)
    if rule == "min-sr-ns":
        return tau / float(M)
    if rule == "ie":
        return tau.copy()
    if rule == "min-sr-s":
        return min_sr_s(tau)
    raise ValueError(f"unknown q-delta rule {rule!r}")


class Collocation:
    def __init__(self, M: int, rule: str = "clamped"):
        self.M = M
        self.tau = radau_right_nodes(M)
        self.Q = collocation_matrix(self.tau)
        self.rule = rule

    def qdelta(self, k: int) -> np.ndarray:
        return qdelta(self.tau, k, self.rule)


def dsdc_step(u_n, f_E, f_I, solve, coll: Collocation, K: int, dt: float,
              norms=None, residuals=None):
    """One dSDC step t_n -> t_n + dt (Algorithm 2 with Eq. (7)).

    f_E(u), f_I(u): explicit/implicit right-hand sides; solve(alpha, beta)
    returns u with u - alpha f_I(u) = beta.  If ``residuals`` is a list, the
    per-sweep residual norms (``norms(r)``, max over updated nodes) are
    appended to it, one entry per sweep.
    """
    M, Q = coll.M, coll.Q
    E0 = f_E(u_n)
    I0 = f_I(u_n)
    u = [u_n] * M
    E = [E0] * M
    I = [I0] * M

    def update(m, k):
        quad = sum(Q[m, j] * (I[j] + E[j]) for j in range(M))
        coll_rhs = u_n + dt * quad
        alpha = dt * coll.qdelta(k + 1)[m]
        beta = coll_rhs - alpha * I[m]
        return solve(alpha, beta), coll_rhs - u[m]

    for k in range(K - 1):
        results = [update(m, k) for m in range(M)]          # the parallel loop
        if residuals is not None:
            residuals.append(np.max(np.stack([norms(r) for _, r in results]), axis=0))
        u = [x for x, _ in results]
        E = [f_E(x) for x in u]
        I = [f_I(x) for x in u]
    u_last, r_last = update(M - 1, K - 1)                   # last sweep, node M only
    if residuals is not None:
        residuals.append(norms(r_last))
    return u_last


def swe_step(swe, u_n, coll: Collocation, K: int, dt: float, residuals=None):
    """One dSDC step of the shallow-water problem, f_I = L_g, f_E = T_E."""
    return dsdc_step(u_n, swe.explicit, swe.linear, swe.solve, coll, K, dt,
                     norms=swe.field_norms, residuals=residuals)


def swe_run(swe, u0, coll: Collocation, K: int, dt: float, nsteps: int):
    u = u0
    for _ in range(nsteps):
        u = swe_step(swe, u, coll, K, dt)
    return u
