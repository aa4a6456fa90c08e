"""Pins of the oracle's reference integrators (CPU only): serial IMEX SDC
(Algorithm 1, Eq. (6)) and IMEX-o2 (Sec. 3.2).

* The first serial sweep is IMEX Euler stepped across the node intervals
  (forward Euler on f_E, backward Euler on f_I), written out independently.
* Enough serial sweeps reach the collocation solution, computed as one dense
  linear solve of the collocation system.
* K serial sweeps are of order min(K, 2M - 1); IMEX-o2 of order 2: observed
  orders against an independent high-accuracy integration (scipy DOP853).
* IMEX-o2's limits: with f_I = 0 and linear f_E = B one step is Heun's
  polynomial I + dt B + (dt B)^2 / 2; with f_E = 0 and skew-symmetric f_I it
  conserves the norm (Crank-Nicolson is a Cayley transform).
"""
import numpy as np
import pytest
from scipy.integrate import solve_ivp

import swe_inputs as si
from oracle import integrators as oi
from oracle import sdc, sht, swe


def _linear(n, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n))
    A = -0.5 * (A @ A.T) / n - 0.1 * np.eye(n)                      # damped, stiff-ish
    B = 0.3 * rng.standard_normal((n, n)) / np.sqrt(n)
    return A, B


def _solver(A):
    n = A.shape[0]
    return lambda alpha, beta: np.linalg.solve(np.eye(n) - alpha * A, beta)


@pytest.mark.parametrize("M", [2, 3, 4])
def test_first_serial_sweep_is_imex_euler_over_the_nodes(M):
    n = 5
    A, B = _linear(n, M)
    f_I = lambda x: A @ x
    f_E = lambda x: B @ x + 0.1 * np.sin(x)
    solve = _solver(A)
    coll = sdc.Collocation(M)
    u_n = np.linspace(0.5, 1.5, n)
    dt = 0.4
    got = oi.imex_sdc_step(u_n, f_E, f_I, solve, coll, 1, dt)
    x, t_prev = u_n, 0.0
    for tm in coll.tau:
        h = dt * (tm - t_prev)
        x = np.linalg.solve(np.eye(n) - h * A, x + h * f_E(x))
        t_prev = tm
    np.testing.assert_allclose(got, x, rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("implicit", ["euler", "lu"])
@pytest.mark.parametrize("M", [2, 3, 4])
def test_serial_sweeps_converge_to_collocation(M, implicit):
    n = 4
    A, B = _linear(n, 10 + M)
    coll = sdc.Collocation(M)
    u_n = np.array([1.0, -0.5, 0.25, 2.0])
    dt = 0.2
    # collocation system U = 1 (x) u_n + dt (Q (x) (A + B)) U
    big = np.eye(M * n) - dt * np.kron(coll.Q, A + B)
    U = np.linalg.solve(big, np.tile(u_n, M))
    got = oi.imex_sdc_step(u_n, lambda x: B @ x, lambda x: A @ x, _solver(A), coll, 60, dt, implicit)
    np.testing.assert_allclose(got, U[-n:], rtol=1e-12, atol=1e-13)


def test_lu_weights_two_nodes_closed_form():
    """M = 2 (tau = 1/3, 1; Q = [[5/12, -1/12], [3/4, 1/4]]): Q^T = L U with
    L = [[1, 0], [-1/5, 1]], U = [[5/12, 3/4], [0, 2/5]], so the implicit weights
    are U^T = [[5/12, 0], [3/4, 2/5]]."""
    np.testing.assert_allclose(oi.lu_weights(sdc.Collocation(2).Q), [[5 / 12, 0.0], [3 / 4, 2 / 5]], atol=1e-15)


@pytest.mark.parametrize("M", [3, 4, 8])
def test_lu_weights_make_the_stiff_limit_nilpotent(M):
    """With q^Delta = U^T, q^Delta^{-1} Q = L^T is unit upper triangular, so the
    stiff-limit sweep matrix I - q^Delta^{-1} Q is strictly upper triangular
    (checked by a generic solve) and its M-th power vanishes; q^Delta is lower
    triangular."""
    Q = sdc.Collocation(M).Q
    Qd = oi.lu_weights(Q)
    assert np.all(np.triu(Qd, 1) == 0.0)
    K = np.eye(M) - np.linalg.solve(Qd, Q)
    assert np.abs(np.tril(K)).max() < 1e-13
    assert np.abs(np.linalg.matrix_power(K, M)).max() < 1e-14


def _nonlinear_problem():
    A = np.array([[-1.0, 2.0], [-2.0, -1.0]])
    f_I = lambda x: A @ x
    f_E = lambda x: np.array([np.sin(x[1]), -0.5 * x[0] * x[1]])
    rhs = lambda t, x: f_I(x) + f_E(x)
    u0 = np.array([1.0, 0.5])
    T = 1.0
    ref = solve_ivp(rhs, (0.0, T), u0, method="DOP853", rtol=1e-13, atol=1e-15).y[:, -1]
    return A, f_I, f_E, u0, T, ref


def _observed_order(step, nsteps_list):
    A, f_I, f_E, u0, T, ref = _nonlinear_problem()
    errs = []
    for ns in nsteps_list:
        x = u0
        for _ in range(ns):
            x = step(x, f_E, f_I, _solver(A), T / ns)
        errs.append(np.linalg.norm(x - ref))
    return np.log2(errs[0] / errs[1])


@pytest.mark.parametrize("implicit", ["euler", "lu"])
@pytest.mark.parametrize("K,order", [(1, 1), (2, 2), (3, 3)])
def test_serial_sdc_order(K, order, implicit):
    coll = sdc.Collocation(3)
    p = _observed_order(lambda x, fe, fi, so, dt: oi.imex_sdc_step(x, fe, fi, so, coll, K, dt, implicit), [16, 32])
    assert abs(p - order) < 0.3, p


def test_imex2_order_two():
    p = _observed_order(oi.imex2_step, [32, 64])
    assert abs(p - 2.0) < 0.2, p


def test_imex2_limits():
    n = 4
    rng = np.random.default_rng(3)
    B = rng.standard_normal((n, n))
    u = rng.standard_normal(n)
    dt = 0.3
    zero = lambda x: np.zeros_like(x)
    got = oi.imex2_step(u, lambda x: B @ x, zero, lambda al, b: b, dt)
    heun = u + dt * B @ u + 0.5 * dt * dt * B @ (B @ u)
    np.testing.assert_allclose(got, heun, rtol=1e-14, atol=1e-14)
    S = rng.standard_normal((n, n))
    S = S - S.T                                                      # skew-symmetric
    x = u.copy()
    for _ in range(50):
        x = oi.imex2_step(x, zero, lambda y: S @ y, _solver(S), dt)
    assert abs(np.linalg.norm(x) - np.linalg.norm(u)) < 1e-13 * np.linalg.norm(u)


def test_swe_first_serial_sweep_is_imex_euler():
    T, J, L = 10, 16, 32
    o = swe.SWE(sht.Grid(T, J, L), swe.default_physics())
    wl = si.Workload("i", 0, T, J, L, 3, 1, 600.0, 1, 1, (100.0, 100.0))
    u = swe.initial_state(wl, o)
    coll = sdc.Collocation(3)
    got = oi.imex_sdc_step(u, o.explicit, o.linear, o.solve, coll, 1, 600.0)
    x, t_prev = u, 0.0
    for tm in coll.tau:
        h = 600.0 * (tm - t_prev)
        x = o.solve(h, x + h * o.explicit(x))
        t_prev = tm
    scale = np.abs(x).max(axis=1, keepdims=True)
    assert np.all(np.abs(got - x) <= 1e-13 * scale)
