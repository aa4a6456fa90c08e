"""Pins of the oracle's discrete adjoint (CPU only).

* T_E is exactly linear + quadratic in the state, so the central difference
  (T_E(u + v) - T_E(u - v)) / 2 is its exact tangent: the dot-product test
  <J v, w> = <v, J^T w> then holds to rounding with no truncation error.
* Every transform building block passes its own dot-product test.
* With linear f_I and f_E the dSDC step is a linear map A; its adjoint must be
  A^T, built column by column from the forward step.
* The full gradient of the height loss agrees with central finite
  differences along seeded directions.
"""
import numpy as np
import pytest

import swe_inputs as si
from oracle import adjoint as adj
from oracle import sdc, sht, swe


def rdot(a, b):
    return float(np.real(np.vdot(a, b)))


def _setup(T=10, J=16, L=32):
    g = sht.Grid(T, J, L)
    s = swe.SWE(g, swe.default_physics())
    wl = si.Workload("adj", 0, T, J, L, 3, 3, 600.0, 1, 1, (100.0, 100.0))
    return s, swe.initial_state(wl, s)


def _rand(shape, rng):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def test_building_block_transposes():
    g = sht.Grid(9, 14, 30)
    rng = np.random.default_rng(2)
    F = _rand((g.J, g.T + 1), rng)
    r = rng.standard_normal((g.J, g.L))
    assert abs(rdot(r, g.fourier_to_grid(F)) - rdot(adj.fourier_to_grid_T(g, r), F)) < 1e-11
    f = rng.standard_normal((g.J, g.L))
    Fb = _rand((g.J, g.T + 1), rng)
    assert abs(rdot(Fb, g.grid_to_fourier(f)) - rdot(adj.grid_to_fourier_T(g, Fb), f)) < 1e-12
    c = _rand(g.ncoef, rng)
    for tab in ("p", "h"):
        X = _rand((g.J, g.T + 1), rng)
        assert abs(rdot(X, g.synth(c, tab)) - rdot(adj.synth_T(g, X, tab), c)) < 1e-11
        wts = rng.uniform(0.1, 1.0, g.J)
        cb = _rand(g.ncoef, rng)
        assert abs(rdot(cb, g.analyse(X, wts, tab)) - rdot(adj.analyse_T(g, cb, wts, tab), X)) < 1e-11


@pytest.mark.parametrize("T,J,L", [(10, 16, 32), (21, 32, 64)])
def test_explicit_tendency_dot_product_exact(T, J, L):
    s, u = _setup(T, J, L)
    rng = np.random.default_rng(T)
    scale = np.abs(u).max(axis=1, keepdims=True)
    v = _rand(u.shape, rng) * scale
    w = _rand(u.shape, rng)
    Jv = (s.explicit(u + v) - s.explicit(u - v)) / 2.0        # exact: T_E is quadratic
    lhs = rdot(w, Jv)
    rhs = rdot(adj.explicit_vjp(s, u, w), v)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_linear_step_adjoint_is_transpose():
    """f_I = A, f_E = B linear: the step is a matrix; its VJP must be that matrix transposed."""
    A = np.array([[0.0, -1.5, 0.2], [1.5, 0.0, 0.0], [0.1, 0.0, -0.4]])
    B = np.array([[-0.2, 0.3, 0.0], [0.05, -0.1, 0.2], [0.0, 0.1, -0.3]])
    n = 3
    f_I = lambda x: A @ x
    f_E = lambda x: B @ x
    solve = lambda al, b: np.linalg.solve(np.eye(n) - al * A, b)
    solveT = lambda al, b: np.linalg.solve((np.eye(n) - al * A).T, b)
    for M, K in [(3, 3), (4, 5), (1, 1), (2, 4)]:
        coll = sdc.Collocation(M)
        step = lambda x: sdc.dsdc_step(x, f_E, f_I, solve, coll, K, 0.3)
        Amat = np.stack([step(e) for e in np.eye(n)], axis=1)
        for e in np.eye(n):
            got = adj.dsdc_step_vjp(np.zeros(n), e, f_E, lambda x, a: B.T @ a, f_I, lambda x: A.T @ x, solve,
                                    solveT, coll, K, 0.3)
            np.testing.assert_allclose(got, Amat.T @ e, atol=1e-14)


@pytest.mark.parametrize("M,K", [(3, 3), (4, 5), (2, 1)])
def test_step_adjoint_against_finite_differences(M, K):
    s, u = _setup()
    rng = np.random.default_rng(M * 10 + K)
    coll = sdc.Collocation(M)
    ub = _rand(u.shape, rng)
    d = _rand(u.shape, rng) * np.abs(u).max(axis=1, keepdims=True)
    eps = 1e-6
    jd = (sdc.swe_step(s, u + eps * d, coll, K, 600.0) - sdc.swe_step(s, u - eps * d, coll, K, 600.0)) / (2 * eps)
    lhs = rdot(ub, jd)
    rhs = rdot(adj.swe_step_vjp(s, u, ub, coll, K, 600.0), d)
    assert abs(lhs - rhs) <= 1e-8 * abs(lhs)


def test_loss_gradient_against_finite_differences():
    s, u = _setup()
    coll = sdc.Collocation(3)
    rng = np.random.default_rng(7)
    target = s.height_grid(u) + rng.standard_normal((s.grid.J, s.grid.L))
    loss, grad = adj.loss_and_gradient(s, u, coll, 3, 600.0, 3, target)
    assert np.all(grad[:, :s.grid.T + 1].imag == 0)          # m = 0: no imaginary DOFs
    for i in range(4):
        d = _rand(u.shape, rng) * np.abs(u).max(axis=1, keepdims=True)
        d[:, :s.grid.T + 1] = d[:, :s.grid.T + 1].real
        eps = 1e-6
        lp = adj.height_loss(s, sdc.swe_run(s, u + eps * d, coll, 3, 600.0, 3), target)
        lm = adj.height_loss(s, sdc.swe_run(s, u - eps * d, coll, 3, 600.0, 3), target)
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - rdot(grad, d)) <= 1e-6 * abs(fd), (fd, rdot(grad, d))
