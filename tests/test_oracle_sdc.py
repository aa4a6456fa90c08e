"""Pins of the oracle's collocation data and dSDC step (CPU only).

The checks compare with textbook Radau IIA tables, exact polynomial
integration, dense collocation solves computed independently of the sweep,
the Pade stability function, IMEX Euler, the paper's performance model
(Table 1 and the printed speedup S = 3.25), conservation of mass and a
steady zonal flow.
"""
import math
import os

import numpy as np
import pytest

import swe_inputs as si
from oracle import sdc, sht, swe

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _radau_golden():
    tabs = {}
    cur = None
    for line in open(os.path.join(GOLDEN, "radau_iia.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        key, rest = line.split(" ", 1)
        vals = [eval(v, {"sqrt": math.sqrt}) for v in rest.split(";")]
        if key == "M":
            cur = {"a": []}
            tabs[int(vals[0])] = cur
        elif key == "a":
            cur["a"].append(vals)
        else:
            cur[key] = vals
    return tabs


@pytest.mark.parametrize("M", [2, 3])
def test_radau_iia_textbook_tables(M):
    ref = _radau_golden()[M]
    coll = sdc.Collocation(M)
    np.testing.assert_allclose(coll.tau, ref["c"], atol=1e-15)
    np.testing.assert_allclose(coll.Q, np.array(ref["a"]), atol=2e-15)


@pytest.mark.parametrize("M", range(1, 9))
def test_collocation_matrix_exactness(M):
    coll = sdc.Collocation(M)
    tau, Q = coll.tau, coll.Q
    assert tau[-1] == 1.0 and np.all(np.diff(tau) > 0) and tau[0] > 0
    np.testing.assert_allclose(Q.sum(axis=1), tau, atol=1e-13)
    for p in range(M):                                   # degree <= M-1 exact on every row
        np.testing.assert_allclose(Q @ tau ** p, tau ** (p + 1) / (p + 1), atol=1e-12)
    for p in range(2 * M - 1):                           # Radau quadrature: degree 2M-2 on [0, 1]
        assert abs(Q[-1] @ tau ** p - 1.0 / (p + 1)) < 1e-12


def test_min_sr_flex_coefficients():
    coll = sdc.Collocation(4, "clamped")
    for k in range(1, 8):
        np.testing.assert_allclose(coll.qdelta(k), coll.tau / min(k, 4))
    lit = sdc.Collocation(4, "literal")
    np.testing.assert_allclose(lit.qdelta(6), lit.tau / 6)


def _dahlquist_step_error(rule, M, z):
    """|dSDC step (K = M) - collocation solution| on y' = z y over dt = 1, y(0) = 1."""
    coll = sdc.Collocation(M, rule)
    u = sdc.dsdc_step(np.array([1.0]), lambda v: 0.0 * v, lambda v: z * v, lambda al, b: b / (1.0 - al * z),
                      coll, M, 1.0)
    U = np.linalg.solve(np.eye(M) - z * coll.Q, np.ones(M))
    return abs(u[0] - U[-1])


@pytest.mark.parametrize("M", [2, 3, 4])
def test_min_sr_flex_exact_in_the_stiff_limit(M):
    """MIN-SR-FLEX: in the stiff limit a sweep's error operator tends to I - D_k^{-1} Q,
    and the product over k = 1..M of these vanishes, so M sweeps reach the
    collocation solution; the implicit-Euler diagonal does not."""
    z = -1e9
    assert _dahlquist_step_error("clamped", M, z) < 1e-13
    assert _dahlquist_step_error("literal", M, z) < 1e-13
    assert _dahlquist_step_error("ie", M, z) > 1e-10


@pytest.mark.parametrize("M", [2, 3])
def test_min_sr_ns_gains_an_order_in_the_non_stiff_limit(M):
    """MIN-SR-NS: Q - diag(tau / M) is nilpotent, so in the non-stiff limit M sweeps
    leave an O(z^{M+2}) error against the collocation solution; a diagonal
    without that property (implicit Euler, tau_m) leaves O(z^{M+1})."""
    def slope(rule):
        return np.log2(_dahlquist_step_error(rule, M, -0.02) / _dahlquist_step_error(rule, M, -0.01))
    assert slope("min-sr-ns") > M + 1.8
    assert abs(slope("ie") - (M + 1)) < 0.2


def test_implicit_euler_diagonal_sweeps_from_t_n():
    """Every sweep of the implicit-Euler diagonal is, at k = 0, one IMEX Euler step
    from t_n to t_n + tau_m dt (the FLEX first sweep), and its fixed point is the
    collocation solution (checked on the IMEX oscillator)."""
    A = np.array([[0.0, -2.0], [2.0, 0.0]])
    B = np.array([[-0.3, 0.1], [-0.2, -0.1]])
    f_E, f_I, solve = _linear_problem(A, B)
    u0 = np.array([1.0, 0.5])
    for M in (2, 4):
        coll = sdc.Collocation(M, "ie")
        dt = 0.1
        got = sdc.dsdc_step(u0, f_E, f_I, solve, coll, 1, dt)
        want = np.linalg.solve(np.eye(2) - dt * A, u0 + dt * (B @ u0))      # tau_M = 1
        np.testing.assert_allclose(got, want, rtol=1e-14)
        got = sdc.dsdc_step(u0, f_E, f_I, solve, coll, 80, dt)
        np.testing.assert_allclose(got, _dense_collocation(A + B, u0, coll.Q, dt), rtol=1e-12)


def test_min_sr_s_two_nodes_closed_form():
    """M = 2 (tau = 1/3, 1): det(xQ - D) = det(Q)(x - 1)^2 reduces to d1 d2 = 1/6 and
    3 d1 + 5 d2 = 4, whose increasing positive root is ((4 - sqrt 6)/6, (4 + sqrt 6)/10)."""
    d = sdc.Collocation(2, "min-sr-s").qdelta(1)
    np.testing.assert_allclose(d, [(4 - np.sqrt(6)) / 6, (4 + np.sqrt(6)) / 10], rtol=1e-13)


@pytest.mark.parametrize("M", [2, 3, 4, 5, 8])
def test_min_sr_s_stiff_limit_nilpotent(M):
    """MIN-SR-S: positive, increasing, the same in every sweep, and the stiff-limit
    sweep matrix I - D^{-1} Q nilpotent -- checked through its eigenvalues (a
    different computation from the characteristic-polynomial root the oracle
    solves for: a nilpotent perturbation of size eps spreads them by about
    eps^(1/M)) and through its M-th power."""
    coll = sdc.Collocation(M, "min-sr-s")
    d = coll.qdelta(3)
    assert np.all(d > 0) and np.all(np.diff(d) > 0)
    np.testing.assert_array_equal(d, coll.qdelta(1))
    K = np.eye(M) - coll.Q / d[:, None]
    assert np.abs(np.linalg.eigvals(K)).max() < 1e-12 ** (1.0 / M) * 10
    assert np.abs(np.linalg.matrix_power(K, M)).max() < 1e-10


def test_unknown_qdelta_rule_is_rejected():
    with pytest.raises(ValueError):
        sdc.Collocation(3, "min-sr-x").qdelta(1)


def _linear_problem(A, B):
    """u' = A u (implicit) + B u (explicit), u real vector."""
    n = A.shape[0]
    f_I = lambda u: A @ u
    f_E = lambda u: B @ u
    solve = lambda alpha, beta: np.linalg.solve(np.eye(n) - alpha * A, beta)
    return f_E, f_I, solve


def _dense_collocation(A, u0, Q, dt):
    """Node-M value of the collocation solution u = 1 (x) u0 + dt (Q (x) A) u, dense solve."""
    M, n = Q.shape[0], A.shape[0]
    big = np.eye(M * n) - dt * np.kron(Q, A)
    U = np.linalg.solve(big, np.tile(u0, M))
    return U[-n:]


@pytest.mark.parametrize("M", [2, 3])
def test_sweeps_converge_to_radau_stability_function(M):
    """Many sweeps on y' = lambda y reach R(dt lambda), the (M-1, M) Pade approximant."""
    ref = _radau_golden()[M]
    lam = -0.7 + 0.4j
    A = np.array([[lam.real, -lam.imag], [lam.imag, lam.real]])
    f_E, f_I, solve = _linear_problem(A, np.zeros((2, 2)))
    coll = sdc.Collocation(M)
    dt = 0.5
    u0 = np.array([1.0, 0.0])
    u = sdc.dsdc_step(u0, f_E, f_I, solve, coll, 60, dt)
    z = dt * lam
    R = np.polyval(ref["Rnum"][::-1], z) / np.polyval(ref["Rden"][::-1], z)
    np.testing.assert_allclose(u[0] + 1j * u[1], R, atol=1e-13)


@pytest.mark.parametrize("M", [1, 3, 4, 5])
def test_imex_sweeps_converge_to_collocation(M):
    """Implicit A + explicit B (an oscillator with damping): the sweep's fixed point
    is the collocation solution of A + B, from a dense solve."""
    A = np.array([[0.0, -2.0], [2.0, 0.0]])
    B = np.array([[-0.3, 0.1], [-0.2, -0.1]])
    f_E, f_I, solve = _linear_problem(A, B)
    coll = sdc.Collocation(M)
    dt = 0.2
    u0 = np.array([0.3, -1.1])
    u = sdc.dsdc_step(u0, f_E, f_I, solve, coll, 80, dt)
    np.testing.assert_allclose(u, _dense_collocation(A + B, u0, coll.Q, dt), atol=1e-13)


def _small_swe(T=10, J=16, L=32):
    g = sht.Grid(T, J, L)
    s = swe.SWE(g, swe.default_physics())
    wl = si.Workload("small", 0, T, J, L, 3, 3, 600.0, 1, 1, (100.0, 100.0))
    return s, swe.initial_state(wl, s)


def test_first_sweep_is_imex_euler():
    """With one sweep (q(1) = 1, u_j^0 = u_n) the node-M update is IMEX Euler over dt:
    u - dt L_g u = u_n + dt T_E(u_n)."""
    s, u0 = _small_swe()
    coll = sdc.Collocation(3)
    dt = 600.0
    u1 = sdc.swe_step(s, u0, coll, 1, dt)
    rhs = u0 + dt * s.explicit(u0)
    # independent closed-form 2x2 elimination per mode
    beta = dt
    phi = (rhs[0] - beta * s.phys.phibar * rhs[2]) / (1 + beta ** 2 * s.phys.phibar * s.lam)
    div = rhs[2] + beta * s.lam * phi
    np.testing.assert_allclose(u1[0], phi, atol=1e-12 * np.abs(phi).max())
    np.testing.assert_allclose(u1[1], rhs[1], atol=1e-14 * np.abs(rhs[1]).max())
    np.testing.assert_allclose(u1[2], div, atol=1e-12 * np.abs(div).max())


def _perf_golden():
    rows = []
    for line in open(os.path.join(GOLDEN, "perf_model.txt")):
        if line.strip() and not line.startswith("#"):
            M, K, r, S, tol = line.split()
            rows.append((int(M), int(K), float(r), float(S), float(tol)))
    return rows


@pytest.mark.parametrize("M,K", [(3, 3), (4, 4), (4, 5), (2, 1)])
def test_cost_counts_match_table_1(M, K):
    """Algorithm 2 performs 1 + (K-1) M explicit evaluations and (K-1) M + 1 solves per step."""
    s, u0 = _small_swe(T=5, J=8, L=16)
    coll = sdc.Collocation(M)
    s.n_explicit = s.n_solve = 0
    sdc.swe_step(s, u0, coll, K, 100.0)
    assert s.n_explicit == 1 + (K - 1) * M
    assert s.n_solve == (K - 1) * M + 1


def test_performance_model_speedup_printed_value():
    """The per-step counts of Algorithm 2 fed into Table 1's cost model give the printed S."""
    for M, K, r, S_printed, tol in _perf_golden():
        s, u0 = _small_swe(T=5, J=8, L=16)
        s.n_explicit = s.n_solve = 0
        sdc.swe_step(s, u0, sdc.Collocation(M), K, 100.0)
        cE, cS = 1.0, 1.0                              # S does not depend on them when r fixed
        ctE = r * (cE + cS)
        evals_after_init = s.n_explicit - 1            # the k = 0 evaluation is shared
        solves_in_sweeps = s.n_solve - 1               # the last-node solve is shared
        seq = cE + evals_after_init * cE + solves_in_sweeps * (cS + ctE) + cS
        par = cE + (K - 1) * (cE + cS + ctE) + cS
        assert abs(seq / par - S_printed) <= tol


def test_mass_is_conserved_over_steps():
    s, u0 = _small_swe()
    coll = sdc.Collocation(3)
    u = sdc.swe_run(s, u0, coll, 3, 600.0, 5)
    assert abs(u[0, 0] - u0[0, 0]) <= 1e-14 * abs(u0[0, 0]) + 1e-12
    assert abs(u[2, 0]) < 1e-25 and abs(u[1, 0]) < 1e-25


def test_steady_zonal_flow_survives_steps():
    T, J, L = 10, 16, 32
    g = sht.Grid(T, J, L)
    phys = swe.default_physics()
    s = swe.SWE(g, phys)
    u0 = np.zeros((3, g.ncoef), complex)
    u0[1, 1] = 2 * 20.0 / phys.a / math.sqrt(1.5)
    c = -(phys.a * phys.omega * 20.0 + 200.0)
    u0[0, 2] = c * (2.0 / 3.0) / math.sqrt(2.5)
    u = sdc.swe_run(s, u0, sdc.Collocation(4), 4, 900.0, 4)
    # div starts at zero: measure it against the vorticity scale
    ref = np.abs(u0).max(axis=1)
    ref[2] = ref[1]
    for f in range(3):
        assert np.abs(u[f] - u0[f]).max() <= 1e-12 * ref[f]


def test_sweeps_converge_to_nonlinear_collocation():
    """T = 5: many sweeps reproduce the collocation solution of the full nonlinear
    problem, solved here by Newton's method on all M x 3 x ncoef unknowns."""
    from scipy.optimize import root
    T, J, L, M = 5, 8, 16, 3
    g = sht.Grid(T, J, L)
    s = swe.SWE(g, swe.default_physics())
    wl = si.Workload("tiny", 0, T, J, L, M, 3, 600.0, 1, 1, (100.0, 100.0))
    u0 = swe.initial_state(wl, s)
    coll = sdc.Collocation(M)
    dt = 300.0
    u_sdc = sdc.swe_step(s, u0, coll, 40, dt)
    nc = g.ncoef
    scale = np.abs(u0).max(axis=1)[:, None]

    def pack(U):
        return np.concatenate([(U.real / scale).ravel(), (U.imag / scale).ravel()])

    def unpack(x):
        h = x.size // 2
        re = x[:h].reshape(M, 3, nc) * scale
        im = x[h:].reshape(M, 3, nc) * scale
        return re + 1j * im

    def residual(x):
        U = unpack(x)
        F = np.stack([s.rhs(U[j]) for j in range(M)])
        R = U - u0[None] - dt * np.einsum("mj,jfc->mfc", coll.Q, F)
        return pack(R)

    sol = root(residual, pack(np.stack([u0] * M)), method="hybr", tol=1e-14)
    u_col = unpack(sol.x)[-1]
    for f in range(3):
        np.testing.assert_allclose(u_sdc[f], u_col[f], atol=1e-11 * np.abs(u0[f]).max())


def test_order_of_accuracy_linearised_regime():
    """Small-amplitude seeded state at T = 21: errors at dt, dt/2, dt/4 against dt/16
    fall with slope ~ min(K, 2M-1) = 3 for M = 3, K = 3 (one order per sweep)."""
    T, J, L = 21, 32, 64
    g = sht.Grid(T, J, L)
    s = swe.SWE(g, swe.default_physics())
    wl = si.Workload("ord", 0, T, J, L, 3, 3, 600.0, 1, 1, (100.0, 100.0))
    u0 = swe.initial_state(wl, s)
    coll = sdc.Collocation(3)
    horizon = 7200.0
    runs = {}
    for div in (1, 2, 4, 16):
        dt = 1800.0 / div
        runs[div] = sdc.swe_run(s, u0, coll, 3, dt, int(round(horizon / dt)))
    ref = runs[16]
    errs = [np.abs(runs[d][1] - ref[1]).max() for d in (1, 2, 4)]
    slopes = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(2.5 < sl < 4.2 for sl in slopes), (errs, slopes)


def test_residual_first_sweep_closed_form_and_convergence():
    """Before sweep 1 every u_j^0 = u_n, so R_m^0 = dt tau_m F(u_n); after many
    sweeps the collocation residual of node M vanishes."""
    s, u0 = _small_swe(T=5, J=8, L=16)
    coll = sdc.Collocation(3)
    dt = 200.0
    res = []
    sdc.swe_step(s, u0, coll, 30, dt, residuals=res)
    F = s.rhs(u0)
    expect = np.max(np.stack([s.field_norms(dt * t * F) for t in coll.tau]), axis=0)
    np.testing.assert_allclose(res[0], expect, rtol=1e-12)
    assert len(res) == 30
    assert np.all(res[-1] <= 1e-10 * res[0])
