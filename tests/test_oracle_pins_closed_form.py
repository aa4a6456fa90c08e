"""Closed-form pins of the oracle pieces that no other test fixes independently (CPU only).

* The Parseval-weighted residual norm (``SWE.field_norms``) against the grid
  L2 norm of the same band-limited field, (1/2pi) int int f^2 dlambda dmu,
  evaluated by Gauss quadrature in mu and the trapezoidal rule in lambda on
  values built from scipy's associated Legendre functions and explicit
  cos/sin sums (no oracle transform involved).
* The dSDC step (Algorithm 2 with Eq. (7)) on one gravity-wave mode with
  T_E = 0 against the closed-form matrix exponential of the linear system
  d(Phi', div)/dt = A (Phi', div), A = [[0, -Phibar], [lambda_n, 0]]
  (Eq. (4)'s L_g in spectral form): a rotation at omega = sqrt(Phibar lambda_n).
  One step's error falls with slope min(K, 2M - 1) + 1 in dt and the error at
  a fixed time with slope min(K, 2M - 1) (one order per sweep, capped at the
  Radau IIA collocation order 2M - 1).
* The normalised Legendre table at the largest truncation, T511 on 768 Gauss
  latitudes: Gauss orthonormality, and the polar rows (where the unscaled
  sectoral start Pbar_m^m underflows for large m) against 40-digit values.
"""
import math

import numpy as np
import pytest
import scipy.special as sps

import swe_inputs as si
from oracle import sdc, sht, swe


# ---------------------------------------------------------------------------
# residual norm = grid L2 norm (Parseval on the sphere)
# ---------------------------------------------------------------------------
def _pbar_scipy(n, m, x):
    norm = math.sqrt((2 * n + 1) / 2.0 * math.factorial(n - m) / math.factorial(n + m))
    return (-1) ** m * norm * sps.lpmv(m, n, x)


def _grid_values(T, coef, mu, lam):
    """f(mu_j, lambda_k) = sum_{m=-T..T} sum_n c_n^m Pbar_n^m(mu) e^{i m lambda}, c^{-m} = conj(c^m)."""
    f = np.zeros((mu.size, lam.size))
    for m in range(T + 1):
        for n in range(m, T + 1):
            c = coef[si.order_offset(T, m) + n - m]
            p = _pbar_scipy(n, m, mu)[:, None]
            if m == 0:
                f += p * c.real
            else:
                f += 2.0 * p * (c.real * np.cos(m * lam)[None, :] - c.imag * np.sin(m * lam)[None, :])
    return f


@pytest.mark.parametrize("T,J,L,seed", [(6, 10, 20, 0), (12, 20, 40, 1), (21, 32, 64, 2)])
def test_field_norms_equal_grid_l2_norm(T, J, L, seed):
    g = sht.Grid(T, J, L)
    s = swe.SWE(g, swe.default_physics())
    rng = np.random.default_rng([2403, seed])
    r = rng.standard_normal((3, g.ncoef)) + 1j * rng.standard_normal((3, g.ncoef))
    r[:, s.m == 0] = r[:, s.m == 0].real                  # real m = 0 coefficients
    r[1] *= 1e-5                                          # fields of different scales
    mu, w = sps.roots_legendre(J)                         # scipy's own Gauss rule
    lam = 2.0 * np.pi * np.arange(L) / L
    norms = s.field_norms(r)
    for f in range(3):
        vals = _grid_values(T, r[f], mu, lam)
        # f^2 has degree <= 2T <= 2J - 1 in mu and wavenumber <= 2T < L: both rules are exact
        l2 = math.sqrt(np.sum(w[:, None] * vals ** 2) / L)
        assert abs(norms[f] - l2) <= 1e-12 * l2, (f, norms[f], l2)


def test_field_norms_detect_a_single_order():
    """An m > 0 mode counts twice (its -m partner), an m = 0 mode once."""
    T = 4
    g = sht.Grid(T, 6, 12)
    s = swe.SWE(g, swe.default_physics())
    r = np.zeros((3, g.ncoef), complex)
    r[0, si.order_offset(T, 0) + 2] = 3.0
    r[1, si.order_offset(T, 3) + 1] = 3.0 + 4.0j
    nrm = s.field_norms(r)
    assert nrm[0] == pytest.approx(3.0, rel=1e-15)
    assert nrm[1] == pytest.approx(5.0 * math.sqrt(2.0), rel=1e-15)
    assert nrm[2] == 0.0


# ---------------------------------------------------------------------------
# one gravity-wave mode against exp(dt A)
# ---------------------------------------------------------------------------
def _mode_problem(n0=7, m0=3):
    T, J, L = 10, 16, 32
    g = sht.Grid(T, J, L)
    s = swe.SWE(g, swe.default_physics())
    idx = si.order_offset(T, m0) + n0 - m0
    lam_n = n0 * (n0 + 1) / si.RADIUS ** 2
    phibar = si.GRAVITY * si.MEAN_DEPTH
    om = math.sqrt(phibar * lam_n)
    u0 = np.zeros((3, g.ncoef), complex)
    u0[0, idx] = 1000.0 + 300.0j
    u0[1, idx] = 3e-5 - 1e-5j
    u0[2, idx] = 2e-6 - 1e-6j

    def exact(t):
        c, sn = math.cos(om * t), math.sin(om * t)
        E = np.array([[c, -phibar * sn / om], [lam_n * sn / om, c]])
        return E @ np.array([u0[0, idx], u0[2, idx]])

    return s, u0, idx, om, exact


def _mode_error(u, idx, ex, u0):
    return max(abs(u[0, idx] - ex[0]) / abs(ex[0]), abs(u[2, idx] - ex[1]) / abs(ex[1]))


@pytest.mark.parametrize("M,K", [(1, 1), (2, 2), (3, 2), (3, 3), (2, 4), (4, 4), (4, 5)])
def test_single_mode_matches_matrix_exponential_with_sdc_order(M, K):
    s, u0, idx, om, exact = _mode_problem()
    coll = sdc.Collocation(M)
    zero = lambda u: np.zeros_like(u)                     # T_E = 0: only L_g acts
    p = min(K, 2 * M - 1)
    # one step: local error ~ dt^(p+1)
    fs = np.array([0.4, 0.2, 0.1, 0.05]) if p + 1 >= 5 else np.array([0.2, 0.1, 0.05, 0.025])
    loc = []
    for f in fs:
        dt = f / om
        u = sdc.dsdc_step(u0, zero, s.linear, s.solve, coll, K, dt)
        loc.append(_mode_error(u, idx, exact(dt), u0))
        # the vorticity of the mode is untouched by L_g
        assert abs(u[1, idx] - u0[1, idx]) <= 1e-15 * abs(u0[1, idx])
    slope = np.polyfit(np.log(fs), np.log(loc), 1)[0]
    assert abs(slope - (p + 1)) < 0.45, (loc, slope)
    # fixed time 2 / omega: global error ~ dt^p
    ns = np.array([4, 8, 16, 32]) if p < 4 else np.array([8, 16, 32, 64])
    glob = []
    for nst in ns:
        dt = 2.0 / om / nst
        u = u0
        for _ in range(nst):
            u = sdc.dsdc_step(u, zero, s.linear, s.solve, coll, K, dt)
        glob.append(_mode_error(u, idx, exact(2.0 / om), u0))
    gslope = -np.polyfit(np.log(ns), np.log(glob), 1)[0]
    assert abs(gslope - p) < 0.6, (glob, gslope)


def test_single_mode_many_sweeps_is_radau_iia_not_the_exponential():
    """With K large the step is the collocation (Radau IIA) solution: its error
    against exp(dt A) is the R(z) - e^z defect, of order dt^(2M) per step, and
    the step stays norm-contracting (|R(i omega dt)| < 1)."""
    s, u0, idx, om, exact = _mode_problem()
    M = 3
    coll = sdc.Collocation(M)
    zero = lambda u: np.zeros_like(u)
    errs = []
    fs = np.array([0.8, 0.4, 0.2])
    for f in fs:
        dt = f / om
        u = sdc.dsdc_step(u0, zero, s.linear, s.solve, coll, 40, dt)
        errs.append(_mode_error(u, idx, exact(dt), u0))
    slope = np.polyfit(np.log(fs), np.log(errs), 1)[0]
    assert abs(slope - 2 * M) < 0.4, (errs, slope)


# ---------------------------------------------------------------------------
# the Legendre table at T511 on 768 Gauss latitudes
# ---------------------------------------------------------------------------
T511_ORDERS = (0, 1, 2, 63, 200, 255, 300, 400, 450, 500, 511)


@pytest.fixture(scope="module")
def t511_table():
    mu, w = sht.gauss_grid(768)
    return mu, w, sht.legendre_pbar(511, mu, orders=set(T511_ORDERS))


def test_pbar_gauss_orthonormal_t511(t511_table):
    mu, w, P = t511_table
    for m in T511_ORDERS:
        G = (P[m].T * w) @ P[m]
        np.testing.assert_allclose(G, np.eye(G.shape[0]), atol=1e-12)


def test_pbar_polar_rows_t511_against_extended_precision(t511_table):
    """At the latitudes closest to the pole the sectoral start of large orders
    underflows; the table must still hold every entry to 1e-12 absolute (the
    functions are of unit L2 norm; some 500 recurrence steps of rounding reach
    ~2e-13 at the polar row for small m), or 1e-12 relative where an entry
    exceeds 1, checked against 40-digit values of the
    normalised function from its Jacobi-polynomial form in mpmath."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    mu, w, P = t511_table

    def pbar_mp(n, m, x):
        # Pbar_n^m = sqrt((2n+1)/2 (n-m)!/(n+m)!) (1-x^2)^(m/2) (n+m)!/(2^m n!) P_{n-m}^{(m,m)}(x),
        # with the Jacobi polynomial from its hypergeometric series in (1-x)/2 (fast near the pole)
        x = mp.mpf(x)
        norm = mp.sqrt((2 * n + 1) / mp.mpf(2) * mp.factorial(n - m) / mp.factorial(n + m))
        dm = mp.factorial(n + m) / (mp.mpf(2) ** m * mp.factorial(n))
        return norm * (1 - x * x) ** (mp.mpf(m) / 2) * dm * mp.jacobi(n - m, m, m, x)

    for j in (0, 1, 5, 20):
        for m in (2, 63, 255, 511):
            for n in sorted({m, m + 1, (m + 512) // 2, 512}):
                ref = float(pbar_mp(n, m, mu[j]))
                assert abs(P[m][j, n - m] - ref) <= 1e-12 * max(1.0, abs(ref)), (j, m, n, P[m][j, n - m], ref)
