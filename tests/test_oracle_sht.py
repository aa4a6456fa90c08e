"""Pins of the oracle's spherical-harmonic transform and tendencies (CPU only).

Each check compares the oracle with something other than itself: library
routines (scipy Gauss nodes, scipy associated Legendre functions, numpy FFT),
closed forms, or a brute-force evaluation of Eq. (4) by symbolic calculus.
"""
import math

import numpy as np
import pytest
import scipy.special as sps

import swe_inputs as si
from oracle import sht, swe


def _grid(T, J, L):
    return sht.Grid(T, J, L)


def _pbar_scipy(n, m, x):
    """Normalised Pbar_n^m from scipy's lpmv (which carries the Condon-Shortley phase)."""
    norm = math.sqrt((2 * n + 1) / 2.0 * math.factorial(n - m) / math.factorial(n + m))
    return (-1) ** m * norm * sps.lpmv(m, n, x)


@pytest.mark.parametrize("J", [2, 3, 12, 48, 192, 384, 768])
def test_gauss_nodes_are_legendre_roots(J):
    mu, w = sht.gauss_grid(J)
    assert np.all(np.diff(mu) < 0), "north to south ordering"
    assert abs(w.sum() - 2.0) < 1e-14
    x, wr = sps.roots_legendre(J)
    np.testing.assert_allclose(mu, x[::-1], rtol=0, atol=1e-14)
    np.testing.assert_allclose(w, wr[::-1], rtol=5e-9, atol=0)   # scipy's own error reaches ~2e-9
    # |P_J'| reaches J^2/2 at the poles, so a correctly rounded node leaves |P_J| ~ J^2 ulp
    assert np.max(np.abs(sps.eval_legendre(J, mu))) < 2e-16 * J * J + 1e-14
    for p in range(0, 2 * J, max(1, (2 * J) // 16)):           # exact up to degree 2J-1
        exact = 0.0 if p % 2 else 2.0 / (p + 1)
        assert abs(np.sum(w * mu ** p) - exact) < 1e-14


@pytest.mark.parametrize("J", [48, 384, 768])
def test_gauss_nodes_against_extended_precision(J):
    """Nodes and weights against a 40-digit Newton refinement (mpmath)."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    mu, w = sht.gauss_grid(J)
    for i in sorted({0, 1, 2, J // 3, J // 2 - 1, J - 1}):
        r = mp.mpf(mu[i])
        for _ in range(6):
            dp = J * (r * mp.legendre(J, r) - mp.legendre(J - 1, r)) / (r * r - 1)
            r = r - mp.legendre(J, r) / dp
        dp = J * (r * mp.legendre(J, r) - mp.legendre(J - 1, r)) / (r * r - 1)
        wt = 2 / ((1 - r * r) * dp * dp)
        assert abs(float(mu[i] - r)) < 2e-16
        assert abs(float((w[i] - wt) / wt)) < 5e-12


def test_pbar_closed_forms_low_degree():
    mu = np.linspace(-0.99, 0.99, 23)
    s = np.sqrt(1 - mu ** 2)
    P = sht.legendre_pbar(3, mu)
    closed = {
        (0, 0): np.full_like(mu, 1 / math.sqrt(2)),
        (1, 0): math.sqrt(1.5) * mu,
        (1, 1): math.sqrt(0.75) * s,
        (2, 0): math.sqrt(5 / 8) * (3 * mu ** 2 - 1),
        (2, 1): math.sqrt(15 / 4) * mu * s,
        (2, 2): math.sqrt(15 / 16) * s ** 2,
    }
    for (n, m), ref in closed.items():
        np.testing.assert_allclose(P[m][:, n - m], ref, rtol=1e-14, atol=1e-15)


def test_pbar_against_scipy_lpmv():
    T = 20
    mu = np.linspace(-0.98, 0.98, 17)
    P = sht.legendre_pbar(T, mu)
    for m in range(T + 1):
        for n in range(m, T + 2):
            ref = _pbar_scipy(n, m, mu)
            np.testing.assert_allclose(P[m][:, n - m], ref, rtol=1e-11, atol=1e-12)


@pytest.mark.parametrize("T,J", [(31, 48), (127, 192)])
def test_pbar_gauss_orthonormal(T, J):
    mu, w = sht.gauss_grid(J)
    P = sht.legendre_pbar(T, mu)
    for m in range(0, T + 1, 3):
        G = (P[m].T * w) @ P[m]
        np.testing.assert_allclose(G, np.eye(G.shape[0]), atol=1e-13)


def test_h_is_derivative_of_pbar():
    T = 12
    mu = np.linspace(-0.9, 0.9, 11)
    d = 1e-6
    P = sht.legendre_pbar(T, mu)
    H = sht.legendre_h(T, P)
    Pp = sht.legendre_pbar(T, mu + d)
    Pm = sht.legendre_pbar(T, mu - d)
    for m in range(T + 1):
        fd = (1 - mu ** 2)[:, None] * (Pp[m] - Pm[m])[:, : T + 1 - m] / (2 * d)
        np.testing.assert_allclose(H[m], fd, rtol=0, atol=2e-7)


def test_dft_matches_numpy_fft():
    T, J, L = 10, 4, 24
    g = _grid(T, J, L)
    rng = np.random.default_rng(1)
    f = rng.standard_normal((J, L))
    F = g.grid_to_fourier(f)
    ref = np.fft.rfft(f, axis=1)[:, : T + 1] / L
    np.testing.assert_allclose(F, ref, atol=1e-14)
    Fh = rng.standard_normal((J, T + 1)) + 1j * rng.standard_normal((J, T + 1))
    Fh[:, 0] = Fh[:, 0].real
    full = np.zeros((J, L // 2 + 1), complex)
    full[:, : T + 1] = Fh
    np.testing.assert_allclose(g.fourier_to_grid(Fh), np.fft.irfft(full, n=L, axis=1) * L, atol=1e-12)


@pytest.mark.parametrize("T,J,L", [(5, 8, 16), (31, 48, 96), (42, 64, 128)])
def test_scalar_round_trip(T, J, L):
    g = _grid(T, J, L)
    n, m = si.degree_order_arrays(T)
    rng = np.random.default_rng(T)
    c = rng.standard_normal(g.ncoef) + 1j * rng.standard_normal(g.ncoef)
    c[m == 0] = c[m == 0].real
    c2 = g.grid_to_spec(g.spec_to_grid(c))
    assert np.max(np.abs(c2 - c)) < 1e-13 * np.max(np.abs(c))


def _single(T, n, m, value):
    c = np.zeros(si.ncoef(T), complex)
    c[si.order_offset(T, m) + n - m] = value
    return c


def test_wind_closed_forms():
    """Solid-body rotation, a divergent zonal flow and an m=1 rotation, closed forms of U, V."""
    T, J, L = 6, 12, 24
    g = _grid(T, J, L)
    phys = swe.Physics(2.0, 0.7, 1.3, 1.1)
    s = swe.SWE(g, phys)
    a, u0 = phys.a, 3.0
    mu = g.mu[:, None]
    lam = g.lam[None, :]
    # zeta = 2 u0 mu / a  ->  U = u0 (1 - mu^2), V = 0
    zeta = _single(T, 1, 0, 2 * u0 / a / math.sqrt(1.5))
    U, V = s.wind_fourier(zeta, np.zeros_like(zeta))
    np.testing.assert_allclose(g.fourier_to_grid(U), u0 * (1 - mu ** 2) + 0 * lam, atol=1e-13)
    np.testing.assert_allclose(g.fourier_to_grid(V), 0 * mu * lam, atol=1e-13)
    # chi = c mu  (div = -2 chi / a^2)  ->  U = 0, V = (c/a)(1 - mu^2)
    cc = 1.7
    div = _single(T, 1, 0, -2.0 / a ** 2 * cc / math.sqrt(1.5))
    U, V = s.wind_fourier(np.zeros_like(div), div)
    np.testing.assert_allclose(g.fourier_to_grid(U), 0 * mu * lam, atol=1e-13)
    np.testing.assert_allclose(g.fourier_to_grid(V), cc / a * (1 - mu ** 2) + 0 * lam, atol=1e-13)
    # psi = c sqrt(1-mu^2) cos(lambda) = c * 2/sqrt(3) Pbar_1^1 Re e^{i lam}; the (1,1)
    # coefficient of a real field carries half the amplitude (f = 2 Re f_1 e^{i lam})
    psi11 = cc / (2 * math.sqrt(0.75))
    zeta = _single(T, 1, 1, -2.0 / a ** 2 * psi11)
    U, V = s.wind_fourier(zeta, np.zeros_like(zeta))
    sq = np.sqrt(1 - mu ** 2)
    np.testing.assert_allclose(g.fourier_to_grid(U), cc / a * mu * sq * np.cos(lam), atol=1e-13)
    np.testing.assert_allclose(g.fourier_to_grid(V), -cc / a * sq * np.sin(lam), atol=1e-13)


def _tc2_state(T, phys, u0):
    """Steady zonal flow u = u0 cos(lat) in gradient-wind balance:
    Phi' = -(a Omega u0 + u0^2/2) mu^2 + const (derived from f u + u^2 tan/a = -(1/a) dPhi/dlat)."""
    u = np.zeros((3, si.ncoef(T)), complex)
    u[1, 1] = 2 * u0 / phys.a / math.sqrt(1.5)
    c = -(phys.a * phys.omega * u0 + u0 ** 2 / 2)
    u[0, 2] = c * (2.0 / 3.0) / math.sqrt(2.5)           # mu^2 = 1/3 + (2/3) P_2
    u[0, 0] = c / 3.0 * math.sqrt(2.0)
    return u


@pytest.mark.parametrize("T,J,L", [(5, 8, 16), (31, 48, 96)])
def test_steady_zonal_flow_is_fixed_point(T, J, L):
    g = _grid(T, J, L)
    phys = swe.default_physics()
    s = swe.SWE(g, phys)
    u = _tc2_state(T, phys, 20.0)
    rhs = s.rhs(u)
    scale = np.abs(s.explicit(u)).max(axis=1) + np.abs(s.linear(u)).max(axis=1)
    # per field, relative to the size of the cancelling terms
    assert np.abs(rhs[1]).max() <= 1e-13 * scale.max()
    assert np.abs(rhs[2]).max() <= 1e-13 * scale[2]
    assert np.abs(rhs[0]).max() <= 1e-13 * (np.abs(u[0]).max() * phys.omega)


def _explicit_linear_part(s, u, eps=1.0):
    """The linear part of T_E (which is exactly linear + quadratic in u)."""
    return (4 * s.explicit(eps * u) - s.explicit(2 * eps * u)) / (2 * eps)


def test_linear_coriolis_closed_form():
    """L_c in spectral form for a small random (zeta, div) state:
    L_c(zeta)_n = -(2 Om/a^2) i m psi_n + (2 Om/a^2)[(n^2-1) eps_n chi_{n-1} + n(n+2) eps_{n+1} chi_{n+1}]
    L_c(div)_n  = -(2 Om/a^2)[(n^2-1) eps_n psi_{n-1} + n(n+2) eps_{n+1} psi_{n+1}] - (2 Om/a^2) i m chi_n
    (derived from -div(f V), curl(f V) with f = 2 Om mu and mu Pbar_n = eps_{n+1} Pbar_{n+1} + eps_n Pbar_{n-1})."""
    T, J, L = 12, 20, 40
    g = _grid(T, J, L)
    phys = swe.Physics(2.0, 0.7, 1.3, 1.1)
    s = swe.SWE(g, phys)
    n, m = si.degree_order_arrays(T)
    rng = np.random.default_rng(5)
    u = np.zeros((3, g.ncoef), complex)
    for f in (1, 2):
        c = rng.standard_normal(g.ncoef) + 1j * rng.standard_normal(g.ncoef)
        c[m == 0] = c[m == 0].real
        c[n == 0] = 0
        u[f] = c
    lin = _explicit_linear_part(s, u)
    psi = s.streamfunction(u[1])
    chi = s.streamfunction(u[2])
    k = 2 * phys.omega / phys.a ** 2
    ref_z = np.zeros(g.ncoef, complex)
    ref_d = np.zeros(g.ncoef, complex)
    for i in range(g.ncoef):
        nn, mm = n[i], m[i]
        cpl_psi = 0j
        cpl_chi = 0j
        if nn - 1 >= mm:
            e = sht.epsilon(nn, mm)
            cpl_psi += (nn * nn - 1) * e * psi[i - 1]
            cpl_chi += (nn * nn - 1) * e * chi[i - 1]
        if nn + 1 <= T:
            e = sht.epsilon(nn + 1, mm)
            cpl_psi += nn * (nn + 2) * e * psi[i + 1]
            cpl_chi += nn * (nn + 2) * e * chi[i + 1]
        ref_z[i] = -k * 1j * mm * psi[i] + k * cpl_chi
        ref_d[i] = -k * cpl_psi - k * 1j * mm * chi[i]
    scale = np.abs(ref_z).max() + np.abs(ref_d).max()
    np.testing.assert_allclose(lin[1], ref_z, atol=1e-12 * scale)
    np.testing.assert_allclose(lin[2], ref_d, atol=1e-12 * scale)
    np.testing.assert_allclose(lin[0], 0, atol=1e-12 * scale)


def test_mass_tendency_vanishes():
    T, J, L = 21, 32, 64
    g = _grid(T, J, L)
    s = swe.SWE(g, swe.default_physics())
    wl = si.Workload("x", 0, T, J, L, 3, 3, 600.0, 1, 1, (100.0, 100.0))
    u = swe.initial_state(wl, s)
    te = s.explicit(u)
    assert abs(te[0, 0]) <= 1e-15 * np.abs(te[0]).max()
    assert abs(te[2, 0]) <= 1e-15 * np.abs(te[2]).max()
    assert abs(te[1, 0]) <= 1e-15 * np.abs(te[1]).max()


def test_explicit_tendency_brute_force_symbolic():
    """T_E of Eq. (4) by symbolic calculus in (lambda, latitude) on the primitive
    (u, v, Phi') equations, projected with an independent fine quadrature, against
    the oracle's transform-method T_E at T = 3."""
    sp = pytest.importorskip("sympy")
    T, J, L = 3, 8, 16
    g = _grid(T, J, L)
    phys = swe.Physics(2.0, 0.7, 1.3, 1.1)
    s = swe.SWE(g, phys)
    n_arr, m_arr = si.degree_order_arrays(T)
    rng = np.random.default_rng(11)
    u = np.zeros((3, g.ncoef), complex)
    for f in range(3):
        c = 0.3 * (rng.standard_normal(g.ncoef) + 1j * rng.standard_normal(g.ncoef))
        c[m_arr == 0] = c[m_arr == 0].real
        if f > 0:
            c[n_arr == 0] = 0
        u[f] = c
    psi = s.streamfunction(u[1])
    chi = s.streamfunction(u[2])

    lam, th = sp.symbols("lam th", real=True)
    x = sp.sin(th)

    def pbar_sym(n, m):
        norm = sp.sqrt(sp.Rational(2 * n + 1, 2) * sp.factorial(n - m) / sp.factorial(n + m))
        # sympy's assoc_legendre carries (-1)^m; write (1-x^2)^{m/2} as cos(th)^m
        Pnm = sp.diff(sp.legendre(n, sp.Symbol("z")), sp.Symbol("z"), m).subs(sp.Symbol("z"), x)
        return norm * sp.cos(th) ** m * Pnm

    def field(c):
        expr = 0
        for i in range(c.size):
            n, m = int(n_arr[i]), int(m_arr[i])
            w = 1 if m == 0 else 2
            re, im = float(c[i].real), float(c[i].imag)
            expr += w * (re * sp.cos(m * lam) - im * sp.sin(m * lam)) * pbar_sym(n, m)
        return expr

    a = phys.a
    f = 2 * phys.omega * sp.sin(th)
    PSI, CHI, PH = field(psi), field(chi), field(u[0])
    uu = -sp.diff(PSI, th) / a + sp.diff(CHI, lam) / (a * sp.cos(th))
    vv = sp.diff(PSI, lam) / (a * sp.cos(th)) + sp.diff(CHI, th) / a
    adv = lambda q: uu / (a * sp.cos(th)) * sp.diff(q, lam) + vv / a * sp.diff(q, th)
    ut = f * vv - (adv(uu) - uu * vv * sp.tan(th) / a)
    vt = -f * uu - (adv(vv) + uu * uu * sp.tan(th) / a)
    divV = (sp.diff(uu, lam) + sp.diff(vv * sp.cos(th), th)) / (a * sp.cos(th))
    pt = -adv(PH) - PH * divV
    zt = (sp.diff(vt, lam) - sp.diff(ut * sp.cos(th), th)) / (a * sp.cos(th))
    dt = (sp.diff(ut, lam) + sp.diff(vt * sp.cos(th), th)) / (a * sp.cos(th))
    fns = [sp.lambdify((lam, th), e, "numpy") for e in (pt, zt, dt)]

    # independent projection: 40 Gauss points in mu, 32 uniform longitudes
    xq, wq = sps.roots_legendre(40)
    thq = np.arcsin(xq)
    lq = 2 * np.pi * np.arange(32) / 32
    LL, TT = np.meshgrid(lq, thq)
    ref = np.zeros((3, g.ncoef), complex)
    for fi, fn in enumerate(fns):
        vals = np.broadcast_to(fn(LL, TT), LL.shape)
        Fm = np.fft.fft(vals, axis=1) / 32          # e^{-i m lam} coefficients
        for i in range(g.ncoef):
            n, m = int(n_arr[i]), int(m_arr[i])
            ref[fi, i] = np.sum(wq * Fm[:, m] * _pbar_scipy(n, m, xq))
    got = s.explicit(u)
    for fi in range(3):
        scale = np.abs(ref[fi]).max()
        np.testing.assert_allclose(got[fi], ref[fi], atol=1e-11 * scale)
