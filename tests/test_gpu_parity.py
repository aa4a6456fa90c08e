"""CUDA path against the FP64 oracle, element by element, through the C ABI.

The FP64 bar is the relative L2 distance per field: <= 1e-12 for one tendency
or transform, <= 1e-11 after a run (the accuracy target the FP64 path is held
to).  Inputs are the oracle's seeded initial states, passed to the GPU.
"""
import math

import numpy as np
import pytest

import swe_inputs as si
from oracle import sdc as osdc
from oracle import sht, swe
from tests.helpers import rel_l2, to_numpy

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_EVAL = 1e-12
TOL_RUN = 1e-11


def _solver(T, J, L, M, K, dt, precision=0, **kw):
    from paper_2403_20135_gb300 import Solver
    return Solver(T, J, L, M, K, dt, si.RADIUS, si.OMEGA, si.GRAVITY, si.MEAN_DEPTH, precision=precision, **kw)


def _oracle(T, J, L):
    g = sht.Grid(T, J, L)
    return swe.SWE(g, swe.default_physics())


def _wl(T, J, L, M=3, K=3, dt=600.0, idx=0, nb=1):
    return si.Workload("case", idx, T, J, L, M, K, dt, 1, nb, (100.0, 100.0))


def _cuda(u):
    return torch.from_numpy(np.ascontiguousarray(u)).to("cuda")


# sizes: several latitude chunks and a ragged tail (J/2 = 17, 24, 50 vs 64-wide
# chunks), odd/even truncations, nlon with radix 8, 4, 2, 3 stages
CASES = [(5, 8, 16), (21, 34, 72), (31, 48, 96), (42, 64, 128), (63, 100, 192)]


@pytest.mark.parametrize("T,J,L", CASES)
def test_tendency_matches_oracle(T, J, L):
    o = _oracle(T, J, L)
    u0 = swe.initial_state(_wl(T, J, L), o)
    ref = o.explicit(u0)
    s = _solver(T, J, L, 3, 3, 600.0)
    got = to_numpy(s.tendency(_cuda(u0)))
    err = rel_l2(got, ref)
    assert np.all(err <= TOL_EVAL), err


def test_tendency_batch_is_per_state():
    T, J, L = 31, 48, 96
    o = _oracle(T, J, L)
    states = np.stack([swe.initial_state(_wl(T, J, L, idx=i), o) for i in range(3)])
    s = _solver(T, J, L, 3, 3, 600.0)
    got = to_numpy(s.tendency(_cuda(states)))
    for b in range(3):
        assert np.all(rel_l2(got[b], o.explicit(states[b])) <= TOL_EVAL)


@pytest.mark.parametrize("T,J,L", [(31, 48, 96), (63, 100, 192)])
def test_scalar_transforms_match_oracle(T, J, L):
    o = _oracle(T, J, L)
    s = _solver(T, J, L, 2, 2, 600.0)
    n, m = si.degree_order_arrays(T)
    rng = np.random.default_rng(3)
    c = rng.standard_normal(o.grid.ncoef) + 1j * rng.standard_normal(o.grid.ncoef)
    c[m == 0] = c[m == 0].real
    grid = to_numpy(s.spec_to_grid(_cuda(c)))
    ref = o.grid.spec_to_grid(c)
    assert np.max(np.abs(grid - ref)) <= 1e-13 * np.max(np.abs(ref))
    f = rng.standard_normal((J, L))
    spec = to_numpy(s.grid_to_spec(torch.from_numpy(f).to("cuda")))
    ref = o.grid.grid_to_spec(f)
    assert np.max(np.abs(spec - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_grid_and_collocation_data_match_oracle():
    T, J, L = 127, 192, 384
    s = _solver(T, J, L, 4, 4, 300.0)
    mu, w = s.grid_coords()
    omu, ow = sht.gauss_grid(J)
    np.testing.assert_allclose(mu, omu, atol=2e-16)
    np.testing.assert_allclose(w, ow, rtol=2e-12)
    for M in range(1, 9):
        sm = _solver(5, 8, 16, M, 2, 100.0)
        tau, Q = sm.collocation()
        c = osdc.Collocation(M)
        np.testing.assert_allclose(tau, c.tau, atol=1e-15)
        np.testing.assert_allclose(Q, c.Q, atol=1e-14)


@pytest.mark.parametrize("M,K", [(3, 3), (4, 5), (1, 1), (2, 4), (8, 2)])
def test_one_step_and_residuals_match_oracle(M, K):
    T, J, L = 21, 34, 72
    o = _oracle(T, J, L)
    wl = _wl(T, J, L, M, K, 600.0)
    u0 = swe.initial_state(wl, o)
    res = []
    ref = osdc.swe_step(o, u0, osdc.Collocation(M), K, 600.0, residuals=res)
    s = _solver(T, J, L, M, K, 600.0)
    out, r = s.step(_cuda(u0), residuals=True)
    assert np.all(rel_l2(to_numpy(out), ref) <= TOL_EVAL * 10)
    np.testing.assert_allclose(r, np.stack(res), rtol=1e-10)


@pytest.mark.parametrize("rule", ["literal", "min-sr-ns", "ie", "min-sr-s"])
def test_qdelta_rules_match_oracle(rule):
    import paper_2403_20135_gb300 as pkg
    code = {"literal": pkg.SDC_QDELTA_LITERAL, "min-sr-ns": pkg.SDC_QDELTA_MIN_SR_NS,
            "ie": pkg.SDC_QDELTA_IMPLICIT_EULER, "min-sr-s": pkg.SDC_QDELTA_MIN_SR_S}[rule]
    T, J, L, M, K = 21, 34, 72, 3, 5
    o = _oracle(T, J, L)
    u0 = swe.initial_state(_wl(T, J, L, M, K), o)
    ref = osdc.swe_step(o, u0, osdc.Collocation(M, rule), K, 600.0)
    clamped = osdc.swe_step(o, u0, osdc.Collocation(M, "clamped"), K, 600.0)
    s = _solver(T, J, L, M, K, 600.0, qdelta_rule=code)
    out, r = s.step(_cuda(u0), residuals=True)
    res = []
    osdc.swe_step(o, u0, osdc.Collocation(M, rule), K, 600.0, residuals=res)
    got = to_numpy(out)
    assert np.all(rel_l2(got, ref) <= TOL_EVAL * 10)
    res = np.stack(res)
    # late sweeps of the fast-converging rules reach residuals near the rounding
    # level of the state: per field, an absolute floor of 1e-12 x the first sweep's
    assert np.all(np.abs(r - res) <= 1e-10 * np.abs(res) + 1e-12 * res[0]), (r, res)
    assert np.any(rel_l2(got, clamped) > 1e-9)          # the rules differ


def test_qdelta_rule_switch_and_bad_value():
    import paper_2403_20135_gb300 as pkg
    from paper_2403_20135_gb300 import _lib
    T, J, L, M, K = 21, 34, 72, 3, 3
    o = _oracle(T, J, L)
    u0 = swe.initial_state(_wl(T, J, L, M, K), o)
    s = _solver(T, J, L, M, K, 600.0)
    first = to_numpy(s.step(_cuda(u0)))                  # captures the default graph
    assert s.lib.sdc_set_option(s.h, _lib.SDC_OPT_QDELTA_RULE, 7) == _lib.SDC_EINVAL
    s.set_qdelta_rule(pkg.SDC_QDELTA_MIN_SR_NS)
    got = to_numpy(s.step(_cuda(u0)))
    ref = osdc.swe_step(o, u0, osdc.Collocation(M, "min-sr-ns"), K, 600.0)
    assert np.all(rel_l2(got, ref) <= TOL_EVAL * 10)
    s.set_qdelta_rule(pkg.SDC_QDELTA_CLAMPED)
    np.testing.assert_array_equal(to_numpy(s.step(_cuda(u0))), first)


def test_t31_workload_full_run():
    """The T31 48x96 workload, M=3, K=3, dt=600 s, all 20 steps."""
    wl = si.WORKLOADS["t31"]
    o = _oracle(wl.T, wl.nlat, wl.nlon)
    u0 = swe.initial_state(wl, o)
    ref = osdc.swe_run(o, u0, osdc.Collocation(wl.nodes), wl.sweeps, wl.dt, wl.nsteps)
    s = _solver(wl.T, wl.nlat, wl.nlon, wl.nodes, wl.sweeps, wl.dt)
    got = to_numpy(s.run(_cuda(u0), wl.nsteps))
    err = rel_l2(got, ref)
    assert np.all(err <= TOL_RUN), err


def test_t127_workload_first_steps():
    """The T127 192x384 workload (M=4, K=4, dt=300 s), first 5 steps."""
    wl = si.WORKLOADS["t127"]
    o = _oracle(wl.T, wl.nlat, wl.nlon)
    u0 = swe.initial_state(wl, o)
    ref = osdc.swe_run(o, u0, osdc.Collocation(wl.nodes), wl.sweeps, wl.dt, 5)
    s = _solver(wl.T, wl.nlat, wl.nlon, wl.nodes, wl.sweeps, wl.dt)
    got = to_numpy(s.run(_cuda(u0), 5))
    assert np.all(rel_l2(got, ref) <= TOL_RUN)


def test_t255_workload_one_step():
    """The benchmarked T255 384x768 workload (M=4, K=5, dt=150 s): one full step
    in the launch configuration the benchmark times, against the oracle."""
    wl = si.WORKLOADS["t255"]
    o = _oracle(wl.T, wl.nlat, wl.nlon)
    u0 = swe.initial_state(wl, o)
    ref = osdc.swe_step(o, u0, osdc.Collocation(wl.nodes), wl.sweeps, wl.dt)
    s = _solver(wl.T, wl.nlat, wl.nlon, wl.nodes, wl.sweeps, wl.dt)
    st = _cuda(u0)
    got = to_numpy(s.run(st, 1))
    assert np.all(rel_l2(got, ref) <= TOL_RUN)


def test_t255_steady_zonal_flow_and_mass():
    """At the benchmarked size: a balanced zonal flow stays fixed and the mean
    height is conserved to rounding over 10 steps (properties at any size)."""
    wl = si.WORKLOADS["t255"]
    s = _solver(wl.T, wl.nlat, wl.nlon, wl.nodes, wl.sweeps, wl.dt)
    a, om, u0 = si.RADIUS, si.OMEGA, 20.0
    st = s.empty_state()
    st[1, 1] = 2 * u0 / a / math.sqrt(1.5)
    c = -(a * om * u0 + u0 ** 2 / 2)
    st[0, 2] = c * (2.0 / 3.0) / math.sqrt(2.5)
    ref = st.clone()
    s.run(st, 10)
    d = (st - ref).abs().amax(dim=1).cpu().numpy()
    scale = ref.abs().amax(dim=1).cpu().numpy()
    scale[2] = scale[1]
    assert np.all(d <= 1e-12 * scale), (d, scale)
    # mass: the (0,0) coefficient of Phi' of a seeded state
    o_mu, _ = s.grid_coords()
    x = s.initial_state(wl)
    m0 = x[0, 0].item()
    s.run(x, 10)
    assert abs(x[0, 0].item() - m0) <= 1e-13 * abs(m0) + 1e-9
    assert abs(x[2, 0].item()) < 1e-18


def test_zero_steps_and_counters():
    T, J, L, M, K = 21, 34, 72, 4, 3
    s = _solver(T, J, L, M, K, 300.0)
    o = _oracle(T, J, L)
    u0 = _cuda(swe.initial_state(_wl(T, J, L, M, K), o))
    before = u0.clone()
    s.run(u0, 0)
    assert torch.equal(u0, before)
    e0, s0, _ = s.counters()
    s.run(u0, 3)
    e1, s1, l1 = s.counters()
    assert e1 - e0 == 3 * (1 + (K - 1) * M)          # Table 1
    assert s1 - s0 == 3 * ((K - 1) * M + 1)
    # E0 (one state, 3 kernels), K - 1 batches of M states split into two
    # concurrent chains of 3 kernels each, and K sweeps (epilogue inside)
    assert s.launches_per_step() == 3 + 6 * (K - 1) + K
    s.set_chains(1)
    assert s.launches_per_step() == 4 * K             # K tendency batches x 3 kernels + K sweeps


def test_invalid_shapes_raise():
    s = _solver(21, 34, 72, 3, 3, 300.0)
    with pytest.raises(ValueError):
        s.step(torch.zeros((3, 10), dtype=torch.complex128, device="cuda"))
    with pytest.raises(ValueError):
        s.tendency(torch.zeros((4, 3, s.ncoef), dtype=torch.complex128, device="cuda")[:, :, :5])
    from paper_2403_20135_gb300 import SdcError
    with pytest.raises(SdcError):
        s.tendency(torch.zeros((4, 3, s.ncoef), dtype=torch.complex128, device="cuda"))


def test_nan_state_reports_divergence_and_context_stays_usable():
    """Failure injected on the host: a NaN coefficient in the input state makes the
    residual norms non-finite, sdc_step (residuals requested) returns
    SDC_EDIVERGED, and the next step of a good state is unaffected."""
    from paper_2403_20135_gb300 import SdcError
    from paper_2403_20135_gb300._lib import SDC_EDIVERGED
    T, J, L, M, K = 21, 34, 72, 3, 3
    o = _oracle(T, J, L)
    u0 = swe.initial_state(_wl(T, J, L, M, K), o)
    bad = u0.copy()
    bad[1, 7] = complex(np.nan, 0.0)
    s = _solver(T, J, L, M, K, 600.0)
    with pytest.raises(SdcError) as err:
        s.step(_cuda(bad), residuals=True)
    assert err.value.status == SDC_EDIVERGED
    got = to_numpy(s.step(_cuda(u0), residuals=True)[0])
    ref = osdc.swe_step(o, u0, osdc.Collocation(M), K, 600.0)
    assert np.all(rel_l2(got, ref) <= TOL_EVAL * 10)
