"""The seeded workloads at their stated run lengths, through the C ABI (GPU only).

* T127 on 192 x 384, M = 4, K = 4, dt = 300 s: 200 steps (Algorithm 2 iterated
  over the whole horizon) against the FP64 oracle, rel. L2 <= 1e-11 per field.
* T255 on 384 x 768, M = 4, K = 5, dt = 150 s: 20 steps against the oracle, in
  FP64 (<= 1e-11) and in every mixed mode (within the derived rounding bound);
  and the fixed-error criterion the precision form is judged by: after the
  500-step horizon the FP32 and 3-piece split-BF16 modes stay below that run's
  FP64 discretisation error (FP64 at dt against FP64 at dt/4, both on the GPU).
  Over 20 steps that discretisation error (7.6e-7 in vorticity) lies below the
  FP32 rounding floor, so the criterion is only meaningful over the horizon.
* T127 differentiation form, 96 steps with 8 snapshots: the gradient of the
  height misfit against central differences along 16 seeded directions
  (<= 1e-6), and the dot-product test of the whole step's adjoint,
  <w, J v> = <J^T w, v> to <= 1e-12, with J v taken exactly from the step's
  polynomial structure (below).
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

TOL_RUN = 1e-11
_ORACLE = {}


def _solver(wl, precision=0, dt=None):
    from paper_2403_20135_gb300 import Solver
    return Solver(wl.T, wl.nlat, wl.nlon, wl.nodes, wl.sweeps, wl.dt if dt is None else dt, si.RADIUS,
                  si.OMEGA, si.GRAVITY, si.MEAN_DEPTH, precision=precision)


def _cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda")


def _oracle_run(key, nsteps):
    """(initial state, oracle state after nsteps) of a seeded workload, computed once."""
    if (key, nsteps) not in _ORACLE:
        wl = si.WORKLOADS[key]
        o = swe.SWE(sht.Grid(wl.T, wl.nlat, wl.nlon), swe.default_physics())
        u0 = swe.initial_state(wl, o)
        u = osdc.swe_run(o, u0, osdc.Collocation(wl.nodes), wl.sweeps, wl.dt, nsteps)
        _ORACLE[(key, nsteps)] = (u0, u)
    return _ORACLE[(key, nsteps)]


def test_t127_workload_full_run_matches_oracle():
    wl = si.WORKLOADS["t127"]
    u0, ref = _oracle_run("t127", wl.nsteps)
    s = _solver(wl)
    got = to_numpy(s.run(_cuda(u0), wl.nsteps))
    s.sync()
    err = rel_l2(got, ref)
    print(f"T127 {wl.nsteps} steps: rel L2 per field (phi, zeta, div) {err}")
    assert np.all(err <= TOL_RUN), err
    # the global mean of h is conserved to rounding over the run
    assert abs(got[0, 0] - u0[0, 0]) <= 1e-13 * abs(u0[0, 0]) + 1e-10


T255_STEPS = 20


def _t255_fp64_increments():
    """Per field, the sum over the T255_STEPS FP64 steps (GPU) of the relative
    change of the state in one step, ||u_{k+1} - u_k|| / ||u_k||."""
    if "t255_incr" not in _ORACLE:
        wl = si.WORKLOADS["t255"]
        u0, _ = _oracle_run("t255", T255_STEPS)
        s = _solver(wl)
        x = _cuda(u0)
        prev = to_numpy(x)
        tot = np.zeros(3)
        for _ in range(T255_STEPS):
            s.run(x, 1)
            cur = to_numpy(x)
            tot += rel_l2(cur, prev)
            prev = cur
        _ORACLE["t255_incr"] = tot
    return _ORACLE["t255_incr"]


def test_t255_workload_fp64_matches_oracle():
    wl = si.WORKLOADS["t255"]
    u0, ref = _oracle_run("t255", T255_STEPS)
    s = _solver(wl)
    got = to_numpy(s.run(_cuda(u0), T255_STEPS))
    s.sync()
    err = rel_l2(got, ref)
    print(f"T255 FP64 {T255_STEPS} steps: rel L2 per field {err}")
    assert np.all(err <= TOL_RUN), err


@pytest.mark.parametrize("name,precision", [("fp32", 1), ("bf16x3", 2), ("bf16x6", 3)])
def test_t255_workload_mixed_modes_against_oracle(name, precision):
    """20 steps of each mixed mode against the oracle.  The bound: every step
    moves the state by its increment, which carries the tendencies' relative
    rounding error (the per-tendency bound of the mixed tests); over the run
    these add up to that bound times the summed relative increments."""
    from tests.test_gpu_mixed import bound
    wl = si.WORKLOADS["t255"]
    u0, ref = _oracle_run("t255", T255_STEPS)
    s = _solver(wl, precision)
    got = to_numpy(s.run(_cuda(u0), T255_STEPS))
    s.sync()
    err = rel_l2(got, ref)
    tol = bound(precision, wl.T, wl.nlat, wl.nlon) * np.maximum(1.0, _t255_fp64_increments())
    print(f"T255 {name} {T255_STEPS} steps: rel L2 vs oracle {err} (bound {tol})")
    assert np.all(np.isfinite(err))
    assert np.all(err <= tol), (err, tol)


HORIZON = si.WORKLOADS["t255"].nsteps


def _t255_horizon_fp64():
    """FP64 GPU state after the 500-step horizon, and the FP64 discretisation
    error there (FP64 at dt against FP64 at dt/4)."""
    if "t255_h" not in _ORACLE:
        wl = si.WORKLOADS["t255"]
        s = _solver(wl)
        u0 = s.initial_state(wl)
        a = to_numpy(s.run(u0.clone(), HORIZON))
        q = _solver(wl, dt=wl.dt / 4)
        b = to_numpy(q.run(u0.clone(), 4 * HORIZON))
        q.sync()
        _ORACLE["t255_h"] = (u0, a, rel_l2(a, b))
    return _ORACLE["t255_h"]


@pytest.mark.parametrize("name,precision", [("fp32", 1), ("bf16x6", 3)])
def test_t255_fixed_error_over_horizon(name, precision):
    """The precision form's accuracy gate: after the 500-step horizon a mixed
    mode's per-field error against the FP64 GPU path stays below that run's
    FP64 discretisation error.  (BF16x3 does not meet it and is not claimed to.)"""
    wl = si.WORKLOADS["t255"]
    u0, a, edisc = _t255_horizon_fp64()
    s = _solver(wl, precision)
    got = to_numpy(s.run(u0.clone(), HORIZON))
    s.sync()
    err = rel_l2(got, a)
    print(f"T255 {name} {HORIZON} steps: rel L2 vs FP64 {err}; FP64 discretisation error {edisc}")
    assert np.all(err < edisc), (err, edisc)


# ---------------------------------------------------------------------------
# differentiation form
# ---------------------------------------------------------------------------
def _rdot(a, b):
    return float(np.real(np.vdot(a, b)))


def test_differentiation_workload_sixteen_directions():
    """T127, M = 4, K = 4, dt = 300 s, 96 steps, 8 snapshots: the gradient of
    0.5 ||h(T) - h_target||^2 against central differences (eps = 1e-6 relative
    to the state's scale) along 16 seeded directions, rel. error <= 1e-6."""
    wl = si.WORKLOADS["t127adj"]
    s = _solver(wl)
    u0 = s.initial_state(wl)
    nsteps = wl.nsteps
    dp, dz, dd = si.direction(wl, 0, si.PURPOSE_TARGET)
    up = u0.clone()
    up += 1e-3 * _cuda(np.stack([dp, dz, dd]))
    s.run(up, nsteps)
    target = si.MEAN_DEPTH + s.spec_to_grid(up[0].contiguous()) / si.GRAVITY
    loss, g = s.adjoint_run(u0, nsteps, target, nsnapshots=8)
    gn = to_numpy(g)
    eps = 1e-6
    worst = 0.0
    for k in range(16):
        d = np.stack(si.direction(wl, k))
        vals = []
        for sign in (1.0, -1.0):
            x = u0 + sign * eps * _cuda(d)
            s.run(x, nsteps)
            h = si.MEAN_DEPTH + s.spec_to_grid(x[0].contiguous()) / si.GRAVITY
            vals.append(0.5 * float(((h - target) ** 2).sum()))
        fd = (vals[0] - vals[1]) / (2 * eps)
        rel = abs(fd - _rdot(gn, d)) / abs(fd)
        worst = max(worst, rel)
        assert rel <= 1e-6, (k, fd, _rdot(gn, d))
    print(f"differentiation form: 16 directions, worst rel. error {worst:.2e}")


def test_whole_step_dot_product():
    """<w, J v> = <J^T w, v> for one step of the differentiation workload.

    T_E is quadratic and each of the K sweeps evaluates it on the previous
    iterate, so one step is a polynomial of degree 2^K in the state.  Along a
    line u + eps v the odd part (f(u + eps v) - f(u - eps v)) / 2 is then an odd
    polynomial of degree < 2^K in eps, and its linear coefficient, J v, is fixed
    exactly by 2^(K-1) symmetric evaluations (here at the positive Chebyshev
    points of degree 2^K); only rounding separates it from the tangent."""
    wl = si.WORKLOADS["t127adj"]
    s = _solver(wl)
    u0 = s.initial_state(wl)
    un = to_numpy(u0)
    scale = np.abs(un).max(axis=1, keepdims=True)
    v = np.stack(si.direction(wl, 3))
    rng = np.random.default_rng(17)
    w = (rng.standard_normal(un.shape) + 1j * rng.standard_normal(un.shape)) / scale
    n, m = si.degree_order_arrays(wl.T)
    w[:, m == 0] = w[:, m == 0].real                      # m = 0 coefficients are real
    npts = 2 ** (wl.sweeps - 1)
    t = np.cos((2 * np.arange(1, npts + 1) - 1) * np.pi / (4 * npts))
    h = 0.05
    odd = []
    for ti in t:
        fp = to_numpy(s.run(u0 + h * ti * _cuda(v), 1))
        fm = to_numpy(s.run(u0 - h * ti * _cuda(v), 1))
        odd.append(0.5 * (fp - fm))
    V = np.stack([t ** (2 * k + 1) for k in range(npts)], axis=1)   # odd powers 1, 3, ..., 2^K - 1
    alpha = np.linalg.solve(V.T, np.eye(npts)[:, 0])                # c_1 = sum_i alpha_i odd(t_i)
    jv = sum(a * o for a, o in zip(alpha, odd)) / h
    jtw = to_numpy(s.step_adjoint(u0, _cuda(w)))
    lhs, rhs = _rdot(w, jv), _rdot(jtw, v)
    rel = abs(lhs - rhs) / abs(lhs)
    print(f"whole-step dot-product test: <w, Jv> = {lhs:.16e}, <J^T w, v> = {rhs:.16e}, rel {rel:.2e}")
    assert rel <= 1e-12, (lhs, rhs, rel)
