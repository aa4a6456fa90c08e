"""CUDA discrete adjoint against the oracle's adjoint and against
derivative-free checks, through the C ABI (GPU only).

* J_E^T against the oracle element by element, and the GPU dot-product test
  with the exact central-difference tangent of the quadratic T_E;
* the step adjoint against the oracle's;
* loss + gradient of the height misfit over several steps against the oracle,
  independent of the checkpoint budget, and against central finite
  differences at the T127 differentiation workload;
* the number of recomputed forward steps equals the optimal binomial
  checkpointing cost (computed here independently).
"""
import numpy as np
import pytest

import swe_inputs as si
from oracle import adjoint as oadj
from oracle import sdc as osdc
from oracle import sht, swe
from tests.helpers import rel_l2, to_numpy

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _solver(T, J, L, M, K, dt, precision=0, **kw):
    from paper_2403_20135_gb300 import Solver
    return Solver(T, J, L, M, K, dt, si.RADIUS, si.OMEGA, si.GRAVITY, si.MEAN_DEPTH, precision=precision, **kw)


def _oracle(T, J, L):
    return swe.SWE(sht.Grid(T, J, L), swe.default_physics())


def _cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda")


def _rand(shape, rng):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def rdot(a, b):
    return float(np.real(np.vdot(a, b)))


@pytest.mark.parametrize("T,J,L", [(21, 34, 72), (31, 48, 96), (63, 100, 192)])
def test_tendency_adjoint_matches_oracle(T, J, L):
    o = _oracle(T, J, L)
    wl = si.Workload("a", 0, T, J, L, 3, 3, 600.0, 1, 1, (100.0, 100.0))
    u = swe.initial_state(wl, o)
    rng = np.random.default_rng(T)
    a = _rand(u.shape, rng)
    a[:, :T + 1] = a[:, :T + 1].real
    ref = oadj.explicit_vjp(o, u, a)
    s = _solver(T, J, L, 3, 3, 600.0)
    got = to_numpy(s.tendency_adjoint(_cuda(u), _cuda(a)))
    assert np.all(rel_l2(got, ref) <= 1e-12), rel_l2(got, ref)


def test_tendency_adjoint_dot_product_on_gpu():
    T, J, L = 42, 64, 128
    o = _oracle(T, J, L)
    wl = si.Workload("a", 1, T, J, L, 4, 3, 600.0, 1, 1, (100.0, 100.0))
    u = swe.initial_state(wl, o)
    rng = np.random.default_rng(3)
    v = _rand(u.shape, rng) * np.abs(u).max(axis=1, keepdims=True)
    w = _rand(u.shape, rng)
    s = _solver(T, J, L, 4, 3, 600.0)
    batch = _cuda(np.stack([u + v, u - v]))
    te = to_numpy(s.tendency(batch))
    jv = (te[0] - te[1]) / 2.0                     # exact tangent of the quadratic T_E
    jtw = to_numpy(s.tendency_adjoint(_cuda(u), _cuda(w)))
    lhs, rhs = rdot(w, jv), rdot(jtw, v)
    assert abs(lhs - rhs) <= 1e-11 * abs(lhs)


@pytest.mark.parametrize("M,K", [(3, 3), (4, 5), (1, 1), (2, 4)])
def test_step_adjoint_matches_oracle(M, K):
    T, J, L = 21, 34, 72
    o = _oracle(T, J, L)
    wl = si.Workload("a", 0, T, J, L, M, K, 600.0, 1, 1, (100.0, 100.0))
    u = swe.initial_state(wl, o)
    rng = np.random.default_rng(M + 7 * K)
    ub = _rand(u.shape, rng)
    ref = oadj.swe_step_vjp(o, u, ub, osdc.Collocation(M), K, 600.0)
    s = _solver(T, J, L, M, K, 600.0)
    got = to_numpy(s.step_adjoint(_cuda(u), _cuda(ub)))
    assert np.all(rel_l2(got, ref) <= 1e-11), rel_l2(got, ref)


@pytest.mark.parametrize("rule", ["min-sr-ns", "ie", "min-sr-s"])
def test_step_adjoint_other_qdelta_rules(rule):
    import paper_2403_20135_gb300 as pkg
    code = {"min-sr-ns": pkg.SDC_QDELTA_MIN_SR_NS, "ie": pkg.SDC_QDELTA_IMPLICIT_EULER,
            "min-sr-s": pkg.SDC_QDELTA_MIN_SR_S}[rule]
    T, J, L, M, K = 21, 34, 72, 3, 4
    o = _oracle(T, J, L)
    wl = si.Workload("a", 0, T, J, L, M, K, 600.0, 1, 1, (100.0, 100.0))
    u = swe.initial_state(wl, o)
    ub = _rand(u.shape, np.random.default_rng(11))
    ref = oadj.swe_step_vjp(o, u, ub, osdc.Collocation(M, rule), K, 600.0)
    s = _solver(T, J, L, M, K, 600.0, qdelta_rule=code)
    got = to_numpy(s.step_adjoint(_cuda(u), _cuda(ub)))
    assert np.all(rel_l2(got, ref) <= 1e-11), rel_l2(got, ref)


def _dp_cost(n, s):
    """Independent evaluation of the optimal checkpointing cost (memoised recursion)."""
    from functools import lru_cache

    @lru_cache(maxsize=None)
    def C(n, s):
        if n <= 1:
            return 0
        if s == 0:
            return n * (n - 1) // 2
        return min(m + C(n - m, s - 1) + C(m, s) for m in range(1, n))
    return C(n, s)


def test_loss_gradient_matches_oracle_any_checkpoint_budget():
    wl = si.WORKLOADS["t31"]
    o = _oracle(wl.T, wl.nlat, wl.nlon)
    u0 = swe.initial_state(wl, o)
    rng = np.random.default_rng(11)
    target = o.height_grid(u0) + rng.standard_normal((wl.nlat, wl.nlon))
    nsteps = 6
    loss_ref, grad_ref = oadj.loss_and_gradient(o, u0, osdc.Collocation(wl.nodes), wl.sweeps, wl.dt, nsteps, target)
    s = _solver(wl.T, wl.nlat, wl.nlon, wl.nodes, wl.sweeps, wl.dt)
    ht = torch.from_numpy(target).to("cuda")
    grads = []
    for nsnap in (1, 2, 3, 32):
        loss, g = s.adjoint_run(_cuda(u0), nsteps, ht, nsnapshots=nsnap)
        assert abs(loss - loss_ref) <= 1e-11 * abs(loss_ref)
        assert np.all(rel_l2(to_numpy(g), grad_ref) <= 1e-10), rel_l2(to_numpy(g), grad_ref)
        grads.append(to_numpy(g))
        ub = torch.zeros_like(_cuda(u0))
        _, nfwd = s.run_adjoint(_cuda(u0), nsteps, ub, nsnapshots=nsnap)
        assert nfwd == _dp_cost(nsteps, nsnap - 1)
    for g in grads[1:]:
        np.testing.assert_array_equal(g, grads[0])      # the schedule changes no arithmetic


def test_zero_steps_loss_gradient():
    T, J, L = 21, 34, 72
    o = _oracle(T, J, L)
    wl = si.Workload("a", 0, T, J, L, 3, 3, 600.0, 1, 1, (100.0, 100.0))
    u0 = swe.initial_state(wl, o)
    target = o.height_grid(u0) * 0.99
    s = _solver(T, J, L, 3, 3, 600.0)
    loss, g = s.adjoint_run(_cuda(u0), 0, torch.from_numpy(target).to("cuda"), 1)
    assert abs(loss - oadj.height_loss(o, u0, target)) <= 1e-12 * loss
    assert np.all(rel_l2(to_numpy(g)[:1], oadj.height_loss_seed(o, u0, target)[:1]) <= 1e-12)


def test_differentiation_workload_finite_differences():
    """T127 192x384, M=4, K=4, dt=300 s (the differentiation workload), 8 steps,
    4 snapshots: central differences along 4 seeded directions, rel. err <= 1e-6."""
    wl = si.WORKLOADS["t127adj"]
    s = _solver(wl.T, wl.nlat, wl.nlon, wl.nodes, wl.sweeps, wl.dt)
    u0 = s.initial_state(wl)
    nsteps = 8
    # target: the run of a perturbed initial state
    dp, dz, dd = si.direction(wl, 0, si.PURPOSE_TARGET)
    up = u0.clone()
    up += 1e-3 * torch.from_numpy(np.stack([dp, dz, dd])).to("cuda")
    s.run(up, nsteps)
    target = si.MEAN_DEPTH + s.spec_to_grid(up[0].contiguous()) / si.GRAVITY
    loss, g = s.adjoint_run(u0, nsteps, target, nsnapshots=4)
    gn = to_numpy(g)
    for k in range(4):
        dp, dz, dd = si.direction(wl, k)
        d = np.stack([dp, dz, dd])
        eps = 1e-6
        vals = []
        for sign in (1.0, -1.0):
            x = u0 + sign * eps * _cuda(d)
            s.run(x, nsteps)
            h = si.MEAN_DEPTH + s.spec_to_grid(x[0].contiguous()) / si.GRAVITY
            vals.append(0.5 * float(((h - target) ** 2).sum()))
        fd = (vals[0] - vals[1]) / (2 * eps)
        assert abs(fd - rdot(gn, d)) <= 1e-6 * abs(fd), (k, fd, rdot(gn, d))


def test_autograd_function():
    from paper_2403_20135_gb300.autograd import height_loss, sdc_run
    T, J, L = 21, 34, 72
    o = _oracle(T, J, L)
    wl = si.Workload("a", 0, T, J, L, 3, 3, 600.0, 1, 1, (100.0, 100.0))
    u0 = swe.initial_state(wl, o)
    target = o.height_grid(u0) * 0.999
    s = _solver(T, J, L, 3, 3, 600.0)
    x = _cuda(u0).requires_grad_(True)
    loss = height_loss(x, s, 4, torch.from_numpy(target).to("cuda"), 2)
    loss.backward()
    _, gref = oadj.loss_and_gradient(o, u0, osdc.Collocation(3), 3, 600.0, 4, target)
    assert np.all(rel_l2(to_numpy(x.grad), gref) <= 1e-10)
    # SdcRun: gradient of a linear functional of the final state
    x2 = _cuda(u0).requires_grad_(True)
    y = sdc_run(x2, s, 3, 2)
    rng = np.random.default_rng(5)
    wv = _cuda(_rand(u0.shape, rng))
    (y.real * wv.real + y.imag * wv.imag).sum().backward()
    ref = u0 * 0
    ub = to_numpy(wv)
    states = [u0]
    for _ in range(3):
        states.append(osdc.swe_step(o, states[-1], osdc.Collocation(3), 3, 600.0))
    for n in range(2, -1, -1):
        ub = oadj.swe_step_vjp(o, states[n], ub, osdc.Collocation(3), 3, 600.0)
    assert np.all(rel_l2(to_numpy(x2.grad), ub) <= 1e-10)
