"""The largest combined form at full size: T511 on a 768 x 1536 Gauss grid,
M = 4, K = 5, dt = 75 s (GPU only).  No oracle run at this size (too slow);
the checks are properties that hold at any size and comparisons between the
GPU's own precisions:

* every mixed mode stays within the rounding bound of the mixed tests at
  T = 511 (per tendency, times the number of steps) of the FP64 run;
* the global mean of Phi' (the (0, 0) coefficient) is conserved to rounding;
* the checkpointed adjoint with 16 snapshots recomputes exactly the optimal
  binomial number of forward steps, and its gradient agrees with a central
  finite difference along a seeded direction.
"""
import numpy as np
import pytest

import swe_inputs as si
from tests.helpers import rel_l2, to_numpy
from tests.test_gpu_mixed import bound

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

WL = si.WORKLOADS["t511"]


def _solver(precision=0):
    from paper_2403_20135_gb300 import Solver
    return Solver.for_workload(WL, precision=precision)


def _dp_cost(n, s):
    from functools import lru_cache

    @lru_cache(maxsize=None)
    def C(n, s):
        if n <= 1:
            return 0
        if s == 0:
            return n * (n - 1) // 2
        return min(m + C(n - m, s - 1) + C(m, s) for m in range(1, n))
    return C(n, s)


def test_t511_precisions_and_mass():
    s64 = _solver()
    u0 = s64.initial_state(WL)
    ref = u0.clone()
    s64.run(ref, 2)
    s64.sync()
    mass0 = u0[0, 0].real.item()
    assert abs(ref[0, 0].real.item() - mass0) <= 1e-12 * abs(mass0) + 1e-9
    refn = to_numpy(ref)
    for prec in (1, 2, 3):
        sm = _solver(prec)
        x = u0.clone()
        sm.run(x, 2)
        sm.sync()
        err = rel_l2(to_numpy(x), refn)
        print(f"T511 precision {prec}: rel L2 vs FP64 after 2 steps {err}")
        assert np.all(err <= 2 * bound(prec, WL.T, WL.nlat, WL.nlon)), (prec, err)   # 2 steps
        sm.close()


def test_t511_checkpointed_adjoint():
    s = _solver()
    u0 = s.initial_state(WL)
    ub = torch.zeros_like(u0)
    ub[0] = 1.0
    nsteps, nsnap = 24, 16
    _, nfwd = s.run_adjoint(u0, nsteps, ub, nsnapshots=nsnap)
    assert nfwd == _dp_cost(nsteps, nsnap - 1)
    # gradient of the height misfit after 2 steps against a central difference
    dp, dz, dd = si.direction(WL, 0, si.PURPOSE_TARGET)
    up = u0.clone()
    up += 1e-3 * torch.from_numpy(np.stack([dp, dz, dd])).to("cuda")
    s.run(up, 2)
    target = si.MEAN_DEPTH + s.spec_to_grid(up[0].contiguous()) / si.GRAVITY
    loss, g = s.adjoint_run(u0, 2, target, nsnapshots=16)
    dp, dz, dd = si.direction(WL, 1)
    d = torch.from_numpy(np.stack([dp, dz, dd])).to("cuda")
    eps = 1e-6
    vals = []
    for sign in (1.0, -1.0):
        x = u0 + sign * eps * d
        s.run(x, 2)
        h = si.MEAN_DEPTH + s.spec_to_grid(x[0].contiguous()) / si.GRAVITY
        vals.append(0.5 * float(((h - target) ** 2).sum()))
    fd = (vals[0] - vals[1]) / (2 * eps)
    an = float(torch.real(torch.vdot(g.flatten(), d.flatten())))
    assert abs(fd - an) <= 1e-6 * abs(fd), (fd, an)


def test_t511_fp32_step_adjoint_close_to_fp64():
    """The FP32-mode reversed step at T511 (transposed transforms in FP32 on the
    state-batched kernels) against the FP64 reversed step, same seeded state and
    seed u-bar, within the FP32 per-tendency bound at this truncation."""
    u0 = _solver().initial_state(WL)
    ub = u0 / (u0.abs() ** 2).sum(dim=1, keepdim=True)   # each field weighted by its own scale
    ref = to_numpy(_solver(0).step_adjoint(u0, ub))
    got = to_numpy(_solver(1).step_adjoint(u0, ub))
    err = rel_l2(got, ref)
    assert np.all(err <= bound(1, WL.T, WL.nlat, WL.nlon)), err


def test_t511_tensor_core_five_states():
    """Five node states at T511 in the 3-piece mode (64 projection and 48
    synthesis columns per tile, the longest groups).  The batch's tendencies
    against the FP64 context's, within the per-tendency bound."""
    from paper_2403_20135_gb300 import Solver
    s64 = Solver(WL.T, WL.nlat, WL.nlon, 5, 3, WL.dt, si.RADIUS, si.OMEGA, si.GRAVITY, si.MEAN_DEPTH, precision=0)
    u0 = s64.initial_state(WL)
    batch = torch.stack([u0 * f for f in (0.5, 0.75, 1.0, 1.5, 2.0)]).contiguous()
    ref = to_numpy(s64.tendency(batch))
    s64.close()
    sm = Solver(WL.T, WL.nlat, WL.nlon, 5, 3, WL.dt, si.RADIUS, si.OMEGA, si.GRAVITY, si.MEAN_DEPTH, precision=3)
    got = to_numpy(sm.tendency(batch))
    sm.sync()
    for b in range(5):
        err = rel_l2(got[b], ref[b])
        assert np.all(err <= bound(3, WL.T, WL.nlat, WL.nlon)), (b, err)


def test_t511_fp32_chains_equal_one_chain():
    """Two state chains at the largest size, where the FP32 Legendre table
    (202 MB) streams from HBM: steps and reversed steps equal the one-chain
    results bit for bit."""
    a = _solver(1)
    b = _solver(1)
    a.set_chains(1)
    b.set_chains(2)
    u0 = a.initial_state(WL)
    np.testing.assert_array_equal(to_numpy(a.run(u0.clone(), 2)), to_numpy(b.run(u0.clone(), 2)))
    ub = torch.ones_like(u0)
    np.testing.assert_array_equal(to_numpy(a.step_adjoint(u0, ub)), to_numpy(b.step_adjoint(u0, ub)))
