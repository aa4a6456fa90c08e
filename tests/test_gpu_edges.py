"""Edge cases of sizes and parameters on the GPU (GPU only): the smallest
truncations, the longest rings and the most latitudes the C ABI accepts, the
largest node count in the adjoint and the largest sweep count, each against
the oracle (FP64 bar) or the mixed-mode bound."""
import numpy as np
import pytest

import swe_inputs as si
from oracle import adjoint as oadj
from oracle import sdc as osdc
from oracle import sht, swe
from tests.helpers import rel_l2, to_numpy
from tests.test_gpu_mixed import bound

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_EVAL = 1e-12


def _solver(T, J, L, M=3, K=3, dt=600.0, precision=0):
    from paper_2403_20135_gb300 import Solver
    return Solver(T, J, L, M, K, dt, si.RADIUS, si.OMEGA, si.GRAVITY, si.MEAN_DEPTH, precision=precision)


def _state(T, J, L, M=3, K=3):
    o = swe.SWE(sht.Grid(T, J, L), swe.default_physics())
    return o, swe.initial_state(si.Workload("e", 0, T, J, L, M, K, 600.0, 1, 1, (100.0, 100.0)), o)


def _cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda")


@pytest.mark.parametrize("T,J,L", [(1, 2, 4), (2, 4, 8), (3, 6, 12)])
def test_smallest_truncations(T, J, L):
    o, u = _state(T, J, L)
    ref = o.explicit(u)
    s = _solver(T, J, L)
    assert np.all(rel_l2(to_numpy(s.tendency(_cuda(u))), ref) <= TOL_EVAL)
    got = to_numpy(s.run(_cuda(u), 2))
    s.sync()
    assert np.all(rel_l2(got, osdc.swe_run(o, u, osdc.Collocation(3), 3, 600.0, 2)) <= 1e-11)
    for prec in (1, 3):
        sm = _solver(T, J, L, precision=prec)
        err = rel_l2(to_numpy(sm.tendency(_cuda(u))), ref)
        sm.sync()
        assert np.all(err <= bound(prec, T, J, L)), (prec, err)


def test_longest_rings():
    from paper_2403_20135_gb300 import SdcError
    T, J = 21, 34
    o, u = _state(T, J, 2304)
    ref = o.explicit(u)
    with pytest.raises(SdcError) as e:
        _solver(T, J, 2304)                  # the FP64 ring stops at 2048 longitudes
    assert e.value.status == 6
    for prec in (1, 3):
        err = rel_l2(to_numpy(_solver(T, J, 2304, precision=prec).tendency(_cuda(u))), ref)
        assert np.all(err <= bound(prec, T, J, 2304)), (prec, err)
    o2, u2 = _state(T, J, 2048)
    assert np.all(rel_l2(to_numpy(_solver(T, J, 2048).tendency(_cuda(u2))), o2.explicit(u2)) <= TOL_EVAL)


def test_most_latitudes():
    T, J, L = 21, 2048, 64
    o, u = _state(T, J, L)
    ref = o.explicit(u)
    assert np.all(rel_l2(to_numpy(_solver(T, J, L).tendency(_cuda(u))), ref) <= TOL_EVAL)
    for prec in (1, 3):
        err = rel_l2(to_numpy(_solver(T, J, L, precision=prec).tendency(_cuda(u))), ref)
        assert np.all(err <= bound(prec, T, J, L)), (prec, err)


def test_eight_nodes_step_adjoint():
    T, J, L, M, K, dt = 10, 16, 32, 8, 3, 600.0
    o, u = _state(T, J, L, M, K)
    rng = np.random.default_rng(8)
    ub = rng.standard_normal(u.shape) + 1j * rng.standard_normal(u.shape)
    ub[:, :T + 1] = ub[:, :T + 1].real
    ref = oadj.swe_step_vjp(o, u, ub, osdc.Collocation(M), K, dt)
    got = to_numpy(_solver(T, J, L, M, K, dt).step_adjoint(_cuda(u), _cuda(ub)))
    assert np.all(rel_l2(got, ref) <= 1e-11), rel_l2(got, ref)


def test_most_sweeps():
    T, J, L, M, K = 5, 8, 16, 3, 64
    o, u = _state(T, J, L, M, K)
    ref = osdc.swe_run(o, u, osdc.Collocation(M), K, 600.0, 1)
    got = to_numpy(_solver(T, J, L, M, K).run(_cuda(u), 1))
    assert np.all(rel_l2(got, ref) <= 1e-11), rel_l2(got, ref)
