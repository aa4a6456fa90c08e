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


@pytest.mark.parametrize("T,J,L", [(15, 24, 48), (47, 72, 144)])
def test_odd_padded_ring_lengths(T, J, L):
    """Ring lengths whose padded length (one spare element per 16) is odd: 48
    and 144 longitudes give 51 and 153, so the FP32 ring kernels' second
    scratch array starts on an 8-byte boundary and their input copies and
    output staging take the 8-byte branches (generic pass plans; 48 = 16 x 3,
    144 = 16 x 9).  FP32 tendency and run against the oracle within the mixed
    bound, the FP32-mode adjoint against the FP64 one."""
    o, u = _state(T, J, L, M=4, K=4)
    ref = o.explicit(u)
    s32 = _solver(T, J, L, M=4, K=4, dt=300.0, precision=1)
    err = rel_l2(to_numpy(s32.tendency(_cuda(np.stack([u, 0.5 * u])))[0]), ref)
    assert np.all(err <= bound(1, T, J, L)), err
    s64 = _solver(T, J, L, M=4, K=4, dt=300.0)
    a = to_numpy(s64.run(_cuda(u), 3))
    b = to_numpy(s32.run(_cuda(u), 3))
    assert np.all(rel_l2(b, a) <= 30 * bound(1, T, J, L)), rel_l2(b, a)
    rng = np.random.default_rng(11)
    target = torch.from_numpy(o.height_grid(u) + rng.standard_normal((J, L))).to("cuda")
    ref_loss, ref_g = s64.adjoint_run(_cuda(u), 2, target, nsnapshots=2)
    loss, g = s32.adjoint_run(_cuda(u), 2, target, nsnapshots=2)
    s32.sync()
    assert abs(loss - ref_loss) <= 1e-5 * abs(ref_loss), (loss, ref_loss)
    assert np.all(rel_l2(to_numpy(g), to_numpy(ref_g)) <= 1e-5), rel_l2(to_numpy(g), to_numpy(ref_g))
