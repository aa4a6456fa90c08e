"""The paper's reference integrators on the GPU against the oracle (GPU only):
serial IMEX SDC (Algorithm 1, Eq. (6)) and IMEX-o2 (Sec. 3.2), selected with
SDC_OPT_METHOD on the same context as dSDC and sharing its T_E kernels."""
import numpy as np
import pytest

import swe_inputs as si
from oracle import integrators as oi
from oracle import sdc as osdc
from oracle import sht, swe
from tests.helpers import rel_l2, to_numpy

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-11


def _setup(T, J, L, M, K, dt, method, precision=0):
    from paper_2403_20135_gb300 import Solver
    o = swe.SWE(sht.Grid(T, J, L), swe.default_physics())
    wl = si.Workload("r", 0, T, J, L, M, K, dt, 1, 1, (100.0, 100.0))
    u = swe.initial_state(wl, o)
    s = Solver(T, J, L, M, K, dt, si.RADIUS, si.OMEGA, si.GRAVITY, si.MEAN_DEPTH, precision=precision,
               method=method)
    return o, u, s


def _cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda")


@pytest.mark.parametrize("T,J,L,M,K", [(21, 34, 72, 3, 3), (31, 48, 96, 4, 5), (21, 34, 72, 2, 1)])
def test_serial_sdc_matches_oracle(T, J, L, M, K):
    from paper_2403_20135_gb300 import SDC_METHOD_SERIAL_SDC
    o, u, s = _setup(T, J, L, M, K, 600.0, SDC_METHOD_SERIAL_SDC)
    ref = oi.swe_imex_sdc_run(o, u, osdc.Collocation(M), K, 600.0, 2)
    got = to_numpy(s.run(_cuda(u), 2))
    s.sync()
    assert np.all(rel_l2(got, ref) <= TOL), rel_l2(got, ref)
    ev, sol, _ = s.counters()
    assert ev == 2 * K * M and sol == 2 * K * M
    assert s.launches_per_step() == 5 * K * M          # E0 + K M node kernels + (K M - 1) tendencies


@pytest.mark.parametrize("M,K", [(3, 3), (4, 5)])
def test_serial_sdc_lu_weights_match_oracle(M, K):
    """Serial IMEX SDC with the LU implicit weights (SDC_OPT_SERIAL_IMPLICIT)
    against the oracle, and the two weight choices give different steps."""
    from paper_2403_20135_gb300 import SDC_METHOD_SERIAL_SDC, SDC_SERIAL_IMPLICIT_EULER, SDC_SERIAL_IMPLICIT_LU
    T, J, L = 21, 34, 72
    o, u, s = _setup(T, J, L, M, K, 600.0, SDC_METHOD_SERIAL_SDC)
    s.set_serial_implicit(SDC_SERIAL_IMPLICIT_LU)
    ref = oi.swe_imex_sdc_run(o, u, osdc.Collocation(M), K, 600.0, 2, implicit="lu")
    got = to_numpy(s.run(_cuda(u), 2))
    s.sync()
    assert np.all(rel_l2(got, ref) <= TOL), rel_l2(got, ref)
    s.set_serial_implicit(SDC_SERIAL_IMPLICIT_EULER)
    euler = to_numpy(s.run(_cuda(u), 2))
    assert np.any(rel_l2(euler, got) > 1e-9)


@pytest.mark.parametrize("T,J,L", [(21, 34, 72), (31, 48, 96)])
def test_imex2_matches_oracle(T, J, L):
    from paper_2403_20135_gb300 import SDC_METHOD_IMEX2
    o, u, s = _setup(T, J, L, 4, 4, 300.0, SDC_METHOD_IMEX2)
    ref = oi.swe_imex2_run(o, u, 300.0, 4)
    got = to_numpy(s.run(_cuda(u), 4))
    s.sync()
    assert np.all(rel_l2(got, ref) <= TOL), rel_l2(got, ref)
    assert s.launches_per_step() == 11
    ev, sol, _ = s.counters()
    assert ev == 8 and sol == 8


def test_switching_methods_on_one_context():
    from paper_2403_20135_gb300 import SDC_METHOD_DSDC, SDC_METHOD_IMEX2, SDC_METHOD_SERIAL_SDC
    T, J, L, M, K, dt = 21, 34, 72, 3, 3, 600.0
    o, u, s = _setup(T, J, L, M, K, dt, SDC_METHOD_DSDC)
    coll = osdc.Collocation(M)
    refs = {SDC_METHOD_DSDC: osdc.swe_run(o, u, coll, K, dt, 1),
            SDC_METHOD_SERIAL_SDC: oi.swe_imex_sdc_run(o, u, coll, K, dt, 1),
            SDC_METHOD_IMEX2: oi.swe_imex2_run(o, u, dt, 1)}
    for method in (SDC_METHOD_SERIAL_SDC, SDC_METHOD_IMEX2, SDC_METHOD_DSDC, SDC_METHOD_IMEX2):
        s.set_method(method)
        got = to_numpy(s.run(_cuda(u), 1))
        s.sync()
        assert np.all(rel_l2(got, refs[method]) <= TOL), (method, rel_l2(got, refs[method]))


def test_reference_methods_refuse_adjoint_and_residuals():
    from paper_2403_20135_gb300 import SDC_METHOD_SERIAL_SDC, SdcError
    o, u, s = _setup(21, 34, 72, 3, 3, 600.0, SDC_METHOD_SERIAL_SDC)
    x = _cuda(u)
    with pytest.raises(SdcError) as e:
        s.step(x, residuals=True)
    assert e.value.status == 6
    with pytest.raises(SdcError) as e:
        s.step_adjoint(x, torch.ones_like(x))
    assert e.value.status == 6
    with pytest.raises(SdcError):
        s.set_method(7)


@pytest.mark.parametrize("method", [1, 2])
def test_reference_methods_in_fp32(method):
    """The FP32 transforms serve the reference integrators too; after a few
    steps they stay within the FP32 tendency bound of the FP64 path."""
    T, J, L = 42, 64, 128
    o, u, s64 = _setup(T, J, L, 3, 3, 300.0, method)
    _, _, s32 = _setup(T, J, L, 3, 3, 300.0, method, precision=1)
    a = to_numpy(s64.run(_cuda(u), 3))
    b = to_numpy(s32.run(_cuda(u), 3))
    s32.sync()
    assert np.all(rel_l2(b, a) <= 1e-5), rel_l2(b, a)
