"""Programmatic dependent launch in the step graphs (SDC_OPT_PDL) changes when
a kernel is scheduled, not what it computes: every kernel waits for its
predecessors' completion before it touches their results, so steps, steps
with residuals, retaped steps and reversed steps equal the results without
it bit for bit, in every precision and with one or two chains (GPU only)."""
import numpy as np
import pytest

import swe_inputs as si
from tests.helpers import to_numpy

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _pair(wl, precision, chains):
    from paper_2403_20135_gb300 import Solver
    a = Solver.for_workload(wl, precision=precision)
    b = Solver.for_workload(wl, precision=precision)
    a.set_chains(chains)
    b.set_chains(chains)
    a.set_pdl(0)
    b.set_pdl(1)
    return a, b


@pytest.mark.parametrize("precision,chains", [(0, 1), (0, 2), (1, 1), (1, 2), (2, 1), (3, 1)])
def test_pdl_equals_serial_launches(precision, chains):
    wl = si.Workload("p", 2, 63, 100, 192, 4, 4, 300.0, 1, 1, (100.0, 100.0))
    a, b = _pair(wl, precision, chains)
    u0 = a.initial_state(wl)
    np.testing.assert_array_equal(to_numpy(a.run(u0.clone(), 3)), to_numpy(b.run(u0.clone(), 3)))
    ra, rb = a.step(u0.clone(), residuals=True)[1], b.step(u0.clone(), residuals=True)[1]
    np.testing.assert_array_equal(np.asarray(ra), np.asarray(rb))
    if precision <= 1:
        ub = torch.ones_like(u0)
        np.testing.assert_array_equal(to_numpy(a.step_adjoint(u0, ub)), to_numpy(b.step_adjoint(u0, ub)))


def test_pdl_other_integrators_and_odd_nodes():
    from paper_2403_20135_gb300 import SDC_METHOD_IMEX2, SDC_METHOD_SERIAL_SDC
    wl = si.Workload("p", 2, 31, 48, 96, 3, 3, 600.0, 1, 1, (100.0, 100.0))
    a, b = _pair(wl, 1, 2)
    u0 = a.initial_state(wl)
    np.testing.assert_array_equal(to_numpy(a.run(u0.clone(), 2)), to_numpy(b.run(u0.clone(), 2)))
    for method in (SDC_METHOD_SERIAL_SDC, SDC_METHOD_IMEX2):
        a.set_method(method)
        b.set_method(method)
        np.testing.assert_array_equal(to_numpy(a.run(u0.clone(), 2)), to_numpy(b.run(u0.clone(), 2)))


def test_pdl_option_errors():
    from paper_2403_20135_gb300 import SdcError, Solver
    s = Solver(21, 34, 72, 3, 3, 600.0, si.RADIUS, si.OMEGA, si.GRAVITY, si.MEAN_DEPTH)
    for bad in (-1, 2):
        with pytest.raises(SdcError) as e:
            s.set_pdl(bad)
        assert e.value.status == 1


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_multi_step_graph_equals_single_steps(precision):
    """sdc_run captures four steps per graph for long runs (the remainder runs
    on the one-step graph): nine steps in one call equal nine one-step calls
    bit for bit."""
    from paper_2403_20135_gb300 import Solver
    wl = si.Workload("p", 2, 31, 48, 96, 3, 3, 600.0, 1, 1, (100.0, 100.0))
    s = Solver.for_workload(wl, precision=precision)
    u0 = s.initial_state(wl)
    a = to_numpy(s.run(u0.clone(), 9))
    x = u0.clone()
    for _ in range(9):
        s.run(x, 1)
    np.testing.assert_array_equal(a, to_numpy(x))
