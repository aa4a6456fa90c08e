"""Concurrent state chains per tendency batch (SDC_OPT_CHAINS = 2 to 4) change
the schedule, not the arithmetic: steps and reversed steps equal the one-chain
results bit for bit, also where the batch splits unevenly (GPU only)."""
import numpy as np
import pytest

import swe_inputs as si
from tests.helpers import to_numpy

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,chains", [(0, 2), (1, 2), (0, 4), (1, 3), (1, 4)])
def test_chains_equal_one_chain(precision, chains):
    from paper_2403_20135_gb300 import Solver
    wl = si.Workload("c", 2, 63, 100, 192, 4, 4, 300.0, 1, 1, (100.0, 100.0))
    s1 = Solver.for_workload(wl, precision=precision)
    s1.set_chains(1)
    s2 = Solver.for_workload(wl, precision=precision)
    s2.set_chains(chains)
    u0 = s1.initial_state(wl)
    a = to_numpy(s1.run(u0.clone(), 3))
    b = to_numpy(s2.run(u0.clone(), 3))
    np.testing.assert_array_equal(a, b)
    ub = torch.ones_like(u0)
    np.testing.assert_array_equal(to_numpy(s1.step_adjoint(u0, ub)), to_numpy(s2.step_adjoint(u0, ub)))
    # an odd node count splits the batch unevenly
    wl3 = si.Workload("c", 2, 31, 48, 96, 3, 3, 600.0, 1, 1, (100.0, 100.0))
    t1 = Solver.for_workload(wl3, precision=precision)
    t1.set_chains(1)
    t2 = Solver.for_workload(wl3, precision=precision)
    t2.set_chains(chains)
    v0 = t1.initial_state(wl3)
    np.testing.assert_array_equal(to_numpy(t1.run(v0.clone(), 2)), to_numpy(t2.run(v0.clone(), 2)))


def test_chains_option_errors():
    from paper_2403_20135_gb300 import SdcError, Solver
    s = Solver(21, 34, 72, 3, 3, 600.0, si.RADIUS, si.OMEGA, si.GRAVITY, si.MEAN_DEPTH)
    for bad in (0, 5):
        with pytest.raises(SdcError) as e:
            s.set_chains(bad)
        assert e.value.status == 1
