"""On-the-fly Legendre recurrence of the FP32 synthesis (SDC_OPT_LEGENDRE),
through the C ABI (GPU only).

The recurrence regenerates the normalised Legendre functions row by row in
FP32-pair arithmetic from FP64 seeds instead of reading the FP32 table, so
its rows equal the table's FP32 roundings up to an occasional last-bit
difference.  Checks: one tendency against the oracle within the FP32 bound of
the mixed tests, against the table path far inside that bound, whole runs
against the FP64 path (the fixed-error gate over the 500-step T255 horizon),
and the option's error returns.
"""
import numpy as np
import pytest

import swe_inputs as si
from oracle import sht, swe
from tests.helpers import rel_l2, to_numpy
from tests.test_gpu_mixed import bound

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _solver(T, J, L, M=4, K=3, dt=300.0, precision=1, recurrence=True):
    import paper_2403_20135_gb300 as pkg
    s = pkg.Solver(T, J, L, M, K, dt, si.RADIUS, si.OMEGA, si.GRAVITY, si.MEAN_DEPTH, precision=precision)
    if recurrence:
        s.set_legendre(pkg.SDC_LEGENDRE_RECURRENCE)
    return s


def _cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda")


@pytest.mark.parametrize("T,J,L", [(21, 34, 72), (63, 100, 192), (255, 384, 768)])
def test_recurrence_tendency_matches_oracle_and_table(T, J, L):
    o = swe.SWE(sht.Grid(T, J, L), swe.default_physics())
    wl = si.Workload("r", 2, T, J, L, 4, 3, 300.0, 1, 1, (100.0, 100.0))
    u = swe.initial_state(wl, o)
    batch = np.stack([u, 0.5 * u, 2.0 * u, u])
    rec = _solver(T, J, L)
    tab = _solver(T, J, L, recurrence=False)
    got = to_numpy(rec.tendency(_cuda(batch)))
    ref_tab = to_numpy(tab.tendency(_cuda(batch)))
    one = to_numpy(rec.tendency(_cuda(u)))                # the batch of one state (E0's launch)
    rec.sync()
    for b, f in enumerate((1.0, 0.5, 2.0, 1.0)):
        ref = o.explicit(f * u)
        err = rel_l2(got[b], ref)
        print(f"T{T} state {b}: recurrence vs oracle {err}, vs table {rel_l2(got[b], ref_tab[b])}")
        assert np.all(err <= bound(1, T, J, L)), err
        # the same contraction on rows that differ from the table's by at most
        # a last bit: far inside the rounding bound
        assert np.all(rel_l2(got[b], ref_tab[b]) <= 0.1 * bound(1, T, J, L))
    assert np.all(rel_l2(one, o.explicit(u)) <= bound(1, T, J, L))


def test_recurrence_fixed_error_over_horizon():
    """The T255 precision form with the recurrence: after the 500-step horizon
    the per-field error against the FP64 GPU path stays below the FP64
    discretisation error, as with the table."""
    wl = si.WORKLOADS["t255"]
    import paper_2403_20135_gb300 as pkg
    s64 = pkg.Solver.for_workload(wl, precision=0)
    u0 = s64.initial_state(wl)
    a = to_numpy(s64.run(u0.clone(), wl.nsteps))
    q = pkg.Solver(wl.T, wl.nlat, wl.nlon, wl.nodes, wl.sweeps, wl.dt / 4, si.RADIUS, si.OMEGA, si.GRAVITY,
                   si.MEAN_DEPTH, precision=0)
    edisc = rel_l2(a, to_numpy(q.run(u0.clone(), 4 * wl.nsteps)))
    rec = pkg.Solver.for_workload(wl, precision=1)
    rec.set_legendre(pkg.SDC_LEGENDRE_RECURRENCE)
    got = to_numpy(rec.run(u0.clone(), wl.nsteps))
    rec.sync()
    err = rel_l2(got, a)
    print(f"T255 FP32 recurrence, {wl.nsteps} steps: rel L2 vs FP64 {err}; discretisation error {edisc}")
    assert np.all(err < edisc), (err, edisc)


def test_recurrence_t511_close_to_fp64():
    wl = si.WORKLOADS["t511"]
    import paper_2403_20135_gb300 as pkg
    s64 = pkg.Solver.for_workload(wl, precision=0)
    u0 = s64.initial_state(wl)
    ref = to_numpy(s64.run(u0.clone(), 2))
    s64.close()
    rec = pkg.Solver.for_workload(wl, precision=1)
    rec.set_legendre(pkg.SDC_LEGENDRE_RECURRENCE)
    got = to_numpy(rec.run(u0.clone(), 2))
    rec.sync()
    err = rel_l2(got, ref)
    print(f"T511 FP32 recurrence, 2 steps: rel L2 vs FP64 {err}")
    assert np.all(err <= 2 * bound(1, wl.T, wl.nlat, wl.nlon)), err


def test_recurrence_option_errors():
    import paper_2403_20135_gb300 as pkg
    from paper_2403_20135_gb300 import SdcError
    s64 = _solver(21, 34, 72, precision=0, recurrence=False)
    with pytest.raises(SdcError) as e:
        s64.set_legendre(pkg.SDC_LEGENDRE_RECURRENCE)
    assert e.value.status == 6                            # SDC_EUNSUPPORTED
    s32 = _solver(21, 34, 72, recurrence=False)
    with pytest.raises(SdcError) as e:
        s32.set_legendre(7)
    assert e.value.status == 1                            # SDC_EINVAL
    # switching back and forth gives back the table path's result bit for bit
    o = swe.SWE(sht.Grid(21, 34, 72), swe.default_physics())
    u = _cuda(swe.initial_state(si.Workload("r", 0, 21, 34, 72, 4, 3, 300.0, 1, 1, (100.0, 100.0)), o))
    before = to_numpy(s32.run(u.clone(), 2))
    s32.set_legendre(pkg.SDC_LEGENDRE_RECURRENCE)
    s32.run(u.clone(), 1)
    s32.set_legendre(pkg.SDC_LEGENDRE_TABLE)
    np.testing.assert_array_equal(to_numpy(s32.run(u.clone(), 2)), before)
