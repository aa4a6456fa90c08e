"""Mixed-precision transforms against the FP64 oracle (GPU only).

FP32: Legendre contractions and ring FFTs in FP32.  Split-BF16 on the tensor
cores (tcgen05): 2 pieces / 3 products or 3 pieces / 6 products with FP32
accumulation.  The implicit solves and the quadrature stay FP64 in every mode.

Tolerance, from the arithmetic (not fitted to measurements).  Each output
coefficient of one tendency ends a chain of roundings: the synthesis sum over
at most T + 1 degrees, log2 L butterfly stages of the inverse FFT, the grid
products, log2 L stages of the forward FFT and the projection sum over J/2
latitude pairs, N = (T + 1) + 2 log2 L + J/2 rounded terms in all.
Independent roundings of relative size u add up to about u sqrt(N) of the
terms' magnitude (the probabilistic bound for sums of Higham and Mary, 2019).
The vorticity and divergence tendencies carry one horizontal derivative of the
products (factors m and n eps_n up to T + 1 against the undifferentiated
field), which multiplies the relative error by up to T + 1.  Bound per field:

    rel L2 <= u (T + 1) sqrt(N),

with u the relative error of one product in the mode: binary32's unit
roundoff 2^-24 (FP32); 2^-15 for two BF16 pieces (16 significant bits, each
operand within 2^-17, the dropped low x low product within 2^-16); 2^-22 for
three pieces (operands within 2^-25, the three dropped products within
2^-23, plus the FP32 accumulation's 2^-24).  A run of n steps changes the
state by dt T_E per step, a small fraction of it, through contractive solves,
so its relative error stays below n times one tendency's bound.
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

UNIT = {1: 2.0 ** -24, 2: 2.0 ** -15, 3: 2.0 ** -22}     # precision -> relative error of one product


def bound(precision, T, J, L):
    n_chain = (T + 1) + 2 * math.log2(L) + J / 2
    return UNIT[precision] * (T + 1) * math.sqrt(n_chain)


def _solver(T, J, L, M, K, dt, precision):
    from paper_2403_20135_gb300 import Solver
    return Solver(T, J, L, M, K, dt, si.RADIUS, si.OMEGA, si.GRAVITY, si.MEAN_DEPTH, precision=precision)


def _cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda")


@pytest.mark.parametrize("precision", [1, 2, 3])
@pytest.mark.parametrize("T,J,L", [(21, 34, 72), (63, 100, 192), (255, 384, 768)])
def test_mixed_tendency_accuracy(precision, T, J, L):
    o = swe.SWE(sht.Grid(T, J, L), swe.default_physics())
    wl = si.Workload("m", 2, T, J, L, 4, 3, 300.0, 1, 1, (100.0, 100.0))
    u = swe.initial_state(wl, o)
    ref = o.explicit(u)
    s = _solver(T, J, L, 4, 3, 300.0, precision)
    batch = _cuda(np.stack([u, 0.5 * u, u, 2.0 * u]))      # B = 4 states in one launch
    got = to_numpy(s.tendency(batch))
    s.sync()
    for b, f in enumerate((1.0, 0.5, 1.0, 2.0)):
        refb = ref if f == 1.0 else o.explicit(f * u)
        err = rel_l2(got[b], refb)
        print(f"precision {precision} T{T} state {b}: rel L2 per field {err}")
        assert np.all(err <= bound(precision, T, J, L)), (precision, b, err)
    one = to_numpy(s.tendency(_cuda(u)))                   # B = 1 launch
    s.sync()
    assert np.all(rel_l2(one, ref) <= bound(precision, T, J, L))


@pytest.mark.parametrize("precision", [1, 2])
@pytest.mark.parametrize("J", [600, 1202])
def test_mixed_tendency_many_latitudes(precision, J):
    """Long latitude rows: the FP32 synthesis switches to fewer row splits per
    latitude block (300 and 601 northern latitudes), the projection's K loop
    and the tensor-core K chunks run much longer than at the bench size, and
    601 is odd (scalar projection loads)."""
    T, L = 21, 64
    o = swe.SWE(sht.Grid(T, J, L), swe.default_physics())
    wl = si.Workload("m", 2, T, J, L, 4, 3, 300.0, 1, 1, (100.0, 100.0))
    u = swe.initial_state(wl, o)
    ref = o.explicit(u)
    s = _solver(T, J, L, 4, 3, 300.0, precision)
    got = to_numpy(s.tendency(_cuda(np.stack([u, 2.0 * u]))))
    s.sync()
    assert np.all(rel_l2(got[0], ref) <= bound(precision, T, J, L)), rel_l2(got[0], ref)
    assert np.all(rel_l2(got[1], o.explicit(2.0 * u)) <= bound(precision, T, J, L))


@pytest.mark.parametrize("precision", [2, 3])
def test_tensor_core_step_close_to_oracle(precision):
    T, J, L, M, K, dt = 42, 64, 128, 4, 5, 300.0
    o = swe.SWE(sht.Grid(T, J, L), swe.default_physics())
    wl = si.Workload("m", 2, T, J, L, M, K, dt, 1, 1, (100.0, 100.0))
    u = swe.initial_state(wl, o)
    ref = osdc.swe_run(o, u, osdc.Collocation(M), K, dt, 3)
    s = _solver(T, J, L, M, K, dt, precision)
    got = to_numpy(s.run(_cuda(u), 3))
    s.sync()
    assert np.all(rel_l2(got, ref) <= 3 * bound(precision, T, J, L)), rel_l2(got, ref)   # 3 steps


def test_tensor_core_modes_order_of_accuracy():
    """The 3-piece split is at least 10x more accurate than the 2-piece split and
    within 2x of the FP32 SIMT path (the FP32 floor)."""
    T, J, L = 127, 192, 384
    o = swe.SWE(sht.Grid(T, J, L), swe.default_physics())
    wl = si.Workload("m", 1, T, J, L, 4, 3, 300.0, 1, 3, (50.0, 150.0))
    u = swe.initial_state(wl, o)
    ref = o.explicit(u)
    e = {}
    for p in (1, 2, 3):
        s = _solver(T, J, L, 4, 3, 300.0, p)
        e[p] = rel_l2(to_numpy(s.tendency(_cuda(u))), ref).max()
        s.sync()
    assert e[3] * 10 <= e[2], e
    assert e[3] <= 2 * e[1], e


@pytest.mark.parametrize("precision", [1, 3])
def test_mixed_adjoint_close_to_fp64_adjoint(precision):
    """The discrete adjoint in a mixed mode (the retape records FP32 grid fields,
    the transposed transforms run in FP32; sweeps and solves stay FP64): loss
    and gradient of a 3-step height misfit against the FP64 context's."""
    T, J, L, M, K, dt = 42, 64, 128, 4, 4, 300.0
    o = swe.SWE(sht.Grid(T, J, L), swe.default_physics())
    wl = si.Workload("m", 2, T, J, L, M, K, dt, 1, 1, (100.0, 100.0))
    u = swe.initial_state(wl, o)
    rng = np.random.default_rng(5)
    target = torch.from_numpy(o.height_grid(u) + rng.standard_normal((J, L))).to("cuda")
    ref_loss, ref_g = _solver(T, J, L, M, K, dt, 0).adjoint_run(_cuda(u), 3, target, nsnapshots=2)
    loss, g = _solver(T, J, L, M, K, dt, precision).adjoint_run(_cuda(u), 3, target, nsnapshots=2)
    assert abs(loss - ref_loss) <= 1e-5 * abs(ref_loss), (loss, ref_loss)
    err = rel_l2(to_numpy(g), to_numpy(ref_g))
    print(f"precision {precision}: gradient rel L2 vs FP64 adjoint {err}")
    assert np.all(err <= 1e-5), err


@pytest.mark.parametrize("precision", [2, 3])
def test_tensor_core_eight_states(precision):
    """The largest batch (eight node states: 80 projection and 64 synthesis
    columns per tile) and odd latitude-pair counts (J2 = 17, 25)."""
    for T, J, L in ((21, 34, 72), (31, 50, 96)):
        o = swe.SWE(sht.Grid(T, J, L), swe.default_physics())
        wl = si.Workload("m", 3, T, J, L, 8, 3, 300.0, 1, 1, (100.0, 100.0))
        u = swe.initial_state(wl, o)
        facs = np.linspace(0.5, 2.0, 8)
        s = _solver(T, J, L, 8, 3, 300.0, precision)
        got = to_numpy(s.tendency(_cuda(np.stack([f * u for f in facs]))))
        s.sync()
        for b, f in enumerate(facs):
            err = rel_l2(got[b], o.explicit(f * u))
            assert np.all(err <= bound(precision, T, J, L)), (T, b, err)
