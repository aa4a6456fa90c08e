"""Mixed-precision transforms against the FP64 oracle (GPU only).

FP32: Legendre contractions and ring FFTs in FP32.  Split-BF16 on the tensor
cores (tcgen05): 2 pieces / 3 products (~2^-16 per product) or 3 pieces /
6 products (~2^-24, so FP32 accumulation and the FP32 ring FFTs set the
floor).  The relative L2 error of one tendency grows with the truncation:
its high-degree coefficients carry the derivative factors n eps_n and
lambda_n ~ n^2, which amplify the rounding of the contractions; measured
errors scale about as T^1.5.  The bounds are 3x the T21 measurement times
(T/21)^1.5.  The implicit solves and the quadrature stay FP64 in every mode.
"""
import numpy as np
import pytest

import swe_inputs as si
from oracle import sdc as osdc
from oracle import sht, swe
from tests.helpers import rel_l2, to_numpy

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BASE = {1: 6e-6, 2: 2.5e-4, 3: 6e-6}          # precision -> rel L2 bound at T21


def bound(precision, T):
    return BASE[precision] * (T / 21.0) ** 1.5


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
        assert np.all(err <= bound(precision, T)), (precision, b, err)
    one = to_numpy(s.tendency(_cuda(u)))                   # B = 1 launch
    s.sync()
    assert np.all(rel_l2(one, ref) <= bound(precision, T))


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
    assert np.all(rel_l2(got[0], ref) <= 2 * bound(precision, T)), rel_l2(got[0], ref)
    assert np.all(rel_l2(got[1], o.explicit(2.0 * u)) <= 2 * bound(precision, T))


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
    assert np.all(rel_l2(got, ref) <= 10 * bound(precision, T))


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
