"""The allocation-free spectral-to-grid entry point (sdc_spec_to_grid_static).

It exists for callers that cannot call cudaMalloc (host applications that own
all device memory, latency-critical loops that cannot afford an allocation's
device synchronisation, processes under a fixed device-memory budget): it
needs no context and keeps its intermediate data in a static 2 MiB device
array.  Its output must equal the context-based sdc_spec_to_grid's, within
the transform tolerance of the other tests, call after call (the shared
array keeps the previous call's contents).  This file is collected last.
"""
import ctypes

import numpy as np
import pytest

import swe_inputs as si


def _lib():
    import paper_2403_20135_gb300 as pkg
    return pkg.load()


def test_static_transform_rejects_oversize_and_null():
    lib = _lib()
    from paper_2403_20135_gb300 import _lib as L
    fake = ctypes.c_void_p(256)
    # T511 on 768 latitudes needs 384*2*512 complex doubles: beyond the 2 MiB array
    assert lib.sdc_spec_to_grid_static(511, 768, 1536, fake, fake, None) == L.SDC_EUNSUPPORTED
    assert lib.sdc_spec_to_grid_static(255, 384, 768, None, fake, None) == L.SDC_EINVAL
    assert lib.sdc_spec_to_grid_static(255, 383, 768, fake, fake, None) == L.SDC_EINVAL
    assert lib.sdc_spec_to_grid_static(255, 384, 700, fake, fake, None) == L.SDC_EINVAL


@pytest.mark.gpu
def test_static_transform_matches_context_transform_twice():
    torch = pytest.importorskip("torch")
    from paper_2403_20135_gb300 import Solver
    lib = _lib()
    rng = np.random.default_rng(7)
    for T, J, L in [(63, 100, 192), (63, 100, 192), (255, 384, 768), (21, 34, 72)]:
        s = Solver(T, J, L, 2, 2, 300.0, si.RADIUS, si.OMEGA, si.GRAVITY, si.MEAN_DEPTH)
        n, m = si.degree_order_arrays(T)
        c = rng.standard_normal(s.ncoef) + 1j * rng.standard_normal(s.ncoef)
        c[m == 0] = c[m == 0].real
        spec = torch.from_numpy(c).to("cuda")
        ref = s.spec_to_grid(spec)
        out = torch.full((J, L), float("nan"), dtype=torch.float64, device="cuda")
        stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        for _ in range(2):                                     # two calls in a row
            out.fill_(float("nan"))
            st = lib.sdc_spec_to_grid_static(T, J, L, ctypes.c_void_p(spec.data_ptr()),
                                             ctypes.c_void_p(out.data_ptr()), stream)
            assert st == 0
            torch.cuda.synchronize()
            # the single-evaluation tolerance of the parity tests (relative to the
            # field's maximum; the static path generates its own Gauss nodes)
            diff = (out - ref).abs().max().item()
            assert diff <= 1e-12 * ref.abs().max().item(), (T, diff)
        s.close()
