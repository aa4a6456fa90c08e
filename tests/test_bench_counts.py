"""The algorithmic work counts bench.py divides by (CPU only), against the
per-unit figures stated with the kernels: at T255 (33,152 extended rows,
192 latitude pairs, L = 768) one node evaluation is 16 next J2 flops of
synthesis (4 complex fields x 2 real FMA per row and latitude), 20 next J2
of projection (5 fields) and 9 complex FFTs of 5 L log2 L flops plus 60 L of
products per ring pair; the FP64 step adds the sweeps' quadrature and solves."""
import math

import pytest

import bench
import swe_inputs as si


def test_stage_flops_per_node_evaluation():
    wl = si.WORKLOADS["t255"]
    nxt, J2, L = 256 * 259 // 2, 192, 768
    assert nxt == 33152
    assert bench.stage_flops(wl, "synthesis", 1) == 16.0 * nxt * J2
    assert bench.stage_flops(wl, "analysis", 1) == 20.0 * nxt * J2
    assert bench.stage_flops(wl, "ring", 1) == pytest.approx((9 * 5.0 * L * math.log2(L) + 60.0 * L) * J2)
    assert bench.stage_flops(wl, "synthesis", 4) == 4 * bench.stage_flops(wl, "synthesis", 1)
    with pytest.raises(ValueError):
        bench.stage_flops(wl, "unknown", 1)


def test_sweep_counts():
    wl = si.WORKLOADS["t255"]
    nc, M = 256 * 257 // 2, 4
    # all M nodes updated, tendencies of M projected states: (12 M + 24) M + 8 M + 36 M per mode
    assert bench.sweep_flops(wl, M, M) == nc * ((12.0 * M + 24.0) * M + 8.0 * M + 36.0 * M)
    # bytes: u_n, M iterates, M outputs (3 fields x 16 B) and 10 values per projected state
    assert bench.sweep_bytes(wl, True, M, 8) == nc * ((1 + 2 * M) * 3 * 16.0 + M * 10 * 8)
    assert bench.sweep_bytes(wl, False, 1, 16) == nc * ((1 + M + 1) * 3 * 16.0 + 10 * 16)
