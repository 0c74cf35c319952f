"""Host-side arithmetic of bench.py (no GPU): the solve-level effective bandwidth."""
import pytest

import bench


def test_solve_level_bytes():
    V, nsrc, k = 38416, 16, 400
    r = bench.solve_level(V, nsrc, k, 162.6, 6687.8)
    field = 96 * V
    assert r["bytes_by_kernel"]["stencil"] == k * bench_stencil_launch(V, nsrc)
    assert r["bytes_by_kernel"]["update"] == (k - 1) * 16 * field * nsrc
    assert r["bytes_by_kernel"]["recombination"] == k * 2 * field * nsrc + 2 * 192 * V * nsrc
    assert r["bytes_per_step"] == sum(r["bytes_by_kernel"].values())
    assert r["achieved"] == pytest.approx(r["bytes_per_step"] / 0.1626 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 6687.8)
    assert 0.55 < r["frac"] < 0.59          # 617 GB in 162.6 ms against 6687.8 GB/s


def bench_stencil_launch(V, nsrc):
    return V * (8 * 96 * nsrc + 288)        # the roofline's algorithmic bytes of one stencil launch
