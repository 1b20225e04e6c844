"""The benchmark's work model, on the CPU: the FP32 lane-operation and FP64
operation counts per spinor-step that the roofline divides by the measured time,
the normalisation degrees of the step groups, and the launch count of a solve,
each against the figures the kernels' formulation gives (Sec. III step, grouped
as the kernels group it)."""
import pytest

import bench


@pytest.mark.parametrize("G,DF", [(16, 5), (8, 6), (4, 7), (2, 9)])
def test_group_normalisation_degrees(G, DF):
    assert bench.tan_norm_degree(G) == DF


@pytest.mark.parametrize("tdeg,G,strips,ops", [
    (1, 16, True, 12.75 + 31 / 16),   # LZS samples 3, 4, 5, 7 of the benchmark
    (2, 16, True, 14.5 + 31 / 16),    # samples 0, 1, 2
    (2, 8, True, 14.5 + 32 / 8),      # sample 6
    (1, 16, False, 19 + 31 / 16),     # contiguous tiles, tan degree 1
    (2, 16, False, 19 + 31 / 16),     # contiguous tiles: 17 + DT + (26 + DF)/G
])
def test_exact_group_ops(tdeg, G, strips, ops):
    assert bench.ops_mixed(2, 1, group=G, strips=strips, tdeg=tdeg) == pytest.approx(ops)


def test_exact_single_step_ops():
    # 32 + dc + ds, 4.5 fewer on row strips
    assert bench.ops_mixed(3, 2, group=1) == 37
    assert bench.ops_mixed(3, 2, group=1, strips=True) == 32.5


def test_strang_and_magnus_ops():
    assert bench.ops_strang(2, 1, group=16, strips=True, tdeg=2) == pytest.approx(13.9375)
    assert bench.ops_strang(2, 1, group=16, strips=False, tdeg=2) == pytest.approx(24 + 31 / 16)
    assert bench.ops_strang(2, 2, group=1, strips=True) == pytest.approx(31 + 8 / 4)
    assert bench.ops_magnus4(2, 1, group=8, strips=True, tdeg=2) == pytest.approx(26.5)
    assert bench.ops_magnus4(2, 1, group=1) == 43


def test_fp64_ops():
    assert bench.ops_fp64(5, 5, strips=True) == 16.25
    assert bench.ops_fp64(5, 5, strips=False) == 18.0


@pytest.mark.parametrize("n,strips,launches", [
    (2048, True, 3),   # 13 waves of 4-row strips, the last wave's 288 tiles in 2-row strips
    (1024, True, 3),   # 912 4-row tiles, 224 2-row tiles
    (4096, True, 2),   # 16384 tiles fill 53.9 waves: the last wave is more than half full
    (256, True, 2),    # 64 tiles, at most half a wave: all in 2-row strips, one launch
    (2048, False, 2),  # contiguous tiles: one evolve launch
])
def test_launches_per_solve(n, strips, launches):
    assert bench.launches_per_solve(n, strips, 152) == launches
