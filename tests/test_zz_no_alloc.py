"""The allocation-free density entry point (dsp_density_noalloc).

It serves callers that cannot call cudaMalloc (a host application that owns
the device memory through its own allocator, or a loop where an allocation's
device synchronisation is not allowed).  Checked through the C ABI against
the existing dsp_reduce_density on two calls in a row (plus a repeat of the
first, so stale contents of the shared static scratch would show).  This file
is collected last on purpose.
"""
import numpy as np
import pytest
import torch

from paper_1607_03062_gb300 import binding as B
from paper_1607_03062_gb300 import workloads as W

pytestmark = pytest.mark.gpu

# same tolerances as the parity tests: density relative error
TOL_REL = {"fp64": 1e-10, "fp32_mixed": 1e-4}


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1607_03062_gb300 import build
    build.build()
    B.lib()
    torch.cuda.set_device(0)


def _solved(grid, pulse, steps, prec):
    g = B.Grid(grid["nx"], grid["ny"], grid["px"], grid["py"], prec)
    a_mid, a_in, a_out, dt = B.sample_pulse(pulse, steps)
    g.set_pulse(a_mid, dt, a_in, a_out)
    g.evolve(steps)
    g.project()
    n_ref = g.density()
    return g, n_ref


def test_noalloc_matches_reduce_density_on_consecutive_calls():
    cases = [
        ({"nx": 300, "ny": 170, "px": (-4.0, 4.0), "py": (-3.0, 5.0)},
         W.sin2_pulse(1.0, 1.55, 5.0), 1500, "fp64"),
        ({"nx": 1024, "ny": 999, "px": (-6.0, 6.0), "py": (-6.0, 6.0)},
         W.gauss_pulse(2.0, 1.55, 1.0), 1200, "fp32_mixed"),
    ]
    solved = [(_solved(grid, pulse, steps, prec), grid, prec)
              for grid, pulse, steps, prec in cases]
    stream = torch.cuda.current_stream().cuda_stream
    for (g, n_ref), grid, prec in solved + solved[:1]:
        n = B.density_noalloc(g.map.data_ptr(), prec, grid["nx"], grid["ny"], grid["px"],
                              grid["py"], stream)
        assert n > 0
        assert abs(n - n_ref) <= TOL_REL[prec] * n_ref, (prec, n, n_ref)
        if prec == "fp64":  # same values, same summation order
            assert n == n_ref
    for (g, _), _, _ in solved:
        g.close()


def test_noalloc_above_1024_tiles_and_at_the_maximum_size():
    """2048 tiles (the final sum then strides: each of its 1024 threads adds two
    tile sums before the tree) against dsp_reduce_density, bitwise for an FP64
    map, on two calls in a row; and a map of exactly DSP_NOALLOC_MAX_POINTS
    points (a 256 MB float map of zeros) is accepted and sums to 0."""
    grid = {"nx": 2048, "ny": 1024, "px": (-5.0, 5.0), "py": (-4.0, 4.0)}
    (g, n_ref), = [_solved(grid, W.sin2_pulse(1.5, 1.55, 2.0), 120, "fp64")]
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        n = B.density_noalloc(g.map.data_ptr(), "fp64", grid["nx"], grid["ny"], grid["px"],
                              grid["py"], stream)
        assert n == n_ref and n > 0
    g.close()
    side = 8192
    assert side * side == 67108864  # DSP_NOALLOC_MAX_POINTS
    zeros = torch.zeros(side * side, dtype=torch.float32, device="cuda")
    assert B.density_noalloc(zeros.data_ptr(), "fp32_mixed", side, side, (-1, 1), (-1, 1),
                             stream) == 0.0
    del zeros


def test_noalloc_refuses_maps_beyond_its_static_scratch():
    with pytest.raises(B.DSPError) as e:
        B.density_noalloc(16, "fp32_mixed", 8193, 8192, (-1, 1), (-1, 1))
    assert e.value.code == -1
