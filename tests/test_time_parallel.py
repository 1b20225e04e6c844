"""Time-parallel solve (dsp_solve_segmented): the same steps grouped into
segments whose operator products are formed in parallel and then multiplied
in time order.  Checked against the FP64 oracle with the parity tolerances,
and against the sequential solve."""
import numpy as np
import pytest
import torch

from paper_1607_03062_gb300 import binding as B
from paper_1607_03062_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {"fp64": (1e-9, 1e-10), "fp32_mixed": (1e-5, 1e-4)}


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1607_03062_gb300 import build
    build.build()
    B.lib()
    torch.cuda.set_device(0)


def _solve(grid, table, prec, scheme="exact", valley=1, segments=None):
    a_mid, a_in, a_out, dt = table
    g = B.Grid(grid["nx"], grid["ny"], grid["px"], grid["py"], prec, scheme, valley)
    g.set_pulse(a_mid, dt, a_in, a_out)
    m, n = g.solve() if segments is None else g.solve_segmented(segments)
    torch.cuda.synchronize()
    out = m.double().cpu().numpy().copy()
    g.close()
    return out, n


@pytest.mark.parametrize("prec", ["fp64", "fp32_mixed"])
def test_segmented_sin2_64_against_oracle(orc, prec):
    cfg = W.config_sin2_64()
    g = cfg["grid"]
    a_mid, a_in, a_out, dt = orc.pulse_table(cfg["pulse"], cfg["steps"])
    ref, _, _, nref = orc.solve_grid(g["nx"], g["ny"], g["px"], g["py"], a_mid, dt, a_in, a_out)
    m, n = _solve(g, B.sample_pulse(cfg["pulse"], cfg["steps"]), prec, segments=0)
    tp, tn = TOL[prec]
    assert np.abs(m - ref).max() <= tp
    assert abs(n - nref) <= tn * nref
    ms, ns = _solve(g, B.sample_pulse(cfg["pulse"], cfg["steps"]), prec)
    assert np.abs(m - ms).max() <= (1e-12 if prec == "fp64" else 2e-6)


@pytest.mark.parametrize("prec", ["fp64", "fp32_mixed"])
@pytest.mark.parametrize("scheme,valley,segments", [("exact", -1, 7), ("strang_xy", 1, 13),
                                                    ("exact", 1, 1), ("exact", 1, 1500)])
def test_segmented_ragged_against_oracle(orc, prec, scheme, valley, segments):
    """Uneven segments (1500 steps in 7 or 13), one segment, one step per segment."""
    grid = {"nx": 67, "ny": 45, "px": (-3.0, 5.0), "py": (-2.5, 3.5)}
    pulse = W.sin2_pulse(2.0, 1.2, 4.0, eps=0.6)
    a_mid, a_in, a_out, dt = orc.pulse_table(pulse, 1500)
    ref, _, _, nref = orc.solve_grid(67, 45, grid["px"], grid["py"], a_mid, dt, a_in, a_out,
                                     scheme=scheme, valley=valley)
    m, n = _solve(grid, B.sample_pulse(pulse, 1500), prec, scheme, valley, segments)
    tp, tn = TOL[prec]
    assert np.abs(m - ref).max() <= tp
    assert abs(n - nref) <= tn * nref


def test_segmented_needs_a_fresh_grid():
    g = B.Grid(16, 16, (-1, 1), (-1, 1), "fp64")
    a_mid, a_in, a_out, dt = B.sample_pulse(W.sin2_pulse(1.0, 1.55, 2.0), 100)
    g.set_pulse(a_mid, dt, a_in, a_out)
    g.evolve(10)
    with pytest.raises(B.DSPError) as e:
        g.solve_segmented(4)
    assert e.value.code == -4
    with pytest.raises(B.DSPError) as e:
        B.solve_segmented(g.h, -1, g.map.data_ptr())
    assert e.value.code == -1
    g.close()
