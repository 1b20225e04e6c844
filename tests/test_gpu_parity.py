"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle.

Tolerances (per point |c+|^2 absolute, density relative):
  FP64        1e-9 and 1e-10 -- both sides are FP64; the difference is rounding
              order and the series-vs-libm evaluation of cos/sin, O(1e-16) per
              step, accumulated over <= 1e5 unitary steps.
  FP32_MIXED  1e-5 and 1e-4 -- the accuracy target for the mixed path.
"""
import math

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


def run_gpu(grid, table, precision="fp32_mixed", scheme="exact", valley=1, pieces=None):
    a_mid, a_in, a_out, dt = table
    g = B.Grid(grid["nx"], grid["ny"], grid["px"], grid["py"], precision, scheme, valley)
    g.set_pulse(a_mid, dt, a_in, a_out)
    if pieces is None:
        m, n = g.solve()
    else:
        for p in pieces:
            g.evolve(p)
        m = g.project()
        n = g.density()
    torch.cuda.synchronize()
    out = m.double().cpu().numpy().copy()
    g.close()
    return out, n


def run_oracle(orc, grid, table, scheme="exact", valley=1):
    a_mid, a_in, a_out, dt = table
    cp, _, _, n = orc.solve_grid(grid["nx"], grid["ny"], grid["px"], grid["py"], a_mid, dt, a_in,
                                 a_out, scheme=scheme, valley=valley)
    return cp, n


def assert_close(prec, m, n, ref, nref):
    tp, tn = TOL[prec]
    err = np.abs(m - ref).max()
    assert err <= tp, f"{prec}: max |c+|^2 error {err:.3e} > {tp}"
    if nref > 0:
        rel = abs(n - nref) / nref
        assert rel <= tn, f"{prec}: density relative error {rel:.3e} > {tn}"
    else:
        assert abs(n) <= 1e-12


@pytest.mark.parametrize("prec", ["fp64", "fp32_mixed"])
def test_sin2_64_full_map(orc, prec):
    """64x64 grid on [-4,4]^2, 5-cycle sin^2 pulse, 2000 steps: every point."""
    cfg = W.config_sin2_64()
    tab = orc.pulse_table(cfg["pulse"], cfg["steps"])
    ref, nref = run_oracle(orc, cfg["grid"], tab)
    m, n = run_gpu(cfg["grid"], B.sample_pulse(cfg["pulse"], cfg["steps"]), prec)
    assert_close(prec, m, n, ref, nref)


@pytest.mark.parametrize("prec", ["fp64", "fp32_mixed"])
@pytest.mark.parametrize("scheme,valley", [("exact", 1), ("exact", -1), ("strang_xy", 1),
                                           ("strang_xy", -1)])
def test_ragged_tiles_and_chunks(orc, prec, scheme, valley):
    """67x45 points (3 tiles, ragged tail), asymmetric box, elliptical pulse,
    1500 steps evolved in pieces that straddle the 1024-step table chunks."""
    grid = {"nx": 67, "ny": 45, "px": (-3.0, 5.0), "py": (-2.5, 3.5)}
    pulse = W.sin2_pulse(2.0, 1.2, 4.0, eps=0.6)
    n_steps = 1500
    ref, nref = run_oracle(orc, grid, orc.pulse_table(pulse, n_steps), scheme, valley)
    m, n = run_gpu(grid, B.sample_pulse(pulse, n_steps), prec, scheme, valley,
                   pieces=[700, 1, 799])
    assert_close(prec, m, n, ref, nref)


@pytest.mark.parametrize("prec", ["fp64", "fp32_mixed"])
@pytest.mark.parametrize("scheme", ["exact", "strang_xy"])
def test_pieces_equal_one_launch_bitwise(prec, scheme):
    """Pieces that end on multiples of 16 steps give bitwise the one-launch result;
    a boundary inside a step group changes rounding only (bitwise where the
    library takes every step alone: FP64, or group_steps == 1)."""
    grid = {"nx": 100, "ny": 37, "px": (-4, 4), "py": (-4, 4)}
    tab = B.sample_pulse(W.gauss_pulse(2.0, 1.55, 1.0), 3100)
    g = B.Grid(100, 37, grid["px"], grid["py"], prec, scheme)
    g.set_pulse(tab[0], tab[3], tab[1], tab[2])
    group = B.get_info(g.h)["group_steps"]
    g.close()
    m1, n1 = run_gpu(grid, tab, prec, scheme)
    m2, n2 = run_gpu(grid, tab, prec, scheme, pieces=[1024, 992, 16, 1068])
    assert np.array_equal(m1, m2) and n1 == n2
    m3, n3 = run_gpu(grid, tab, prec, scheme, pieces=[1023, 1, 1, 2075])
    if group == 1:
        assert np.array_equal(m1, m3) and n1 == n3
    else:
        assert np.abs(m1 - m3).max() <= 1e-6 and abs(n1 - n3) <= 1e-6 * n1


# 5-cycle sin^2 pulse on [-4, 4]^2 (theta_max ~ 128 / n_steps): the step count
# picks the FP32-mixed group size G, the largest of 16, 8, 4, 2 with G theta_max
# within the group angle: 0.27 for EXACT and STRANG_XY, 0.2 for MAGNUS4.
GROUP_ANGLE = {"exact": 0.27, "strang_xy": 0.27, "magnus4": 0.2}
GROUP_STEPS = {1: 800, 2: 1300, 4: 2500, 8: 5000, 16: 10000}
GROUP_STEPS_MAGNUS4 = {1: 1000, 2: 1600, 4: 3000, 8: 6000, 16: 12000}


def group_steps(scheme, G):
    return (GROUP_STEPS_MAGNUS4 if scheme == "magnus4" else GROUP_STEPS)[G]


@pytest.mark.parametrize("scheme", ["exact", "strang_xy"])
@pytest.mark.parametrize("G", sorted(GROUP_STEPS))
def test_step_groups_vs_oracle_and_pieces(orc, G, scheme):
    """Each FP32-mixed group size, EXACT and STRANG_XY: the library reports it,
    the result meets the oracle at the FP32-mixed tolerance, pieces ending on
    multiples of 16 are bitwise the one-launch result, and boundaries inside
    groups (the ragged single steps at both ends of a launch) change rounding
    only."""
    grid = {"nx": 48, "ny": 40, "px": (-4, 4), "py": (-4, 4)}
    pulse = W.sin2_pulse(1.0, 1.55, 5.0, eps=0.4)
    n = GROUP_STEPS[G]
    tab = B.sample_pulse(pulse, n)
    g = B.Grid(48, 40, grid["px"], grid["py"], "fp32_mixed", scheme)
    g.set_pulse(tab[0], tab[3], tab[1], tab[2])
    info = B.get_info(g.h)
    g.close()
    assert info["group_steps"] == G
    a = GROUP_ANGLE[scheme]
    assert G * info["theta_max"] <= a and (G == 16 or 2 * G * info["theta_max"] > a)
    ref, nref = run_oracle(orc, grid, orc.pulse_table(pulse, n), scheme)
    m1, n1 = run_gpu(grid, tab, "fp32_mixed", scheme)
    assert_close("fp32_mixed", m1, n1, ref, nref)
    cut = [16 * 19, 16 * 25, n - 16 * 44]
    m2, n2 = run_gpu(grid, tab, "fp32_mixed", scheme, pieces=cut)
    assert np.array_equal(m1, m2) and n1 == n2
    m3, n3 = run_gpu(grid, tab, "fp32_mixed", scheme, pieces=[299, 5, 3, n - 307])
    assert_close("fp32_mixed", m3, n3, ref, nref)
    if G == 1:
        assert np.array_equal(m1, m3) and n1 == n3
    else:
        assert np.abs(m1 - m3).max() <= 1e-6


def _strip_vs_contiguous(grid, tab, pieces=None, valley=1, rows=None, segmented=False,
                         scheme="exact", prec="fp32_mixed"):
    """The same grid solved on each tiling the test hook selects -- automatic (row
    strips, the last wave of a launch in 2-row strips), 4-row strips only, and
    contiguous tiles: (map, density) of each, in that order."""
    out = []
    for tiling in (1, 2, 0):
        g = B.Grid(grid["nx"], grid["ny"], grid["px"], grid["py"], prec, scheme, valley,
                   rows=rows)
        B.test_tiling(g.h, tiling)
        info = B.get_info(g.h)
        strips = tiling != 0
        assert info["n_tiles"] == ((g.nx // 256) * -(-g.ny // 4) if strips
                                   else -(-(g.nx * g.ny) // 1024))
        assert info["row_strips"] == (1 if strips else 0)
        g.set_pulse(tab[0], tab[3], tab[1], tab[2])
        if segmented:
            m, n = g.solve_segmented(0)
        elif pieces is None:
            m, n = g.solve()
        else:
            for p_ in pieces:
                g.evolve(p_)
            m = g.project()
            n = g.density()
        torch.cuda.synchronize()
        out.append((m.double().cpu().numpy().copy(), n))
        g.close()
    (m1, n1), (m2, n2), (m3, n3) = out
    assert np.array_equal(m1, m2) and n1 == n2, "last-wave split vs 4-row strips"
    return out[0], out[2]


def test_last_wave_split_mixes_strip_heights():
    """A 512 x 700 grid: 350 strip tiles leave a last wave of 46 on this GPU's 304
    slots, so a launch runs rows 0-607 in 4-row strips and rows 608-699 in 2-row
    strips; EXACT FP32-mixed in groups of 16, both precisions of EXACT, and
    STRANG_XY: bitwise the 4-row-only and contiguous results."""
    grid = {"nx": 512, "ny": 700, "px": (-4, 4), "py": (-4, 4)}
    tab = B.sample_pulse(W.sin2_pulse(1.0, 1.55, 5.0, eps=0.4), 12000)
    for prec, scheme in (("fp32_mixed", "exact"), ("fp64", "exact"), ("fp32_mixed", "strang_xy")):
        (m1, n1), (m2, n2) = _strip_vs_contiguous(grid, tab, scheme=scheme, prec=prec)
        assert np.array_equal(m1, m2) and n1 == n2, (prec, scheme)


@pytest.mark.parametrize("scheme", ["exact", "strang_xy", "magnus4"])
@pytest.mark.parametrize("G", sorted(GROUP_STEPS))
def test_row_strips_bitwise_equal_contiguous_tiles(orc, G, scheme):
    """FP32-mixed grids whose nx is a multiple of 256 evolve on row strips (4
    rows x 256 columns per CTA, the per-step momentum work shared); in every
    scheme, every group size gives the contiguous tiling's map and density bit
    for bit, on a grid whose last strip hangs over the last row (10 rows), and
    the map meets the oracle."""
    grid = {"nx": 512, "ny": 10, "px": (-4, 4), "py": (-4, 4)}
    pulse = W.sin2_pulse(1.0, 1.55, 5.0, eps=0.4)
    n = group_steps(scheme, G)
    sample = B.sample_pulse_gauss if scheme == "magnus4" else B.sample_pulse
    tab = sample(pulse, n)
    (m1, n1), (m2, n2) = _strip_vs_contiguous(grid, tab, scheme=scheme)
    assert np.array_equal(m1, m2) and n1 == n2
    if G in (1, 16):
        if scheme == "magnus4":
            a, a_in, a_out, dt = orc.pulse_table_gauss(pulse, n)
            ref, _, _, nref = orc.solve_grid(512, 10, grid["px"], grid["py"], a, dt, a_in,
                                             a_out, scheme="magnus4")
        else:
            ref, nref = run_oracle(orc, grid, orc.pulse_table(pulse, n), scheme)
        assert_close("fp32_mixed", m1, n1, ref, nref)


@pytest.mark.parametrize("prec,scheme", [("fp64", "exact"), ("fp64", "strang_xy"),
                                         ("fp32_mixed", "exact"), ("fp32_mixed", "strang_xy"),
                                         ("fp32_mixed", "magnus4")])
def test_row_strips_pieces_valley_band_segmented(orc, scheme, prec):
    """Row strips against contiguous tiles, bit for bit (FP64 MAGNUS4 has no
    strip path): ragged pieces (steps alone at both ends of each launch, chunk
    boundaries crossed), valley K-, a band of a larger grid, and the
    time-parallel solve (segments start from the identity column); the FP64
    strips also against the oracle."""
    grid = {"nx": 256, "ny": 23, "px": (-3.0, 5.0), "py": (-2.5, 3.5)}
    pulse = W.sin2_pulse(2.0, 1.2, 4.0, eps=0.6)
    sample = B.sample_pulse_gauss if scheme == "magnus4" else B.sample_pulse
    tab = sample(pulse, 5000)
    for kw in ({"pieces": [299, 5, 3, 4693]}, {"valley": -1, "pieces": [1024, 3976]},
               {"rows": (7, 19)}, {"segmented": True}):
        (m1, n1), (m2, n2) = _strip_vs_contiguous(grid, tab, scheme=scheme, prec=prec, **kw)
        assert np.array_equal(m1, m2) and n1 == n2, kw
    if prec == "fp64":
        (m, n), _ = _strip_vs_contiguous(grid, tab, scheme=scheme, prec=prec)
        ref, nref = run_oracle(orc, grid, orc.pulse_table(pulse, 5000), scheme)
        assert_close("fp64", m, n, ref, nref)


@pytest.mark.parametrize("prec", ["fp64", "fp32_mixed"])
def test_runs_are_deterministic(prec):
    grid = {"nx": 300, "ny": 200, "px": (-4, 4), "py": (-4, 4)}
    tab = B.sample_pulse(W.sin2_pulse(1.0, 1.55, 5.0), 800)
    m1, n1 = run_gpu(grid, tab, prec)
    m2, n2 = run_gpu(grid, tab, prec)
    assert np.array_equal(m1, m2) and n1 == n2


def test_batch_equals_alone_bitwise():
    """One launch over several grids (both precisions, different sizes, pulses and
    step counts) gives bitwise the results of each grid alone."""
    specs = [({"nx": 64, "ny": 64, "px": (-4, 4), "py": (-4, 4)}, W.sin2_pulse(1.0, 1.55, 5.0),
              1200, "fp32_mixed"),
             ({"nx": 130, "ny": 33, "px": (-6, 6), "py": (-3, 3)}, W.gauss_pulse(3.0, 1.1, 1.0),
              900, "fp32_mixed"),
             ({"nx": 50, "ny": 70, "px": (-2, 5), "py": (-4, 4)}, W.sin2_pulse(2.0, 0.9, 3.0, 0.3),
              1500, "fp64")]
    alone = []
    for grid, pulse, n, prec in specs:
        alone.append(run_gpu(grid, B.sample_pulse(pulse, n), prec))
    gs = []
    for grid, pulse, n, prec in specs:
        g = B.Grid(grid["nx"], grid["ny"], grid["px"], grid["py"], prec)
        a_mid, a_in, a_out, dt = B.sample_pulse(pulse, n)
        g.set_pulse(a_mid, dt, a_in, a_out)
        gs.append(g)
    steps = [s[2] for s in specs]
    B.evolve_batch([g.h for g in gs], [500, 500, 500])
    B.evolve_batch([g.h for g in gs], [s - 500 for s in steps])
    for g, (m_ref, n_ref) in zip(gs, alone):
        m = g.project()
        n = g.density()
        torch.cuda.synchronize()
        assert np.array_equal(m.double().cpu().numpy(), m_ref) and n == n_ref
        g.close()


# |c+|^2 of a state that is exactly the negative-energy spinor: 0, up to the
# projection's rounding -- double-float for FP64 (~1e-30), FP32 for FP32-mixed
# (whose map is a float: c+ itself is off by a few float ulps, ~1e-7, so |c+|^2
# by ~1e-14).
ZERO = {"fp64": 1e-15, "fp32_mixed": 1e-13}


@pytest.mark.parametrize("prec", ["fp64", "fp32_mixed"])
def test_zero_steps_and_single_point(orc, prec):
    """No steps: |c+|^2 = 0 when A_in = A_out.  A 1x1 grid is the point p = 0
    (the P -> (0+, 0) limit of the spinors), here under a zero field."""
    grid = {"nx": 5, "ny": 3, "px": (-1, 1), "py": (-1, 1)}
    m, n = run_gpu(grid, (np.zeros((0, 2)), np.zeros(2), np.zeros(2), 0.0), prec)
    assert np.abs(m).max() <= ZERO[prec] and abs(n) <= ZERO[prec]
    one = {"nx": 1, "ny": 1, "px": (-1, 1), "py": (-1, 1)}
    tab = B.sample_pulse(W.sin2_pulse(0.5, 1.55, 2.0), 300)
    ref, nref = run_oracle(orc, one, orc.pulse_table(W.sin2_pulse(0.5, 1.55, 2.0), 300))
    m, n = run_gpu(one, tab, prec)
    assert abs(m[0, 0] - ref[0, 0]) <= TOL[prec][0]


def test_constant_field_landau_zener_on_gpu(orc):
    """The LZ workload through the GPU, FP32-mixed, against the oracle (whose LZ
    closed-form agreement is pinned on the CPU)."""
    E0, T = 1.0, 60.0
    pulse = W.const_field_pulse(E0, T)
    grid = {"nx": 128, "ny": 40, "px": (-40.0, 40.0), "py": (-2.0, 2.0)}
    n = 6000
    ref, nref = run_oracle(orc, grid, orc.pulse_table(pulse, n))
    m, dens = run_gpu(grid, B.sample_pulse(pulse, n), "fp32_mixed")
    assert_close("fp32_mixed", m, dens, ref, nref)


def test_argument_and_order_errors():
    g = B.Grid(8, 8, (-1, 1), (-1, 1), "fp32_mixed")
    with pytest.raises(B.DSPError) as e:  # no pulse yet
        g.evolve(1)
    assert e.value.code == -4
    big = np.full((10, 2), 0.0)
    with pytest.raises(B.DSPError) as e:  # dt * max|p + A| > pi
        g.set_pulse(big, 3.0, [0, 0], [0, 0])
    assert e.value.code == -5
    bad = np.zeros((10, 2))
    bad[3, 1] = np.nan
    with pytest.raises(B.DSPError) as e:
        g.set_pulse(bad, 0.01, [0, 0], [0, 0])
    assert e.value.code == -1
    g.set_pulse(np.zeros((10, 2)), 0.01, [0, 0], [0, 0])
    with pytest.raises(B.DSPError) as e:  # past the end
        g.evolve(11)
    assert e.value.code == -4
    g.evolve(4)
    with pytest.raises(B.DSPError) as e:  # project before the end
        g.project()
    assert e.value.code == -4
    with pytest.raises(B.DSPError) as e:  # no projection yet
        g.density()
    assert e.value.code == -4
    g.evolve(6)
    g.project()
    assert abs(g.density()) < ZERO["fp32_mixed"]
    g.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32_mixed"])
def test_host_buffer_entry_point_matches_device_path(prec):
    grid = {"nx": 96, "ny": 80, "px": (-4, 4), "py": (-4, 4)}
    a_mid, a_in, a_out, dt = B.sample_pulse(W.sin2_pulse(1.0, 1.55, 5.0), 1000)
    m_dev, n_dev = run_gpu(grid, (a_mid, a_in, a_out, dt), prec)
    h = B.create_grid(96, 80, (-4, 4), (-4, 4), prec)
    out = np.zeros((80, 96), dtype=np.float64 if prec == "fp64" else np.float32)
    n = B.solve_host(h, a_mid, dt, a_in, a_out, out)
    B.destroy_grid(h)
    assert np.array_equal(out.astype(np.float64), m_dev) and n == n_dev


@pytest.mark.parametrize("prec", ["fp64", "fp32_mixed"])
def test_checkpoint_resume_bitwise(prec):
    grid = {"nx": 70, "ny": 30, "px": (-4, 4), "py": (-4, 4)}
    tab = B.sample_pulse(W.sin2_pulse(1.5, 1.55, 4.0), 1400)
    m_ref, n_ref = run_gpu(grid, tab, prec)
    a_mid, a_in, a_out, dt = tab
    h1 = B.create_grid(70, 30, (-4, 4), (-4, 4), prec)
    B.set_pulse(h1, a_mid, dt, a_in, a_out)
    B.evolve(h1, 608)  # a multiple of 16: resuming meets the same step groups
    buf = np.zeros(B.state_bytes(70, 30, prec), dtype=np.uint8)
    cur = B.save_state(h1, buf)
    B.destroy_grid(h1)
    h2 = B.create_grid(70, 30, (-4, 4), (-4, 4), prec)
    B.set_pulse(h2, a_mid, dt, a_in, a_out)
    B.load_state(h2, buf, cur)
    B.evolve(h2, 1400 - cur)
    out = np.zeros((30, 70), dtype=np.float64 if prec == "fp64" else np.float32)
    mp = torch.from_numpy(out).cuda()
    B.project(h2, mp.data_ptr())
    n = B.reduce_density(h2)
    B.destroy_grid(h2)
    assert np.array_equal(mp.cpu().numpy().astype(np.float64), m_ref) and n == n_ref


@pytest.mark.parametrize("prec,sample", [("fp64", 0)] + [("fp32_mixed", k) for k in range(8)])
def test_lzs_2048_full_size_sampled(orc, prec, sample):
    """The 2048x2048, 1e5-step LZS workload in the launch configuration the
    benchmark times, every seeded (omega, E0) sample in FP32-mixed (they run at
    different series degrees and step-group sizes: groups of 8 for the one with
    theta_max > 0.025, of 16 for the others) and the first in FP64 (11 s a solve).  384 seeded points, a
    band around p_y = 0 and the 128 largest |c+|^2 of the map, checked one by one."""
    cfg = W.config_lzs_2048(sample)
    g = cfg["grid"]
    tab_o = orc.pulse_table(cfg["pulse"], cfg["steps"])
    m, n = run_gpu(g, B.sample_pulse(cfg["pulse"], cfg["steps"]), prec)
    idx = W.sample_points(g["nx"], g["ny"], 384, seed=11 + sample)
    # points where pairs are likely: around p_y = 0 along the field, and the map's maxima
    xs = orc.grid_nodes(*g["px"], g["nx"])
    ys = orc.grid_nodes(*g["py"], g["ny"])
    band = np.arange(g["nx"] // 2 - 8, g["nx"] // 2 + 8) * g["nx"] + np.arange(0, g["nx"], 128)[:, None]
    top = np.argsort(m.ravel())[-128:]
    idx = np.unique(np.concatenate([idx, band.ravel(), top]))
    r = orc.solve_points(xs[idx % g["nx"]], ys[idx // g["nx"]], *tab_o[:1], tab_o[3], tab_o[1],
                         tab_o[2])
    err = np.abs(m.ravel()[idx] - r["cplus2"]).max()
    assert r["cplus2"].max() > 0.05
    assert err <= TOL[prec][0], f"{prec}: max sampled error {err:.3e}"
    assert np.all(np.isfinite(m)) and m.min() >= 0.0 and m.max() <= 1.0 + 1e-6
    assert n > 0


def test_long_run_4e6_steps_fp32_mixed(orc):
    """A run 44 times longer than the benchmark's: 4.4e6 steps of a 20-cycle
    pulse (theta_max ~ 3e-4, each point turning through ~750 rad).  FP32-mixed in
    groups of 16 against the oracle on the four central rows and 64 seeded points,
    one by one: the error does not grow with the length of the run (measured
    1.4e-6, as at 1e5 steps)."""
    grid = {"nx": 32, "ny": 32, "px": (-3.0, 3.0), "py": (-3.0, 3.0)}
    pulse = W.sin2_pulse(0.5, 0.5, 20.0)
    n = 4_400_000
    tab = B.sample_pulse(pulse, n)
    g = B.Grid(32, 32, grid["px"], grid["py"], "fp32_mixed")
    g.set_pulse(tab[0], tab[3], tab[1], tab[2])
    info = B.get_info(g.h)
    m, _ = g.solve()
    torch.cuda.synchronize()
    m = m.double().cpu().numpy().ravel()
    g.close()
    assert info["group_steps"] == 16 and info["theta_max"] < 3e-4
    idx = np.unique(np.concatenate([np.arange(14 * 32, 18 * 32), W.sample_points(32, 32, 64, seed=3)]))
    a_mid, a_in, a_out, dt = orc.pulse_table(pulse, n)
    xs = orc.grid_nodes(-3.0, 3.0, 32)
    r = orc.solve_points(xs[idx % 32], xs[idx // 32], a_mid, dt, a_in, a_out)
    assert r["cplus2"].max() > 0.1
    err = np.abs(m[idx] - r["cplus2"]).max()
    assert err <= TOL["fp32_mixed"][0], f"max error {err:.3e} over 4.4e6 steps"


def _sampled_parity(orc, cfg, prec, n_sample=256, seed=5, band_rows=8):
    """Full-size solve on the GPU; seeded points plus a band around p_y = 0
    (where pairs are likely) recomputed one by one by the oracle."""
    g = cfg["grid"]
    m, n = run_gpu(g, B.sample_pulse(cfg["pulse"], cfg["steps"]), prec)
    tab = orc.pulse_table(cfg["pulse"], cfg["steps"])
    idx = W.sample_points(g["nx"], g["ny"], n_sample, seed=seed)
    rows = np.arange(g["ny"] // 2 - band_rows // 2, g["ny"] // 2 + band_rows // 2)
    cols = np.linspace(0, g["nx"] - 1, 24).astype(int)
    idx = np.unique(np.concatenate([idx, (rows[:, None] * g["nx"] + cols[None, :]).ravel()]))
    xs = orc.grid_nodes(*g["px"], g["nx"])
    ys = orc.grid_nodes(*g["py"], g["ny"])
    r = orc.solve_points(xs[idx % g["nx"]], ys[idx // g["nx"]], tab[0], tab[3], tab[1], tab[2])
    err = np.abs(m.ravel()[idx] - r["cplus2"]).max()
    assert err <= TOL[prec][0], f"{prec}: sampled max error {err:.3e}"
    assert np.all(np.isfinite(m)) and m.min() >= 0.0 and m.max() <= 1.0 + 1e-6
    return m, n, r


@pytest.mark.parametrize("prec", ["fp64", "fp32_mixed"])
@pytest.mark.parametrize("E0", [0.5, 2.0, 5.0])
def test_gauss_1024_full_size_sampled(orc, prec, E0):
    """1024x1024 on [-8,8]^2, Gaussian pulse (tau = 4 cycles), 3e4 steps."""
    _sampled_parity(orc, W.config_gauss_1024(E0), prec)


def test_two_colour_4096_both_precisions(orc):
    """4096x4096 on [-12,12]^2, two-colour elliptical pulse, 2e5 steps, in FP64
    (about two and a half minutes) and FP32-mixed.  Each map against the oracle
    on 448 seeded and central-row points, one by one; FP32-mixed against the
    FP64 map at every one of the 16.8 M points and in density."""
    cfg = W.config_two_colour_4096()
    m64, n64, r64 = _sampled_parity(orc, cfg, "fp64", n_sample=352, band_rows=4)
    m32, n32, r32 = _sampled_parity(orc, cfg, "fp32_mixed", n_sample=352, band_rows=4)
    err = float(np.abs(m32 - m64).max())
    rel = abs(n32 - n64) / n64
    print(f"two-colour 4096^2: FP32-mixed vs FP64 every point {err:.3e}, density {rel:.3e}")
    assert err <= TOL["fp32_mixed"][0], f"FP32-mixed vs FP64, every point: {err:.3e}"
    assert rel <= TOL["fp32_mixed"][1], f"density relative {rel:.3e}"


def _every_point_vs_fp64(orc, sample, expect_group):
    """One LZS sample at full size (2048^2 x 1e5 steps), solved in both
    precisions in the benchmark's launch configuration.  FP64 against the
    oracle on 384 seeded points plus the map's 128 largest values (1e-9);
    FP32-mixed against that FP64 map at EVERY point (1e-5) and in density
    (1e-4 relative), so a regression at the few sensitive points of the LZS
    fringes, which sampling misses, fails here."""
    cfg = W.config_lzs_2048(sample)
    g = cfg["grid"]
    tab = B.sample_pulse(cfg["pulse"], cfg["steps"])
    gr = B.Grid(g["nx"], g["ny"], g["px"], g["py"], "fp32_mixed")
    gr.set_pulse(tab[0], tab[3], tab[1], tab[2])
    group = B.get_info(gr.h)["group_steps"]
    gr.close()
    assert group == expect_group
    m64, n64 = run_gpu(g, tab, "fp64")
    m32, n32 = run_gpu(g, tab, "fp32_mixed")
    tab_o = orc.pulse_table(cfg["pulse"], cfg["steps"])
    idx = W.sample_points(g["nx"], g["ny"], 384, seed=31 + sample)
    idx = np.unique(np.concatenate([idx, np.argsort(m64.ravel())[-128:]]))
    xs = orc.grid_nodes(*g["px"], g["nx"])
    ys = orc.grid_nodes(*g["py"], g["ny"])
    r = orc.solve_points(xs[idx % g["nx"]], ys[idx // g["nx"]], tab_o[0], tab_o[3], tab_o[1],
                         tab_o[2])
    e64 = float(np.abs(m64.ravel()[idx] - r["cplus2"]).max())
    err = np.abs(m32 - m64)
    e32 = float(err.max())
    rel = abs(n32 - n64) / n64
    worst = np.unravel_index(int(np.argmax(err)), err.shape)
    print(f"LZS sample {sample} (groups of {group}): FP64 vs oracle {e64:.3e}; FP32-mixed vs "
          f"FP64 every point {e32:.3e} at row/col {worst}, density {rel:.3e}")
    assert e64 <= TOL["fp64"][0], f"sample {sample}: FP64 vs oracle {e64:.3e}"
    assert e32 <= TOL["fp32_mixed"][0], (
        f"sample {sample}: FP32-mixed vs FP64 at every point: max {e32:.3e} at {worst}")
    assert rel <= TOL["fp32_mixed"][1], f"sample {sample}: density relative {rel:.3e}"


def test_lzs_sample6_every_point_vs_fp64(orc):
    """The sample with the largest theta_max (0.027, groups of 8, G theta_max =
    0.214): the worst per-point FP32-mixed error of the eight (4.3e-6 measured
    over every point, in groups of 4 and of 8 alike)."""
    _every_point_vs_fp64(orc, 6, expect_group=8)


def test_lzs_sample1_every_point_vs_fp64(orc):
    """A sample whose groups of 16 need the 0.27 group angle (G theta_max =
    0.211; groups of 8 under 0.2)."""
    _every_point_vs_fp64(orc, 1, expect_group=16)


def test_lzs_sample3_every_point_vs_fp64(orc):
    """The groups-of-16 sample with the largest per-point error (5.2e-6)."""
    _every_point_vs_fp64(orc, 3, expect_group=16)


@pytest.mark.parametrize("prec", ["fp64", "fp32_mixed"])
def test_row_bands_bitwise_equal_full_grid(prec):
    """A 300x257 grid cut into 3 ragged row bands (86, 86, 85 rows: tiles that
    straddle rows, a ragged last tile in every band), each solved as its own
    band grid: the band maps put together are bitwise the full-grid map, and
    the band densities summed in rank order match the full density to rounding
    (the tile partial sums are grouped differently)."""
    from paper_1607_03062_gb300 import shard
    grid = {"nx": 300, "ny": 257, "px": (-4.0, 4.0), "py": (-3.0, 5.0)}
    tab = B.sample_pulse(W.sin2_pulse(1.5, 1.3, 4.0, eps=0.3), 1700)
    m_full, n_full = run_gpu(grid, tab, prec)
    maps, dens = [], []
    for r in range(3):
        band = shard.band_grid(grid, r, 3)
        g = B.Grid(band["nx"], band["ny"], band["px"], band["py"], prec, rows=band["rows"])
        info = B.get_info(g.h)
        assert (info["row_begin"], info["ny_total"], info["ny"]) == (
            band["rows"][0], 257, band["rows"][1] - band["rows"][0])
        g.set_pulse(tab[0], tab[3], tab[1], tab[2])
        m, n = g.solve()
        torch.cuda.synchronize()
        maps.append(m.double().cpu().numpy().copy())
        dens.append(n)
        g.close()
    assert np.array_equal(np.concatenate(maps), m_full)
    total = shard.combine_densities(dens)
    assert total == (dens[0] + dens[1]) + dens[2]  # rank order, left to right
    assert abs(total - n_full) <= 1e-12 * n_full


def test_evolve_batch_reports_a_failing_member_on_that_grid():
    """Two grids in one batched launch, the second with its first A(t) chunk
    withheld: its bounded waits run out and its next synchronising call returns
    DSP_E_TIMEOUT (and stays latched), while the first grid, which shared the
    launch, projects and reduces normally to the result it has alone."""
    grid = {"nx": 32, "ny": 32, "px": (-2, 2), "py": (-2, 2)}  # one CTA each
    tab = B.sample_pulse(W.sin2_pulse(1.0, 1.55, 2.0), 3000)
    m_alone, n_alone = run_gpu(grid, tab, "fp32_mixed")
    g1 = B.Grid(32, 32, grid["px"], grid["py"], "fp32_mixed")
    g2 = B.Grid(32, 32, grid["px"], grid["py"], "fp32_mixed")
    for g in (g1, g2):
        g.set_pulse(tab[0], tab[3], tab[1], tab[2])
    B.test_withhold_next_copy(g2.h)
    B.evolve_batch([g1.h, g2.h], [3000, 3000])
    m1 = g1.project()
    n1 = g1.density()
    assert np.array_equal(m1.double().cpu().numpy(), m_alone) and n1 == n_alone
    g2.project()
    with pytest.raises(B.DSPError) as e:
        g2.density()
    assert e.value.code == -6
    with pytest.raises(B.DSPError) as e:
        g2.evolve(0)
    assert e.value.code == -6
    g1.close()
    g2.close()
    m, n = run_gpu(grid, tab, "fp32_mixed")  # the context still works
    assert n == n_alone


@pytest.mark.parametrize("prec", ["fp64", "fp32_mixed"])
def test_dropping_the_final_state_keeps_map_and_density(prec):
    """With the final state not kept, dsp_solve writes the same map and density
    bitwise; the state is then gone (project, solve and save_state refuse with
    DSP_E_STATE) until the next set_pulse."""
    grid = {"nx": 90, "ny": 70, "px": (-4, 4), "py": (-4, 4)}
    tab = B.sample_pulse(W.sin2_pulse(1.0, 1.55, 5.0), 1300)
    m_ref, n_ref = run_gpu(grid, tab, prec)
    g = B.Grid(90, 70, grid["px"], grid["py"], prec)
    B.set_keep_final_state(g.h, False)
    g.set_pulse(tab[0], tab[3], tab[1], tab[2])
    m, n = g.solve()
    torch.cuda.synchronize()
    assert np.array_equal(m.double().cpu().numpy(), m_ref) and n == n_ref
    for call in (g.project, g.solve,
                 lambda: B.save_state(g.h, np.zeros(B.state_bytes(90, 70, prec), np.uint8))):
        with pytest.raises(B.DSPError) as e:
            call()
        assert e.value.code == -4
    assert g.density() == n_ref  # the partial sums of the last projection are still there
    g.set_pulse(tab[0], tab[3], tab[1], tab[2])
    m, n = g.solve()
    torch.cuda.synchronize()
    assert np.array_equal(m.double().cpu().numpy(), m_ref) and n == n_ref
    g.close()


@pytest.mark.parametrize("offset", [1e-4, 1e-12, 1e-15])
def test_standalone_projection_matches_fused_near_p_out_zero(orc, offset):
    """A_out != 0 (the paper pulse with phi = pi/3) and a grid placed so that one
    node sits at p + A_out ~ (offset, 0): at 1e-15 eV that point takes the FP64
    form of the projection, at larger offsets the double-float form.  The
    projection-only launch (after evolving in pieces) and the projection fused
    into the last evolve launch give the same bits in both precisions, every
    value is a probability, and FP32-mixed meets FP64.  At offset 1e-4 the FP64
    map also meets the oracle at every point (closer to zero the two pulse
    samplers' 1e-15 difference in A_out alone turns the projection direction by
    ~1e-15/offset)."""
    pulse = W.paper_pulse(phi=math.pi / 3)
    steps = 4000
    tab = B.sample_pulse(pulse, steps)
    ax, ay = tab[2]
    assert abs(ax) > 1e-3 and ay == 0.0
    h = 0.01
    grid = {"nx": 33, "ny": 31, "px": (-ax - 16.5 * h + offset, -ax + 16.5 * h + offset),
            "py": (-15.5 * h, 15.5 * h)}
    maps = {}
    for prec in ("fp64", "fp32_mixed"):
        m1, n1 = run_gpu(grid, tab, prec)
        m2, n2 = run_gpu(grid, tab, prec, pieces=[1600, 2400])
        assert np.array_equal(m1, m2) and n1 == n2
        assert np.all(np.isfinite(m1)) and m1.min() >= 0.0 and m1.max() <= 1.0 + 1e-6
        maps[prec] = m1
    assert np.abs(maps["fp32_mixed"] - maps["fp64"]).max() <= TOL["fp32_mixed"][0]
    if offset >= 1e-4:
        ref, nref = run_oracle(orc, grid, orc.pulse_table(pulse, steps))
        m, n = run_gpu(grid, tab, "fp64")
        assert_close("fp64", m, n, ref, nref)


@pytest.mark.parametrize("prec", ["fp64", "fp32_mixed"])
@pytest.mark.parametrize("phi", [0.0, math.pi / 3])
def test_paper_laser_pulse_map(orc, prec, phi):
    """Sec. IV pulse (Fig. 1 parameters in eV units).  With phi = 0 the field is
    odd about T/2, so A_out = 0; phi = pi/3 gives A_out != 0, so the projection
    uses a shifted momentum.  Whole 64x64 map on [-0.5,0.5]^2."""
    pulse = W.paper_pulse(phi=phi)
    grid = {"nx": 64, "ny": 64, "px": (-0.5, 0.5), "py": (-0.5, 0.5)}
    steps = 20000
    tab_o = orc.pulse_table(pulse, steps)
    if phi != 0.0:
        assert abs(tab_o[2][0]) > 1e-3
    ref, nref = run_oracle(orc, grid, tab_o)
    m, n = run_gpu(grid, B.sample_pulse(pulse, steps), prec)
    assert ref.max() > 1e-3
    assert_close(prec, m, n, ref, nref)


# ----------------------------------------------------------------------------------------
# Fourth-order Magnus scheme (two Gauss points per step)
# ----------------------------------------------------------------------------------------

@pytest.mark.parametrize("prec", ["fp64", "fp32_mixed"])
@pytest.mark.parametrize("valley", [1, -1])
def test_magnus4_ragged_against_oracle(orc, prec, valley):
    grid = {"nx": 67, "ny": 45, "px": (-3.0, 5.0), "py": (-2.5, 3.5)}
    pulse = W.sin2_pulse(2.0, 1.2, 4.0, eps=0.6)
    n = 1500
    a, a_in, a_out, dt = orc.pulse_table_gauss(pulse, n)
    ref, _, _, nref = orc.solve_grid(67, 45, grid["px"], grid["py"], a, dt, a_in, a_out,
                                     scheme="magnus4", valley=valley)
    m, dens = run_gpu(grid, B.sample_pulse_gauss(pulse, n), prec, "magnus4", valley,
                      pieces=[600, 1, 899])
    assert_close(prec, m, dens, ref, nref)


@pytest.mark.parametrize("G", sorted(GROUP_STEPS_MAGNUS4))
def test_magnus4_step_groups_vs_oracle_and_pieces(orc, G):
    """FP32-mixed MAGNUS4 in each group size: the library reports it, the result meets the oracle at the
    FP32-mixed tolerance, pieces ending on multiples of 16 are bitwise the
    one-launch result, and boundaries inside groups change rounding only."""
    grid = {"nx": 48, "ny": 40, "px": (-4, 4), "py": (-4, 4)}
    pulse = W.sin2_pulse(1.0, 1.55, 5.0, eps=0.4)
    n = GROUP_STEPS_MAGNUS4[G]
    tab = B.sample_pulse_gauss(pulse, n)
    g = B.Grid(48, 40, grid["px"], grid["py"], "fp32_mixed", "magnus4")
    g.set_pulse(tab[0], tab[3], tab[1], tab[2])
    info = B.get_info(g.h)
    g.close()
    assert info["group_steps"] == G
    a, a_in, a_out, dt = orc.pulse_table_gauss(pulse, n)
    ref, _, _, nref = orc.solve_grid(48, 40, grid["px"], grid["py"], a, dt, a_in, a_out,
                                     scheme="magnus4")
    m1, n1 = run_gpu(grid, tab, "fp32_mixed", "magnus4")
    assert_close("fp32_mixed", m1, n1, ref, nref)
    m2, n2 = run_gpu(grid, tab, "fp32_mixed", "magnus4", pieces=[16 * 19, 16 * 25, n - 16 * 44])
    assert np.array_equal(m1, m2) and n1 == n2
    m3, n3 = run_gpu(grid, tab, "fp32_mixed", "magnus4", pieces=[299, 5, 3, n - 307])
    assert_close("fp32_mixed", m3, n3, ref, nref)
    if G == 1:
        assert np.array_equal(m1, m3) and n1 == n3
    else:
        assert np.abs(m1 - m3).max() <= 1e-6


@pytest.mark.parametrize("prec", ["fp64", "fp32_mixed"])
def test_magnus4_reaches_midpoint_accuracy_with_fewer_steps(orc, prec):
    """Against a converged oracle reference, MAGNUS4 with 500 steps is far more
    accurate than the midpoint scheme with 2000 steps (fourth vs second order)."""
    cfg = W.config_sin2_64()
    g = cfg["grid"]
    a, a_in, a_out, dt = orc.pulse_table_gauss(cfg["pulse"], 16000)
    ref, _, _, _ = orc.solve_grid(g["nx"], g["ny"], g["px"], g["py"], a, dt, a_in, a_out,
                                  scheme="magnus4")
    m4, _ = run_gpu(g, B.sample_pulse_gauss(cfg["pulse"], 500), prec, "magnus4")
    mid, _ = run_gpu(g, B.sample_pulse(cfg["pulse"], 2000), prec, "exact")
    err4, err2 = np.abs(m4 - ref).max(), np.abs(mid - ref).max()
    assert err4 < 0.1 * err2, (err4, err2)


@pytest.mark.parametrize("prec", ["fp64", "fp32_mixed"])
def test_magnus4_segmented_and_served(orc, prec):
    grid = {"nx": 48, "ny": 40, "px": (-4.0, 4.0), "py": (-4.0, 4.0)}
    pulse = W.sin2_pulse(1.5, 1.3, 3.0, eps=0.2)
    n = 900
    a, a_in, a_out, dt = orc.pulse_table_gauss(pulse, n)
    ref, _, _, nref = orc.solve_grid(48, 40, grid["px"], grid["py"], a, dt, a_in, a_out,
                                     scheme="magnus4")
    tab = B.sample_pulse_gauss(pulse, n)
    g = B.Grid(48, 40, grid["px"], grid["py"], prec, "magnus4")
    g.set_pulse(tab[0], tab[3], tab[1], tab[2])
    m, dens = g.solve_segmented(0)
    torch.cuda.synchronize()
    assert_close(prec, m.double().cpu().numpy(), dens, ref, nref)
    g.close()
    m_alone, n_alone = run_gpu(grid, tab, prec, "magnus4")
    srv = B.server_create(1 << 30, 4, 250)
    rid = B.server_submit(srv, B.make_request(grid, n, tab[3], tab[1], tab[2], prec, "magnus4",
                                              keep_map=True), tab[0])
    for _ in range(100):
        act, q, f = B.server_step(srv)
        if act == 0 and q == 0:
            break
    out = np.zeros((40, 48), dtype=np.float64 if prec == "fp64" else np.float32)
    state, dens_s, _ = B.server_query(srv, rid, out)
    B.server_destroy(srv)
    assert state == "done" and dens_s == n_alone
    assert np.array_equal(out.astype(np.float64), m_alone)


def test_device_wait_timeout_is_reported_and_context_survives():
    """A launch whose first A(t) chunk is never copied: every CTA's bounded
    mbarrier wait runs out, the kernel flags it and returns; the host reports
    DSP_E_TIMEOUT and the CUDA context keeps working for a fresh grid."""
    import time
    grid = {"nx": 32, "ny": 32, "px": (-2, 2), "py": (-2, 2)}  # one CTA
    tab = B.sample_pulse(W.sin2_pulse(1.0, 1.55, 2.0), 3000)
    g = B.Grid(32, 32, grid["px"], grid["py"], "fp32_mixed")
    g.set_pulse(tab[0], tab[3], tab[1], tab[2])
    B.test_withhold_next_copy(g.h)
    t0 = time.perf_counter()
    with pytest.raises(B.DSPError) as e:
        g.solve()
    assert e.value.code == -6
    assert time.perf_counter() - t0 < 30.0
    with pytest.raises(B.DSPError) as e:  # the grid stays latched
        g.evolve(0)
    assert e.value.code == -6
    g.close()
    torch.cuda.synchronize()  # the context is fine
    m, n = run_gpu(grid, tab, "fp32_mixed")
    assert np.isfinite(n) and n > 0
