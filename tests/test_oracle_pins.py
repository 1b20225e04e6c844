"""Pins of the FP64 oracle to things other than itself (CPU only).

Each test ties one part of the oracle to a closed form, a library routine, an
invariant the paper states, or brute force, chosen so that a plausible slip (a
dropped term, a wrong sign or index, a swapped spinor, the wrong time sample)
fails at least one of them.
"""
import math

import numpy as np
import pytest
import scipy.linalg

from paper_1607_03062_gb300 import workloads as W

SX = np.array([[0, 1], [1, 0]], dtype=complex)
SY = np.array([[0, -1j], [1j, 0]], dtype=complex)


# ----------------------------------------------------------------------------------------
# One step (Sec. III closed form) against a generic matrix exponential.
# ----------------------------------------------------------------------------------------

@pytest.mark.parametrize("valley", [1, -1])
def test_step_matrix_equals_expm(orc, valley):
    rng = np.random.default_rng(11)
    for _ in range(50):
        Px, Py = rng.uniform(-20, 20, size=2)
        dt = rng.uniform(1e-4, 0.15)
        H = valley * (Px * SX + Py * SY)
        ref = scipy.linalg.expm(-1j * dt * H)
        got = orc.step_matrix(Px, Py, dt, "exact", valley)
        assert np.abs(got - ref).max() < 2e-14


def test_step_matrix_zero_momentum_is_identity(orc):
    got = orc.step_matrix(0.0, 0.0, 0.3, "exact", 1)
    assert np.abs(got - np.eye(2)).max() == 0.0


@pytest.mark.parametrize("valley", [1, -1])
def test_strang_xy_equals_product_of_expms(orc, valley):
    rng = np.random.default_rng(12)
    for _ in range(30):
        Px, Py = rng.uniform(-10, 10, size=2)
        dt = rng.uniform(1e-4, 0.1)
        X = scipy.linalg.expm(-1j * valley * dt / 2 * Px * SX)
        Y = scipy.linalg.expm(-1j * valley * dt * Py * SY)
        ref = X @ Y @ X
        got = orc.step_matrix(Px, Py, dt, "strang_xy", valley)
        assert np.abs(got - ref).max() < 2e-14
        # and it differs from the exact exponential at O(dt^3) (sx, sy do not commute)
        ex = orc.step_matrix(Px, Py, dt, "exact", valley)
        assert np.abs(got - ex).max() < 0.5 * (dt * math.hypot(Px, Py)) ** 3 + 1e-14


# ----------------------------------------------------------------------------------------
# Free spinors (Sec. II): eigenvectors of valley*sigma.P, orthogonal, normalised.
# ----------------------------------------------------------------------------------------

@pytest.mark.parametrize("valley", [1, -1])
def test_spinors_are_energy_eigenstates(orc, valley):
    rng = np.random.default_rng(13)
    for _ in range(50):
        Px, Py = rng.uniform(-5, 5, size=2)
        E = math.hypot(Px, Py)
        H = valley * (Px * SX + Py * SY)
        u, v = orc.spinors(Px, Py, valley)
        assert np.abs(H @ u - E * u).max() < 1e-13
        assert np.abs(H @ v + E * v).max() < 1e-13
        assert abs(np.vdot(u, v)) < 1e-15
        assert abs(np.vdot(u, u) - 1) < 1e-15 and abs(np.vdot(v, v) - 1) < 1e-15


# ----------------------------------------------------------------------------------------
# Whole evolutions.
# ----------------------------------------------------------------------------------------

def _c1(orc, steps=2000, E0=1.0):
    cfg = W.config_sin2_64()
    pulse = W.sin2_pulse(E0, 1.55, 5.0)
    return orc.pulse_table(pulse, steps), cfg


def test_unitarity_norm_conserved(orc):
    """Sec. III: every step is unitary, so |psi|^2 = 1 and |c+|^2 + |c-|^2 = 1."""
    (a_mid, a_in, a_out, dt), _ = _c1(orc)
    rng = np.random.default_rng(1)
    px, py = rng.uniform(-4, 4, size=(2, 200))
    for scheme in ("exact", "strang_xy"):
        r = orc.solve_points(px, py, a_mid, dt, a_in, a_out, scheme=scheme)
        assert np.abs(r["norm2"] - 1).max() < 1e-12
        assert np.abs(r["cplus2"] + r["cminus2"] - 1).max() < 1e-12


def test_zero_field_gives_no_pairs(orc):
    """A = 0: the initial negative-energy state is stationary, so |c+|^2 = 0 (a
    swapped u/v would give 1)."""
    a_mid, a_in, a_out, dt = orc.pulse_table(W.zero_pulse(20.0), 1000)
    cp, cm, nr, n = orc.solve_grid(16, 12, (-4, 4), (-3, 3), a_mid, dt, a_in, a_out)
    assert cp.max() < 1e-28 and n < 1e-28
    assert np.abs(cm - 1).max() < 1e-12


def test_strang_xy_zero_field_residue_scales_dt4(orc):
    """The sx/sy split is not exact even for constant P: |c+|^2 = O((dt E)^4)."""
    px, py = np.array([1.3, -0.7]), np.array([0.9, 2.1])
    res = []
    for n in (400, 800):
        a_mid, a_in, a_out, dt = orc.pulse_table(W.zero_pulse(10.0), n)
        r = orc.solve_points(px, py, a_mid, dt, a_in, a_out, scheme="strang_xy")
        res.append(r["cplus2"])
    ratio = res[0] / res[1]
    assert np.all(res[0] > 0) and np.all((ratio > 12) & (ratio < 20))


def test_x_line_is_a_sigma_x_eigenproblem(orc):
    """p_y = 0 with an x field: H ~ sigma_x for all t, so the sigma_x state is kept
    and |c+|^2 is 1 exactly when sign(P_x) differs between t_i and t_f."""
    E0, T = 1.0, 30.0
    a_mid, a_in, a_out, dt = orc.pulse_table(W.const_field_pulse(E0, T), 3000)
    px = np.array([-20.0, -14.5, -10.0, -3.0, 0.7, 9.0, 14.9, 16.0])
    py = np.zeros_like(px)
    r = orc.solve_points(px, py, a_mid, dt, a_in, a_out)
    flip = np.sign(px + a_in[0]) != np.sign(px + a_out[0])
    assert np.abs(r["cplus2"] - flip.astype(float)).max() < 1e-13


@pytest.mark.parametrize("E0", [1.0, 2.0])
def test_landau_zener_closed_form(orc, E0):
    """Constant field: |c+|^2 -> exp(-pi p_y^2 / E0) at p_x = 0 as T grows."""
    py = np.linspace(0.0, 1.5 * math.sqrt(E0), 7)
    px = np.zeros_like(py)
    errs = []
    for T in (50.0, 100.0, 200.0):
        a_mid, a_in, a_out, dt = orc.pulse_table(W.const_field_pulse(E0, T), int(T / 0.01))
        r = orc.solve_points(px, py, a_mid, dt, a_in, a_out)
        errs.append(np.abs(r["cplus2"] - np.exp(-math.pi * py ** 2 / E0)).max())
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1e-5


def test_constant_field_density_rate(orc):
    """Integrating the LZ probability over the swept momenta, with degeneracy 4 and
    the (2 pi)^2 measure: n -> E0^(3/2) T / pi^2.  Pins the density prefactor,
    the grid spacing and the cell-centred nodes."""
    E0 = 1.0
    rel = []
    for T in (30.0, 60.0):
        a_mid, a_in, a_out, dt = orc.pulse_table(W.const_field_pulse(E0, T), int(T / 0.02))
        half = E0 * T / 2 + 6.0
        nx, ny = int(2 * half / 0.1), 60
        _, _, _, n = orc.solve_grid(nx, ny, (-half, half), (-3.0, 3.0), a_mid, dt, a_in, a_out)
        expect = E0 ** 1.5 * T / math.pi ** 2
        rel.append(abs(n - expect) / expect)
    assert rel[1] < rel[0] and rel[1] < 0.03


def test_weak_field_first_order_perturbation(orc):
    """First-order adiabatic perturbation theory for a weak x field:
    |c+|^2 ~ p_y^2/(4|p|^4) |int E_x(t) exp(2i|p|t) dt|^2 with E_x = -dA_x/dt."""
    E0, om = 1e-3, 1.55
    pulse = W.sin2_pulse(E0, om, 5.0)
    T = pulse["T"]
    a_mid, a_in, a_out, dt = orc.pulse_table(pulse, 20000)
    px = np.array([0.3, 0.5, 0.775, 0.6, -0.7])
    py = np.array([0.4, 0.3, 0.1, -0.5, 0.2])
    r = orc.solve_points(px, py, a_mid, dt, a_in, a_out)
    t = np.linspace(0.0, T, 200001)
    Ex = -(E0 / om) * ((math.pi / T) * np.sin(2 * math.pi * t / T) * np.sin(om * t)
                       + om * np.sin(math.pi * t / T) ** 2 * np.cos(om * t))
    pm = np.hypot(px, py)
    I = np.array([np.trapezoid(Ex * np.exp(2j * m * t), t) for m in pm])
    pt = py ** 2 / (4 * pm ** 4) * np.abs(I) ** 2
    assert np.abs(r["cplus2"] / pt - 1).max() < 1e-4


def test_momentum_symmetries(orc):
    """x-linear pulse: |c+(px,-py)| = |c+(px,py)|.  A(T-t) = -A(t) (integer-cycle
    sin^2; Gaussian with T = 6 tau): |c+(-p)| = |c+(p)|, exact in the discrete
    midpoint scheme on the cell-centred grid.  A wrong midpoint (A at t_n)
    breaks the second."""
    for pulse, n in ((W.sin2_pulse(1.0, 1.55, 5.0), 2000), (W.gauss_pulse(2.0, 1.55, 4.0), 4000)):
        a_mid, a_in, a_out, dt = orc.pulse_table(pulse, n)
        cp, _, _, _ = orc.solve_grid(24, 20, (-4, 4), (-4, 4), a_mid, dt, a_in, a_out)
        assert np.abs(cp - cp[::-1, :]).max() < 1e-12
        assert np.abs(cp - cp[::-1, ::-1]).max() < 1e-12
        assert cp.max() > 1e-3  # non-trivial


def test_valleys_give_the_same_probability(orc):
    (a_mid, a_in, a_out, dt), _ = _c1(orc)
    rng = np.random.default_rng(5)
    px, py = rng.uniform(-4, 4, size=(2, 100))
    for scheme in ("exact", "strang_xy"):
        kp = orc.solve_points(px, py, a_mid, dt, a_in, a_out, scheme=scheme, valley=1)
        km = orc.solve_points(px, py, a_mid, dt, a_in, a_out, scheme=scheme, valley=-1)
        assert np.abs(kp["cplus2"] - km["cplus2"]).max() < 1e-12


def test_second_order_convergence(orc):
    """Sec. III: local O(dt^3), so global O(dt^2).  Error against a dt/32 run on a
    16-point sub-grid; log-log slope 2.0 +- 0.1."""
    pulse = W.sin2_pulse(1.0, 1.55, 5.0)
    rng = np.random.default_rng(2)
    px, py = rng.uniform(-2, 2, size=(2, 16))

    def amp(n):
        a_mid, a_in, a_out, dt = orc.pulse_table(pulse, n)
        r = orc.solve_points(px, py, a_mid, dt, a_in, a_out, want_psi=True)
        return r["psi"], dt

    ref, _ = amp(64000)
    errs, dts = [], []
    for n in (500, 1000, 2000):
        psi, dt = amp(n)
        errs.append(np.abs(psi - ref).max())
        dts.append(dt)
    slope = np.polyfit(np.log(dts), np.log(errs), 1)[0]
    assert abs(slope - 2.0) < 0.1

    # Teeth: sampling A at the left end of each step (a plausible slip) is only
    # first order, and this measurement sees it.
    left_errs = []
    for n in (500, 1000, 2000):
        a_mid, a_in, a_out, dt = orc.pulse_table(pulse, n)
        a_left = np.array([orc.pulse_A(pulse, k * dt) for k in range(n)])
        r = orc.solve_points(px, py, a_left, dt, a_in, a_out, want_psi=True)
        left_errs.append(np.abs(r["psi"] - ref).max())
    left_slope = np.polyfit(np.log(dts), np.log(left_errs), 1)[0]
    assert left_slope < 1.5


def test_points_are_independent(orc):
    """Sec. III: each momentum is independent -- any subset or thread count gives
    bitwise the same per-point result as the whole grid."""
    (a_mid, a_in, a_out, dt), _ = _c1(orc, steps=500)
    cp, _, _, _ = orc.solve_grid(10, 7, (-4, 4), (-4, 4), a_mid, dt, a_in, a_out, nthreads=3)
    xs, ys = orc.grid_nodes(-4, 4, 10), orc.grid_nodes(-4, 4, 7)
    idx = [3, 17, 40, 69]
    r = orc.solve_points(xs[np.array(idx) % 10], ys[np.array(idx) // 10], a_mid, dt, a_in,
                         a_out, nthreads=1)
    assert np.array_equal(r["cplus2"], cp.ravel()[idx])


def test_density_sum_matches_exact_summation(orc):
    rng = np.random.default_rng(3)
    x = rng.uniform(0, 1, size=100_003)
    got = orc.density(x, 0.01, 0.02)
    ref = 4.0 / (2 * math.pi) ** 2 * 0.01 * 0.02 * math.fsum(x)
    assert abs(got - ref) / ref < 1e-14


# ----------------------------------------------------------------------------------------
# Pulse tables (the workload inputs).
# ----------------------------------------------------------------------------------------

def test_pulse_table_samples_midpoints_and_ends(orc):
    pulse = W.sin2_pulse(1.0, 1.55, 5.0)
    a_mid, a_in, a_out, dt = orc.pulse_table(pulse, 200)
    assert dt == pytest.approx(pulse["T"] / 200, rel=1e-15)
    T, om = pulse["T"], pulse["omega"]
    t = (np.arange(200) + 0.5) * dt
    ref = (1.0 / om) * np.sin(math.pi * t / T) ** 2 * np.sin(om * t)
    assert np.abs(a_mid[:, 0] - ref).max() < 1e-15 and np.abs(a_mid[:, 1]).max() == 0
    assert np.abs(a_in).max() < 1e-15 and np.abs(a_out).max() < 1e-15


def test_gaussian_and_two_colour_tables(orc):
    g = W.gauss_pulse(2.0, 1.55, 4.0, eps=0.3)
    assert g["T"] == pytest.approx(6 * 4 * 2 * math.pi / 1.55)
    for t in (0.0, 7.3, g["t0"], 60.0):
        A = orc.pulse_A(g, t)
        env = math.exp(-((t - g["t0"]) / g["tau"]) ** 2)
        assert A[0] == pytest.approx((2.0 / 1.55) * env * math.sin(1.55 * t), abs=1e-15)
        assert A[1] == pytest.approx(0.3 * (2.0 / 1.55) * env * math.cos(1.55 * t), abs=1e-15)
    tc = W.two_colour_pulse(3.0, 1.55, 10.0, 0.5, math.pi / 3)
    t = 11.0
    env = math.sin(math.pi * t / tc["T"]) ** 2
    ax = env * (3 / 1.55 * math.sin(1.55 * t) + 3 / 3.1 * math.sin(3.1 * t + math.pi / 3))
    ay = env * 0.5 * (3 / 1.55 * math.cos(1.55 * t) + 3 / 3.1 * math.cos(3.1 * t + math.pi / 3))
    assert np.allclose(orc.pulse_A(tc, t), [ax, ay], atol=1e-15, rtol=0)


def test_const_field_is_minus_dA_dt(orc):
    p = W.const_field_pulse(1.7, 40.0)
    h = 1e-3
    for t in (1.0, 20.0, 39.0):
        E = -(orc.pulse_A(p, t + h)[0] - orc.pulse_A(p, t - h)[0]) / (2 * h)
        assert E == pytest.approx(1.7, rel=1e-10)


def test_paper_pulse_field_is_minus_dA_dt(orc):
    """Sec. IV Eq. (elec_field): the oracle integrates E_x into A_x = -int E_x.  The
    field is restated here piecewise (rise sin^2, flat, continuous cos^2 fall)
    and compared with -dA/dt by central differences."""
    p = W.paper_pulse()
    T, w, E0 = p["T"], p["omega"], p["E0"]
    Or, Of = p["Omega_rise"], p["Omega_fall"]

    def field(t):
        if t < math.pi / (2 * Or):
            env = math.sin(Or * t) ** 2
        elif t > T - math.pi / (2 * Of):
            env = math.cos(Of * (t - T + math.pi / (2 * Of))) ** 2
        else:
            env = 1.0
        return E0 * env * math.cos(w * t)

    h = 0.05
    for t in (37.0, 150.0, 400.0, 700.0, 830.0):
        E = -(orc.pulse_A(p, t + h)[0] - orc.pulse_A(p, t - h)[0]) / (2 * h)
        assert E == pytest.approx(field(t), rel=1e-5, abs=1e-9)
    assert abs(orc.pulse_A(p, 0.0)[0]) == 0.0


def test_paper_fig1_parameters_in_ev_units():
    """Sec. IV prints the Fig. 1 pulse in SI units; tests/golden/ holds the values
    and their eV-unit conversions (hbar = v_F = e = 1)."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "paper_fig1_parameters.txt")
    vals = {}
    for line in open(path):
        line = line.split("#")[0].strip()
        if line:
            k, v = line.split("=")
            vals[k.strip()] = float(v)
    p = W.paper_pulse(vals["nu_hz"], vals["E0_V_per_m"], vals["periods"],
                      vals["Omega_rise_per_s"], vals["Omega_fall_per_s"])
    assert p["omega"] == pytest.approx(vals["hbar_omega_eV"], rel=1e-3)
    assert p["E0"] == pytest.approx(vals["e_E0_hbar_vF_eV2"], rel=1e-3)
    assert p["Omega_rise"] == pytest.approx(vals["hbar_Omega_eV"], rel=1e-3)
    assert p["T"] == pytest.approx(vals["duration_hbar_per_eV"], rel=1e-3)
    assert W.VF_MPS == vals["v_F_m_per_s"]


def test_zero_momentum_point_is_defined(orc):
    """At P = 0 the free spinors are undefined; the oracle takes the limit
    P -> (0+, 0): still orthonormal, and a zero-field run from p = 0 stays put."""
    u, v = orc.spinors(0.0, 0.0, 1)
    assert abs(np.vdot(u, v)) < 1e-15 and abs(np.vdot(v, v) - 1) < 1e-15
    a_mid, a_in, a_out, dt = orc.pulse_table(W.zero_pulse(5.0), 100)
    r = orc.solve_points(np.array([0.0]), np.array([0.0]), a_mid, dt, a_in, a_out)
    assert r["cplus2"][0] == 0.0 and abs(r["norm2"][0] - 1) < 1e-15


# ----------------------------------------------------------------------------------------
# Fourth-order Magnus scheme (the higher-order decomposition of Sec. III).
# ----------------------------------------------------------------------------------------

@pytest.mark.parametrize("valley", [1, -1])
def test_magnus4_step_equals_expm_of_its_definition(orc, valley):
    """exp(dt/2 (A1 + A2) - sqrt(3) dt^2/12 [A1, A2]), A_k = -i valley sigma.P_k,
    built here as matrices and exponentiated by scipy."""
    rng = np.random.default_rng(21)
    for _ in range(40):
        P1 = rng.uniform(-8, 8, size=2)
        P2 = P1 + rng.uniform(-0.5, 0.5, size=2)
        dt = rng.uniform(1e-3, 0.1)
        A1 = -1j * valley * (P1[0] * SX + P1[1] * SY)
        A2 = -1j * valley * (P2[0] * SX + P2[1] * SY)
        W_ = 0.5 * dt * (A1 + A2) - math.sqrt(3) * dt * dt / 12 * (A1 @ A2 - A2 @ A1)
        ref = scipy.linalg.expm(W_)
        got = orc.step_matrix_magnus4(P1, P2, dt, valley)
        assert np.abs(got - ref).max() < 2e-14


def test_magnus4_gauss_table_points(orc):
    pulse = W.sin2_pulse(1.0, 1.55, 5.0)
    a, a_in, a_out, dt = orc.pulse_table_gauss(pulse, 300)
    c = (0.5 - math.sqrt(3) / 6, 0.5 + math.sqrt(3) / 6)
    for n in (0, 17, 299):
        assert np.allclose(a[n, 0:2], orc.pulse_A(pulse, (n + c[0]) * dt), atol=1e-16, rtol=0)
        assert np.allclose(a[n, 2:4], orc.pulse_A(pulse, (n + c[1]) * dt), atol=1e-16, rtol=0)


def test_magnus4_is_fourth_order_and_unitary(orc):
    """Global error O(dt^4) (slope 4.0 +- 0.3) against a fine reference; the
    midpoint scheme converges to the same solution at O(dt^2)."""
    pulse = W.sin2_pulse(1.0, 1.55, 5.0)
    rng = np.random.default_rng(22)
    px, py = rng.uniform(-2, 2, size=(2, 12))

    def psi(n, scheme):
        if scheme == "magnus4":
            a, a_in, a_out, dt = orc.pulse_table_gauss(pulse, n)
        else:
            a, a_in, a_out, dt = orc.pulse_table(pulse, n)
        r = orc.solve_points(px, py, a, dt, a_in, a_out, scheme=scheme, want_psi=True)
        assert np.abs(r["norm2"] - 1).max() < 1e-12
        return r["psi"], dt

    ref, _ = psi(16000, "magnus4")
    errs, dts = [], []
    for n in (250, 500, 1000):
        p_, dt = psi(n, "magnus4")
        errs.append(np.abs(p_ - ref).max())
        dts.append(dt)
    slope = np.polyfit(np.log(dts), np.log(errs), 1)[0]
    assert abs(slope - 4.0) < 0.3
    mid, _ = psi(64000, "exact")
    assert np.abs(mid - ref).max() < 1e-6


def test_magnus4_valleys_and_zero_field(orc):
    a, a_in, a_out, dt = orc.pulse_table_gauss(W.zero_pulse(10.0), 500)
    cp, _, _, _ = orc.solve_grid(9, 7, (-3, 3), (-2, 2), a, dt, a_in, a_out, scheme="magnus4")
    assert cp.max() < 1e-28
    a, a_in, a_out, dt = orc.pulse_table_gauss(W.sin2_pulse(1.5, 1.2, 4.0, eps=0.4), 800)
    rng = np.random.default_rng(23)
    px, py = rng.uniform(-3, 3, size=(2, 40))
    kp = orc.solve_points(px, py, a, dt, a_in, a_out, scheme="magnus4", valley=1)
    km = orc.solve_points(px, py, a, dt, a_in, a_out, scheme="magnus4", valley=-1)
    assert np.abs(kp["cplus2"] - km["cplus2"]).max() < 1e-12
