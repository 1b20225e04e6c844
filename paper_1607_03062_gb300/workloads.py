"""Seeded synthetic workloads: grids, pulse parameters and request streams.

This module holds only the *inputs* of a solve -- grid extents, step counts and
the parameters of the vector-potential pulse -- plus the seeded random draws
that pick them.  It contains none of the method's arithmetic: the pulse A(t)
itself is evaluated independently by the CUDA library's host sampler and by
the oracle, from the parameter dictionaries built here.

Units throughout: hbar = v_F = e = 1, energy and momentum in eV, time in hbar/eV.

Pulse dictionaries (``kind`` plus parameters, all floats):
  * ``sin2``        A = (E0/w) sin^2(pi t/T) (sin wt, eps cos wt), t in [0, T]
  * ``gauss``       A = (E0/w) exp(-(t-t0)^2/tau^2) (sin wt, eps cos wt)
  * ``two_colour``  A = sin^2(pi t/T) sum_k (E0/(k w)) (sin(k w t + ph_k), eps cos(...)),
                    k = 1, 2; ph_1 = 0, ph_2 = phase2
  * ``const_field`` A_x = -E0 (t - T/2): a constant field E_x = E0 (Landau-Zener)
  * ``paper``       Sec. IV Eq. (elec_field): E_x with sin^2 rise, flat top and
                    cos^2 fall, A_x = -int_0^t E_x
  * ``zero``        A = 0
"""
from __future__ import annotations

import math

import numpy as np

TWO_PI = 2.0 * math.pi
# Conversion constants for the paper's physical-unit workload (Sec. IV):
# hbar in eV*s and hbar*v_F in eV*m with v_F = 1.093e6 m/s (Sec. I).
HBAR_EVS = 6.582119569e-16
VF_MPS = 1.093e6
HBAR_VF_EVM = HBAR_EVS * VF_MPS


def sin2_pulse(E0: float, omega: float, cycles: float, eps: float = 0.0) -> dict:
    return {"kind": "sin2", "E0": E0, "omega": omega, "T": cycles * TWO_PI / omega, "eps": eps}


def gauss_pulse(E0: float, omega: float, tau_cycles: float, eps: float = 0.0) -> dict:
    """Gaussian envelope of width tau = tau_cycles periods, centred at t0 = 3 tau,
    lasting T = 6 tau (so A(T - t) = -A(t) when omega*T is a multiple of 2 pi)."""
    tau = tau_cycles * TWO_PI / omega
    return {"kind": "gauss", "E0": E0, "omega": omega, "T": 6.0 * tau, "tau": tau,
            "t0": 3.0 * tau, "eps": eps}


def two_colour_pulse(E0: float, omega: float, cycles: float, eps: float, phase2: float) -> dict:
    return {"kind": "two_colour", "E0": E0, "omega": omega, "T": cycles * TWO_PI / omega,
            "eps": eps, "phase2": phase2}


def const_field_pulse(E0: float, T: float) -> dict:
    return {"kind": "const_field", "E0": E0, "T": T}


def zero_pulse(T: float) -> dict:
    return {"kind": "zero", "T": T}


def paper_pulse(nu_hz: float = 10e12, E0_vpm: float = 1.0e7, periods: float = 5.5,
                Omega_rise_hz: float = 7.85e12, Omega_fall_hz: float = 7.85e12,
                phi: float = 0.0) -> dict:
    """The laser pulse of Sec. IV (Fig. 1 parameters by default) in eV units.

    hbar*omega = 2 pi nu hbar; the field enters as e E0 hbar v_F (eV^2); the
    envelope frequencies as hbar*Omega (eV); the duration as periods/nu (in
    hbar/eV: seconds / hbar)."""
    omega = TWO_PI * nu_hz * HBAR_EVS
    return {"kind": "paper", "E0": E0_vpm * HBAR_VF_EVM, "omega": omega,
            "T": periods / nu_hz / HBAR_EVS, "Omega_rise": Omega_rise_hz * HBAR_EVS,
            "Omega_fall": Omega_fall_hz * HBAR_EVS, "phi": phi}


def grid(n: int, extent: float, ny: int | None = None) -> dict:
    """Square momentum box [-extent, extent]^2 with n (x) by ny (y) cell-centred nodes."""
    return {"nx": n, "ny": n if ny is None else ny, "px": (-extent, extent),
            "py": (-extent, extent)}


# --------------------------------------------------------------------------------------
# The five reference workloads.
# --------------------------------------------------------------------------------------

def config_sin2_64() -> dict:
    """64x64 grid on [-4,4]^2, 5-cycle sin^2 x-linear pulse, w = 1.55, E0 = 1, 2000 steps."""
    return {"name": "sin2_64x64_2000", "grid": grid(64, 4.0),
            "pulse": sin2_pulse(1.0, 1.55, 5.0), "steps": 2000}


def config_gauss_1024(E0: float) -> dict:
    """1024x1024 on [-8,8]^2, Gaussian x-linear pulse (tau = 4 cycles), 3e4 steps."""
    return {"name": f"gauss_1024x1024_E0_{E0:g}", "grid": grid(1024, 8.0),
            "pulse": gauss_pulse(E0, 1.55, 4.0), "steps": 30000}


def lzs_scan_samples(count: int = 8, seed: int = 1607) -> list[tuple[float, float]]:
    """(omega, E0) draws for the Landau-Zener-Stueckelberg scan: omega ~ U[0.5, 3],
    E0 ~ U[0.2, 6], from numpy's default_rng(seed)."""
    rng = np.random.default_rng(seed)
    om = rng.uniform(0.5, 3.0, size=count)
    e0 = rng.uniform(0.2, 6.0, size=count)
    return [(float(a), float(b)) for a, b in zip(om, e0)]


def config_lzs_2048(sample: int = 0, n: int = 2048, steps: int = 100_000) -> dict:
    """2048x2048 on [-10,10]^2, 20-cycle sin^2 x-linear pulse, seeded (omega, E0), 1e5 steps."""
    omega, E0 = lzs_scan_samples()[sample]
    return {"name": f"lzs_{n}x{n}_{steps}_s{sample}", "grid": grid(n, 10.0),
            "pulse": sin2_pulse(E0, omega, 20.0), "steps": steps, "omega": omega, "E0": E0}


def config_two_colour_4096(n: int = 4096, steps: int = 200_000) -> dict:
    """4096x4096 on [-12,12]^2, two-colour (w, 2w) elliptical pulse, 2e5 steps."""
    return {"name": f"two_colour_{n}x{n}_{steps}", "grid": grid(n, 12.0),
            "pulse": two_colour_pulse(3.0, 1.55, 10.0, 0.5, math.pi / 3.0), "steps": steps}


def serving_requests(count: int = 256, seed: int = 1607, rate_hz: float = 50.0,
                     sizes=(128, 256, 512, 1024), steps_range=(1000, 100_000),
                     extent: float = 8.0) -> list[dict]:
    """Seeded Poisson request stream: exponential inter-arrival gaps at ``rate_hz``,
    grid N uniform in ``sizes``, ellipticity ~ U[0,1], omega ~ U[0.8, 2.5],
    E0 ~ U[0.5, 4], steps uniform integer in ``steps_range``; 5-cycle sin^2
    envelope on [-extent, extent]^2."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_hz, size=count)
    arrivals = np.cumsum(gaps) - gaps[0]
    ns = rng.choice(np.asarray(sizes), size=count)
    eps = rng.uniform(0.0, 1.0, size=count)
    om = rng.uniform(0.8, 2.5, size=count)
    e0 = rng.uniform(0.5, 4.0, size=count)
    st = rng.integers(steps_range[0], steps_range[1] + 1, size=count)
    reqs = []
    for k in range(count):
        reqs.append({"id": k, "arrival_s": float(arrivals[k]), "grid": grid(int(ns[k]), extent),
                     "pulse": sin2_pulse(float(e0[k]), float(om[k]), 5.0, float(eps[k])),
                     "steps": int(st[k])})
    return reqs


def sample_points(nx: int, ny: int, count: int, seed: int = 7) -> np.ndarray:
    """Seeded flat indices (row-major, x fastest) of grid points to compare one by one."""
    rng = np.random.default_rng(seed)
    total = nx * ny
    count = min(count, total)
    return np.sort(rng.choice(total, size=count, replace=False))
