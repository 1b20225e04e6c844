"""FP64 CPU oracle for the split-operator massless-Dirac solve (arXiv 1607.03062).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  It wraps the plain C
file ``dirac_oracle.c`` (libm sin/cos/sqrt, C99 complex double, OpenMP over
points) through ctypes and shares nothing with the CUDA library.

Paper passages each function follows:
  * ``pulse_table``   -- Sec. III Eq. (approx_time): A sampled at step midpoints;
                         Sec. II: asymptotic A_in, A_out.
  * ``spinors``       -- Sec. II Eq. (free_spin1..4), normalised to 1.
  * ``step_matrix``   -- Sec. III closed form I cos(dt E) - i sigma.P sin(dt E)/E.
  * ``step_matrix_magnus4``, ``pulse_table_gauss`` -- the fourth-order Magnus
                         decomposition (Sec. III notes that other decompositions
                         would raise the order of the midpoint rule).
  * ``solve_points`` / ``solve_grid`` -- Sec. III Eq. (ev_op_dt) product of steps,
                         then the projection of Sec. II Eq. (pair_prod_homo).
  * ``density``       -- Sec. II Eq. (pair_prod_homo) with degeneracy 4.

Every function is pinned by ``tests/test_oracle_pins.py`` to closed forms,
library routines or invariants (no function here is "parity unpinned" except
the paper pulse's Fig. 1 map, whose printed image is absent).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dirac_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

PULSE_KINDS = {"zero": 0, "sin2": 1, "gauss": 2, "two_colour": 3, "const_field": 4, "paper": 5}
SCHEMES = {"exact": 0, "strang_xy": 1, "magnus4": 2}


class _Pulse(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int32),
        ("pad", ctypes.c_int32),
        ("E0", ctypes.c_double),
        ("omega", ctypes.c_double),
        ("T", ctypes.c_double),
        ("tau", ctypes.c_double),
        ("t0", ctypes.c_double),
        ("eps", ctypes.c_double),
        ("phase2", ctypes.c_double),
        ("Omega_rise", ctypes.c_double),
        ("Omega_fall", ctypes.c_double),
        ("phi", ctypes.c_double),
    ]


def build(force: bool = False) -> str:
    """Compile dirac_oracle.c with gcc (-O2, OpenMP, no FP contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            d, i32, i64, p = ctypes.c_double, ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p
            lib.orc_pulse_table.argtypes = [ctypes.POINTER(_Pulse), i64, p, p, p, ctypes.POINTER(d)]
            lib.orc_pulse_table.restype = ctypes.c_int
            lib.orc_pulse_table_gauss.argtypes = [ctypes.POINTER(_Pulse), i64, p, p, p,
                                                  ctypes.POINTER(d)]
            lib.orc_pulse_table_gauss.restype = ctypes.c_int
            lib.orc_step_matrix_magnus4.argtypes = [d, d, d, d, d, ctypes.c_int, p]
            lib.orc_step_matrix_magnus4.restype = None
            lib.orc_pulse_A.argtypes = [ctypes.POINTER(_Pulse), d, p]
            lib.orc_pulse_A.restype = None
            lib.orc_step_matrix.argtypes = [d, d, d, ctypes.c_int, ctypes.c_int, p]
            lib.orc_step_matrix.restype = None
            lib.orc_spinor_u.argtypes = [d, d, ctypes.c_int, p]
            lib.orc_spinor_u.restype = None
            lib.orc_spinor_v.argtypes = [d, d, ctypes.c_int, p]
            lib.orc_spinor_v.restype = None
            lib.orc_solve_points.argtypes = [i64, p, p, ctypes.c_int, ctypes.c_int, p, i64, d, p, p,
                                             p, p, p, p, ctypes.c_int]
            lib.orc_solve_points.restype = ctypes.c_int
            lib.orc_solve_grid.argtypes = [i32, i32, d, d, d, d, ctypes.c_int, ctypes.c_int, p, i64,
                                           d, p, p, p, p, p, ctypes.POINTER(d), ctypes.c_int]
            lib.orc_solve_grid.restype = ctypes.c_int
            lib.orc_density.argtypes = [i64, p, d, d]
            lib.orc_density.restype = d
            lib.orc_grid_node.argtypes = [d, d, ctypes.c_int, ctypes.c_int]
            lib.orc_grid_node.restype = d
            lib.orc_max_threads.argtypes = []
            lib.orc_max_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _pulse_struct(spec: dict) -> _Pulse:
    s = _Pulse()
    s.kind = PULSE_KINDS[spec["kind"]]
    for name in ("E0", "omega", "T", "tau", "t0", "eps", "phase2", "Omega_rise", "Omega_fall",
                 "phi"):
        setattr(s, name, float(spec.get(name, 0.0)))
    return s


def pulse_A(spec: dict, t: float) -> np.ndarray:
    """A(t) of the pulse described by ``spec`` (a workload dict with its own T)."""
    out = np.zeros(2)
    s = _pulse_struct(spec)
    _load().orc_pulse_A(ctypes.byref(s), float(t), _ptr(out))
    return out


def pulse_table(spec: dict, n_steps: int):
    """(a_mid[n_steps, 2], a_in[2], a_out[2], dt) with A at step midpoints."""
    a_mid = np.zeros((max(n_steps, 0), 2))
    a_in = np.zeros(2)
    a_out = np.zeros(2)
    dt = ctypes.c_double(0.0)
    s = _pulse_struct(spec)
    rc = _load().orc_pulse_table(ctypes.byref(s), int(n_steps), _ptr(a_mid), _ptr(a_in),
                                 _ptr(a_out), ctypes.byref(dt))
    if rc != 0:
        raise ValueError("bad pulse spec")
    return a_mid, a_in, a_out, dt.value


def pulse_table_gauss(spec: dict, n_steps: int):
    """(a_gauss[n_steps, 4], a_in, a_out, dt): A at the two Gauss points of each
    step, t_n + (1/2 -/+ sqrt(3)/6) dt, for the fourth-order Magnus scheme."""
    a = np.zeros((max(n_steps, 0), 4))
    a_in = np.zeros(2)
    a_out = np.zeros(2)
    dt = ctypes.c_double(0.0)
    s = _pulse_struct(spec)
    rc = _load().orc_pulse_table_gauss(ctypes.byref(s), int(n_steps), _ptr(a), _ptr(a_in),
                                       _ptr(a_out), ctypes.byref(dt))
    if rc != 0:
        raise ValueError("bad pulse spec")
    return a, a_in, a_out, dt.value


def step_matrix_magnus4(P1, P2, dt: float, valley: int = 1):
    out = np.zeros(8)
    _load().orc_step_matrix_magnus4(float(P1[0]), float(P1[1]), float(P2[0]), float(P2[1]),
                                    float(dt), int(valley), _ptr(out))
    return (out[0::2] + 1j * out[1::2]).reshape(2, 2)


def _table(a_mid, scheme):
    """Steps of a table: [n, 2] midpoint samples, or [n, 4] Gauss pairs (magnus4)."""
    w = 4 if scheme == "magnus4" else 2
    a = np.ascontiguousarray(a_mid, dtype=np.float64).reshape(-1, w)
    return a, a.shape[0]


def step_matrix(Px: float, Py: float, dt: float, scheme: str = "exact", valley: int = 1):
    out = np.zeros(8)
    _load().orc_step_matrix(float(Px), float(Py), float(dt), SCHEMES[scheme], int(valley),
                            _ptr(out))
    return (out[0::2] + 1j * out[1::2]).reshape(2, 2)


def spinors(Px: float, Py: float, valley: int = 1):
    """Normalised (u, v): positive- and negative-energy spinors of valley*sigma.P."""
    u = np.zeros(4)
    v = np.zeros(4)
    lib = _load()
    lib.orc_spinor_u(float(Px), float(Py), int(valley), _ptr(u))
    lib.orc_spinor_v(float(Px), float(Py), int(valley), _ptr(v))
    return u[0::2] + 1j * u[1::2], v[0::2] + 1j * v[1::2]


def solve_points(px, py, a_mid, dt, a_in, a_out, scheme="exact", valley=1, nthreads=0,
                 want_psi=False):
    """Evolve each point (px[k], py[k]); returns dict of |c+|^2, |c-|^2, |psi|^2 (and psi)."""
    px = np.ascontiguousarray(px, dtype=np.float64).ravel()
    py = np.ascontiguousarray(py, dtype=np.float64).ravel()
    a_mid, n_steps = _table(a_mid, scheme)
    a_in = np.ascontiguousarray(a_in, dtype=np.float64)
    a_out = np.ascontiguousarray(a_out, dtype=np.float64)
    n = px.size
    cp = np.zeros(n)
    cm = np.zeros(n)
    nr = np.zeros(n)
    psi = np.zeros((n, 4)) if want_psi else None
    rc = _load().orc_solve_points(n, _ptr(px), _ptr(py), SCHEMES[scheme], int(valley),
                                  _ptr(a_mid), n_steps, float(dt), _ptr(a_in),
                                  _ptr(a_out), _ptr(cp), _ptr(cm), _ptr(nr), _ptr(psi),
                                  int(nthreads))
    if rc != 0:
        raise ValueError(f"orc_solve_points failed ({rc})")
    out = {"cplus2": cp, "cminus2": cm, "norm2": nr}
    if want_psi:
        out["psi"] = psi[:, 0::2] + 1j * psi[:, 1::2]
    return out


def grid_nodes(lo: float, hi: float, n: int) -> np.ndarray:
    lib = _load()
    return np.array([lib.orc_grid_node(float(lo), float(hi), int(n), i) for i in range(n)])


def solve_grid(nx, ny, px_range, py_range, a_mid, dt, a_in, a_out, scheme="exact", valley=1,
               nthreads=0):
    """Whole cell-centred grid; returns (cplus2[ny, nx], cminus2, norm2, density)."""
    a_mid, n_steps = _table(a_mid, scheme)
    a_in = np.ascontiguousarray(a_in, dtype=np.float64)
    a_out = np.ascontiguousarray(a_out, dtype=np.float64)
    cp = np.zeros((ny, nx))
    cm = np.zeros((ny, nx))
    nr = np.zeros((ny, nx))
    dens = ctypes.c_double(0.0)
    rc = _load().orc_solve_grid(int(nx), int(ny), float(px_range[0]), float(px_range[1]),
                                float(py_range[0]), float(py_range[1]), SCHEMES[scheme],
                                int(valley), _ptr(a_mid), n_steps, float(dt), _ptr(a_in),
                                _ptr(a_out), _ptr(cp), _ptr(cm), _ptr(nr), ctypes.byref(dens),
                                int(nthreads))
    if rc != 0:
        raise ValueError(f"orc_solve_grid failed ({rc})")
    return cp, cm, nr, dens.value


def density(cplus2, hx: float, hy: float) -> float:
    c = np.ascontiguousarray(cplus2, dtype=np.float64).ravel()
    return _load().orc_density(c.size, _ptr(c), float(hx), float(hy))


def max_threads() -> int:
    return _load().orc_max_threads()
