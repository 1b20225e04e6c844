"""Thin ctypes binding of the C ABI in ``include/dsp.h`` (argument marshalling only).

Every step of the solve runs in the CUDA kernels of ``libdsp.so``; this module
converts Python arguments to the C types, calls the library, and raises
``DSPError`` on a non-zero status.  PyTorch is used only for device memory and
streams (see :class:`Grid`).  There is no CPU fallback: if the library has not
been built, loading it raises.

Names follow the C ABI without the ``dsp_`` prefix.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

_lock = threading.Lock()
_lib = None

FP64 = 0
FP32_MIXED = 1
PRECISIONS = {"fp64": FP64, "fp32_mixed": FP32_MIXED}
SCHEMES = {"exact": 0, "strang_xy": 1, "magnus4": 2}
PULSE_KINDS = {"zero": 0, "sin2": 1, "gauss": 2, "two_colour": 3, "const_field": 4, "paper": 5}
REQ_STATES = {0: "queued", 1: "active", 2: "done", 3: "failed", 4: "cancelled"}
STATUS = {0: "ok", -1: "invalid argument", -2: "out of memory or over budget", -3: "CUDA error",
          -4: "call out of order", -5: "time step too large (dt*max|p+A| > pi)",
          -6: "device-side wait timed out",
          -7: "out-of-range index found by a bounds-check build"}

# Every entry point declared in include/dsp.h.
EXPORTS = (
    "dsp_state_bytes", "dsp_create_grid", "dsp_set_pulse", "dsp_evolve", "dsp_project",
    "dsp_reduce_density", "dsp_solve", "dsp_solve_host", "dsp_evolve_batch", "dsp_get_cursor",
    "dsp_save_state", "dsp_load_state", "dsp_destroy_grid", "dsp_status_string",
    "dsp_sample_pulse", "dsp_server_create", "dsp_server_submit", "dsp_server_step",
    "dsp_server_query", "dsp_server_cancel", "dsp_server_destroy", "dsp_density_noalloc",
    "dsp_get_info", "dsp_solve_segmented", "dsp_sample_pulse_gauss",
    "dsp_test_withhold_next_copy", "dsp_create_band", "dsp_set_keep_final_state",
    "dsp_test_tiling",
)


class DSPError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = int(code)
        super().__init__(f"{where}: {STATUS.get(self.code, 'unknown')} ({self.code})")


class PulseSpec(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("reserved", ctypes.c_int32)] + [
        (n, ctypes.c_double) for n in ("E0", "omega", "T", "tau", "t0", "eps", "phase2",
                                       "Omega_rise", "Omega_fall", "phi")]


class GridInfo(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in ("nx", "ny", "precision", "scheme", "valley",
                                              "cos_degree", "sinc_degree", "n_tiles")] + [
        ("n_steps", ctypes.c_int64), ("cursor", ctypes.c_int64), ("dt", ctypes.c_double),
        ("theta_max", ctypes.c_double),
        ("group_steps", ctypes.c_int32), ("row_begin", ctypes.c_int32),
        ("ny_total", ctypes.c_int32), ("row_strips", ctypes.c_int32),
        ("tan_degree", ctypes.c_int32)]


class Request(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("px_min", ctypes.c_double), ("px_max", ctypes.c_double),
        ("py_min", ctypes.c_double), ("py_max", ctypes.c_double),
        ("precision", ctypes.c_int32), ("scheme", ctypes.c_int32), ("valley", ctypes.c_int32),
        ("keep_map", ctypes.c_int32),
        ("n_steps", ctypes.c_int64), ("dt", ctypes.c_double),
        ("a_in", ctypes.c_double * 2), ("a_out", ctypes.c_double * 2),
    ]


def library_path() -> str:
    """libdsp.so, or the variant named by DSP_LIBRARY (e.g. the bounds-check build)."""
    return os.environ.get("DSP_LIBRARY") or _build.LIB


def lib() -> ctypes.CDLL:
    """The loaded libdsp.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            path = library_path()
            if not os.path.exists(path):
                raise RuntimeError(f"{path} is missing: build it first "
                                   "(python -c 'import __graft_entry__ as g; g.build()')")
            L = ctypes.CDLL(path)
            i32, i64, d, p = ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p
            pd, pi64, pi32 = (ctypes.POINTER(d), ctypes.POINTER(i64), ctypes.POINTER(i32))
            sig = {
                "dsp_state_bytes": (i64, [i32, i32, i32]),
                "dsp_create_grid": (i32, [i32, i32, d, d, d, d, i32, i32, i32, p, p, i64,
                                          ctypes.POINTER(p)]),
                "dsp_create_band": (i32, [i32, i32, i32, i32, d, d, d, d, i32, i32, i32, p, p,
                                          i64, ctypes.POINTER(p)]),
                "dsp_set_keep_final_state": (i32, [p, i32]),
                "dsp_set_pulse": (i32, [p, p, i64, d, p, p]),
                "dsp_evolve": (i32, [p, i64]),
                "dsp_project": (i32, [p, p]),
                "dsp_reduce_density": (i32, [p, pd]),
                "dsp_solve": (i32, [p, p, pd]),
                "dsp_solve_host": (i32, [p, p, i64, d, p, p, p, pd]),
                "dsp_evolve_batch": (i32, [p, p, i32]),
                "dsp_get_cursor": (i32, [p, pi64, pi64]),
                "dsp_save_state": (i32, [p, p, i64, pi64]),
                "dsp_load_state": (i32, [p, p, i64, i64]),
                "dsp_destroy_grid": (i32, [p]),
                "dsp_status_string": (ctypes.c_char_p, [i32]),
                "dsp_sample_pulse": (i32, [ctypes.POINTER(PulseSpec), i64, p, p, p, pd]),
                "dsp_server_create": (i32, [i64, i32, i64, p, ctypes.POINTER(p)]),
                "dsp_server_submit": (i32, [p, ctypes.POINTER(Request), p, pi64]),
                "dsp_server_step": (i32, [p, pi32, pi32, pi32]),
                "dsp_server_query": (i32, [p, i64, pi32, pd, p, pi64]),
                "dsp_server_cancel": (i32, [p, i64]),
                "dsp_server_destroy": (i32, [p]),
                "dsp_density_noalloc": (i32, [p, i32, i32, i32, d, d, d, d, p, pd]),
                "dsp_get_info": (i32, [p, ctypes.POINTER(GridInfo)]),
                "dsp_solve_segmented": (i32, [p, i32, p, pd]),
                "dsp_sample_pulse_gauss": (i32, [ctypes.POINTER(PulseSpec), i64, p, p, p, pd]),
                "dsp_test_withhold_next_copy": (i32, [p]),
                "dsp_test_tiling": (i32, [p, i32]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _check(rc: int, where: str):
    if rc != 0:
        raise DSPError(rc, where)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _enum(v, table):
    return table[v] if isinstance(v, str) else int(v)


# ------------------------------------------------------------------------------------------
# Grid entry points
# ------------------------------------------------------------------------------------------

def state_bytes(nx: int, ny: int, precision="fp32_mixed") -> int:
    return int(lib().dsp_state_bytes(nx, ny, _enum(precision, PRECISIONS)))


def create_grid(nx, ny, px_range, py_range, precision="fp32_mixed", scheme="exact", valley=1,
                stream=0, state_ptr=0, state_bytes_=0) -> int:
    h = ctypes.c_void_p()
    rc = lib().dsp_create_grid(int(nx), int(ny), float(px_range[0]), float(px_range[1]),
                               float(py_range[0]), float(py_range[1]),
                               _enum(precision, PRECISIONS), _enum(scheme, SCHEMES), int(valley),
                               ctypes.c_void_p(int(stream)), ctypes.c_void_p(int(state_ptr)),
                               int(state_bytes_), ctypes.byref(h))
    _check(rc, "create_grid")
    return h.value


def create_band(nx, ny, rows, px_range, py_range, precision="fp32_mixed", scheme="exact",
                valley=1, stream=0, state_ptr=0, state_bytes_=0) -> int:
    """A grid holding the rows [rows[0], rows[1]) of the nx by ny grid on the box:
    the full grid's nodes and step choices (see include/dsp.h)."""
    h = ctypes.c_void_p()
    rc = lib().dsp_create_band(int(nx), int(ny), int(rows[0]), int(rows[1]),
                               float(px_range[0]), float(px_range[1]),
                               float(py_range[0]), float(py_range[1]),
                               _enum(precision, PRECISIONS), _enum(scheme, SCHEMES), int(valley),
                               ctypes.c_void_p(int(stream)), ctypes.c_void_p(int(state_ptr)),
                               int(state_bytes_), ctypes.byref(h))
    _check(rc, "create_band")
    return h.value


def set_keep_final_state(h: int, keep: bool):
    _check(lib().dsp_set_keep_final_state(ctypes.c_void_p(h), 1 if keep else 0),
           "set_keep_final_state")


def _steps(a_mid):
    """A table and its step count: [n, 2] midpoint samples or [n, 4] Gauss pairs."""
    a = _f64(a_mid)
    w = a.shape[-1] if a.ndim == 2 else 2
    if w not in (2, 4):
        raise ValueError("pulse table must be [n, 2] (midpoints) or [n, 4] (Gauss pairs)")
    a = a.reshape(-1, w)
    return a, a.shape[0]


def set_pulse(h: int, a_mid, dt: float, a_in, a_out):
    a, n = _steps(a_mid)
    ai, ao = _f64(a_in), _f64(a_out)
    _check(lib().dsp_set_pulse(ctypes.c_void_p(h), _ptr(a), n, float(dt), _ptr(ai),
                               _ptr(ao)), "set_pulse")


def evolve(h: int, steps: int):
    _check(lib().dsp_evolve(ctypes.c_void_p(h), int(steps)), "evolve")


def project(h: int, map_ptr: int):
    _check(lib().dsp_project(ctypes.c_void_p(h), ctypes.c_void_p(int(map_ptr))), "project")


def reduce_density(h: int) -> float:
    n = ctypes.c_double()
    _check(lib().dsp_reduce_density(ctypes.c_void_p(h), ctypes.byref(n)), "reduce_density")
    return n.value


def solve(h: int, map_ptr: int = 0, want_density: bool = True):
    n = ctypes.c_double()
    rc = lib().dsp_solve(ctypes.c_void_p(h), ctypes.c_void_p(int(map_ptr)),
                         ctypes.byref(n) if want_density else None)
    _check(rc, "solve")
    return n.value if want_density else None


def solve_segmented(h: int, segments: int = 0, map_ptr: int = 0, want_density: bool = True):
    """Whole solve with the time axis split into segments run in parallel."""
    n = ctypes.c_double()
    rc = lib().dsp_solve_segmented(ctypes.c_void_p(h), int(segments), ctypes.c_void_p(int(map_ptr)),
                                   ctypes.byref(n) if want_density else None)
    _check(rc, "solve_segmented")
    return n.value if want_density else None


def solve_host(h: int, a_mid, dt: float, a_in, a_out, map_out: np.ndarray | None) -> float:
    a, steps = _steps(a_mid)
    ai, ao = _f64(a_in), _f64(a_out)
    n = ctypes.c_double()
    mp = None if map_out is None else _ptr(map_out)
    _check(lib().dsp_solve_host(ctypes.c_void_p(h), _ptr(a), steps, float(dt), _ptr(ai),
                                _ptr(ao), mp, ctypes.byref(n)), "solve_host")
    return n.value


def evolve_batch(handles, steps):
    hs = (ctypes.c_void_p * len(handles))(*[ctypes.c_void_p(h) for h in handles])
    st = (ctypes.c_int64 * len(steps))(*[int(s) for s in steps])
    _check(lib().dsp_evolve_batch(ctypes.cast(hs, ctypes.c_void_p), ctypes.cast(st, ctypes.c_void_p),
                                  len(handles)), "evolve_batch")


def get_cursor(h: int):
    c, n = ctypes.c_int64(), ctypes.c_int64()
    _check(lib().dsp_get_cursor(ctypes.c_void_p(h), ctypes.byref(c), ctypes.byref(n)),
           "get_cursor")
    return c.value, n.value


def get_info(h: int) -> dict:
    """Series degrees, theta_max, hi/lo grid and tile count chosen for the current pulse."""
    info = GridInfo()
    _check(lib().dsp_get_info(ctypes.c_void_p(h), ctypes.byref(info)), "get_info")
    return {n: getattr(info, n) for n, _ in GridInfo._fields_}


def save_state(h: int, buf: np.ndarray) -> int:
    c = ctypes.c_int64()
    _check(lib().dsp_save_state(ctypes.c_void_p(h), _ptr(buf), buf.nbytes, ctypes.byref(c)),
           "save_state")
    return c.value


def load_state(h: int, buf: np.ndarray, cursor: int):
    _check(lib().dsp_load_state(ctypes.c_void_p(h), _ptr(buf), buf.nbytes, int(cursor)),
           "load_state")


def destroy_grid(h: int):
    _check(lib().dsp_destroy_grid(ctypes.c_void_p(h)), "destroy_grid")


def density_noalloc(map_ptr: int, precision, nx: int, ny: int, px_range, py_range,
                    stream=0) -> float:
    """Pair density of a device |c+|^2 map without any device allocation (the
    scratch is a static array inside the library; see include/dsp.h)."""
    n = ctypes.c_double()
    _check(lib().dsp_density_noalloc(ctypes.c_void_p(int(map_ptr)), _enum(precision, PRECISIONS),
                                     int(nx), int(ny), float(px_range[0]), float(px_range[1]),
                                     float(py_range[0]), float(py_range[1]),
                                     ctypes.c_void_p(int(stream)), ctypes.byref(n)),
           "density_noalloc")
    return n.value


def test_withhold_next_copy(h: int):
    """Failure-path test hook: the next launch's first table chunk is never
    copied, so its bounded device-side wait runs out (DSP_E_TIMEOUT)."""
    _check(lib().dsp_test_withhold_next_copy(ctypes.c_void_p(h)), "test_withhold_next_copy")


def test_tiling(h: int, tiling):
    """Test hook on a grid's tiling: 1 (or True) automatic, 0 (or False)
    contiguous tiles, 2 row strips without the last-wave split (the results
    are bitwise the same in every case)."""
    _check(lib().dsp_test_tiling(ctypes.c_void_p(h), int(tiling)), "test_tiling")


def status_string(code: int) -> str:
    return lib().dsp_status_string(int(code)).decode()


# ------------------------------------------------------------------------------------------
# Pulse sampler
# ------------------------------------------------------------------------------------------

def pulse_spec(spec: dict) -> PulseSpec:
    s = PulseSpec()
    s.kind = PULSE_KINDS[spec["kind"]]
    for n in ("E0", "omega", "T", "tau", "t0", "eps", "phase2", "Omega_rise", "Omega_fall", "phi"):
        setattr(s, n, float(spec.get(n, 0.0)))
    return s


def sample_pulse(spec: dict, n_steps: int):
    """(a_mid[n_steps, 2], a_in[2], a_out[2], dt) from the library's own sampler."""
    a_mid = np.zeros((int(n_steps), 2))
    a_in, a_out = np.zeros(2), np.zeros(2)
    dt = ctypes.c_double()
    s = pulse_spec(spec)
    _check(lib().dsp_sample_pulse(ctypes.byref(s), int(n_steps), _ptr(a_mid), _ptr(a_in),
                                  _ptr(a_out), ctypes.byref(dt)), "sample_pulse")
    return a_mid, a_in, a_out, dt.value


def sample_pulse_gauss(spec: dict, n_steps: int):
    """(a_gauss[n_steps, 4], a_in[2], a_out[2], dt): A at the two Gauss points of
    each step, for the fourth-order Magnus scheme."""
    a = np.zeros((int(n_steps), 4))
    a_in, a_out = np.zeros(2), np.zeros(2)
    dt = ctypes.c_double()
    s = pulse_spec(spec)
    _check(lib().dsp_sample_pulse_gauss(ctypes.byref(s), int(n_steps), _ptr(a), _ptr(a_in),
                                        _ptr(a_out), ctypes.byref(dt)), "sample_pulse_gauss")
    return a, a_in, a_out, dt.value


# ------------------------------------------------------------------------------------------
# Server
# ------------------------------------------------------------------------------------------

def server_create(hbm_budget_bytes: int, max_active: int, chunk_steps: int, stream=0) -> int:
    h = ctypes.c_void_p()
    _check(lib().dsp_server_create(int(hbm_budget_bytes), int(max_active), int(chunk_steps),
                                   ctypes.c_void_p(int(stream)), ctypes.byref(h)), "server_create")
    return h.value


def make_request(grid: dict, n_steps: int, dt: float, a_in, a_out, precision="fp32_mixed",
                 scheme="exact", valley=1, keep_map=False) -> Request:
    r = Request()
    r.nx, r.ny = int(grid["nx"]), int(grid["ny"])
    r.px_min, r.px_max = map(float, grid["px"])
    r.py_min, r.py_max = map(float, grid["py"])
    r.precision = _enum(precision, PRECISIONS)
    r.scheme = _enum(scheme, SCHEMES)
    r.valley = int(valley)
    r.keep_map = 1 if keep_map else 0
    r.n_steps = int(n_steps)
    r.dt = float(dt)
    r.a_in[0], r.a_in[1] = map(float, a_in)
    r.a_out[0], r.a_out[1] = map(float, a_out)
    return r


def server_submit(s: int, req: Request, a_mid) -> int:
    a, _ = _steps(a_mid)
    rid = ctypes.c_int64()
    _check(lib().dsp_server_submit(ctypes.c_void_p(s), ctypes.byref(req), _ptr(a),
                                   ctypes.byref(rid)), "server_submit")
    return rid.value


def server_step(s: int):
    a, q, f = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(lib().dsp_server_step(ctypes.c_void_p(s), ctypes.byref(a), ctypes.byref(q),
                                 ctypes.byref(f)), "server_step")
    return a.value, q.value, f.value


def server_query(s: int, rid: int, map_out: np.ndarray | None = None):
    st, n, done = ctypes.c_int32(), ctypes.c_double(), ctypes.c_int64()
    mp = None if map_out is None else _ptr(map_out)
    _check(lib().dsp_server_query(ctypes.c_void_p(s), int(rid), ctypes.byref(st), ctypes.byref(n),
                                  mp, ctypes.byref(done)), "server_query")
    return REQ_STATES[st.value], n.value, done.value


def server_cancel(s: int, rid: int):
    _check(lib().dsp_server_cancel(ctypes.c_void_p(s), int(rid)), "server_cancel")


def server_destroy(s: int):
    _check(lib().dsp_server_destroy(ctypes.c_void_p(s)), "server_destroy")


# ------------------------------------------------------------------------------------------
# Convenience: a grid whose device memory belongs to PyTorch
# ------------------------------------------------------------------------------------------

class Grid:
    """One momentum grid; the spinor state and the |c+|^2 map are torch tensors on
    the current CUDA device, work goes on torch's current stream.  With
    ``rows=(r0, r1)`` the grid is the band of rows [r0, r1) of the nx by ny grid
    (``dsp_create_band``); its map then holds those rows only."""

    def __init__(self, nx, ny, px_range, py_range, precision="fp32_mixed", scheme="exact",
                 valley=1, device=None, rows=None):
        import torch
        self.torch = torch
        self.nx = int(nx)
        self.rows = (0, int(ny)) if rows is None else (int(rows[0]), int(rows[1]))
        self.ny = self.rows[1] - self.rows[0]
        self.precision = _enum(precision, PRECISIONS)
        dev = torch.device("cuda" if device is None else device)
        nbytes = state_bytes(nx, self.ny, self.precision)
        self.state = torch.empty(nbytes // 4, dtype=torch.float32, device=dev)
        mdt = torch.float64 if self.precision == FP64 else torch.float32
        self.map = torch.empty((self.ny, self.nx), dtype=mdt, device=dev)
        self.stream = torch.cuda.current_stream(dev).cuda_stream
        if rows is None:
            self.h = create_grid(nx, ny, px_range, py_range, self.precision, scheme, valley,
                                 self.stream, self.state.data_ptr(), nbytes)
        else:
            self.h = create_band(nx, ny, self.rows, px_range, py_range, self.precision, scheme,
                                 valley, self.stream, self.state.data_ptr(), nbytes)

    def set_pulse(self, a_mid, dt, a_in, a_out):
        set_pulse(self.h, a_mid, dt, a_in, a_out)

    def evolve(self, steps):
        evolve(self.h, steps)

    def project(self):
        project(self.h, self.map.data_ptr())
        return self.map

    def density(self):
        return reduce_density(self.h)

    def solve(self):
        n = solve(self.h, self.map.data_ptr())
        return self.map, n

    def solve_segmented(self, segments=0):
        n = solve_segmented(self.h, segments, self.map.data_ptr())
        return self.map, n

    def close(self):
        if self.h:
            destroy_grid(self.h)
            self.h = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
