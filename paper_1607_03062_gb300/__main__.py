"""Command line: one solve on the GPU, printed as a JSON line.

    python -m paper_1607_03062_gb300 --workload sin2_64 --precision fp64
    python -m paper_1607_03062_gb300 --spec my_pulse.json --grid 512 --extent 6 --steps 20000 \
        --scheme magnus4 --out map.npy

``--spec`` reads a pulse dictionary (see ``workloads.py``: kind, E0, omega, T, ...).
The |c+|^2 map can be written with ``--out`` (numpy .npy, [ny][nx]).  ``--sample k``
picks the k-th seeded (omega, E0) draw of the LZS scan.  ``--vs-fp64`` also solves
the same grid in FP64 and reports the FP32-mixed map's error over every point:

    python -m paper_1607_03062_gb300 --workload lzs_2048 --sample 6 --vs-fp64
"""
from __future__ import annotations

import argparse
import json
import sys
import time

import numpy as np

from . import binding as B
from . import workloads as W

WORKLOADS = {
    "sin2_64": lambda k: W.config_sin2_64(),
    "gauss_1024": lambda k: W.config_gauss_1024(2.0),
    "lzs_2048": lambda k: W.config_lzs_2048(k),
    "two_colour_4096": lambda k: W.config_two_colour_4096(),
    "paper": lambda k: {"name": "paper_pulse_fig1", "grid": W.grid(256, 0.5),
                        "pulse": W.paper_pulse(), "steps": 20000},
}


def main(argv=None):
    ap = argparse.ArgumentParser(prog="python -m paper_1607_03062_gb300")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="sin2_64")
    ap.add_argument("--spec", help="JSON file with a pulse dictionary (overrides the workload's)")
    ap.add_argument("--grid", type=int, help="points per axis")
    ap.add_argument("--extent", type=float, help="momentum box [-extent, extent]^2 (eV)")
    ap.add_argument("--steps", type=int)
    ap.add_argument("--precision", choices=sorted(B.PRECISIONS), default="fp32_mixed")
    ap.add_argument("--scheme", choices=sorted(B.SCHEMES), default="exact")
    ap.add_argument("--valley", type=int, choices=(1, -1), default=1)
    ap.add_argument("--segmented", type=int, default=-1,
                    help="time-parallel solve with this many segments (0 = automatic)")
    ap.add_argument("--out", help="write the |c+|^2 map to this .npy file")
    ap.add_argument("--sample", type=int, default=0,
                    help="seeded (omega, E0) draw of the LZS scan (lzs_2048 only), 0..7")
    ap.add_argument("--vs-fp64", action="store_true",
                    help="also solve in FP64 and report the map's error over every point")
    ap.add_argument("--reproject", type=int, default=0, metavar="N",
                    help="after the solve, project the final state N more times (the "
                         "projection-only launch) and report its time and bytes per second")
    a = ap.parse_args(argv)

    import torch

    cfg = WORKLOADS[a.workload](a.sample)
    if a.spec:
        with open(a.spec) as f:
            cfg["pulse"] = json.load(f)
        cfg["name"] = "custom"
    g = cfg["grid"]
    if a.grid or a.extent:
        g = W.grid(a.grid or g["nx"], a.extent or g["px"][1])
    steps = a.steps or cfg["steps"]
    sample = B.sample_pulse_gauss if a.scheme == "magnus4" else B.sample_pulse
    a_mid, a_in, a_out, dt = sample(cfg["pulse"], steps)
    grid = B.Grid(g["nx"], g["ny"], g["px"], g["py"], a.precision, a.scheme, a.valley)
    grid.set_pulse(a_mid, dt, a_in, a_out)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    if a.segmented >= 0:
        m, n = grid.solve_segmented(a.segmented)
    else:
        m, n = grid.solve()
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    info = B.get_info(grid.h)
    if a.out:
        np.save(a.out, m.cpu().numpy())
    out = {"workload": cfg["name"], "grid": [g["nx"], g["ny"]], "steps": steps,
           "precision": a.precision, "scheme": a.scheme, "valley": a.valley,
           "density_eV2": n, "max_cplus2": float(m.max().item()), "wall_s": wall,
           "spinor_steps_per_s": g["nx"] * g["ny"] * steps / wall,
           "series_degrees": [info["cos_degree"], info["sinc_degree"]],
           "group_steps": info["group_steps"], "theta_max": info["theta_max"],
           "row_strips": info["row_strips"]}
    if a.reproject > 0:
        # the standalone projection: reads the 32-byte state of every point, writes
        # the map (4 or 8 bytes) and one double per 256-point granule
        times = []
        for _ in range(a.reproject):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            grid.project()
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
        pts = g["nx"] * g["ny"]
        nbytes = pts * (32 + (8 if a.precision == "fp64" else 4)) + 8 * ((pts + 255) // 256)
        t = float(np.median(times))
        out["reproject"] = {"launches": a.reproject, "median_us": t * 1e6,
                            "algorithmic_bytes": nbytes, "gbs": nbytes / t / 1e9}
    grid.close()
    if a.vs_fp64 and a.precision != "fp64":
        ref = B.Grid(g["nx"], g["ny"], g["px"], g["py"], "fp64", a.scheme, a.valley)
        ref.set_pulse(a_mid, dt, a_in, a_out)
        m64, n64 = ref.solve()
        err = (m.double() - m64).abs().flatten().cpu().numpy()
        k = int(np.argmax(err))
        out["vs_fp64"] = {"max_abs_err": float(err[k]), "at_ix_iy": [k % g["nx"], k // g["nx"]],
                          "p99_9": float(np.quantile(err, 0.999)),
                          "points_above_1e-6": int((err > 1e-6).sum()),
                          "density_rel_err": abs(n - n64) / n64 if n64 else None}
        ref.close()
    print(json.dumps(out))
    return 0


if __name__ == "__main__":
    sys.exit(main())
