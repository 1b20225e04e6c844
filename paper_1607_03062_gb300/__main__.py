"""Command line: one solve on the GPU, printed as a JSON line.

    python -m paper_1607_03062_gb300 --workload sin2_64 --precision fp64
    python -m paper_1607_03062_gb300 --spec my_pulse.json --grid 512 --extent 6 --steps 20000 \
        --scheme magnus4 --out map.npy

``--spec`` reads a pulse dictionary (see ``workloads.py``: kind, E0, omega, T, ...).
The |c+|^2 map can be written with ``--out`` (numpy .npy, [ny][nx]).
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
    "sin2_64": W.config_sin2_64,
    "gauss_1024": lambda: W.config_gauss_1024(2.0),
    "lzs_2048": lambda: W.config_lzs_2048(0),
    "two_colour_4096": W.config_two_colour_4096,
    "paper": lambda: {"name": "paper_pulse_fig1", "grid": W.grid(256, 0.5),
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
    a = ap.parse_args(argv)

    import torch

    cfg = WORKLOADS[a.workload]()
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
    print(json.dumps({"workload": cfg["name"], "grid": [g["nx"], g["ny"]], "steps": steps,
                      "precision": a.precision, "scheme": a.scheme, "valley": a.valley,
                      "density_eV2": n, "max_cplus2": float(m.max().item()), "wall_s": wall,
                      "spinor_steps_per_s": g["nx"] * g["ny"] * steps / wall,
                      "series_degrees": [info["cos_degree"], info["sinc_degree"]],
                      "theta_max": info["theta_max"]}))
    grid.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
