"""The command-line entry point (GPU) and the benchmark's reference arm (CPU)."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_json_line():
    """bench.py --impl reference times the FP64 oracle on a bounded sample."""
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "0", "--grid", "128", "--time-steps", "200"],
                         capture_output=True, text=True, timeout=300, check=True)
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["metric"] == "spinor-steps/s" and line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0


@pytest.mark.gpu
def test_cli_solve_writes_map_and_density(tmp_path, orc):
    from paper_1607_03062_gb300 import workloads as W
    out_npy = tmp_path / "map.npy"
    res = subprocess.run([sys.executable, "-m", "paper_1607_03062_gb300", "--workload", "sin2_64",
                          "--precision", "fp64", "--out", str(out_npy)], cwd=ROOT,
                         capture_output=True, text=True, timeout=300, check=True)
    line = json.loads(res.stdout.strip().splitlines()[-1])
    cfg = W.config_sin2_64()
    g = cfg["grid"]
    a_mid, a_in, a_out, dt = orc.pulse_table(cfg["pulse"], cfg["steps"])
    ref, _, _, nref = orc.solve_grid(g["nx"], g["ny"], g["px"], g["py"], a_mid, dt, a_in, a_out)
    m = np.load(out_npy)
    assert np.abs(m - ref).max() <= 1e-9
    assert abs(line["density_eV2"] - nref) <= 1e-10 * nref


@pytest.mark.gpu
def test_cli_fp32_mixed_against_fp64_map():
    """--vs-fp64 solves the same grid in both precisions and reports the
    FP32-mixed map's error over every point; on the 64^2 case it must sit within
    the FP32-mixed tolerance and agree with a direct comparison of the two maps."""
    res = subprocess.run([sys.executable, "-m", "paper_1607_03062_gb300", "--workload", "sin2_64",
                          "--vs-fp64"], cwd=ROOT, capture_output=True, text=True, timeout=300,
                         check=True)
    line = json.loads(res.stdout.strip().splitlines()[-1])
    v = line["vs_fp64"]
    assert line["precision"] == "fp32_mixed" and line["group_steps"] >= 1
    assert 0.0 < v["max_abs_err"] <= 1e-5 and v["p99_9"] <= v["max_abs_err"]
    assert abs(v["density_rel_err"]) <= 1e-4
    assert 0 <= v["at_ix_iy"][0] < 64 and 0 <= v["at_ix_iy"][1] < 64


def test_reference_arm_under_torchrun_two_ranks():
    """Launched like the N > 1 benchmark: rank 0 prints the only JSON line, the
    other rank exits 0 without work."""
    import socket
    sock = socket.socket()
    sock.bind(("127.0.0.1", 0))
    port = sock.getsockname()[1]
    sock.close()
    out = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1",
                          "--nproc-per-node", "2", "--master-addr", "127.0.0.1",
                          "--master-port", str(port), os.path.join(ROOT, "bench.py"),
                          "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0",
                          "--grid", "64", "--time-steps", "100"],
                         capture_output=True, text=True, timeout=300, check=True)
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
