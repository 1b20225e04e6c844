"""The N > 1 path on CPU: world_size 2 over gloo.  Each rank solves its own row
band of a grid with the oracle, the per-band densities are gathered and
summed in rank order, and the result matches the single-process solve; the
round-robin sample assignment covers every sample once per round."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1607_03062_gb300 import shard
from paper_1607_03062_gb300 import workloads as W


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, grid, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import oracle
    pulse = W.sin2_pulse(1.0, 1.55, 5.0)
    a_mid, a_in, a_out, dt = oracle.pulse_table(pulse, 600)
    band = shard.band_grid(grid, rank, world)
    _, _, _, n = oracle.solve_grid(band["nx"], band["ny"], band["px"], band["py"], a_mid, dt, a_in,
                                   a_out, nthreads=1)
    t = torch.tensor([n, float(rank)], dtype=torch.float64)
    got = [torch.zeros(2, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(got, t)
    wall = torch.tensor([0.1 * (rank + 1)], dtype=torch.float64)
    dist.all_reduce(wall, op=dist.ReduceOp.MAX)
    if rank == 0:
        total = shard.combine_densities([float(g[0]) for g in got])
        with open(out_path, "w") as f:
            f.write(f"{total!r} {float(wall.item())!r}")
    dist.destroy_process_group()


def test_row_bands_cover_the_grid():
    for ny in (1, 7, 64, 101):
        for world in (1, 2, 3, 8):
            bands = [shard.row_band(ny, r, world) for r in range(world)]
            assert bands[0][0] == 0 and bands[-1][1] == ny
            assert all(a[1] == b[0] for a, b in zip(bands, bands[1:]))


def test_round_robin_samples():
    world, n = 2, 8
    seen = [shard.sample_for(step, r, world, n) for step in range(4) for r in range(world)]
    assert sorted(seen) == list(range(8))


def test_two_rank_gloo_density_matches_single_process(tmp_path, orc):
    grid = {"nx": 40, "ny": 33, "px": (-4.0, 4.0), "py": (-4.0, 4.0)}
    out = tmp_path / "out.txt"
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, grid, str(out)), nprocs=2, join=True,
                       start_method="spawn")
    total, wall = map(float, out.read_text().split())
    a_mid, a_in, a_out, dt = orc.pulse_table(W.sin2_pulse(1.0, 1.55, 5.0), 600)
    _, _, _, ref = orc.solve_grid(40, 33, grid["px"], grid["py"], a_mid, dt, a_in, a_out)
    assert abs(total - ref) <= 1e-12 * ref
    assert wall == pytest.approx(0.2)
