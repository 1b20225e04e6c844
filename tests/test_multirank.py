"""The N > 1 path on CPU: world_size 2 over gloo.  Each rank solves its own row
band of a grid with the oracle, from the same band descriptor the library
takes (the full grid plus a row range: the nodes are the full grid's global
rows, never re-derived from the band).  The band maps are gathered and, put
together in rank order, are bitwise the single-process map; the per-band
densities summed in rank order match the single-process density; the
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
    import numpy as np

    from oracle import oracle
    pulse = W.sin2_pulse(1.0, 1.55, 5.0)
    a_mid, a_in, a_out, dt = oracle.pulse_table(pulse, 600)
    band = shard.band_grid(grid, rank, world)
    r0, r1 = band["rows"]
    xs = oracle.grid_nodes(*band["px"], band["nx"])
    ys = oracle.grid_nodes(*band["py"], band["ny"])[r0:r1]  # the full grid's rows
    px = np.tile(xs, r1 - r0)
    py = np.repeat(ys, band["nx"])
    cp = oracle.solve_points(px, py, a_mid, dt, a_in, a_out, nthreads=1)["cplus2"]
    hx = (band["px"][1] - band["px"][0]) / band["nx"]
    hy = (band["py"][1] - band["py"][0]) / band["ny"]
    n = oracle.density(cp, hx, hy)  # this band's share of the full density
    rows_max = -(-grid["ny"] // world)
    buf = torch.zeros(rows_max * grid["nx"] + 2, dtype=torch.float64)
    buf[:cp.size] = torch.from_numpy(cp)
    buf[-2] = n
    buf[-1] = float(r1 - r0)
    got = [torch.zeros_like(buf) for _ in range(world)]
    dist.all_gather(got, buf)
    wall = torch.tensor([0.1 * (rank + 1)], dtype=torch.float64)
    dist.all_reduce(wall, op=dist.ReduceOp.MAX)
    if rank == 0:
        total = shard.combine_densities([float(g[-2]) for g in got])
        maps = [g[:int(g[-1]) * grid["nx"]].numpy() for g in got]
        np.save(out_path + ".map.npy", np.concatenate(maps).reshape(grid["ny"], grid["nx"]))
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


def test_band_descriptor_keeps_the_full_grid():
    grid = {"nx": 40, "ny": 33, "px": (-4.0, 4.0), "py": (-3.0, 5.0)}
    bands = [shard.band_grid(grid, r, 3) for r in range(3)]
    assert [b["rows"] for b in bands] == [(0, 11), (11, 22), (22, 33)]
    for b in bands:
        assert (b["nx"], b["ny"], b["px"], b["py"]) == (40, 33, grid["px"], grid["py"])


def test_two_rank_gloo_band_maps_and_density_match_single_process(tmp_path, orc):
    import numpy as np
    grid = {"nx": 40, "ny": 33, "px": (-4.0, 4.0), "py": (-4.0, 4.0)}
    out = tmp_path / "out.txt"
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, grid, str(out)), nprocs=2, join=True,
                       start_method="spawn")
    total, wall = map(float, out.read_text().split())
    a_mid, a_in, a_out, dt = orc.pulse_table(W.sin2_pulse(1.0, 1.55, 5.0), 600)
    ref_map, _, _, ref = orc.solve_grid(40, 33, grid["px"], grid["py"], a_mid, dt, a_in, a_out)
    banded = np.load(str(out) + ".map.npy")
    assert np.array_equal(banded, ref_map)  # the bands' points are the full grid's, bit for bit
    assert abs(total - ref) <= 1e-12 * ref
    assert wall == pytest.approx(0.2)
