"""Continuous-batching server: each result is the same alone and in any mix
(bitwise), admission respects the device-footprint budget, cancellation
leaves the others untouched, and results match the oracle."""
import numpy as np
import pytest
import torch

from paper_1607_03062_gb300 import binding as B
from paper_1607_03062_gb300 import serve
from paper_1607_03062_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1607_03062_gb300 import build
    build.build()
    B.lib()
    torch.cuda.set_device(0)


def small_stream(count=12, seed=3):
    reqs = W.serving_requests(count=count, seed=seed, rate_hz=1e6, sizes=(16, 40, 64, 100),
                              steps_range=(200, 2500), extent=4.0)
    return serve.prepare(reqs)


def test_alone_equals_mixed_bitwise():
    reqs = small_stream()
    alone = serve.run(reqs, hbm_budget_bytes=1 << 34, max_active=1, chunk_steps=1 << 30,
                      keep_map=True, realtime=False)
    mixed = serve.run(reqs, hbm_budget_bytes=1 << 34, max_active=8, chunk_steps=700,
                      keep_map=True, realtime=False)
    assert mixed["max_active_seen"] > 1
    for k in range(len(reqs)):
        a, m = alone["results"][k], mixed["results"][k]
        assert a["state"] == m["state"] == "done"
        assert a["density"] == m["density"]
        assert np.array_equal(a["map"], m["map"])


def test_server_matches_oracle(orc):
    reqs = small_stream(count=4, seed=9)
    out = serve.run(reqs, hbm_budget_bytes=1 << 34, max_active=4, chunk_steps=500, keep_map=True,
                    realtime=False)
    for k, r in enumerate(reqs):
        g = r["grid"]
        a_mid, a_in, a_out, dt = orc.pulse_table(r["pulse"], r["steps"])
        ref, _, _, nref = orc.solve_grid(g["nx"], g["ny"], g["px"], g["py"], a_mid, dt, a_in, a_out)
        res = out["results"][k]
        assert np.abs(res["map"].astype(np.float64) - ref).max() <= 1e-5
        assert abs(res["density"] - nref) <= 1e-4 * nref


def test_admission_by_footprint():
    """Equal-size requests and a budget of 2.5 footprints: never more than two
    are on the device at once, and all of them finish."""
    reqs = serve.prepare(W.serving_requests(count=8, seed=4, rate_hz=1e6, sizes=(64,),
                                            steps_range=(1000, 1000), extent=4.0))
    fp = 32 * 64 * 64 + 16 * 1000 + 4 * 64 * 64 + 8 * 4 + 16
    seen = []
    out = serve.run(reqs, hbm_budget_bytes=int(2.5 * fp), max_active=8, chunk_steps=400,
                    realtime=False, on_step=lambda a, q, f: seen.append(a + f))
    assert max(seen) == 2
    assert all(v["state"] == "done" for v in out["results"].values())


def test_cancel_leaves_others_unchanged():
    reqs = small_stream(count=5, seed=6)
    ref = serve.run(reqs, hbm_budget_bytes=1 << 34, max_active=5, chunk_steps=300,
                    realtime=False)
    srv = B.server_create(1 << 34, 5, 300)
    ids = []
    for r in reqs:
        a_mid, a_in, a_out, dt = r["table"]
        ids.append(B.server_submit(srv, B.make_request(r["grid"], r["steps"], dt, a_in, a_out),
                                   a_mid))
    B.server_step(srv)
    B.server_cancel(srv, ids[2])
    for _ in range(200):
        a, q, f = B.server_step(srv)
        if a == 0 and q == 0:
            break
    for k, rid in enumerate(ids):
        state, dens, _ = B.server_query(srv, rid)
        if k == 2:
            assert state == "cancelled"
        else:
            assert state == "done" and dens == ref["results"][k]["density"]
    B.server_destroy(srv)


def test_submit_validation():
    srv = B.server_create(1 << 20, 2, 100)
    big = B.make_request({"nx": 1024, "ny": 1024, "px": (-1, 1), "py": (-1, 1)}, 10, 0.01,
                         [0, 0], [0, 0])
    with pytest.raises(B.DSPError) as e:
        B.server_submit(srv, big, np.zeros((10, 2)))
    assert e.value.code == -2
    cfl = B.make_request({"nx": 8, "ny": 8, "px": (-1, 1), "py": (-1, 1)}, 10, 5.0, [0, 0], [0, 0])
    with pytest.raises(B.DSPError) as e:
        B.server_submit(srv, cfl, np.zeros((10, 2)))
    assert e.value.code == -5
    B.server_destroy(srv)
