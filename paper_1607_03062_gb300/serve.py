"""Request loop on top of the C ABI's continuous-batching server.

The scheduling itself (admission by device footprint, one batched launch per
iteration over every admitted request, retirement) is the library's
``dsp_server_*``; this module only replays a stream of requests in wall-clock
time -- each is submitted once its arrival time has passed -- and records when
each one finished.  Latency = finish - arrival, both on the host clock.
"""
from __future__ import annotations

import time

import numpy as np

from . import binding as B


def prepare(requests: list[dict], precision: str = "fp32_mixed") -> list[dict]:
    """Samples each request's pulse table with the library's sampler."""
    out = []
    for r in requests:
        a_mid, a_in, a_out, dt = B.sample_pulse(r["pulse"], r["steps"])
        out.append({**r, "table": (a_mid, a_in, a_out, dt), "precision": precision})
    return out


def run(requests: list[dict], hbm_budget_bytes: int, max_active: int, chunk_steps: int,
        stream: int = 0, keep_map: bool = False, realtime: bool = True,
        on_step=None) -> dict:
    """Replays ``requests`` (sorted by ``arrival_s``) through one server.

    realtime=False submits everything at t = 0 (all arrivals already passed).
    Returns per-request results and latencies plus aggregate figures."""
    srv = B.server_create(hbm_budget_bytes, max_active, chunk_steps, stream)
    try:
        t0 = time.perf_counter()
        ids = {}
        results = {}
        pending = list(range(len(requests)))
        nxt = 0
        steps_iter = 0
        max_active_seen = 0
        while len(results) < len(requests):
            now = time.perf_counter() - t0
            while nxt < len(pending) and (not realtime or requests[pending[nxt]]["arrival_s"] <= now):
                k = pending[nxt]
                r = requests[k]
                a_mid, a_in, a_out, dt = r["table"]
                req = B.make_request(r["grid"], r["steps"], dt, a_in, a_out,
                                     precision=r.get("precision", "fp32_mixed"),
                                     keep_map=keep_map)
                ids[k] = B.server_submit(srv, req, a_mid)
                nxt += 1
            active, queued, finished = B.server_step(srv)
            steps_iter += 1
            max_active_seen = max(max_active_seen, active + finished)
            if on_step is not None:
                on_step(active, queued, finished)
            now = time.perf_counter() - t0
            if finished or active == 0:
                for k, rid in ids.items():
                    if k in results:
                        continue
                    state, dens, _ = B.server_query(srv, rid)
                    if state in ("done", "failed", "cancelled"):
                        m = None
                        if keep_map and state == "done":
                            g = requests[k]["grid"]
                            dtp = np.float64 if requests[k].get("precision") == "fp64" else np.float32
                            m = np.zeros((g["ny"], g["nx"]), dtype=dtp)
                            B.server_query(srv, rid, m)
                        arr = requests[k]["arrival_s"] if realtime else 0.0
                        results[k] = {"state": state, "density": dens, "finish_s": now,
                                      "latency_s": now - arr, "map": m}
            if active == 0 and queued == 0 and nxt < len(pending) and realtime:
                wait = requests[pending[nxt]]["arrival_s"] - (time.perf_counter() - t0)
                if wait > 0:
                    time.sleep(min(wait, 0.05))
        wall = time.perf_counter() - t0
    finally:
        B.server_destroy(srv)
    lat = np.array([results[k]["latency_s"] for k in range(len(requests))])
    work = sum(float(r["grid"]["nx"]) * r["grid"]["ny"] * r["steps"] for r in requests)
    return {"results": results, "wall_s": wall, "spinor_steps": work,
            "throughput": work / wall, "p50_s": float(np.percentile(lat, 50)),
            "p99_s": float(np.percentile(lat, 99)), "iterations": steps_iter,
            "max_active_seen": max_active_seen}
