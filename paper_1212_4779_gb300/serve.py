"""Serving driver: Poisson request traces against resident graphs, run
through the library's continuous-batching server (sg_server_*) and, for
comparison, one query per launch in arrival order.

Latency is completion minus arrival on the host clock; throughput is
requests divided by the time from the first arrival to the last
completion.
"""

from __future__ import annotations

import time
from dataclasses import dataclass

import numpy as np

from . import sg


@dataclass
class Request:
    t_arrival: float  # seconds after the trace start
    graph: int        # index into the resident graphs
    R: int
    k: int
    model: str
    p: float
    seed: int


def poisson_trace(count, rate, seed, graph_models, R_choices=(100, 200), k_range=(10, 100), hash_seed0=100000):
    """`count` requests with exponential inter-arrival times (mean 1/rate),
    target graph uniform over `graph_models` [(model, p), ...], R uniform
    over R_choices, k uniform in k_range, hash seed hash_seed0 + j."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = np.cumsum(rng.exponential(1.0 / rate, size=count))
    out = []
    for j in range(count):
        gi = int(rng.integers(0, len(graph_models)))
        model, p = graph_models[gi]
        out.append(Request(float(t[j]), gi, int(rng.choice(R_choices)), int(rng.integers(k_range[0], k_range[1] + 1)),
                           model, p, hash_seed0 + j))
    return out


def _stats(lat_ms, makespan_s, n):
    lat = np.asarray(lat_ms, dtype=np.float64)
    return {"requests": n, "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "qps": n / makespan_s if makespan_s > 0 else 0.0,
            "makespan_s": makespan_s}


def run_served(graphs, trace, max_running=8, k_cap=128, memory_budget=0, timeout_s=3600.0):
    """Submit each request at its arrival time to a server and collect
    results; returns (stats, {index: (seeds, gains)})."""
    srv = sg.sg_server_create(max_running=max_running, memory_budget=memory_budget, k_cap=k_cap)
    results, lat = {}, []
    try:
        t0 = time.perf_counter()
        pending = {}
        nxt = 0
        while nxt < len(trace) or pending:
            now = time.perf_counter() - t0
            while nxt < len(trace) and trace[nxt].t_arrival <= now:
                r = trace[nxt]
                rid = sg.sg_server_submit(srv, graphs[r.graph].handle, r.R, r.k, r.model, r.p, r.seed)
                pending[rid] = (nxt, r.t_arrival)
                nxt += 1
            for rid in list(pending):
                i, ta = pending[rid]
                done, seeds, gains, _ = sg.sg_server_poll(srv, rid, trace[i].k)
                if done:
                    results[i] = (seeds, gains)
                    lat.append((time.perf_counter() - t0 - ta) * 1e3)
                    del pending[rid]
            if time.perf_counter() - t0 > timeout_s:
                raise TimeoutError("served trace did not finish")
            time.sleep(0.0002)
        makespan = time.perf_counter() - t0 - trace[0].t_arrival
    finally:
        sg.sg_server_destroy(srv)
    return _stats(lat, makespan, len(trace)), results


def run_serial(graphs, trace):
    """One query per launch in arrival order on each graph's own workspace:
    request j starts when it has arrived and request j-1 has finished."""
    import torch

    results, service = {}, []
    for i, r in enumerate(trace):
        torch.cuda.synchronize()
        t = time.perf_counter()
        res = graphs[r.graph].select(r.R, r.k, r.model, r.p, r.seed)
        torch.cuda.synchronize()
        service.append(time.perf_counter() - t)
        results[i] = (res.seeds, res.gains)
    finish, lat = 0.0, []
    for r, s_ in zip(trace, service):
        start = max(r.t_arrival, finish)
        finish = start + s_
        lat.append((finish - r.t_arrival) * 1e3)
    return _stats(lat, finish - trace[0].t_arrival, len(trace)), results
