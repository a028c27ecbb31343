"""Open-loop request driver over the library's job scheduler.

The serving loop itself is native: bc_submit hands a job to the context's
scheduler thread, which admits jobs as execution slots and HBM budget free
up, runs every admitted job on a stream of its own (so the kernels of jobs
that arrive while others run overlap on the device) and retires them by
event; bc_poll hands a finished result back.  This module only generates
arrivals, submits at the arrival times, polls, and reports latency
percentiles and throughput.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Request:
    graph: object          # Graph handle from Context.create_graph
    sources: object = None  # None: exact (all sources); else an int32 array
    opts: dict = field(default_factory=dict)

    def work(self) -> int:
        """Traversed edges of the request: sources x canonical edges."""
        k = self.graph.n if self.sources is None else len(self.sources)
        return int(k) * int(self.graph.m)


@dataclass
class Record:
    arrival: float
    submitted: float
    done: float
    status: int
    work: int
    job: int

    @property
    def latency(self) -> float:
        return self.done - self.arrival


def poisson_arrivals(count: int, rate_per_s: float, seed: int) -> np.ndarray:
    """Arrival times (s, from 0) of a Poisson process: exponential gaps."""
    rs = np.random.default_rng(seed)
    return np.cumsum(rs.exponential(1.0 / rate_per_s, size=count))


def run_open_loop(ctx, requests, arrivals, poll_s: float = 2e-4, results: dict | None = None):
    """Submits request i at arrivals[i] (seconds after the start) and polls
    until every job is done.  Returns one Record per request, in order; with
    `results` given, stores each finished BC vector under its request index."""
    t0 = time.perf_counter()
    pending = {}
    records = [None] * len(requests)
    nxt = 0
    while nxt < len(requests) or pending:
        now = time.perf_counter() - t0
        while nxt < len(requests) and arrivals[nxt] <= now:
            r = requests[nxt]
            job = ctx.submit(r.graph, r.sources, **r.opts)
            pending[job] = (nxt, float(arrivals[nxt]), time.perf_counter() - t0)
            nxt += 1
        for job in list(pending):
            i, arr, sub = pending[job]
            st, bc, _ = ctx.poll(job, requests[i].graph.n)
            if st == 1:  # BC_PENDING
                continue
            done = time.perf_counter() - t0
            records[i] = Record(arr, sub, done, st, requests[i].work(), job)
            if results is not None:
                results[i] = bc
            del pending[job]
        if nxt < len(requests):
            wait = arrivals[nxt] - (time.perf_counter() - t0)
            time.sleep(min(max(wait, 0.0), poll_s) if pending else max(wait, 0.0))
        else:
            time.sleep(poll_s)
    return records


def solo_service_times(ctx, requests, repeats: int = 1):
    """Service time of each request run alone (submit, wait)."""
    out = []
    for r in requests:
        best = None
        for _ in range(repeats):
            t = time.perf_counter()
            job = ctx.submit(r.graph, r.sources, **r.opts)
            ctx.wait(job, r.graph.n)
            dt = time.perf_counter() - t
            best = dt if best is None else min(best, dt)
        out.append(best)
    return np.array(out)


def summarize(records):
    lat = np.array([r.latency for r in records])
    span = max(r.done for r in records) - min(r.arrival for r in records)
    work = sum(r.work for r in records)
    return {
        "requests": len(records),
        "p50_ms": float(np.percentile(lat, 50) * 1e3),
        "p99_ms": float(np.percentile(lat, 99) * 1e3),
        "mean_ms": float(lat.mean() * 1e3),
        "gteps": work / span / 1e9 if span > 0 else None,
        "errors": int(sum(1 for r in records if r.status != 0)),
    }
