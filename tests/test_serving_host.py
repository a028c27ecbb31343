"""Host logic of the open-loop serving driver, without a GPU: the arrival
process, the latency summary, and the submit/poll loop against a fake job
scheduler whose jobs take a fixed service time."""
import time
from dataclasses import dataclass

import numpy as np

from paper_1409_7764_gb300 import serving


@dataclass
class FakeGraph:
    n: int
    m: int


class FakeCtx:
    """submit() starts a job that is done `service` seconds later; poll()
    answers BC_PENDING (1) until then, then (0, bc, stats) once."""

    def __init__(self, service):
        self.service = service
        self.jobs = {}
        self.next = 1
        self.max_in_flight = 0

    def submit(self, g, src=None, **opts):
        job = self.next
        self.next += 1
        self.jobs[job] = (time.perf_counter(), g, src)
        self.max_in_flight = max(self.max_in_flight, len(self.jobs))
        return job

    def poll(self, job, n):
        t, g, src = self.jobs[job]
        if time.perf_counter() - t < self.service:
            return 1, None, None
        del self.jobs[job]
        k = g.n if src is None else len(src)
        return 0, np.full(n, float(k)), {}


def test_poisson_arrivals_are_seeded_exponential_gaps():
    a = serving.poisson_arrivals(20000, 50.0, seed=3)
    b = serving.poisson_arrivals(20000, 50.0, seed=3)
    np.testing.assert_array_equal(a, b)
    gaps = np.diff(np.concatenate([[0.0], a]))
    assert (gaps > 0).all()
    assert abs(gaps.mean() * 50.0 - 1.0) < 0.05            # mean gap 1/rate
    assert abs((gaps < 1 / 50.0).mean() - (1 - np.exp(-1))) < 0.02  # exponential CDF at the mean
    assert not np.array_equal(a, serving.poisson_arrivals(20000, 50.0, seed=4))


def test_request_work_counts_sources_times_edges():
    g = FakeGraph(100, 700)
    assert serving.Request(g).work() == 100 * 700
    assert serving.Request(g, np.arange(7, dtype=np.int32)).work() == 7 * 700


def test_summarize_percentiles_throughput_and_errors():
    recs = [serving.Record(arrival=float(i), submitted=float(i), done=float(i) + 0.001 * (i + 1),
                           status=0 if i != 3 else -5, work=1_000_000_000, job=i + 1)
            for i in range(100)]
    s = serving.summarize(recs)
    lat = np.array([0.001 * (i + 1) for i in range(100)])
    assert s["requests"] == 100 and s["errors"] == 1
    assert abs(s["p50_ms"] - np.percentile(lat, 50) * 1e3) < 1e-9
    assert abs(s["p99_ms"] - np.percentile(lat, 99) * 1e3) < 1e-9
    assert abs(s["mean_ms"] - lat.mean() * 1e3) < 1e-9
    span = (99 + 0.1) - 0.0
    assert abs(s["gteps"] - 100 / span) < 1e-9


def test_open_loop_submits_on_arrival_and_overlaps_jobs():
    ctx = FakeCtx(service=0.03)
    graphs = [FakeGraph(10 + i, 50) for i in range(20)]
    reqs = [serving.Request(g, None if i % 2 else np.arange(3, dtype=np.int32))
            for i, g in enumerate(graphs)]
    arrivals = np.arange(20) * 0.005           # a request every 5 ms, each served in 30 ms
    results = {}
    recs = serving.run_open_loop(ctx, reqs, arrivals, results=results)
    assert len(recs) == 20 and all(r is not None for r in recs)
    assert ctx.max_in_flight > 1               # later requests did not wait for earlier ones
    for i, r in enumerate(recs):
        assert r.status == 0
        assert r.submitted >= r.arrival - 1e-9  # never submitted before it arrives
        assert r.submitted - r.arrival < 0.1    # nor long after
        assert r.latency >= 0.03 - 1e-6         # at least the service time
        assert r.work == reqs[i].work()
        k = graphs[i].n if reqs[i].sources is None else 3
        np.testing.assert_array_equal(results[i], np.full(graphs[i].n, float(k)))
    assert len({r.job for r in recs}) == 20
