"""Host side of the serving loop: the seeded request recipe (Poisson arrivals,
log-uniform sizes and step caps, boxes and rakes) and the latency summary."""
import math
from types import SimpleNamespace

import numpy as np

from paper_2606_02627_gb300 import inputs, serving


def _fields():
    grids = [inputs.cube_grid(33), inputs.Grid((17, 25, 9), (1.0, -2.0, 0.5), (0.5, 0.25, 1.0))]
    return [SimpleNamespace(grid=g) for g in grids]


def test_requests_are_seeded_and_within_bounds():
    fields = _fields()
    a = serving.make_requests(fields, 200, 50.0, seed=7, min_seeds=10, max_seeds=2000, min_steps=5, max_steps=500)
    b = serving.make_requests(fields, 200, 50.0, seed=7, min_seeds=10, max_seeds=2000, min_steps=5, max_steps=500)
    c = serving.make_requests(fields, 200, 50.0, seed=8, min_seeds=10, max_seeds=2000, min_steps=5, max_steps=500)
    assert [r.arrival for r in a] == [r.arrival for r in b]
    assert all(np.array_equal(x.seeds, y.seeds) for x, y in zip(a, b))
    assert [r.arrival for r in a] != [r.arrival for r in c]
    arrivals = np.array([r.arrival for r in a])
    assert np.all(np.diff(arrivals) > 0)
    for r in a:
        assert 10 <= len(r.seeds) <= 2000
        assert 5 <= r.max_steps <= 500
        assert r.shape in ("box", "rake")
        g = fields[r.field].grid
        lo = np.array(g.origin)
        hi = lo + np.array(g.spacing) * (np.array(g.dims) - 1)
        assert r.seeds.dtype == np.float32 and r.seeds.shape[1] == 3
        assert np.all(r.seeds >= lo - 1e-4) and np.all(r.seeds <= hi + 1e-4)
    assert {r.shape for r in a} == {"box", "rake"}
    assert {r.field for r in a} == {0, 1}


def test_poisson_gaps_and_log_uniform_sizes():
    fields = _fields()
    rate = 40.0
    reqs = serving.make_requests(fields, 4000, rate, seed=3, min_seeds=10, max_seeds=1000, min_steps=10,
                                 max_steps=1000)
    gaps = np.diff([0.0] + [r.arrival for r in reqs])
    # exponential gaps: mean 1/rate, coefficient of variation 1
    assert abs(gaps.mean() * rate - 1.0) < 0.06
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.08
    # log-uniform seed counts: log n uniform on [log 10, log 1000]
    logn = np.log([len(r.seeds) for r in reqs])
    assert abs(logn.mean() - 0.5 * (math.log(10) + math.log(1000))) < 0.1
    assert abs(np.median([len(r.seeds) for r in reqs]) - 100) < 15


def test_summary_percentiles():
    reqs = []
    for i in range(101):
        r = serving.Request(i, arrival=float(i), field=0, seeds=np.zeros((1, 3), np.float32), max_steps=1,
                            shape="box")
        r.admitted = r.arrival + 0.001
        r.done = r.arrival + 0.01 * (i + 1)    # latencies 10 ms .. 1010 ms
        r.steps = 5
        reqs.append(r)
    s = serving.summarize(reqs)
    assert s["requests"] == 101
    assert abs(s["p50_ms"] - 510.0) < 1e-6
    assert abs(s["p99_ms"] - np.percentile(np.arange(1, 102) * 10.0, 99)) < 1e-6
    assert abs(s["max_ms"] - 1010.0) < 1e-6
    assert s["particle_steps"] == 505
    assert abs(s["makespan_s"] - (100.0 + 1.01)) < 1e-9
    assert abs(s["queue_ms_p99"] - 1.0) < 1e-6
