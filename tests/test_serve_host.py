"""Serving loop host logic without a GPU: the request stream generator and
the run summary."""
import numpy as np

from paper_2605_10312_gb300 import serve


def test_poisson_requests_stream():
    pools = {"a": np.arange(4000, dtype=np.int32).reshape(-1, 4), "b": np.arange(40000, dtype=np.int32).reshape(-1, 4)}
    reqs = serve.poisson_requests(pools, rate=50.0, nreq=400, nq_range=(10, 1000), seed=3)
    t = np.array([r.arrival for r in reqs])
    assert t[0] == 0.0 and (np.diff(t) >= 0).all()
    gaps = np.diff(t)
    assert abs(gaps.mean() - 1 / 50) < 0.1 / 50 * 5
    n = np.array([r.quartets.shape[0] for r in reqs])
    assert n.min() >= 10 and n.max() <= 1000
    for r in reqs:
        pool = pools[r.mol]
        # a contiguous slice of the molecule's pool
        first = int(np.flatnonzero((pool == r.quartets[0]).all(axis=1))[0])
        assert np.array_equal(pool[first:first + r.quartets.shape[0]], r.quartets)
    again = serve.poisson_requests(pools, rate=50.0, nreq=400, nq_range=(10, 1000), seed=3)
    assert all(np.array_equal(a.quartets, b.quartets) and a.arrival == b.arrival for a, b in zip(reqs, again))
    burst = serve.poisson_requests(pools, rate=50.0, nreq=10, seed=1, burst=True)
    assert all(r.arrival == 0.0 for r in burst)


def test_summary():
    R = serve.Result
    res = [R(0, "ok", 100, 0.0, finished=0.010), R(1, "ok", 300, 0.005, finished=0.020),
           R(2, "timeout", 50, 0.010, finished=0.5), R(3, "rejected", 10, 0.02, finished=0.02)]
    s = serve.summary(res)
    assert s["ok"] == 2 and s["timeout"] == 1 and s["rejected"] == 1
    assert abs(s["p50_ms"] - 12.5) < 1e-9
    assert abs(s["served_quartets_per_s"] - 400 / 0.5) < 1e-6
    assert abs(s["offered_requests_per_s"] - 3 / 0.02) < 1e-6
