"""Serving loop host logic without a GPU: the request stream generator, the
run summary, and the request loop (admission by device-memory footprint,
slots, rejection, bounded waits and timeouts) against fakes of the device
calls."""
import contextlib
import sys
import time

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


# ---------------------------------------------------------------------------
# the request loop against fakes of the device calls (no GPU): streams and
# events that complete after a set time, and a plan whose compute occupies
# its stream for a set duration
# ---------------------------------------------------------------------------
class _FakeStream:
    def __init__(self):
        self.busy_until = 0.0

    def wait_event(self, ev):
        # work queued afterwards starts no earlier than the event
        self.busy_until = max(self.busy_until, ev.t or 0.0)


class _FakeEvent:
    def __init__(self):
        self.t = None

    def record(self, stream):
        self.t = stream.busy_until

    def query(self):
        return time.perf_counter() >= self.t


class _FakeCuda:
    Stream = _FakeStream
    Event = _FakeEvent

    @contextlib.contextmanager
    def stream(self, st):
        yield


class _FakeTorch:
    float64 = "float64"
    cuda = _FakeCuda()

    @staticmethod
    def empty(n, dtype=None, device=None):
        return np.empty(n)


class _Tracker:
    """In-flight plans (computed, not closed), checked against the budget
    and the slot count at every launch."""

    def __init__(self, budget, slots, mol, duration):
        import threading
        self.budget, self.slots, self.mol, self.duration = budget, slots, mol, duration
        self.lock = threading.Lock()   # plans are launched from planner threads
        self.live = set()
        self.plans_of = {}
        self.streams_of = {}
        self.max_live = 0
        self.launch_order = []

    def plan_class(self):
        tr = self

        class FakePlan:
            def __init__(self, basis, quartets, mol=None, stream=None, qbound=None, fp32_below=None, **kw):
                self.q = np.asarray(quartets)
                self.output_count = int(self.q.shape[0])

            def compute(self, out, st):
                with tr.lock:
                    st.busy_until = max(st.busy_until, time.perf_counter()) + tr.duration(self.q)
                    tr.live.add(self)
                    tr.launch_order.append(int(self.q[0, 0]))
                    tr.max_live = max(tr.max_live, len(tr.live))
                    used = sum(serve.Server.footprint(tr.mol, p.q) for p in tr.live)
                    assert used <= tr.budget, "admitted beyond the memory budget"
                    # a request may run as several chunk plans (its id is
                    # the first shell index of its quartets)
                    tr.plans_of.setdefault(int(self.q[0, 0]), []).append(self)
                    tr.streams_of.setdefault(int(self.q[0, 0]), set()).add(id(st))
                    reqs = {int(p.q[0, 0]) for p in tr.live}
                    assert len(reqs) <= tr.slots, "more requests in flight than slots"

            def stats(self):
                return {"fp32_parts": 0}

            def close(self):
                with tr.lock:
                    tr.live.discard(self)
        return FakePlan


class _FakeMol:
    def close(self):
        pass


def _server(monkeypatch, budget, slots, timeout_s, duration):
    monkeypatch.setitem(sys.modules, "torch", _FakeTorch())
    mol = serve.Molecule("m", None, np.zeros((10, 2), dtype=np.int32), np.ones(10), None, mol=_FakeMol(),
                         nsph=np.ones(64, dtype=np.int64))
    tr = _Tracker(budget, slots, mol, duration)
    monkeypatch.setattr(serve.eri, "Plan", tr.plan_class())
    srv = serve.Server(budget_bytes=budget, slots=slots, planners=2, fp32_below=None, timeout_s=timeout_s,
                       poll_s=1e-4)
    srv.molecules["m"] = mol
    return srv, tr, mol


def _requests(sizes, arrivals):
    # the first shell index of a request's quartets is its id (launch order)
    return [serve.Request(i, "m", np.full((n, 4), i, dtype=np.int32), t) for i, (n, t) in
            enumerate(zip(sizes, arrivals))]


def test_admission_holds_the_memory_budget_and_the_slots(monkeypatch):
    """Twelve requests at once, memory for two: never more than two in
    flight, all served, admitted in arrival order (the planner threads
    launch each plan as soon as it is built)."""
    one = serve.Server.footprint(serve.Molecule("m", None, np.zeros((10, 2)), np.ones(10), None,
                                                nsph=np.ones(64, dtype=np.int64)), np.zeros((1000, 4), dtype=np.int32))
    srv, tr, _ = _server(monkeypatch, budget=2 * one + 100, slots=4, timeout_s=5.0, duration=lambda q: 0.05)
    res = srv.serve(_requests([1000] * 12, [0.0] * 12))
    srv.close()
    assert [r.status for r in res] == ["ok"] * 12
    assert tr.max_live == 2
    adm = [r.admitted for r in res]
    assert adm == sorted(adm) and sorted(tr.launch_order) == list(range(12))
    assert all(r.admitted <= r.launched <= r.finished for r in res)


def test_oversize_request_is_rejected_others_served(monkeypatch):
    srv, tr, mol = _server(monkeypatch, budget=300_000, slots=2, timeout_s=5.0, duration=lambda q: 0.005)
    res = srv.serve(_requests([100, 100_000, 100], [0.0, 0.001, 0.002]))
    srv.close()
    assert serve.Server.footprint(mol, np.zeros((100_000, 4), dtype=np.int32)) > 300_000
    assert [r.status for r in res] == ["ok", "rejected", "ok"]


def test_timeout_is_reported_and_the_slot_held_until_the_work_ends(monkeypatch):
    """A request whose work outlasts the timeout is reported as "timeout" at
    the deadline; its slot and memory return only when the device finishes,
    so the next request (one slot, arriving shortly before) launches after
    that and, its latency counted from its arrival, within its timeout."""
    work = {0: 0.30, 1: 0.01}
    srv, tr, _ = _server(monkeypatch, budget=1 << 30, slots=1, timeout_s=0.05,
                         duration=lambda q: work[int(q[0, 0])])
    res = srv.serve(_requests([10, 10], [0.0, 0.27]))
    srv.close()
    assert res[0].status == "timeout" and res[1].status == "ok"
    assert res[0].finished - res[0].arrival < 0.25          # reported at the deadline, not at the end
    assert res[1].launched >= 0.29                          # the slot was held until the work ended



def test_large_request_runs_as_chunk_plans(monkeypatch):
    """A request of more than chunk_quartets quartets runs as ceil(n / chunk)
    plans of contiguous quartet ranges, launched in order on its slot's
    stream and all closed when its work ends; its footprint counts each chunk
    plan's copy of the pair records (the sum of the chunk plans' footprints)."""
    srv, tr, mol = _server(monkeypatch, budget=1 << 30, slots=2, timeout_s=5.0, duration=lambda q: 0.01)
    srv.chunk_quartets = 400
    reqs = _requests([1000, 300], [0.0, 0.0])
    res = srv.serve(reqs)
    srv.close()
    assert [r.status for r in res] == ["ok", "ok"]
    assert srv.chunked == 1
    assert [p.q.shape[0] for p in tr.plans_of[0]] == [333, 333, 334]
    assert len(tr.plans_of[1]) == 1
    assert len(tr.streams_of[0]) == 1
    assert not tr.live
    assert serve.Server.chunks(1000, 400) == [(0, 333), (333, 666), (666, 1000)]
    assert serve.Server.chunks(400, 400) == [(0, 400)] and serve.Server.chunks(7, None) == [(0, 7)]
    whole = serve.Server.footprint(mol, reqs[0].quartets, 400)
    assert whole == sum(serve.Server.footprint(mol, p.q) for p in tr.plans_of[0])


def test_no_chunks_under_load(monkeypatch):
    """With as many requests in flight as chunk_inflight, a large request
    runs as one plan."""
    srv, tr, _ = _server(monkeypatch, budget=1 << 30, slots=4, timeout_s=5.0, duration=lambda q: 0.05)
    srv.chunk_quartets = 400
    srv.chunk_inflight = 1
    res = srv.serve(_requests([100, 1000], [0.0, 0.0]))
    srv.close()
    assert [r.status for r in res] == ["ok", "ok"]
    assert len(tr.plans_of[1]) == 1 and srv.chunked == 0
