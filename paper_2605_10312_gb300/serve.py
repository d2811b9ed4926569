"""Serving loop with continuous batching for ERI requests.

A request is a batch of shell quartets of one registered molecule.  The
server keeps each molecule's basis and Schwarz data resident (pair factors
Q_ab computed once on the device at registration), and runs requests as they
arrive:

  * admission: a request enters when a slot (a CUDA stream) is free and its
    device-memory footprint (output blocks, quartet records, pair data) fits
    in the remaining budget; requests are admitted in arrival order;
  * planning: a pool of host threads builds each admitted request's plan on
    its molecule (eri_plan_on_mol: the molecule's primitive-pair records are
    reused, and the plan's device memory is stream-ordered, so that retiring
    one request never synchronises the device under the others); the native
    planner releases the interpreter lock;
  * execution: the planner thread that built a plan also launches it on
    its slot's stream, so requests that arrive while others are on the
    device overlap with them, and the request loop only admits, polls and
    retires;
  * large requests (off by default): with chunk_quartets set, while fewer
    than chunk_inflight requests are in flight, a request of more than
    chunk_quartets quartets is cut into contiguous chunks whose plans are
    built in parallel on a second pool of host threads, then launched in
    order on the slot's stream into consecutive ranges of one output
    buffer.  Chunk plans add class launches of their own: measured on the
    serving benchmark (with plans of ordered part rounds), chunking every large request cut the burst capacity
    from 194 to 154 requests/s (chunks of 250,000 quartets) and 88
    (100,000) and raised p50 at 50 requests/s from 18 to 22 ms while it cut
    p99 there from 213 to 150 ms; chunking only while fewer than half the
    planner threads were busy kept the capacity (191) but left p99 at 337
    ms;
  * completion: polled with CUDA events; a request that has not finished
    within its timeout is reported with status "timeout" (the host stops
    waiting for it; its memory is reclaimed when the device finishes);
  * precision: quartets whose bound Q_ab Q_cd is below fp32_below run their
    recurrences in FP32 (eri_plan_on_stream with the per-quartet bounds).

Latency is measured from arrival to the completion of the request's work on
the device (host polling granularity included).
"""
from __future__ import annotations

import collections
import concurrent.futures as cf
import dataclasses
import time

import numpy as np

from . import eri, screen

NSPH = np.array([1, 3, 5, 7, 9], dtype=np.int64)


@dataclasses.dataclass
class Molecule:
    key: object
    basis: object
    pairs: np.ndarray     # [npair, 2] shell pairs (a >= b)
    pair_q: np.ndarray    # Schwarz factor per pair (host copy)
    pair_q_dev: object    # the same on the device
    mol: object = None    # eri.Mol: shells and primitive-pair records on the device
    nsph: np.ndarray = None  # spherical components per shell (int64)


@dataclasses.dataclass
class Request:
    rid: int
    mol: object           # registered molecule key
    quartets: np.ndarray  # [n, 4] shell indices
    arrival: float        # seconds after the start of the run


@dataclasses.dataclass
class Result:
    rid: int
    status: str           # "ok", "timeout", "rejected"
    quartets: int
    arrival: float
    admitted: float = float("nan")
    launched: float = float("nan")
    finished: float = float("nan")
    fp32_parts: int = 0
    output: object = None  # device tensor (keep_outputs=True)

    @property
    def latency(self):
        return self.finished - self.arrival


class Server:
    def __init__(self, budget_bytes=8 << 30, slots=8, planners=4, fp32_below=1e-6, timeout_s=10.0,
                 keep_outputs=False, poll_s=50e-6, chunk_quartets=None, chunk_inflight=None):
        import torch
        self.torch = torch
        self.budget = int(budget_bytes)
        self.streams = [torch.cuda.Stream() for _ in range(slots)]
        self.pool = cf.ThreadPoolExecutor(max_workers=planners)
        # chunk plans of large requests (a planner thread waits on them, so
        # they need threads of their own)
        self.chunk_quartets = chunk_quartets
        self.chunk_pool = cf.ThreadPoolExecutor(max_workers=planners)
        # chunking applies while fewer requests than this are in flight
        self.chunk_inflight = chunk_inflight if chunk_inflight is not None else max(1, planners // 2)
        self.chunked = 0  # requests run as several chunk plans
        self.fp32_below = fp32_below
        self.timeout_s = timeout_s
        self.keep_outputs = keep_outputs
        self.poll_s = poll_s
        self.molecules = {}

    def close(self):
        self.pool.shutdown(wait=True)
        self.chunk_pool.shutdown(wait=True)
        for m in self.molecules.values():
            if m.mol is not None:
                m.mol.close()

    # -- molecules ----------------------------------------------------------
    def register(self, key, basis):
        """Keep a molecule resident: Schwarz factors of every shell pair,
        computed on the device."""
        pairs, q = screen.pair_bounds(basis)
        mol = Molecule(key, basis, pairs, q, self.torch.from_numpy(q).to("cuda"), eri.Mol(basis),
                       NSPH[basis.shell_l].astype(np.int64))
        self.molecules[key] = mol
        return mol

    # -- accounting ---------------------------------------------------------
    @staticmethod
    def chunks(n, chunk_quartets):
        """Quartet ranges [lo, hi) of the plans of a request of n quartets."""
        k = 1 if not chunk_quartets or n <= chunk_quartets else -(-n // chunk_quartets)
        cuts = [n * i // k for i in range(k + 1)]
        return list(zip(cuts[:-1], cuts[1:]))

    @staticmethod
    def footprint(mol, quartets, chunk_quartets=None):
        """Device bytes a request holds while it runs: its output blocks, up
        to four quartet-part records per quartet and, per plan (one per
        chunk), a copy of the molecule's pair records."""
        q = np.asarray(quartets)
        ns = mol.nsph if mol.nsph is not None else NSPH[mol.basis.shell_l].astype(np.int64)
        out = int((ns[q[:, 0]] * ns[q[:, 1]] * ns[q[:, 2]] * ns[q[:, 3]]).sum())
        npair = 2 * mol.pairs.shape[0]
        nplan = len(Server.chunks(q.shape[0], chunk_quartets))
        return 8 * out + 4 * 32 * q.shape[0] + nplan * (32 * npair + (1 << 16))

    def bounds(self, mol, quartets):
        return screen.quartet_bounds(mol.pair_q, quartets)

    # -- one request --------------------------------------------------------
    def _build(self, req, stream, lo=0, hi=None):
        """The plan of quartets [lo, hi) of a request."""
        mol = self.molecules[req.mol]
        if lo != 0 or hi is not None:
            req = Request(req.rid, req.mol, req.quartets[lo:hi], req.arrival)
        # a request's class launches spread over the plan's streams (measured:
        # one stream per plan leaves small requests' kernels too narrow to
        # fill the GPU -- capacity 106 against 138 requests/s)
        if self.fp32_below is None:
            return eri.Plan(None, req.quartets, mol=mol.mol, stream=stream)
        qb = self.bounds(mol, req.quartets)
        return eri.Plan(None, req.quartets, qbound=qb, fp32_below=self.fp32_below, mol=mol.mol, stream=stream)

    def _build_and_launch(self, req, stream, chunk=None):
        """On a planner thread: the request's plan, its output buffer and its
        launches on the slot's stream, then an event after them.  Launching
        a plan's few hundred class kernels takes milliseconds of host time,
        which the request loop's thread would otherwise spend once per
        request (measured: it bounded capacity at 167 requests/s with 16
        slots)."""
        torch = self.torch
        ranges = self.chunks(req.quartets.shape[0], chunk)
        if len(ranges) == 1:
            plans = [self._build(req, stream)]
        else:
            futs = [self.chunk_pool.submit(self._build, req, stream, lo, hi) for lo, hi in ranges[1:]]
            plans = [self._build(req, stream, *ranges[0])] + [f.result() for f in futs]
        counts = [p.output_count for p in plans]
        with torch.cuda.stream(stream):
            out = torch.empty(max(1, sum(counts)), dtype=torch.float64, device="cuda")
            off = 0
            for p, c in zip(plans, counts):
                p.compute(out[off:off + c], stream)
                off += c
            ev = torch.cuda.Event()
            ev.record(stream)
        return plans, out, ev, sum(p.stats()["fp32_parts"] for p in plans)

    def run_alone(self, req):
        """The request evaluated by itself (plain plan, default stream
        order): the reference for results in the mix."""
        mol = self.molecules[req.mol]
        if self.fp32_below is None:
            p = eri.Plan(mol.basis, req.quartets)
        else:
            p = eri.Plan(mol.basis, req.quartets, qbound=self.bounds(mol, req.quartets),
                         fp32_below=self.fp32_below)
        out = self.torch.empty(max(1, p.output_count), dtype=self.torch.float64, device="cuda")
        p.compute(out)
        self.torch.cuda.synchronize()
        p.close()
        return out

    # -- the loop -----------------------------------------------------------
    def serve(self, requests):
        """Run a request stream (arrival times relative to the start) to
        completion; returns one Result per request, in request order."""
        torch = self.torch
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        results = {r.rid: Result(r.rid, "ok", int(r.quartets.shape[0]), r.arrival) for r in requests}
        queue = collections.deque()
        free_slots = list(range(len(self.streams)))[::-1]
        free_bytes = self.budget
        planning = {}   # future -> (req, slot, nbytes)
        running = []    # [req, slot, nbytes, plan, out, event, timed_out]
        t0 = time.perf_counter()
        while pending or queue or planning or running:
            now = time.perf_counter() - t0
            progressed = False
            while pending and pending[0].arrival <= now:
                queue.append(pending.popleft())
                progressed = True
            # admission in arrival order while the head fits
            while queue and free_slots:
                req = queue[0]
                # chunk plans only while the planner threads have room
                light = len(planning) + len(running) < self.chunk_inflight
                chunk = self.chunk_quartets if light else None
                nbytes = self.footprint(self.molecules[req.mol], req.quartets, chunk)
                if nbytes > self.budget:
                    queue.popleft()
                    res = results[req.rid]
                    res.status, res.finished = "rejected", now
                    progressed = True
                    continue
                if nbytes > free_bytes:
                    break
                queue.popleft()
                slot = free_slots.pop()
                free_bytes -= nbytes
                if len(self.chunks(req.quartets.shape[0], chunk)) > 1:
                    self.chunked += 1
                results[req.rid].admitted = now
                fut = self.pool.submit(self._build_and_launch, req, self.streams[slot], chunk)
                planning[fut] = (req, slot, nbytes)
                progressed = True
            # plans built and launched by the planner threads
            for fut in [f for f in planning if f.done()]:
                req, slot, nbytes = planning.pop(fut)
                plans, out, ev, fp32_parts = fut.result()
                res = results[req.rid]
                res.launched = time.perf_counter() - t0
                res.fp32_parts = fp32_parts
                running.append([req, slot, nbytes, plans, out, ev, False])
                progressed = True
            # completions (bounded waits)
            still = []
            for item in running:
                req, slot, nbytes, plans, out, ev, timed_out = item
                res = results[req.rid]
                if ev.query():
                    t = time.perf_counter() - t0
                    if not timed_out:
                        res.finished = t
                    for p in plans:
                        p.close()  # stream-ordered: frees after the work on the slot's stream
                    if self.keep_outputs and not timed_out:
                        res.output = out
                    del out
                    free_slots.append(slot)
                    free_bytes += nbytes
                    progressed = True
                    continue
                if not timed_out and time.perf_counter() - t0 - res.arrival > self.timeout_s:
                    res.status, res.finished = "timeout", time.perf_counter() - t0
                    item[6] = True
                still.append(item)
            running = still
            if not progressed:
                time.sleep(self.poll_s)
        return [results[r.rid] for r in requests]


def summary(results, offered_span=None):
    """p50/p99 latency (ms) and throughput of a finished run."""
    ok = [r for r in results if r.status == "ok"]
    lat = np.array([r.latency for r in ok]) * 1e3
    first = min(r.arrival for r in results)
    last = max(r.finished for r in results)
    nq = sum(r.quartets for r in ok)
    arrivals = np.array(sorted(r.arrival for r in results))
    span = offered_span if offered_span is not None else (arrivals[-1] - arrivals[0] if len(arrivals) > 1 else 0.0)
    return {
        "requests": len(results), "ok": len(ok),
        "timeout": sum(r.status == "timeout" for r in results),
        "rejected": sum(r.status == "rejected" for r in results),
        "p50_ms": float(np.percentile(lat, 50)) if len(lat) else None,
        "p99_ms": float(np.percentile(lat, 99)) if len(lat) else None,
        "mean_ms": float(lat.mean()) if len(lat) else None,
        "served_quartets_per_s": nq / max(1e-9, last - first),
        "served_requests_per_s": len(ok) / max(1e-9, last - first),
        "offered_requests_per_s": (len(results) - 1) / span if span > 0 else None,
        "offered_quartets_per_s": sum(r.quartets for r in results) / span if span > 0 else None,
        "fp32_parts": int(sum(r.fp32_parts for r in ok)),
        # where the time of the largest 5% of requests goes: waiting for
        # admission, planning and launching, and the device work
        "largest_5pct": _stages([r for r in ok if r.quartets >= np.percentile([x.quartets for x in ok], 95)])
        if ok else None,
    }


def _stages(rs):
    ms = lambda xs: float(np.mean(xs) * 1e3) if len(xs) else None
    return {"requests": len(rs), "quartets_mean": float(np.mean([r.quartets for r in rs])) if rs else None,
            "admit_ms": ms([r.admitted - r.arrival for r in rs]),
            "plan_launch_ms": ms([r.launched - r.admitted for r in rs]),
            "device_ms": ms([r.finished - r.launched for r in rs])}


def screened_pool(mol, threshold, n, seed):
    """A seeded random sample of n quartets from the molecule's screened
    list (all of them, shuffled, if fewer survive)."""
    from . import synth
    return synth.sample_screened_quartets(mol.pair_q, mol.pairs, threshold, n, seed=seed)


def poisson_requests(pools, rate, nreq, nq_range=(1_000, 1_000_000), seed=0, burst=False):
    """A request stream: exponential inter-arrival times of mean 1/rate (all
    at t = 0 when burst), each request a random molecule of `pools` (key ->
    screened quartet pool) and a seeded slice of its pool whose length is
    log-uniform in nq_range."""
    rng = np.random.default_rng(seed)
    keys = sorted(pools)
    t = 0.0
    out = []
    for rid in range(nreq):
        if not burst and rid:
            t += rng.exponential(1.0 / rate)
        key = keys[int(rng.integers(len(keys)))]
        pool = pools[key]
        n = int(min(pool.shape[0], round(10 ** rng.uniform(np.log10(nq_range[0]), np.log10(nq_range[1])))))
        start = int(rng.integers(0, pool.shape[0] - n + 1))
        out.append(Request(rid, key, np.ascontiguousarray(pool[start:start + n]), 0.0 if burst else t))
    return out
