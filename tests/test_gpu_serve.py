"""Serving loop on the GPU: requests that arrive while others run are
admitted as slots and memory free up; every result in the mix equals the
same request evaluated alone; bounded waits and admission limits."""
import numpy as np
import pytest

from paper_2605_10312_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def server_mod():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2605_10312_gb300 import eri, serve
    eri.library()
    return serve


def _setup(serve, srv, sizes=(2, 3, 4), nq=(200, 4000), nreq=16, rate=2000.0, seed=0):
    pools = {}
    for k, nw in enumerate(sizes):
        mol = srv.register(k, synth.water_cluster(nw, seed=40 + k))
        pools[k] = serve.screened_pool(mol, 1e-10, 20_000, seed=k)
    return serve.poisson_requests(pools, rate=rate, nreq=nreq, nq_range=nq, seed=seed)


@pytest.mark.parametrize("chunk", [None, 1500])
def test_results_alone_equal_results_in_the_mix(server_mod, chunk):
    """chunk 1500: requests of more than 1,500 quartets run as two or three
    chunk plans built in parallel, into one output buffer."""
    serve = server_mod
    srv = serve.Server(budget_bytes=1 << 30, slots=4, planners=3, fp32_below=1e-6, keep_outputs=True,
                       chunk_quartets=chunk, chunk_inflight=100)
    reqs = _setup(serve, srv)
    res = srv.serve(reqs)
    assert all(r.status == "ok" for r in res)
    # overlap: some request was admitted before an earlier one finished
    order = sorted(res, key=lambda r: r.admitted)
    assert any(b.admitted < a.finished for a, b in zip(order, order[1:]))
    assert sum(r.fp32_parts for r in res) > 0
    if chunk:
        assert srv.chunked > 0
    for req, r in zip(reqs, res):
        alone = srv.run_alone(req).cpu().numpy()
        mixed = r.output.cpu().numpy()[: alone.shape[0]]
        # chunked quartets reduce atomically: equal up to summation order
        assert np.allclose(mixed, alone, rtol=1e-13, atol=1e-16), req.rid
    s = serve.summary(res)
    assert s["ok"] == len(reqs) and s["p99_ms"] >= s["p50_ms"] > 0
    srv.close()


def test_admission_by_memory_and_rejection(server_mod):
    serve = server_mod
    probe = serve.Server(budget_bytes=1 << 30, slots=2, planners=1, fp32_below=None)
    reqs = _setup(serve, probe, sizes=(2,), nq=(500, 3000), nreq=6, seed=1)
    sizes = [probe.footprint(probe.molecules[r.mol], r.quartets) for r in reqs]
    probe.pool.shutdown()
    # a budget that holds the largest request alone: requests run one by one
    srv = serve.Server(budget_bytes=max(sizes), slots=4, planners=2, fp32_below=None, keep_outputs=True)
    srv.molecules = dict(probe.molecules)
    res = srv.serve(reqs)
    assert all(r.status == "ok" for r in res)
    # at any admission, the admitted requests still running fit the budget
    for r in res:
        held = sum(s for q, s in zip(res, sizes) if q.admitted <= r.admitted < q.finished)
        assert held <= max(sizes)
    # a budget below the smallest request: everything is rejected, nothing hangs
    tiny = serve.Server(budget_bytes=min(sizes) - 1, slots=2, planners=1, fp32_below=None)
    tiny.molecules = dict(probe.molecules)
    res = tiny.serve(reqs)
    assert all(r.status == "rejected" for r in res)
    tiny.pool.shutdown()
    srv.close()


def test_timeout_status_is_bounded(server_mod):
    serve = server_mod
    srv = serve.Server(budget_bytes=1 << 30, slots=2, planners=1, fp32_below=None, timeout_s=0.0)
    reqs = _setup(serve, srv, sizes=(2,), nq=(2000, 4000), nreq=4, seed=2)
    res = srv.serve(reqs)
    assert all(r.status == "timeout" for r in res)
    srv.close()
