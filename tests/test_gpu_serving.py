"""Continuous-batching fold-in + top-k service (snect_serve_*), through the C ABI.

Each query's result must be the same alone (snect_foldin + snect_topk on the context) and in
a mix of concurrent queries: the kernels and their CTA partition depend only on the query, so
the tolerance is exact equality.  Admission follows the device-memory budget, and requests
staged in the server's pinned pool or from their own copy give the same results.
"""
import math

import numpy as np
import pytest

import snect_synth as S

pytestmark = pytest.mark.gpu


def request_bytes(n, J1):
    """Arena bytes of a request of n cells: cells (8 B), values (4 B) and the fold-in's
    per-256-cell Gram partials, each rounded up to 256 bytes."""
    up = lambda x: -(-x // 256) * 256
    return up(8 * n) + up(4 * n) + up(4 * math.ceil(n / 256) * (J1 * J1 + J1))


@pytest.fixture(scope="module")
def served(gpu_lib):
    import paper_1711_08095_gb300 as snect

    m = S.serving_model(I=(1200, 3000, 5), J=(16, 16, 5))
    idx = np.array([[0, 0, 0], [1, 1, 1]], np.int32)
    c = snect.Snect((1200, 3000, 5), m.G.shape, idx, np.zeros(2, np.float32), np.zeros((0, 2), np.int32),
                    np.zeros(0, np.float32), m.G, m.U, lam=m.lam, lam_g=0.0, lr=0.01, batch=1)
    queries = [S.serving_query(m, q=q, lo=500, hi=15000) for q in range(40)]
    alone = []
    for jk, x, _ in queries:
        u = c.foldin(jk, x)
        i, sc = c.topk(u, 10)
        alone.append((u, i, sc))
    yield m, c, queries, alone
    c.close()


def test_results_are_the_same_alone_and_in_the_mix(served):
    m, c, queries, alone = served
    srv = c.serve(n_slots=6, mem_budget_bytes=64 << 20, max_cells=15000)
    tickets = [srv.submit(jk, x, 10) for jk, x, _ in queries]
    for t, (u0, i0, s0) in zip(tickets, alone):
        u, i, sc, lat = srv.poll(t, 10)
        assert np.array_equal(u, u0) and np.array_equal(i, i0) and np.array_equal(sc, s0)
        assert lat > 0
    st = srv.stats()
    srv.stop()
    assert st["admitted"] == st["completed"] == len(queries)
    assert st["max_concurrent"] > 1  # requests overlapped on the device


@pytest.mark.parametrize("wait_ms", [None, "0"])
def test_requests_beyond_the_pinned_pool(served, wait_ms, monkeypatch):
    """A server keeps four pinned request buffers per slot.  With one slot and 40 requests
    submitted at once, submit waits for buffers to come back as requests complete (the
    default); with SNECT_SERVE_PIN_WAIT_MS=0 most requests find the pool empty and are staged
    at admission from their own copy instead.  Every result is still that of the request
    alone."""
    m, c, queries, alone = served
    if wait_ms is None:
        monkeypatch.delenv("SNECT_SERVE_PIN_WAIT_MS", raising=False)
    else:
        monkeypatch.setenv("SNECT_SERVE_PIN_WAIT_MS", wait_ms)
    srv = c.serve(n_slots=1, mem_budget_bytes=64 << 20, max_cells=15000)
    tickets = [srv.submit(jk, x, 10) for jk, x, _ in queries]
    for t, (u0, i0, s0) in zip(tickets, alone):
        u, i, sc, _ = srv.poll(t, 10)
        assert np.array_equal(u, u0) and np.array_equal(i, i0) and np.array_equal(sc, s0)
    st = srv.stats()
    srv.stop()
    assert st["admitted"] == st["completed"] == len(queries) and st["max_concurrent"] == 1


@pytest.mark.parametrize("fit", [1, 2])
def test_admission_follows_the_memory_budget(served, fit):
    """The requests in flight are carved from one arena of exactly the budget: with room for
    `fit` requests of the largest size and only requests above half of it, never more than
    `fit` run at once, with slots to spare; results stay those of the requests alone."""
    m, c, _, _ = served
    big = [S.serving_query(m, q=100 + q, size=12000 + 250 * q) for q in range(10)]
    alone = [c.foldin(jk, x) for jk, x, _ in big]
    srv = c.serve(n_slots=6, mem_budget_bytes=fit * request_bytes(15000, 16), max_cells=15000)
    tickets = [srv.submit(jk, x, 10) for jk, x, _ in big]
    for t, u0 in zip(tickets, alone):
        u, _, _, _ = srv.poll(t, 10)
        assert np.array_equal(u, u0)
    st = srv.stats()
    srv.stop()
    assert st["completed"] == len(big)
    assert 1 <= st["max_concurrent"] <= fit, st


def test_bad_requests(served):
    """Out-of-range cells and non-finite values fail their own request only.  With one slot,
    the request after a bad one runs on the same stream and must not see its flag."""
    import paper_1711_08095_gb300 as snect

    m, c, queries, _ = served
    with pytest.raises(snect.SnectError):
        c.serve(n_slots=2, mem_budget_bytes=1000, max_cells=15000)  # below one largest request
    srv = c.serve(n_slots=1, mem_budget_bytes=64 << 20, max_cells=1000)
    jk, x, _ = queries[0]
    with pytest.raises(snect.SnectError):
        srv.submit(jk, x, 10)  # more cells than max_cells
    u0 = c.foldin(jk[:50], x[:50])
    bad_cell = jk[:50].copy()
    bad_cell[3, 0] = 10 ** 6
    bad_val = x[:50].copy()
    bad_val[7] = np.nan
    for bj, bx in ((bad_cell, x[:50]), (jk[:50], bad_val)):
        t = srv.submit(bj, bx, 10)
        with pytest.raises(snect.SnectError):
            srv.poll(t, 10)
        t = srv.submit(jk[:50], x[:50], 10)  # the server keeps serving
        u, _, _, _ = srv.poll(t, 10)
        assert np.array_equal(u, u0)
    srv.stop()
