"""Serving loop on the GPU: admission, continuous batching, and that each
query's result is the same alone and in the mix (bit-exact)."""
import time

import numpy as np
import pytest

import workload as W
from tests._helpers import PRF, alloc_outs, load_tables

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2209_03526_gb300")


@pytest.fixture(scope="module")
def served():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = P.Context(0, prf_keys=PRF, serve_max_inflight=8)
    graph = W.edge_graph(20000, 80000, 4, 2, seed=41)
    load_tables(c, graph)
    yield c, graph
    c.close()


def _result_tensors(res):
    out = []
    for g in res["groups"]:
        out.append([P.device_words(p, g["n_elems"]).clone() for p in g["shares"]])
    return out


def test_served_results_equal_alone(served):
    ctx, graph = served
    qs = W.query_mix(graph, 12, seed=42)
    toks = [P.keygen(q["preds"], 32, bytes([i + 1]) * 16) for i, q in enumerate(qs)]
    tickets = []
    pending = list(range(len(qs)))
    results = {}
    # submit in waves: later queries arrive while earlier ones are on the device
    while pending or tickets:
        while pending:
            try:
                tk = ctx.submit(toks[pending[0]])
            except P.OblivgmError as e:
                assert e.status == P.EAGAIN
                break
            tickets.append((tk, pending.pop(0)))
        tk, qi = tickets.pop(0)
        res = ctx.poll(tk, timeout_ms=60000)
        assert res is not None and res["latency_ms"] >= 0
        results[qi] = (tk, _result_tensors(res))
        ctx.release(tk)
    stats = ctx.serve_stats()
    assert stats["completed"] >= len(qs) and stats["reserved_bytes"] == 0
    for qi, (tk, got) in results.items():
        outs = alloc_outs(graph, preds=qs[qi]["preds"])
        ctx.filter_and_combine(tk & 0xFFFFFFFF, toks[qi], outs)
        torch.cuda.synchronize()
        for ga, gb in zip(got, outs):
            for ta, tb in zip(ga, gb):
                assert torch.equal(ta, tb), qi


def test_admission_by_slots(served):
    ctx, graph = served
    q = W.query_mix(graph, 1, seed=43)[0]
    tok = P.keygen(q["preds"], 32, bytes(16))
    tks = []
    rejected = 0
    for _ in range(12):
        try:
            tks.append(ctx.submit(tok))
        except P.OblivgmError as e:
            assert e.status == P.EAGAIN
            rejected += 1
    assert len(tks) == 8 and rejected == 4
    for tk in tks:
        assert ctx.poll(tk, timeout_ms=60000) is not None
        ctx.release(tk)
    with pytest.raises(P.OblivgmError) as e:
        ctx.poll(tks[0], 0)
    assert e.value.status == P.ENOENT


def test_poll_timeout_and_unknown_ticket(served):
    ctx, graph = served
    with pytest.raises(P.OblivgmError) as e:
        ctx.poll(987654321, 0)
    assert e.value.status == P.ENOENT
    q = W.query_mix(graph, 1, seed=44)[0]
    tk = ctx.submit(P.keygen(q["preds"], 32, bytes(16)))
    r = ctx.poll(tk, 0)            # may or may not be done already; must not block
    t0 = time.time()
    r = ctx.poll(tk, 60000)
    assert r is not None and time.time() - t0 < 60
    ctx.release(tk)


def test_admission_by_memory():
    """A query whose output share sets do not fit in the serve arena is not admitted; one that
    fits is, and releasing it returns its bytes."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    g = W.rng(45)
    tab = W.table(W.uniform_attrs(g, 1, 10000, 32), 32, g)
    small = W.table(W.uniform_attrs(g, 1, 1000, 32), 32, g)
    # 1,000-element group needs 12,000 B of outputs; 10,000 elements need 120,000 B
    with P.Context(0, prf_keys=PRF, serve_arena_bytes=50000) as c:
        from tests._helpers import to_dev
        c.load_shares(0, [to_dev(s) for s in tab["shares"]], 32)
        c.load_shares(1, [to_dev(s) for s in small["shares"]], 32)
        big_tok = P.keygen([W.eq_pred(0, 0, 0, 5)], 32, bytes(16))
        with pytest.raises(P.OblivgmError) as e:
            c.submit(big_tok)
        assert e.value.status == P.EAGAIN
        tk = c.submit(P.keygen([W.eq_pred(1, 0, 0, 5)], 32, bytes(16)))
        assert c.serve_stats()["reserved_bytes"] == 12000
        assert c.poll(tk, 60000) is not None
        c.release(tk)
        st = c.serve_stats()
        assert st["reserved_bytes"] == 0 and st["rejected"] == 1 and st["completed"] == 1


def test_poll_waits_at_most_the_context_limit():
    """A negative timeout waits up to the context's poll limit, not without end: with the limit
    at 2 ms a poll on a query that runs for tens of milliseconds returns ETIMEOUT at once; the
    query keeps running and a later poll under the default limit gets its result."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    g = W.rng(46)
    n = 1 << 20
    tab = W.table(W.uniform_attrs(g, 1, n, 32), 32, g)
    preds = [W.range_pred(0, 0, 0, 1000 * k, 0xF0000000) for k in range(8)]   # ~60 ms on one GB300
    with P.Context(0, prf_keys=PRF) as c:
        from tests._helpers import to_dev
        c.load_shares(0, [to_dev(s) for s in tab["shares"]], 32)
        assert c.set_poll_limit(2) == P.POLL_LIMIT_DEFAULT_MS
        tk = c.submit(P.keygen(preds, 32, bytes(16)))
        t0 = time.time()
        with pytest.raises(P.OblivgmError) as e:
            c.poll(tk, -1)
        assert e.value.status == P.ETIMEOUT and time.time() - t0 < 1.0
        with pytest.raises(P.OblivgmError) as e:
            c.poll(tk, 60000)              # a longer timeout is capped by the limit too
        assert e.value.status == P.ETIMEOUT
        assert c.set_poll_limit(P.POLL_LIMIT_DEFAULT_MS) == 2
        r = c.poll(tk, -1)
        assert r is not None and r["groups"][0]["n_elems"] == n
        c.release(tk)
        with pytest.raises(P.OblivgmError) as e:
            c.set_poll_limit(0)
        assert e.value.status == P.EINVAL


def test_a_failed_served_batch_reports_why():
    """When a served batch cannot launch (its workspace allocation is refused through the test
    hook) the poll reports the failure with the launch's own reason, not an empty text."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    g = W.rng(47)
    tab = W.table(W.uniform_attrs(g, 1, 5000, 32), 32, g)
    with P.Context(0, prf_keys=PRF) as c:
        from tests._helpers import to_dev
        c.load_shares(0, [to_dev(s) for s in tab["shares"]], 32)
        tok = P.keygen([W.eq_pred(0, 0, 0, 5)], 32, bytes(16))
        c.test_fail_next_alloc()
        tk = c.submit(tok)
        with pytest.raises(P.OblivgmError) as e:
            c.poll(tk, 60000)
        assert e.value.status == P.ECUDA and "refused" in str(e.value)
        c.release(tk)
        tk = c.submit(tok)                 # the next batch allocates normally
        assert c.poll(tk, 60000) is not None
        c.release(tk)
