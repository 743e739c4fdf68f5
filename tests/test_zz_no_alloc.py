"""The entry point that allocates no device memory.

oblivgm_filter_and_combine_noalloc serves callers that may not allocate GPU
memory while they run (a fixed up-front memory budget, a latency-critical
serving thread).  It keeps its per-call workspace in one fixed device array
inside the library instead of asking the allocator, so it must give exactly
what oblivgm_filter_and_combine gives.  Shares are integers: "within the
tolerance" here means equal word for word.  Two different queries are run one
after the other so the second call reuses the array the first one filled.
This file is named to be collected last.
"""
import numpy as np
import pytest

import workload as W
from tests._helpers import PRF, alloc_outs, load_tables

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2209_03526_gb300")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = P.Context(0, prf_keys=PRF)
    yield c
    c.close()


def _equal(a, b):
    return all(torch.equal(x, y) for ga, gb in zip(a, b) for x, y in zip(ga, gb))


def test_no_alloc_equals_filter_and_combine_on_two_calls_in_a_row(ctx):
    graph = W.edge_graph(10007, 30011, 4, 2, seed=51)     # ragged sizes, vertex and edge tables
    load_tables(ctx, graph)
    bulk = W.bulk_vertex_filter(n_vertices=10007, seed=52)
    queries = [bulk["preds"], W.query_mix(graph, 1, seed=53)[0]["preds"]]
    for call, preds in enumerate(queries):
        toks = P.keygen(preds, 32, bytes([call + 1]) * 16)
        want = alloc_outs(graph, preds=preds)
        ctx.filter_and_combine(40 + call, toks, want)
        got = alloc_outs(graph, preds=preds)
        ctx.filter_and_combine_noalloc(40 + call, toks, got)
        torch.cuda.synchronize()
        ctx.sync()
        assert _equal(got, want), call
        # the result is a real predicate evaluation, not an echo: reconstruct one group
        rec = sum(t.cpu().numpy().view(np.uint32).astype(np.uint64) for t in got[0]) & 0xFFFFFFFF
        assert set(np.unique(rec)) <= {0, 1}


def test_no_alloc_rejects_a_query_larger_than_its_array(ctx):
    graph = W.edge_graph(1000, 3000, 4, 2, seed=54)
    load_tables(ctx, graph)
    preds = [W.range_pred(0, k % 4, 0, 10, 1 << 30) for k in range(40)]   # ~330 KB of workspace
    toks = P.keygen(preds, 32, bytes(16))
    outs = alloc_outs(graph, preds=preds)
    with pytest.raises(P.OblivgmError) as e:
        ctx.filter_and_combine_noalloc(1, toks, outs)
    assert e.value.status == P.ERANGE


def test_no_alloc_calls_back_to_back_on_one_stream(ctx):
    """Two calls with different queries issued one after the other on one stream, with a
    single synchronisation at the end: the second call's workspace upload is ordered after the
    first call's kernel on that stream, so both results equal the ordinary entry point's."""
    graph = W.edge_graph(10007, 30011, 4, 2, seed=56)
    load_tables(ctx, graph)
    queries = [W.bulk_vertex_filter(n_vertices=10007, seed=57)["preds"], W.query_mix(graph, 1, seed=58)[0]["preds"]]
    toks = [P.keygen(q, 32, bytes([call + 7]) * 16) for call, q in enumerate(queries)]
    want = [alloc_outs(graph, preds=q) for q in queries]
    for call, q in enumerate(queries):
        ctx.filter_and_combine(60 + call, toks[call], want[call])
    got = [alloc_outs(graph, preds=q) for q in queries]
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    for call in range(2):
        ctx.filter_and_combine_noalloc(60 + call, toks[call], got[call], stream=s)
    s.synchronize()
    ctx.sync(s)
    torch.cuda.synchronize()
    for call in range(2):
        assert _equal(got[call], want[call]), call


@pytest.mark.filterwarnings("ignore:The CUDA Graph is empty")   # the refused call captures nothing
def test_no_alloc_refuses_a_stream_under_capture(ctx):
    """The call uploads its workspace from a host buffer that lives only for the call, so a
    captured call would replay a copy of freed memory: on a capturing stream it must return
    EINVAL before launching anything, and the context stays usable."""
    graph = W.edge_graph(1000, 3000, 4, 2, seed=59)
    load_tables(ctx, graph)
    preds = [W.eq_pred(0, 0, 0, 5)]
    toks = P.keygen(preds, 32, bytes(16))
    outs = alloc_outs(graph, preds=preds)
    torch.cuda.synchronize()
    launches = ctx.launch_count()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    caught = None
    with torch.cuda.graph(g, stream=s):
        try:
            ctx.filter_and_combine_noalloc(1, toks, outs, stream=s)
        except P.OblivgmError as err:
            caught = err
    assert caught is not None and caught.status == P.EINVAL
    assert ctx.launch_count() == launches
    want = alloc_outs(graph, preds=preds)
    ctx.filter_and_combine(1, toks, want)
    ctx.filter_and_combine_noalloc(1, toks, outs)
    torch.cuda.synchronize()
    ctx.sync()
    assert _equal(outs, want)
