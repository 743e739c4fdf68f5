"""GPU parity at the benchmark workloads' full sizes, in the launch configurations bench.py times.

* triangle + pendant (6 predicates) on the 1,000,000-vertex / 10,000,000-edge graph, as one
  prepared plan (one persistent k_filter launch) replayed from a CUDA graph;
* the first 16 queries of the 256-query mix on that graph with 4 vertex attributes, in one plan;
* one query of the serving mix on the 4,000,000-vertex / 40,000,000-edge graph, through the
  serving loop (submit / poll).

Every element of every group must reconstruct to the plaintext predicates (Def. 2), and sampled
elements -- random ones plus the first, the last and both sides of the tile boundaries near
either end -- must equal the oracle share for share (integer work: bit-exact).
"""
import numpy as np
import pytest

import oracle
import workload as W
from tests._helpers import PRF, from_dev, load_tables, oracle_group

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2209_03526_gb300")


def _seed(i):
    return bytes([i % 256, (i >> 8) % 256]) + bytes(14)


def _sample(n, tile, rng, k=192):
    edges = [t * tile + d for t in (1, 2, n // tile - 1, n // tile) for d in (-1, 0, 1)]
    return np.unique(np.concatenate([[0, n - 1], [e for e in edges if 0 <= e < n], rng.integers(0, n, k)]))


def _groups(preds):
    out = {}
    for p in preds:
        out.setdefault(p["group"], p["table"])
    return out


def _check_query(graph, preds, toks, qid, got, tile, rng):
    """got[g] = (3, n) uint32 shares of group g; every element against plaintext, a sample
    against the oracle."""
    for g, t in _groups(preds).items():
        vals = graph["tables"][t]["values"]
        rec = oracle.reconstruct(got[g])
        assert np.array_equal(rec, oracle.plain_group(preds, g, vals)), g
        sample = _sample(vals.shape[1], tile, rng)
        want = oracle_group(oracle, graph, toks, qid, g, sample, threads=16)
        assert np.array_equal(got[g][:, sample], want), g


def _plan_run(ctx, queries, toks, table_n):
    outs = []
    for q in queries:
        ng = max(p["group"] for p in q["preds"]) + 1
        tab = _groups(q["preds"])
        outs.append([[torch.empty(table_n[tab[g]], dtype=torch.int32, device="cuda") for _ in range(3)]
                     for g in range(ng)])
    qids = list(range(1, len(queries) + 1))
    plan = ctx.plan_create(qids, toks, outs)
    shape = ctx.plan_describe(plan)
    ctx.plan_launch(plan)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        ctx.plan_launch(plan, torch.cuda.current_stream())
    for o in outs:
        for grp in o:
            for t in grp:
                t.fill_(-1)
    g.replay()
    torch.cuda.synchronize()
    ctx.sync()
    ctx.plan_destroy(plan)
    return qids, shape, [[np.stack([from_dev(t) for t in grp]) for grp in o] for o in outs]


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = P.Context(0, prf_keys=PRF)
    c.autotune()
    yield c
    c.close()


def test_triangle_pendant_full_size(ctx):
    graph = W.edge_graph(1_000_000, 10_000_000, 2, 2, seed=3)
    load_tables(ctx, graph)
    table_n = {i: t["values"].shape[1] for i, t in enumerate(graph["tables"])}
    q = W.triangle_pendant(graph, seed=3)
    toks = [P.keygen(q["preds"], 32, _seed(0))]
    qids, shape, got = _plan_run(ctx, [q], toks, table_n)
    assert shape["kernel"] == "k_filter"
    _check_query(graph, q["preds"], toks[0], qids[0], got[0], shape["tile"], W.rng(81))


def test_query_mix_prefix_full_size(ctx):
    graph = W.edge_graph(1_000_000, 10_000_000, 4, 2, seed=4)
    load_tables(ctx, graph)
    table_n = {i: t["values"].shape[1] for i, t in enumerate(graph["tables"])}
    queries = W.query_mix(graph, 256, seed=4)[:16]
    toks = [P.keygen(q["preds"], 32, _seed(i)) for i, q in enumerate(queries)]
    qids, shape, got = _plan_run(ctx, queries, toks, table_n)
    rng = W.rng(82)
    for i, q in enumerate(queries):
        _check_query(graph, q["preds"], toks[i], qids[i], got[i], shape["tile"], rng)


def test_served_query_full_size():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    graph = W.edge_graph(4_000_000, 40_000_000, 4, 2, seed=5)
    with P.Context(0, prf_keys=PRF) as c:
        load_tables(c, graph)
        q = W.query_mix(graph, 200, seed=5)[3]
        toks = P.keygen(q["preds"], 32, _seed(3))
        tk = c.submit(toks)
        res = c.poll(tk, 120000)
        got = {}
        for g, r in enumerate(res["groups"]):
            got[g] = np.stack([P.device_words(p, r["n_elems"]).cpu().numpy().view(np.uint32) for p in r["shares"]])
        c.release(tk)
    _check_query(graph, q["preds"], toks, tk & 0xFFFFFFFF, got, 768, W.rng(83))
