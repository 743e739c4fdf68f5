"""GPU parity: the CUDA path through the C ABI against the CPU oracle, bit-exact.

Integer work only, so the bar is equality of every compared share.  Sizes span
several element tiles and a ragged tail; the full-size bulk filter is checked
on sampled elements against the oracle and on every element against the
plaintext predicates (a property that holds at any size).
"""
import numpy as np
import pytest

import oracle
import workload as W
from tests._helpers import PRF, alloc_outs, from_dev, load_tables, oracle_group, to_dev

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


# ---------------------------------------------------------------- raw DPF / DCF

def _keys(kind, n, alphas, betas, g):
    gen = oracle.dpf_gen if kind == P.KEY_DPF else oracle.dcf_gen
    keys = []
    for a, b in zip(alphas, betas):
        s0 = bytes(g.integers(0, 256, 16, dtype=np.uint8))
        s1 = bytes(g.integers(0, 256, 16, dtype=np.uint8))
        keys.extend(gen(n, a, b, s0, s1))
    return keys


@pytest.mark.parametrize("kind", [P.KEY_DPF, P.KEY_DCF])
@pytest.mark.parametrize("n", [5, 16, 32])
def test_raw_batch_all_pairs(ctx, kind, n):
    g = np.random.default_rng(10 * n + kind)
    top = (1 << n) - 1
    alphas = [0, top, int(g.integers(0, top + 1)), int(g.integers(0, top + 1))]
    betas = [int(v) for v in g.integers(1, 1 << 32, len(alphas))]
    keys = _keys(kind, n, alphas, betas, g)
    pts = [0, top, 1, top - 1]
    for a in alphas:
        pts += [a, (a + 1) & top, (a - 1) & top]
    pts += [int(v) for v in g.integers(0, top + 1, 1000 - len(pts))]
    pts = np.array(pts + [int(v) for v in g.integers(0, top + 1, 37)], dtype=np.uint32)   # ragged: 1037
    d_pts = to_dev(pts)
    out = torch.empty(len(keys) * len(pts), dtype=torch.int32, device="cuda")
    (ctx.eval_dpf_batch if kind == P.KEY_DPF else ctx.eval_dcf_batch)(b"".join(keys), len(keys), d_pts, out,
                                                                       all_pairs=True)
    got = from_dev(out).reshape(len(keys), len(pts))
    for k, key in enumerate(keys):
        assert np.array_equal(got[k], oracle.eval_many(key, pts, kind)), k
    # the two parties' shares reconstruct the function
    for j, (a, b) in enumerate(zip(alphas, betas)):
        rec = (got[2 * j].astype(np.uint64) + got[2 * j + 1]) & 0xFFFFFFFF
        want = np.where(pts == a, b, 0) if kind == P.KEY_DPF else np.where(pts < a, b, 0)
        assert np.array_equal(rec, want)


@pytest.mark.parametrize("kind", [P.KEY_DPF, P.KEY_DCF])
def test_raw_batch_key_per_point(ctx, kind):
    g = np.random.default_rng(77 + kind)
    n = 32
    keys = _keys(kind, n, [int(v) for v in g.integers(0, 1 << 32, 5)], [1] * 5, g)
    pts = g.integers(0, 1 << 32, 3001, dtype=np.uint64).astype(np.uint32)
    kop = g.integers(0, len(keys), 3001).astype(np.uint32)
    kop[7] = len(keys) + 3          # out of range -> 0
    out = torch.empty(len(pts), dtype=torch.int32, device="cuda")
    (ctx.eval_dpf_batch if kind == P.KEY_DPF else ctx.eval_dcf_batch)(b"".join(keys), len(keys), to_dev(pts), out,
                                                                       key_of_point=to_dev(kop))
    got = from_dev(out)
    for i in range(len(pts)):
        want = 0 if kop[i] >= len(keys) else oracle.eval_many(keys[kop[i]], [pts[i]], kind)[0]
        assert got[i] == want, i


def test_raw_batch_rejects_bad_arguments(ctx):
    g = np.random.default_rng(5)
    keys = _keys(P.KEY_DPF, 8, [3], [1], g)
    pts = to_dev(np.arange(10, dtype=np.uint32))
    small = torch.empty(5, dtype=torch.int32, device="cuda")
    with pytest.raises(P.OblivgmError) as e:
        ctx.eval_dpf_batch(b"".join(keys), 2, pts, small, all_pairs=True)
    assert e.value.status == P.ERANGE
    out = torch.empty(20, dtype=torch.int32, device="cuda")
    with pytest.raises(P.OblivgmError):       # a DPF key handed to the DCF entry point
        ctx.eval_dcf_batch(b"".join(keys), 2, pts, out, all_pairs=True)


# ---------------------------------------------------------------- fused filter

def _filter(ctx, wl, tokens, query_id, offset=0):
    outs = alloc_outs(wl, offset=offset)
    ctx.filter_and_combine(query_id, tokens, outs)
    torch.cuda.synchronize()
    ctx.sync()
    return [np.stack([from_dev(t) for t in grp]) for grp in outs]


def test_tiny_path_full_parity_and_matcher(ctx):
    wl = W.tiny_path(seed=1)
    load_tables(ctx, wl)
    toks = P.keygen(wl["preds"], wl["n_bits"], bytes(range(16)))
    got = _filter(ctx, wl, toks, 11)
    vt, et = wl["tables"]
    want_v = oracle_group(oracle, wl, toks, 11, 0, np.arange(1000))
    want_e = oracle_group(oracle, wl, toks, 11, 1, np.arange(4000))
    assert np.array_equal(got[0], want_v)
    assert np.array_equal(got[1], want_e)
    bits_v = oracle.reconstruct(got[0]).astype(bool)
    bits_e = oracle.reconstruct(got[1]).astype(bool)
    plain_v = oracle.plain_group(wl["preds"], 0, vt["values"]).astype(bool)
    plain_e = oracle.plain_group(wl["preds"], 1, et["values"]).astype(bool)
    assert np.array_equal(bits_v, plain_v) and np.array_equal(bits_e, plain_e)
    got_m = oracle.match(1000, wl["edges"], 3, wl["query_edges"], [bits_v, None, None], [None, bits_e])
    want_m = oracle.match(1000, wl["edges"], 3, wl["query_edges"], [plain_v, None, None], [None, plain_e])
    assert got_m == want_m and len(got_m) > 0


@pytest.mark.parametrize("n_vertices", [4099])
def test_bulk_filter_ragged_full_parity(ctx, n_vertices):
    wl = W.bulk_vertex_filter(n_vertices=n_vertices, seed=3)
    load_tables(ctx, wl)
    toks = P.keygen(wl["preds"], 32, bytes(range(3, 19)))
    got = _filter(ctx, wl, toks, 5)
    want = oracle_group(oracle, wl, toks, 5, 0, np.arange(n_vertices), threads=16)
    assert np.array_equal(got[0], want)
    rec = oracle.reconstruct(got[0])
    assert np.array_equal(rec, oracle.plain_group(wl["preds"], 0, wl["tables"][0]["values"]))
    assert rec[wl["target"]] == 1


SCHEDULES = [(1024, 1), (768, 1), (512, 1), (256, 2), (512, 2), (128, 4), (256, 4), (512, 4)]


def test_every_schedule_gives_identical_shares(ctx):
    wl = W.bulk_vertex_filter(n_vertices=3333, seed=4)
    wl["preds"] = [wl["preds"][0], wl["preds"][5], wl["preds"][6]]   # EQ + 2 RANGE keeps it quick
    load_tables(ctx, wl)
    toks = P.keygen(wl["preds"], 32, bytes(16))
    ref = None
    prev = ctx.set_walk_parallel(0)   # the per-element kernel in every launch shape
    try:
        for t, e in SCHEDULES:
            ctx.set_schedule(t, e)
            got = _filter(ctx, wl, toks, 9)[0]
            if ref is None:
                ref = got
                want = oracle_group(oracle, wl, toks, 9, 0, np.arange(3333), threads=16)
                assert np.array_equal(ref, want)
            assert np.array_equal(got, ref), (t, e)
    finally:
        ctx.set_schedule(768, 1)
        ctx.set_walk_parallel(prev)


def test_unaligned_outputs_and_tiny_tables(ctx):
    g = W.rng(21)
    wl = {"tables": [W.table(W.uniform_attrs(g, 2, 1, 32), 32, g), W.table(W.uniform_attrs(g, 1, 7, 32), 32, g)]}
    wl["preds"] = [W.eq_pred(0, 1, 0, int(wl["tables"][0]["values"][1, 0])), W.range_pred(1, 0, 1, 0, 1 << 31),
                   W.eq_pred(1, 0, 1, int(wl["tables"][1]["values"][0, 6]))]
    load_tables(ctx, wl)
    toks = P.keygen(wl["preds"], 32, bytes(range(16)))
    prev = ctx.set_walk_parallel(0)
    try:
        # scalar, uint4 and uint2 stores of the per-element kernel, then the walk-parallel kernel
        for sched, wp in (((512, 1), 0), ((256, 4), 0), ((256, 2), 0), ((768, 1), ALWAYS)):
            ctx.set_schedule(*sched)
            ctx.set_walk_parallel(wp)
            for offset in (0, 1):
                outs = alloc_outs(wl, offset=offset)
                ctx.filter_and_combine(3, toks, outs)
                torch.cuda.synchronize()
                for grp, n in ((0, 1), (1, 7)):
                    got = np.stack([from_dev(t) for t in outs[grp]])
                    assert np.array_equal(got, oracle_group(oracle, wl, toks, 3, grp, np.arange(n))), sched
    finally:
        ctx.set_schedule(768, 1)
        ctx.set_walk_parallel(prev)


ALWAYS = (1 << 64) - 1


def test_walk_parallel_kernel_equals_oracle(ctx):
    """The walk-parallel kernel (one thread per key walk, 40-element tiles) gives the
    oracle's shares: the tiny path query (EQ + RANGE ANDs, two tables), a bulk filter of
    4,099 elements (102 full tiles and a ragged one; EQ and RANGE over n = 32), and a
    batch of queries; the default switch-over picks it for the tiny query and the
    per-element kernel for the large one, with the same shares either way."""
    wl = W.tiny_path(seed=1)
    load_tables(ctx, wl)
    toks = P.keygen(wl["preds"], wl["n_bits"], bytes(range(16)))
    want = [oracle_group(oracle, wl, toks, 11, 0, np.arange(1000)),
            oracle_group(oracle, wl, toks, 11, 1, np.arange(4000))]
    prev = ctx.set_walk_parallel(ALWAYS)
    try:
        ctx.set_walk_parallel(prev)
        outs = alloc_outs(wl)
        plan = ctx.plan_create([11], [toks], [outs])      # 5,000 elements: under the default switch-over
        assert ctx.plan_describe(plan)["kernel"] == "k_filter_wp"
        ctx.plan_destroy(plan)
        for wp in (ALWAYS, 0, prev):
            ctx.set_walk_parallel(wp)
            got = _filter(ctx, wl, toks, 11)
            assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1]), wp
        bulk = W.bulk_vertex_filter(n_vertices=4099, seed=13)
        load_tables(ctx, bulk)
        btoks = P.keygen(bulk["preds"], 32, bytes(range(5, 21)))
        ctx.set_walk_parallel(ALWAYS)
        got = _filter(ctx, bulk, btoks, 6)[0]
        assert np.array_equal(got, oracle_group(oracle, bulk, btoks, 6, 0, np.arange(4099), threads=16))
        ctx.set_walk_parallel(0)
        assert np.array_equal(_filter(ctx, bulk, btoks, 6)[0], got)
        graph = W.edge_graph(700, 3000, 4, 2, seed=71)
        load_tables(ctx, graph)
        qs = W.query_mix(graph, 4, seed=72)
        qtoks = [P.keygen(q["preds"], 32, bytes([i + 3]) * 16) for i, q in enumerate(qs)]
        res = {}
        for wp in (ALWAYS, 0):
            ctx.set_walk_parallel(wp)
            outs = [alloc_outs(graph, preds=q["preds"]) for q in qs]
            ctx.filter_batch(list(range(40, 44)), qtoks, outs)
            ctx.sync()
            res[wp] = [[np.stack([from_dev(t) for t in grp]) for grp in q] for q in outs]
        for qa, qb in zip(res[ALWAYS], res[0]):
            for a, b in zip(qa, qb):
                assert np.array_equal(a, b)
    finally:
        ctx.set_walk_parallel(prev)


def test_empty_table_is_a_no_op(ctx):
    g = W.rng(22)
    wl = {"tables": [W.table(np.zeros((1, 0), dtype=np.uint32), 32, g)]}
    wl["preds"] = [W.eq_pred(0, 0, 0, 5)]
    load_tables(ctx, wl)
    toks = P.keygen(wl["preds"], 32, bytes(16))
    outs = [[torch.empty(0, dtype=torch.int32, device="cuda") for _ in range(3)]]
    ctx.filter_and_combine(1, toks, outs)
    ctx.sync()


def test_batch_equals_each_query_alone(ctx):
    graph = W.edge_graph(5000, 20000, 4, 2, seed=31)
    load_tables(ctx, graph)
    qs = W.query_mix(graph, 6, seed=32)
    toks = [P.keygen(q["preds"], 32, bytes([i]) * 16) for i, q in enumerate(qs)]
    outs_b = [alloc_outs(graph, preds=q["preds"]) for q in qs]
    ctx.filter_batch(list(range(100, 106)), toks, outs_b)
    torch.cuda.synchronize()
    for i, q in enumerate(qs):
        outs_a = alloc_outs(graph, preds=q["preds"])
        ctx.filter_and_combine(100 + i, toks[i], outs_a)
        torch.cuda.synchronize()
        for ga, gb in zip(outs_a, outs_b[i]):
            for ta, tb in zip(ga, gb):
                assert torch.equal(ta, tb)
    # and one query against the oracle on a sample of its first group
    q = qs[0]
    grp_tab = [p["table"] for p in q["preds"] if p["group"] == 0][0]
    n = graph["tables"][grp_tab]["values"].shape[1]
    sample = np.unique(np.concatenate([[0, n - 1], W.rng(3).integers(0, n, 300)]))
    want = oracle_group(oracle, graph, toks[0], 100, 0, sample)
    got = np.stack([from_dev(t) for t in outs_b[0][0]])[:, sample]
    assert np.array_equal(got, want)


def test_bad_tokens_and_missing_tables(ctx):
    wl = W.tiny_path(seed=1)
    load_tables(ctx, wl)
    toks = list(P.keygen(wl["preds"], 16, bytes(16)))
    outs = alloc_outs(wl)
    bad = bytearray(toks[1])
    bad[5] = 3                                  # claims to be server 3's token
    with pytest.raises(P.OblivgmError) as e:
        ctx.filter_and_combine(1, [toks[0], bytes(bad), toks[2]], outs)
    assert e.value.status == P.EINVAL
    with pytest.raises(P.OblivgmError):         # n_groups disagrees with the token
        ctx.filter_and_combine(1, toks, outs[:1])
    other = P.keygen([W.eq_pred(9, 0, 0, 1)], 16, bytes(16))
    with pytest.raises(P.OblivgmError) as e:
        ctx.filter_and_combine(1, other, [outs[0]])
    assert e.value.status == P.ENOENT
    with pytest.raises(P.OblivgmError):         # 32-bit keys on a 16-bit table
        ctx.filter_and_combine(1, P.keygen([W.eq_pred(0, 0, 0, 1)], 32, bytes(16)), [outs[0]])


def test_full_size_bulk_filter_sampled(ctx):
    """1,048,576 vertices x 4 attributes, 8 predicates (the bulk-filter workload at full
    size), autotuned launch shape as the bench uses it: every element reconstructs to the
    plaintext AND, and sampled elements match the oracle share for share."""
    wl = W.bulk_vertex_filter(n_vertices=1 << 20, seed=2)
    load_tables(ctx, wl)
    ctx.autotune()
    toks = P.keygen(wl["preds"], 32, bytes(range(16)))
    got = _filter(ctx, wl, toks, 1)[0]
    rec = oracle.reconstruct(got)
    plain = oracle.plain_group(wl["preds"], 0, wl["tables"][0]["values"])
    assert np.array_equal(rec, plain) and plain.sum() >= 1
    n = 1 << 20
    sample = np.unique(np.concatenate([[0, 1, 1023, 1024, n - 1, wl["target"]],
                                       W.rng(7).integers(0, n, 250)]))
    want = oracle_group(oracle, wl, toks, 1, 0, sample, threads=16)
    assert np.array_equal(got[:, sample], want)


def test_full_size_wide_ranges_many_positives(ctx):
    """A full-size group whose predicates are wide ranges only, so that most elements match:
    2^20 vertices, three 32-bit ranges ANDed (about 62 % of the elements reconstruct to 1).
    Every element against the plaintext, and 1,024 random elements plus the first, the last
    and the elements on both sides of every tile boundary the launch uses near the start and
    the end, share for share against the oracle."""
    n = 1 << 20
    g = W.rng(71)
    vals = W.uniform_attrs(g, 3, n, 32)
    wl = {"tables": [W.table(vals, 32, g)], "preds": [
        W.range_pred(0, 0, 0, 0x10000000, 0xF0000000),
        W.range_pred(0, 1, 0, 0x20000000, 0xFFFFFFFF),     # the domain's last value included
        W.range_pred(0, 2, 0, 0, 0xD0000000)]}             # and its first
    load_tables(ctx, wl)
    ctx.autotune()
    toks = P.keygen(wl["preds"], 32, bytes(range(3, 19)))
    got = _filter(ctx, wl, toks, 5)[0]
    rec = oracle.reconstruct(got)
    plain = oracle.plain_group(wl["preds"], 0, vals)
    assert np.array_equal(rec, plain)
    assert 0.55 < plain.mean() < 0.70
    outs = alloc_outs(wl)
    plan = ctx.plan_create([5], [toks], [outs])
    tile = ctx.plan_describe(plan)["tile"]
    ctx.plan_destroy(plan)
    edges = [t * tile + d for t in (1, 2, 3, n // tile - 1, n // tile) for d in (-1, 0, 1)]
    sample = np.unique(np.concatenate([[0, n - 1], [e for e in edges if 0 <= e < n],
                                       W.rng(72).integers(0, n, 1024)]))
    assert len(sample) >= 1024
    want = oracle_group(oracle, wl, toks, 5, 0, sample, threads=16)
    assert np.array_equal(got[:, sample], want)


def test_plain_path_equals_fused_and_oracle(ctx):
    """The plain per-query path (one launch per key half, global-memory AES tables) gives the
    same shares as the fused kernel and the oracle."""
    wl = W.tiny_path(seed=1)
    load_tables(ctx, wl)
    toks = P.keygen(wl["preds"], 16, bytes(range(16)))
    fused = alloc_outs(wl)
    plain = alloc_outs(wl)
    ctx.filter_and_combine(21, toks, fused)
    ctx.filter_plain(21, toks, plain)
    torch.cuda.synchronize()
    for ga, gb in zip(fused, plain):
        for ta, tb in zip(ga, gb):
            assert torch.equal(ta, tb)
    bulk = W.bulk_vertex_filter(n_vertices=2053, seed=6)
    load_tables(ctx, bulk)
    toks = P.keygen(bulk["preds"], 32, bytes(range(5, 21)))
    plain = alloc_outs(bulk)
    ctx.filter_plain(22, toks, plain)
    torch.cuda.synchronize()
    got = np.stack([from_dev(t) for t in plain[0]])
    assert np.array_equal(got, oracle_group(oracle, bulk, toks, 22, 0, np.arange(2053), threads=16))


@pytest.mark.parametrize("walk_parallel", [False, True])
def test_prepared_plan_and_cuda_graph_replay(ctx, walk_parallel):
    """A prepared batch launched directly, then captured into a CUDA graph and replayed twice,
    gives the shares of filter_batch for the same queries (per-element and walk-parallel plans)."""
    prev = ctx.set_walk_parallel((1 << 64) - 1 if walk_parallel else 0)
    try:
        _plan_and_graph(ctx, walk_parallel)
    finally:
        ctx.set_walk_parallel(prev)


def _plan_and_graph(ctx, walk_parallel):
    graph = W.edge_graph(6000, 20000, 4, 2, seed=61)
    load_tables(ctx, graph)
    qs = W.query_mix(graph, 5, seed=62)
    qids = list(range(200, 205))
    toks = [P.keygen(q["preds"], 32, bytes([i + 7]) * 16) for i, q in enumerate(qs)]
    want = [alloc_outs(graph, preds=q["preds"]) for q in qs]
    ctx.filter_batch(qids, toks, want)
    torch.cuda.synchronize()
    got = [alloc_outs(graph, preds=q["preds"]) for q in qs]

    def same():
        torch.cuda.synchronize()
        return all(torch.equal(a, b) for qa, qb in zip(got, want) for ga, gb in zip(qa, qb) for a, b in zip(ga, gb))

    def clear():
        for q in got:
            for grp in q:
                for t in grp:
                    t.fill_(-1)

    plan = ctx.plan_create(qids, toks, got)
    try:
        d = ctx.plan_describe(plan)
        assert d["kernel"] == ("k_filter_wp" if walk_parallel else "k_filter")
        assert d["tile"] <= (40 if walk_parallel else d["threads"]) and 0 < d["grid"] <= d["items"]
        s = torch.cuda.Stream()
        ctx.plan_launch(plan, s)
        s.synchronize()
        assert same()
        clear()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            ctx.plan_launch(plan, torch.cuda.current_stream())
        for _ in range(2):
            clear()
            g.replay()
            assert same()
        ctx.sync()
    finally:
        ctx.plan_destroy(plan)


def test_expired_device_wait_is_reported_and_context_survives(ctx):
    """A bounded device wait that runs out (the test hook asks the key-staging barrier for
    bytes that never come) is reported as EFAULT_DEVICE by sync, and the next call is correct."""
    wl = W.bulk_vertex_filter(n_vertices=5000, seed=8)
    load_tables(ctx, wl)
    toks = P.keygen(wl["preds"][:2], 32, bytes(16))
    outs = alloc_outs(wl, preds=wl["preds"][:2])
    ctx.test_expire_next_wait(20000)            # 20 ms
    ctx.filter_and_combine(3, toks, outs)
    torch.cuda.synchronize()
    with pytest.raises(P.OblivgmError) as e:
        ctx.sync()
    assert e.value.status == P.EFAULT_DEVICE
    ctx.sync()                                   # the flag was cleared
    ctx.filter_and_combine(3, toks, outs)
    ctx.sync()
    got = np.stack([from_dev(t) for t in outs[0]])
    wl2 = dict(wl)
    wl2["preds"] = wl["preds"][:2]
    sample = np.array([0, 1, 4999, wl["target"]])
    assert np.array_equal(got[:, sample], oracle_group(oracle, wl2, toks, 3, 0, sample))


def test_fetch_unique_matches_oracle(ctx):
    """secFetch case I after a filter: the matched element's index and attributes, share for
    share equal to the oracle's (which runs on its own filter output)."""
    g = W.rng(71)
    n_el, bits = 70001, 32
    vals = W.uniform_attrs(g, 4, n_el, bits)
    wl = {"tables": [W.table(vals, bits, g)]}
    load_tables(ctx, wl)
    target = 54321
    preds = [W.eq_pred(0, 2, 0, int(vals[2, target])), W.range_pred(0, 1, 0, 0, 0xFFFFFFFF)]
    toks = P.keygen(preds, bits, bytes(range(7, 23)))
    outs = alloc_outs(wl, preds=preds)
    ctx.filter_and_combine(31, toks, outs)
    res = torch.empty(3 * 4, dtype=torch.int32, device="cuda")
    ctx.fetch_unique(31, 0, 0, outs[0], [0, 1, 3], res)
    ctx.sync()
    got = from_dev(res).reshape(3, 4)
    x_or = oracle_group(oracle, wl, toks, 31, 0, np.arange(n_el), threads=16)
    want = oracle.fetch_unique(x_or, [(wl["tables"][0]["shares"], bits)], 0, [0, 1, 3], 31, 0, PRF)
    assert np.array_equal(got, want)
    rec = oracle.reconstruct(got)
    assert rec[0] == target and list(rec[1:]) == [vals[a, target] for a in (0, 1, 3)]


@pytest.mark.parametrize("n_el,attrs,offset", [(1, [0], 0), (1003, [], 0), (1003, list(range(11)), 0),
                                             (1003, list(range(11)), 1), (200_001, [3, 9, 1], 0),
                                             (200_001, [3, 9, 1], 1)])
def test_fetch_unique_column_groups_and_sizes(ctx, n_el, attrs, offset):
    """secFetch case I on synthetic result shares (any values: the sums are linear in x):
    no attribute, more attributes than one pass takes (8 columns), one candidate, many CTAs,
    16-byte-aligned result shares (4-candidate loads) and shares one word off (scalar loads)."""
    g = W.rng(72 + n_el)
    bits = 32
    vals = W.uniform_attrs(g, 12, n_el, bits)
    wl = {"tables": [W.table(vals, bits, g)]}
    load_tables(ctx, wl)
    xs = [g.integers(0, 1 << 32, n_el, dtype=np.uint64).astype(np.uint32) for _ in range(3)]
    res = torch.empty(3 * (1 + len(attrs)), dtype=torch.int32, device="cuda")
    dx = [to_dev(np.concatenate([np.zeros(offset, dtype=np.uint32), x]))[offset:] for x in xs]
    ctx.fetch_unique(8, 5, 0, dx, attrs, res)
    ctx.sync()
    got = from_dev(res).reshape(3, 1 + len(attrs))
    want = oracle.fetch_unique(xs, [(wl["tables"][0]["shares"], bits)], 0, attrs, 8, 5, PRF)
    assert np.array_equal(got, want)


def test_fetch_unique_calls_back_to_back(ctx):
    """secFetch case I leaves the context's accumulators at zero for the next call: three calls
    on one stream with different attribute lists and outputs, one synchronisation at the end,
    each equal to the oracle."""
    g = W.rng(74)
    n_el, bits = 30011, 32
    vals = W.uniform_attrs(g, 5, n_el, bits)
    wl = {"tables": [W.table(vals, bits, g)]}
    load_tables(ctx, wl)
    xs = [g.integers(0, 1 << 32, n_el, dtype=np.uint64).astype(np.uint32) for _ in range(3)]
    dx = [to_dev(x) for x in xs]
    calls = [[0, 1, 2, 3, 4], [2], []]
    res = [torch.empty(3 * (1 + len(a)), dtype=torch.int32, device="cuda") for a in calls]
    for q, (attrs, r) in enumerate(zip(calls, res)):
        ctx.fetch_unique(20 + q, q, 0, dx, attrs, r)
    ctx.sync()
    for q, (attrs, r) in enumerate(zip(calls, res)):
        want = oracle.fetch_unique(xs, [(wl["tables"][0]["shares"], bits)], 0, attrs, 20 + q, q, PRF)
        assert np.array_equal(from_dev(r).reshape(3, 1 + len(attrs)), want), q
