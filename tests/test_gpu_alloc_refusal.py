"""Host-side fault injection: a refused device allocation.

oblivgm_test_fail_next_alloc makes the context's next workspace allocation fail
as if the device were out of memory.  Every entry point that allocates must
return ENOMEM without launching anything, and the next call must succeed with
the same shares as a call that was never refused.  Nothing faults on the GPU.
"""
import numpy as np
import pytest

import oracle
import workload as W
from tests._helpers import PRF, alloc_outs, from_dev, load_tables, to_dev

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


def _refused_then_ok(ctx, call):
    ctx.test_fail_next_alloc()
    with pytest.raises(P.OblivgmError) as e:
        call()
    assert e.value.status == P.ENOMEM
    ctx.sync()
    return call()


def test_filter_paths_recover_after_refused_allocation(ctx):
    wl = W.tiny_path(seed=4)
    load_tables(ctx, wl)
    toks = P.keygen(wl["preds"], wl["n_bits"], bytes(range(16)))
    ref = alloc_outs(wl)
    ctx.filter_and_combine(5, toks, ref)
    ctx.sync()
    want = [np.stack([from_dev(t) for t in g]) for g in ref]
    for fn in (ctx.filter_and_combine, ctx.filter_plain):
        outs = alloc_outs(wl)
        _refused_then_ok(ctx, lambda: fn(5, toks, outs))
        ctx.sync()
        for g, grp in enumerate(outs):
            assert np.array_equal(np.stack([from_dev(t) for t in grp]), want[g])


def test_raw_eval_recovers_after_refused_allocation(ctx):
    g = np.random.default_rng(2)
    k0, k1 = oracle.dpf_gen(16, 77, 5, bytes(range(16)), bytes(range(16, 32)))
    pts = to_dev(g.integers(0, 1 << 16, 300, dtype=np.uint64).astype(np.uint32))
    out = torch.empty(2 * 300, dtype=torch.int32, device="cuda")
    _refused_then_ok(ctx, lambda: ctx.eval_dpf_batch(k0 + k1, 2, pts, out, all_pairs=True))
    ctx.sync()
    got = from_dev(out).reshape(2, 300)
    assert np.array_equal(got[0], oracle.eval_many(k0, from_dev(pts), oracle.KIND_DPF))


def test_onehot_shuffle_and_fetch_recover_after_refused_allocation(ctx):
    g = W.rng(3)
    n, N = 6, 200
    vals = W.uniform_attrs(g, 1, N, n)
    hot = W.onehot_table(vals, n, g)
    ctx.load_onehot(0, [to_dev(s) for s in hot["shares"]], n)
    preds = [W.range_pred(0, 0, 0, 5, 40)]
    toks = P.keygen_onehot(preds, n, bytes(range(16)))
    outs = [[torch.empty((N + 31) // 32, dtype=torch.int32, device="cuda") for _ in range(3)]]
    _refused_then_ok(ctx, lambda: ctx.filter_onehot(1, toks, outs))
    ctx.sync()
    shares = [g.integers(0, 1 << 32, (50, 3), dtype=np.uint64).astype(np.uint32) for _ in range(3)]
    ins = [torch.from_numpy(s.view(np.int32)).cuda() for s in shares]
    sh_out = [torch.empty_like(ins[0]) for _ in range(3)]
    seeds = bytes(range(48))
    _refused_then_ok(ctx, lambda: ctx.shuffle(ins, seeds, sh_out))
    ctx.sync()
    want = oracle.shuffle(shares, seeds, oracle.SHUF_ADD)
    for j in range(3):
        assert np.array_equal(sh_out[j].cpu().numpy().view(np.uint32), want[j])
    tab = W.table(W.uniform_attrs(g, 2, N, 16), 16, g)
    ctx.load_shares(0, [to_dev(s) for s in tab["shares"]], 16)
    flags = np.zeros(N, dtype=np.uint32)
    flags[[3, 50]] = 1
    s1 = g.integers(0, 1 << 32, N, dtype=np.uint64).astype(np.uint32)
    s2 = g.integers(0, 1 << 32, N, dtype=np.uint64).astype(np.uint32)
    xs = [s1, s2, flags - s1 - s2]
    fouts = [torch.zeros((N, 3), dtype=torch.int32, device="cuda") for _ in range(3)]
    m = _refused_then_ok(ctx, lambda: ctx.fetch_multi(0, [to_dev(x) for x in xs], [0, 1], seeds, fouts))
    assert m == 2
