"""GPU parity of the one-hot mode (the paper's secEval as written) against the oracle.

Every compared share bit is equal; the reconstruction equals the plaintext
predicates.  The keys stop their trees 7 levels early (a leaf seed gives 2^min(n,7)
bits), so the domains cover the leaf-only keys (n = 1, a 2-bit leaf; n = 5, one
word; n = 6, two words; n = 7, one 128-bit leaf) and the first levels (n = 8, 9);
as to the dot pass they cover one partial word (n = 3), a few words (n = 6),
half a warp of words (n = 9), whole warps of words (n = 10), the staged path
with one warp per 32 elements (n = 12), with two warps and more words than the
persistent grid has CTAs (n = 13, 70,001 elements), and the bench's domain
(n = 16) with a ragged last word and CTAs that each take two words; and a table
loaded from host memory."""
import numpy as np
import pytest

import oracle
import workload as W
from tests._helpers import PRF, from_dev, to_dev

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


def _load(ctx, tid, tab):
    ctx.load_onehot(tid, [to_dev(s) for s in tab["shares"]], tab["bits"])


def _unpack(words, n):
    w = np.asarray(words, dtype=np.uint32)
    bits = (w[:, None] >> np.arange(32, dtype=np.uint32)) & 1
    return bits.reshape(-1)[:n]


def _run(ctx, toks, n_groups, sizes, qid):
    outs = [[torch.full(((sizes[g] + 31) // 32,), -1, dtype=torch.int32, device="cuda") for _ in range(3)]
            for g in range(n_groups)]
    ctx.filter_onehot(qid, toks, outs)
    ctx.sync()
    return [np.stack([_unpack(from_dev(t), sizes[g]) for t in outs[g]]) for g in range(n_groups)], outs


@pytest.mark.parametrize("n,n_elems", [(1, 40), (3, 77), (5, 64), (6, 1000), (7, 500), (8, 257), (9, 1025),
                                        (10, 333), (12, 129)])
def test_onehot_parity(ctx, n, n_elems):
    g = W.rng(100 + n)
    top = (1 << n) - 1
    vals = W.uniform_attrs(g, 2, n_elems, n)
    tab = W.onehot_table(vals, n, g)
    _load(ctx, 0, tab)
    preds = [W.eq_pred(0, 0, 0, int(vals[0, 3])),
             W.range_pred(0, 1, 1, top // 4, top), W.eq_pred(0, 0, 1, int(vals[0, 5])),
             W.range_pred(0, 0, 2, 0, top // 2)]
    toks = P.keygen_onehot(preds, n, bytes([n]) * 16)
    got, outs = _run(ctx, toks, 3, [n_elems] * 3, 17)
    for grp in range(3):
        want = oracle.filter_onehot(toks, 17, PRF, [(tab["shares"], n)], grp, np.arange(n_elems))
        assert np.array_equal(got[grp], want), grp
        assert np.array_equal(oracle.reconstruct_bits(got[grp]), oracle.plain_group(preds, grp, vals))
        # bits past the last element are zero
        last = from_dev(outs[grp][0])[-1]
        if n_elems % 32:
            assert last >> (n_elems % 32) == 0


@pytest.mark.parametrize("n,n_elems", [(13, 70_001), (14, 20_011), (16, 5_003)])
def test_onehot_parity_persistent_grid(ctx, n, n_elems):
    """More 32-element words than the dot pass's persistent grid has CTAs, so CTAs carry
    their copy pipeline from one word into the next.  Every element of every group is
    checked against the plaintext; group 0's shares against the oracle on a sample that
    covers the first words, words across the table and the ragged last word (the
    oracle's EvalAll over 2^16 positions is too slow for all three groups)."""
    g = W.rng(100 + n)
    top = (1 << n) - 1
    vals = W.uniform_attrs(g, 2, n_elems, n)
    tab = W.onehot_table(vals, n, g)
    _load(ctx, 0, tab)
    preds = [W.eq_pred(0, 0, 0, int(vals[0, 3])),
             W.range_pred(0, 1, 1, top // 4, top), W.eq_pred(0, 0, 1, int(vals[0, 5])),
             W.range_pred(0, 0, 2, 0, top // 2)]
    toks = P.keygen_onehot(preds, n, bytes([n]) * 16)
    got, outs = _run(ctx, toks, 3, [n_elems] * 3, 17)
    for grp in range(3):
        assert np.array_equal(oracle.reconstruct_bits(got[grp]), oracle.plain_group(preds, grp, vals)), grp
        last = from_dev(outs[grp][0])[-1]
        assert last >> (n_elems % 32) == 0
    idx = np.unique(np.concatenate([np.arange(0, 64), np.arange(0, n_elems, n_elems // 24),
                                    np.arange(n_elems - 40, n_elems)]))
    want = oracle.filter_onehot(toks, 17, PRF, [(tab["shares"], n)], 0, idx)
    assert np.array_equal(got[0][:, idx], want)


def test_onehot_fig1_example(ctx):
    from tests.test_oracle_matcher import PAPER_RESULTS, Q_EDGES, Q_PREDS, _fig1_graph
    attrs, edges = _fig1_graph()
    g = W.rng(12)
    tab = W.onehot_table(attrs, 6, g)
    _load(ctx, 3, tab)
    preds = [dict(p, table=3) for p in Q_PREDS]
    toks = P.keygen_onehot(preds, 6, bytes(range(16)))
    got, _ = _run(ctx, toks, 5, [9] * 5, 4)
    ok = [oracle.reconstruct_bits(x).astype(bool) for x in got]
    assert oracle.match(9, edges, 5, Q_EDGES, ok, [None] * 4) == PAPER_RESULTS


def test_modes_reject_each_others_tokens(ctx):
    g = W.rng(7)
    vals = W.uniform_attrs(g, 1, 40, 8)
    _load(ctx, 5, W.onehot_table(vals, 8, g))
    ctx.load_shares(5, [to_dev(s) for s in W.table(vals, 8, g)["shares"]], 8)
    t_onehot = P.keygen_onehot([W.eq_pred(5, 0, 0, 1)], 8, bytes(16))
    t_masked = P.keygen([W.eq_pred(5, 0, 0, 1)], 8, bytes(16))
    outs_bits = [[torch.zeros(2, dtype=torch.int32, device="cuda") for _ in range(3)]]
    outs_words = [[torch.zeros(40, dtype=torch.int32, device="cuda") for _ in range(3)]]
    with pytest.raises(P.OblivgmError) as e:
        ctx.filter_onehot(1, t_masked, outs_bits)
    assert e.value.status == P.EINVAL
    with pytest.raises(P.OblivgmError) as e:
        ctx.filter_and_combine(1, t_onehot, outs_words)
    assert e.value.status == P.EINVAL


def test_onehot_many_predicates_on_one_column(ctx):
    """Seven predicates on one attribute column (two streaming passes of up to four),
    in three AND-groups, on a ragged table."""
    n, n_elems = 8, 203
    g = W.rng(31)
    vals = W.uniform_attrs(g, 1, n_elems, n)
    tab = W.onehot_table(vals, n, g)
    _load(ctx, 0, tab)
    v = [int(vals[0, i]) for i in (1, 2, 3)]
    preds = [W.range_pred(0, 0, 0, 10, 250), W.eq_pred(0, 0, 1, v[0]), W.range_pred(0, 0, 0, 0, 200),
             W.range_pred(0, 0, 2, 30, 255), W.eq_pred(0, 0, 0, v[1]), W.range_pred(0, 0, 2, 0, 254),
             W.range_pred(0, 0, 1, 5, 255)]
    preds.sort(key=lambda p: p["group"])
    toks = P.keygen_onehot(preds, n, bytes(range(3, 19)))
    got, _ = _run(ctx, toks, 3, [n_elems] * 3, 29)
    tabs = [(tab["shares"], n)]
    for grp in range(3):
        want = oracle.filter_onehot(toks, 29, PRF, tabs, grp, np.arange(n_elems))
        assert np.array_equal(got[grp], want), grp
        assert np.array_equal(oracle.reconstruct_bits(got[grp]), oracle.plain_group(preds, grp, vals))


def test_onehot_host_loaded_table_equals_device_loaded(ctx):
    """A table loaded from host memory gives the same shares as the same table loaded
    from device memory, with predicates on both attributes."""
    n, n_elems = 12, 3001
    g = W.rng(77)
    top = (1 << n) - 1
    vals = W.uniform_attrs(g, 2, n_elems, n)
    tab = W.onehot_table(vals, n, g)
    preds = [W.eq_pred(0, 1, 0, int(vals[1, 7])), W.range_pred(0, 0, 1, top // 3, top // 2)]
    toks = P.keygen_onehot(preds, n, bytes([9]) * 16)
    _load(ctx, 0, tab)
    want, _ = _run(ctx, toks, 2, [n_elems] * 2, 23)
    host = [torch.from_numpy(np.ascontiguousarray(s_, dtype=np.uint32).view(np.int32)) for s_ in tab["shares"]]
    ctx.load_onehot(0, host, n)
    got, _ = _run(ctx, toks, 2, [n_elems] * 2, 23)
    for grp in range(2):
        assert np.array_equal(got[grp], want[grp]), grp
        assert np.array_equal(oracle.reconstruct_bits(got[grp]), oracle.plain_group(preds, grp, vals)), grp
