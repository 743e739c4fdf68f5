"""The largest queries the boundary accepts, on the GPU, against the oracle.

* 64 predicates (the maximum) folded into one group: the fold runs 63 times
  (re-share steps up to 64 + 63), with AND, XOR and OR mixed; masked mode
  through the per-element kernel, the walk-parallel kernel and the plain path,
  the fresh-key mode and the one-hot mode;
* 64 groups (the maximum) of one predicate each over two tables, 192 output
  arrays, in the masked and in the one-hot mode;
* one predicate more than the maximum, or one group more, is rejected.
"""
import numpy as np
import pytest

import oracle
import workload as W
from tests._helpers import PRF, from_dev, to_dev

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2209_03526_gb300")

SEED = bytes(range(40, 56))
AND, XOR, OR = P.COMBINE_AND, P.COMBINE_XOR, P.COMBINE_OR
ALWAYS = (1 << 64) - 1


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = P.Context(0, prf_keys=PRF)
    yield c
    c.close()


def _outs(sizes):
    return [[torch.full((n,), -1, dtype=torch.int32, device="cuda") for _ in range(3)] for n in sizes]


def _host(outs):
    return [np.stack([from_dev(t) for t in grp]) for grp in outs]


def _preds64(n, vals):
    """64 predicates in group 0: equalities on values present in the table joined by OR,
    every eighth a range joined by XOR, every sixteenth an AND with a wide range"""
    top = (1 << n) - 1
    preds = []
    for p in range(64):
        op = AND if p == 0 else (AND if p % 16 == 0 else XOR if p % 8 == 0 else OR)
        if p % 8 == 0:
            lo = (p * 5) % (top // 2)
            pr = W.range_pred(0, p % 2, 0, lo, lo + top // 4, combine=op)
        else:
            pr = W.eq_pred(0, p % 2, 0, int(vals[p % 2, (37 * p) % vals.shape[1]]), combine=op)
        if op == AND and p > 0:
            pr = W.range_pred(0, p % 2, 0, 1, top - 1, combine=AND)
        preds.append(pr)
    return preds


@pytest.mark.parametrize("path", ["per_element", "walk_parallel", "plain", "fresh", "onehot"])
def test_64_predicates_in_one_group(ctx, path):
    n, n_elems = 8, 1030
    g = W.rng(61)
    vals = W.uniform_attrs(g, 2, n_elems, n)
    preds = _preds64(n, vals)
    plain = oracle.plain_group(preds, 0, vals)
    assert 0 < int(plain.sum()) < n_elems
    if path == "onehot":
        tab = W.onehot_table(vals, n, g)
        ctx.load_onehot(0, [to_dev(s) for s in tab["shares"]], n)
        toks = P.keygen_onehot(preds, n, SEED)
        words = (n_elems + 31) // 32
        outs = [[torch.empty(words, dtype=torch.int32, device="cuda") for _ in range(3)]]
        ctx.filter_onehot(3, toks, outs)
        ctx.sync()
        w = np.stack([from_dev(t) for t in outs[0]]).astype(np.uint32)
        got = ((w[:, :, None] >> np.arange(32, dtype=np.uint32)) & 1).reshape(3, -1)[:, :n_elems]
        want = oracle.filter_onehot(toks, 3, PRF, [(tab["shares"], n)], 0, np.arange(n_elems))
        assert np.array_equal(got, want)
        assert np.array_equal(oracle.reconstruct_bits(got), plain)
        return
    tab = W.table(vals, n, g)
    ctx.load_shares(0, [to_dev(s) for s in tab["shares"]], n)
    outs = _outs([n_elems])
    if path == "fresh":
        L = P.fresh_token_size(preds, n, [n_elems])
        toks = [torch.zeros(L, dtype=torch.uint8, device="cuda") for _ in range(3)]
        ctx.keygen_fresh(preds, n, [n_elems], SEED, toks)
        ctx.filter_fresh(3, toks, outs)
        ctx.sync()
        got = _host(outs)[0]
        sample = np.array([0, 1, 2, 511, 512, 1027, 1028, 1029])
        want = oracle.fresh_direct(preds, n, SEED, 3, PRF, [(tab["shares"], n)], 0, sample, threads=8)
        assert np.array_equal(got[:, sample], want)
        assert np.array_equal(oracle.reconstruct(got), plain)
        return
    toks = P.keygen(preds, n, SEED)
    prev = ctx.set_walk_parallel(ALWAYS if path == "walk_parallel" else 0)
    try:
        if path == "plain":
            ctx.filter_plain(3, toks, outs)
        else:
            ctx.filter_and_combine(3, toks, outs)
        ctx.sync()
    finally:
        ctx.set_walk_parallel(prev)
    got = _host(outs)[0]
    want = oracle.filter_group(toks, 3, PRF, [(tab["shares"], n)], 0, np.arange(n_elems), threads=8)
    assert np.array_equal(got, want)
    assert np.array_equal(oracle.reconstruct(got), plain)


def test_64_groups(ctx):
    n = 10
    g = W.rng(62)
    sizes = (700, 333)
    vals = [W.uniform_attrs(g, 2, sizes[0], n), W.uniform_attrs(g, 1, sizes[1], n)]
    tabs = [W.table(v, n, g) for v in vals]
    for tid, t in enumerate(tabs):
        ctx.load_shares(tid, [to_dev(s) for s in t["shares"]], n)
    preds = []
    for grp in range(64):
        t = grp % 2
        v = vals[t]
        if grp % 3 == 0:
            preds.append(W.range_pred(t, grp % v.shape[0], grp, grp, grp + 300))
        else:
            preds.append(W.eq_pred(t, grp % v.shape[0], grp, int(v[grp % v.shape[0], grp])))
    toks = P.keygen(preds, n, SEED)
    outs = _outs([sizes[grp % 2] for grp in range(64)])
    ctx.filter_and_combine(4, toks, outs)
    ctx.sync()
    got = _host(outs)
    shares = [(t["shares"], n) for t in tabs]
    for grp in range(64):
        want = oracle.filter_group(toks, 4, PRF, shares, grp, np.arange(sizes[grp % 2]))
        assert np.array_equal(got[grp], want), grp
        assert np.array_equal(oracle.reconstruct(got[grp]), oracle.plain_group(preds, grp, vals[grp % 2])), grp
    with pytest.raises(P.OblivgmError) as e:
        P.keygen(preds + [W.eq_pred(0, 0, 64, 1)], n, SEED)      # 65 predicates
    assert e.value.status == P.EINVAL
    with pytest.raises(P.OblivgmError) as e:
        ctx.filter_and_combine(4, toks, outs + _outs([5]))        # 65 groups
    assert e.value.status == P.EINVAL


def test_64_groups_onehot(ctx):
    """64 one-hot groups over two tables of different sizes (22 and 11 packed words), at
    n = 12 so every column goes through the staged dot pass, several passes per column;
    the single fold launch maps its items back to 64 groups of two word counts."""
    n = 12
    g = W.rng(63)
    sizes = (700, 333)
    vals = [W.uniform_attrs(g, 2, sizes[0], n), W.uniform_attrs(g, 1, sizes[1], n)]
    tabs = [W.onehot_table(v, n, g) for v in vals]
    for tid, t in enumerate(tabs):
        ctx.load_onehot(tid, [to_dev(s) for s in t["shares"]], n)
    preds = []
    for grp in range(64):
        t = grp % 2
        v = vals[t]
        if grp % 3 == 0:
            preds.append(W.range_pred(t, grp % v.shape[0], grp, grp, grp + 900))
        else:
            preds.append(W.eq_pred(t, grp % v.shape[0], grp, int(v[grp % v.shape[0], grp])))
    toks = P.keygen_onehot(preds, n, SEED)
    outs = _outs([(sizes[grp % 2] + 31) // 32 for grp in range(64)])
    ctx.filter_onehot(5, toks, outs)
    ctx.sync()
    shares = [(t["shares"], n) for t in tabs]
    for grp in range(64):
        m = sizes[grp % 2]
        words = np.stack([from_dev(x) for x in outs[grp]]).view(np.uint32)
        bits = ((words[:, :, None] >> np.arange(32, dtype=np.uint32)) & 1).reshape(3, -1)[:, :m]
        assert np.array_equal(oracle.reconstruct_bits(bits), oracle.plain_group(preds, grp, vals[grp % 2])), grp
        assert words[0, -1] >> (m % 32) == 0, grp
        # share for share on groups at both ends and in the middle of the fold's item space
        # (the oracle's one-hot filter takes about two seconds a group here)
        if grp in (0, 1, 2, 31, 62, 63):
            want = oracle.filter_onehot(toks, 5, PRF, shares, grp, np.arange(m))
            assert np.array_equal(bits, want), grp
