"""GPU parity of the fresh-key mode (Sec. V-C, one mask and one key triple per value).

* the GPU client's tokens equal the oracle's, byte for byte (ragged N, both
  predicate kinds, two tables);
* the GPU servers' filter on the ORACLE's tokens equals the oracle's filter on
  every element, bit-exact;
* end to end (GPU keygen + GPU filter) at 200,003 elements and n = 32: sampled
  elements equal the oracle's token-free computation from the same seed, and
  every element reconstructs to the plaintext AND;
* degenerate sizes and rejected inputs.
"""
import numpy as np
import pytest

import oracle
import workload as W
from tests._helpers import PRF, from_dev, to_dev

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2209_03526_gb300")

SEED = bytes(range(7, 23))


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = P.Context(0, prf_keys=PRF)
    yield c
    c.close()


def _load(ctx, tables):
    for tid, t in enumerate(tables):
        ctx.load_shares(tid, [to_dev(s) for s in t["shares"]], t["bits"])


def _gpu_tokens(ctx, preds, bits, elems, seed=SEED):
    L = P.fresh_token_size(preds, bits, elems)
    assert L == oracle.fresh_token_len(preds, bits, elems)
    toks = [torch.zeros(L, dtype=torch.uint8, device="cuda") for _ in range(3)]
    ctx.keygen_fresh(preds, bits, elems, seed, toks)
    return toks


def _outs(sizes):
    return [[torch.full((n,), -1, dtype=torch.int32, device="cuda") for _ in range(3)] for n in sizes]


def _two_tables(bits, n0, n1, seed):
    g = W.rng(seed)
    v0 = W.uniform_attrs(g, 2, n0, bits)
    v1 = W.uniform_attrs(g, 3, n1, bits)
    v1[1, ::5] = 9
    return [W.table(v0, bits, g), W.table(v1, bits, g)]


def _preds(tables, bits):
    top = (1 << bits) - 1
    v0 = tables[0]["values"]
    return [W.eq_pred(0, 1, 0, int(v0[1, 3])), W.range_pred(0, 0, 0, top // 4, top - 3),
            W.range_pred(1, 2, 1, 5, top // 2), W.eq_pred(1, 1, 1, 9), W.range_pred(1, 0, 1, 0, top)]


def test_gpu_tokens_equal_oracle_tokens(ctx):
    bits = 12
    tables = _two_tables(bits, 1003, 517, seed=21)
    preds = _preds(tables, bits)
    elems = [1003, 517]
    toks = _gpu_tokens(ctx, preds, bits, elems)
    torch.cuda.synchronize()
    want = oracle.keygen_fresh(preds, bits, elems, SEED)
    for i in range(3):
        got = toks[i].cpu().numpy().tobytes()
        assert got == want[i], i


def test_gpu_filter_on_oracle_tokens(ctx):
    bits = 12
    tables = _two_tables(bits, 1003, 517, seed=22)
    _load(ctx, tables)
    preds = _preds(tables, bits)
    elems = [1003, 517]
    otoks = oracle.keygen_fresh(preds, bits, elems, SEED)
    dtoks = [torch.from_numpy(np.frombuffer(t, dtype=np.uint8).copy()).cuda() for t in otoks]
    outs = _outs([1003, 517])
    ctx.filter_fresh(31, dtoks, outs)
    ctx.sync()
    tabs = [(t["shares"], bits) for t in tables]
    for grp, n in ((0, 1003), (1, 517)):
        want = oracle.filter_fresh(otoks, 31, PRF, tabs, grp, np.arange(n), threads=4)
        got = np.stack([from_dev(x) for x in outs[grp]])
        assert np.array_equal(got, want), grp
        plain = oracle.plain_group(preds, grp, tables[grp]["values"])
        assert np.array_equal(oracle.reconstruct(got), plain)


def test_gpu_fresh_end_to_end_full_size_sampled(ctx):
    bits, n = 32, 200_003
    g = W.rng(23)
    vals = W.uniform_attrs(g, 2, n, bits)
    vals[0, ::97] = 123456789
    tab = W.table(vals, bits, g)
    _load(ctx, [tab])
    preds = [W.eq_pred(0, 0, 0, 123456789), W.range_pred(0, 1, 0, 1 << 30, 3 << 30),
             W.range_pred(0, 1, 1, 0, 1 << 31), W.eq_pred(0, 0, 1, int(vals[0, 5]))]
    toks = _gpu_tokens(ctx, preds, bits, [n])
    outs = _outs([n, n])
    ctx.filter_fresh(77, toks, outs)
    ctx.sync()
    del toks
    sample = np.concatenate([[0, 1, 2, 3, n - 4, n - 3, n - 2, n - 1],
                             np.flatnonzero(vals[0] == 123456789)[:40],
                             g.choice(n, 150, replace=False)])
    for grp in (0, 1):
        got = np.stack([from_dev(x) for x in outs[grp]])
        want = oracle.fresh_direct(preds, bits, SEED, 77, PRF, [(tab["shares"], bits)], grp, sample, threads=8)
        assert np.array_equal(got[:, sample], want), grp
        plain = oracle.plain_group(preds, grp, vals)
        assert np.array_equal(oracle.reconstruct(got), plain)
        assert 0 < int(plain.sum()) < n


def test_gpu_fresh_tiny_and_one_bit_domain(ctx):
    # N = 1 (N4 = 4, three padding words per array) and n = 1
    g = W.rng(24)
    vals = np.array([[1], [0]], dtype=np.uint32)
    tab = W.table(vals, 1, g)
    _load(ctx, [tab])
    preds = [W.eq_pred(0, 0, 0, 1), W.range_pred(0, 1, 0, 0, 0)]
    toks = _gpu_tokens(ctx, preds, 1, [1])
    torch.cuda.synchronize()
    assert [t.cpu().numpy().tobytes() for t in toks] == list(oracle.keygen_fresh(preds, 1, [1], SEED))
    outs = _outs([1])
    ctx.filter_fresh(1, toks, outs)
    ctx.sync()
    got = np.stack([from_dev(x) for x in outs[0]])
    assert oracle.reconstruct(got)[0] == 1


def test_gpu_fresh_rejects_bad_inputs(ctx):
    bits = 12
    tables = _two_tables(bits, 1003, 517, seed=25)
    _load(ctx, tables)
    preds = _preds(tables, bits)
    toks = _gpu_tokens(ctx, preds, bits, [1003, 517])
    # wrong table size in the client's view -> descriptors disagree with the loaded table
    bad = _gpu_tokens(ctx, preds, bits, [1000, 517])
    with pytest.raises(P.OblivgmError) as e:
        ctx.filter_fresh(1, bad, _outs([1003, 517]))
    assert e.value.status == P.EINVAL
    # tokens of different keygen calls mixed
    other = _gpu_tokens(ctx, preds[:2], bits, [1003, 517])
    with pytest.raises(P.OblivgmError):
        ctx.filter_fresh(1, [toks[0], other[1], toks[2]], _outs([1003, 517]))
    # servers out of order
    with pytest.raises(P.OblivgmError):
        ctx.filter_fresh(1, [toks[1], toks[0], toks[2]], _outs([1003, 517]))
    # a buffer that is too small, and an unaligned one
    small = [torch.zeros(100, dtype=torch.uint8, device="cuda") for _ in range(3)]
    with pytest.raises(P.OblivgmError) as e:
        ctx.keygen_fresh(preds, bits, [1003, 517], SEED, small)
    assert e.value.status == P.ERANGE
    L = P.fresh_token_size(preds, bits, [1003, 517])
    big = torch.zeros(L + 16, dtype=torch.uint8, device="cuda")
    with pytest.raises(P.OblivgmError) as e:
        ctx.keygen_fresh(preds, bits, [1003, 517], SEED, [big[1:], toks[1], toks[2]])
    assert e.value.status == P.EINVAL
    # a buffer shorter than the token says it is: rejected before any kernel reads it
    with pytest.raises(P.OblivgmError) as e:
        ctx.filter_fresh(1, [toks[0], toks[1][: L // 2], toks[2]], _outs([1003, 517]))
    assert e.value.status == P.EINVAL
    # the context still works
    ctx.filter_fresh(2, toks, _outs([1003, 517]))
    ctx.sync()
