"""GPU parity of the aggregation ops (Sec. V-D): AND, the paper's "one of" as XOR,
and OR, in every mode, bit-exact against the oracle and equal to the Boolean fold
of the plaintext predicates.

* masked mode: the per-element kernel, the walk-parallel kernel, the plain
  per-query path and the no-allocation entry point;
* fresh-key mode: the GPU client's tokens equal the oracle's byte for byte, and
  the servers' shares equal the oracle's;
* one-hot mode;
* tampered op fields are rejected (EINVAL) and the context keeps working.
"""
import numpy as np
import pytest

import oracle
import workload as W
from tests._helpers import PRF, from_dev, to_dev

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2209_03526_gb300")

SEED = bytes(range(9, 25))
AND, XOR, OR = P.COMBINE_AND, P.COMBINE_XOR, P.COMBINE_OR
ALWAYS = (1 << 64) - 1


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = P.Context(0, prf_keys=PRF)
    yield c
    c.close()


def _preds(n):
    top = (1 << n) - 1
    return [
        W.range_pred(0, 0, 0, 0, top // 2), W.eq_pred(0, 1, 0, 3, combine=XOR), W.eq_pred(0, 0, 0, 5, combine=OR),
        W.range_pred(0, 1, 0, 1, top - 1, combine=AND),
        W.range_pred(0, 0, 1, 2, top // 3), W.range_pred(0, 1, 1, top // 4, top // 2, combine=XOR),
        W.eq_pred(0, 0, 2, 1), W.range_pred(0, 1, 2, top - max(2, top // 16), top, combine=OR),
    ]


def _vals(n, n_elems, seed):
    g = W.rng(seed)
    v = W.uniform_attrs(g, 2, n_elems, n)
    v[0, ::11] = 5
    v[1, ::13] = 3
    v[0, ::17] = 1
    return v, g


def _outs(n_elems, n_groups=3):
    return [[torch.full((n_elems,), -1, dtype=torch.int32, device="cuda") for _ in range(3)] for _ in range(n_groups)]


def _host(outs):
    return [np.stack([from_dev(t) for t in grp]) for grp in outs]


@pytest.mark.parametrize("path", ["per_element", "walk_parallel", "plain", "noalloc"])
def test_masked_mode_ops_equal_oracle(ctx, path):
    n, n_elems = 12, 3001
    vals, g = _vals(n, n_elems, 51)
    tab = W.table(vals, n, g)
    ctx.load_shares(0, [to_dev(s) for s in tab["shares"]], n)
    preds = _preds(n)
    toks = P.keygen(preds, n, SEED)
    outs = _outs(n_elems)
    prev = ctx.set_walk_parallel(ALWAYS if path == "walk_parallel" else 0)
    try:
        if path == "plain":
            ctx.filter_plain(8, toks, outs)
        elif path == "noalloc":
            ctx.filter_and_combine_noalloc(8, toks, outs)
        else:
            ctx.filter_and_combine(8, toks, outs)
        ctx.sync()
    finally:
        ctx.set_walk_parallel(prev)
    got = _host(outs)
    for grp in range(3):
        want = oracle.filter_group(toks, 8, PRF, [(tab["shares"], n)], grp, np.arange(n_elems), threads=8)
        assert np.array_equal(got[grp], want), grp
        plain = oracle.plain_group(preds, grp, vals)
        assert np.array_equal(oracle.reconstruct(got[grp]), plain), grp
        assert 0 < int(plain.sum()) < n_elems


def test_fresh_mode_ops_equal_oracle(ctx):
    n, n_elems = 10, 1203
    vals, g = _vals(n, n_elems, 52)
    tab = W.table(vals, n, g)
    ctx.load_shares(0, [to_dev(s) for s in tab["shares"]], n)
    preds = _preds(n)
    L = P.fresh_token_size(preds, n, [n_elems])
    toks = [torch.zeros(L, dtype=torch.uint8, device="cuda") for _ in range(3)]
    ctx.keygen_fresh(preds, n, [n_elems], SEED, toks)
    torch.cuda.synchronize()
    want_toks = oracle.keygen_fresh(preds, n, [n_elems], SEED)
    for i in range(3):
        assert toks[i].cpu().numpy().tobytes() == want_toks[i], i
    outs = _outs(n_elems)
    ctx.filter_fresh(6, toks, outs)
    ctx.sync()
    got = _host(outs)
    for grp in range(3):
        want = oracle.filter_fresh(want_toks, 6, PRF, [(tab["shares"], n)], grp, np.arange(n_elems), threads=8)
        assert np.array_equal(got[grp], want), grp
        assert np.array_equal(oracle.reconstruct(got[grp]), oracle.plain_group(preds, grp, vals)), grp


def _unpack(words, n):
    w = np.asarray(words, dtype=np.uint32)
    return ((w[:, None] >> np.arange(32, dtype=np.uint32)) & 1).reshape(-1)[:n]


@pytest.mark.parametrize("n,n_elems", [(4, 700), (8, 1500)])
def test_onehot_mode_ops_equal_oracle(ctx, n, n_elems):
    vals, g = _vals(n, n_elems, 53 + n)
    tab = W.onehot_table(vals, n, g)
    ctx.load_onehot(0, [to_dev(s) for s in tab["shares"]], n)
    preds = _preds(n)
    toks = P.keygen_onehot(preds, n, SEED)
    words = (n_elems + 31) // 32
    outs = [[torch.empty(words, dtype=torch.int32, device="cuda") for _ in range(3)] for _ in range(3)]
    ctx.filter_onehot(4, toks, outs)
    ctx.sync()
    for grp in range(3):
        got = np.stack([_unpack(from_dev(t), n_elems) for t in outs[grp]])
        want = oracle.filter_onehot(toks, 4, PRF, [(tab["shares"], n)], grp, np.arange(n_elems))
        assert np.array_equal(got, want), grp
        assert np.array_equal(oracle.reconstruct_bits(got), oracle.plain_group(preds, grp, vals)), grp


def _record_offsets(tok, n):
    dpf, dcf = oracle.key_len(oracle.KIND_DPF, n), oracle.key_len(oracle.KIND_DCF, n)
    offs, off = [], 16
    while off < len(tok):
        offs.append(off)
        off += 24 + (2 * dpf if tok[off] == oracle.PRED_EQ else 4 * dcf)
    return offs


def test_tampered_op_fields_are_rejected(ctx):
    n, n_elems = 12, 500
    vals, g = _vals(n, n_elems, 54)
    tab = W.table(vals, n, g)
    ctx.load_shares(0, [to_dev(s) for s in tab["shares"]], n)
    preds = _preds(n)
    toks = P.keygen(preds, n, SEED)
    offs = _record_offsets(toks[0], n)
    cases = []
    t1 = bytearray(toks[1])
    t1[offs[1] + 20] = OR                                  # servers disagree
    cases.append([toks[0], bytes(t1), toks[2]])
    first = [bytearray(t) for t in toks]
    for t in first:
        t[offs[6] + 20] = XOR                              # op on a group's first predicate
    cases.append([bytes(t) for t in first])
    big = [bytearray(t) for t in toks]
    for t in big:
        t[offs[3] + 20] = 3                                # unknown op
    cases.append([bytes(t) for t in big])
    for bad in cases:
        with pytest.raises(P.OblivgmError) as e:
            ctx.filter_and_combine(2, bad, _outs(n_elems))
        assert e.value.status == P.EINVAL
    outs = _outs(n_elems)
    ctx.filter_and_combine(2, toks, outs)
    ctx.sync()
    assert np.array_equal(oracle.reconstruct(_host(outs)[2]), oracle.plain_group(preds, 2, vals))
