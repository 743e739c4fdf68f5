"""Aggregation of a target's predicates (Sec. V-D): AND, the paper's "one of" written
with XOR, and the inclusive OR, folded left to right in list order.

Pins of the oracle against a plain Boolean definition: the reconstructed shares of
every mode (masked, one-hot, fresh-key from tokens, fresh-key from the seed) equal
numpy's &, != and | over the plaintext predicate bits, on every element of tables
whose two attributes take every value of a small domain together.  The ops are
chosen so that each of them changes the result on some element: a wrong sign or
coefficient in any fold fails.  Tokens carry the op in a field of their own; a
group's first predicate must carry AND, and both key generators (oracle and the
library's host keygen) reject anything else, byte for byte alike.
"""
import numpy as np
import pytest

import oracle
import workload as W

PRF = bytes(range(48))
SEED = bytes(range(3, 19))
AND, XOR, OR = oracle.COMBINE_AND, oracle.COMBINE_XOR, oracle.COMBINE_OR


def _grid(n):
    """Two attributes covering every pair of values of an n-bit domain."""
    a, b = np.meshgrid(np.arange(1 << n), np.arange(1 << n), indexing="ij")
    return np.stack([a.ravel(), b.ravel()]).astype(np.uint32)


def _preds(n):
    top = (1 << n) - 1
    return [
        # group 0: ((a < top/2) XOR (b == 3)) OR (a == 5), then AND b in [1, top - 1]
        W.range_pred(0, 0, 0, 0, top // 2), W.eq_pred(0, 1, 0, 3, combine=XOR), W.eq_pred(0, 0, 0, 5, combine=OR),
        W.range_pred(0, 1, 0, 1, top - 1, combine=AND),
        # group 1: a in [2, 9] XOR b in [4, 12]  (both hold on some elements: XOR != OR)
        W.range_pred(0, 0, 1, 2, 9), W.range_pred(0, 1, 1, 4, 12, combine=XOR),
        # group 2: a == 1 OR b in [top - 2, top]
        W.eq_pred(0, 0, 2, 1), W.range_pred(0, 1, 2, top - 2, top, combine=OR),
    ]


def _check_ops_matter(preds, vals, grp):
    """the group's result under its ops differs from the all-AND result somewhere"""
    plain = oracle.plain_group(preds, grp, vals)
    all_and = oracle.plain_group([dict(p, combine=AND) for p in preds], grp, vals)
    assert not np.array_equal(plain, all_and)
    return plain


def test_plain_group_is_the_boolean_fold():
    vals = _grid(4)
    a, b = vals[0].astype(np.int64), vals[1].astype(np.int64)
    preds = _preds(4)
    want0 = ((((a <= 7) != (b == 3)) | (a == 5)) & (b >= 1) & (b <= 14))
    want1 = ((a >= 2) & (a <= 9)) != ((b >= 4) & (b <= 12))
    want2 = (a == 1) | (b >= 13)
    for grp, w in enumerate((want0, want1, want2)):
        assert np.array_equal(oracle.plain_group(preds, grp, vals), w.astype(np.uint32)), grp


def test_masked_mode_folds_equal_boolean_definition():
    n = 6
    vals = _grid(n)
    g = W.rng(41)
    tab = W.table(vals, n, g)
    preds = _preds(n)
    toks = oracle.keygen(preds, n, SEED)
    for grp in range(3):
        plain = _check_ops_matter(preds, vals, grp)
        got = oracle.filter_group(toks, 9, PRF, [(tab["shares"], n)], grp, np.arange(vals.shape[1]), threads=4)
        assert np.array_equal(oracle.reconstruct(got), plain), grp


def test_onehot_mode_folds_equal_boolean_definition():
    n = 4
    vals = _grid(n)
    g = W.rng(42)
    tab = W.onehot_table(vals, n, g)
    preds = _preds(n)
    toks = oracle.keygen_onehot(preds, n, SEED)
    for grp in range(3):
        plain = _check_ops_matter(preds, vals, grp)
        got = oracle.filter_onehot(toks, 9, PRF, [(tab["shares"], n)], grp, np.arange(vals.shape[1]))
        assert np.array_equal(oracle.reconstruct_bits(got), plain), grp


def test_fresh_mode_folds_equal_boolean_definition_and_direct():
    n = 5
    vals = _grid(n)
    N = vals.shape[1]
    g = W.rng(43)
    tab = W.table(vals, n, g)
    preds = _preds(n)
    toks = oracle.keygen_fresh(preds, n, [N], SEED)
    sample = np.array([0, 1, 2, 33, 100, 500, N - 2, N - 1])
    for grp in range(3):
        plain = _check_ops_matter(preds, vals, grp)
        got = oracle.filter_fresh(toks, 9, PRF, [(tab["shares"], n)], grp, np.arange(N), threads=4)
        assert np.array_equal(oracle.reconstruct(got), plain), grp
        direct = oracle.fresh_direct(preds, n, SEED, 9, PRF, [(tab["shares"], n)], grp, sample)
        assert np.array_equal(direct, got[:, sample]), grp


def _record_offsets(tok, n):
    dpf, dcf = oracle.key_len(oracle.KIND_DPF, n), oracle.key_len(oracle.KIND_DCF, n)
    offs, off = [], 16
    while off < len(tok):
        offs.append(off)
        off += 24 + (2 * dpf if tok[off] == oracle.PRED_EQ else 4 * dcf)
    return offs


def test_token_carries_the_op_and_library_keygen_is_byte_identical():
    P = pytest.importorskip("paper_2209_03526_gb300")
    n = 8
    preds = _preds(n)
    toks = oracle.keygen(preds, n, SEED)
    for t in toks:
        offs = _record_offsets(t, n)
        assert [t[o + 20] for o in offs] == [p["combine"] for p in preds]
        assert all(t[o + 21:o + 24] == bytes(3) for o in offs)
    assert P.keygen(preds, n, SEED) == toks
    assert P.keygen_onehot(_preds(4), 4, SEED) == oracle.keygen_onehot(_preds(4), 4, SEED)
    assert P.fresh_token_size(preds, n, [300]) == oracle.fresh_token_len(preds, n, [300])
    ft = oracle.keygen_fresh(preds, n, [300], SEED)
    for p, pred in enumerate(preds):
        d = ft[0][64 + 32 * p:64 + 32 * (p + 1)]
        assert d[24] == pred["combine"] and d[25:] == bytes(7)


@pytest.mark.parametrize("bad", ["first_xor", "first_or_later_group", "op_3"])
def test_bad_ops_are_rejected_by_both_keygens(bad):
    P = pytest.importorskip("paper_2209_03526_gb300")
    def spoil(preds):
        preds = list(preds)
        if bad == "first_xor":
            preds[0] = dict(preds[0], combine=XOR)
        elif bad == "first_or_later_group":
            preds[4] = dict(preds[4], combine=OR)     # first predicate of group 1
        else:
            preds[1] = dict(preds[1], combine=3)
        return preds

    p8, p4 = _preds(8), _preds(4)
    oracle.keygen(p8, 8, SEED), oracle.keygen_onehot(p4, 4, SEED)   # valid before the change
    p8, p4 = spoil(p8), spoil(p4)
    with pytest.raises(ValueError):
        oracle.keygen(p8, 8, SEED)
    with pytest.raises(ValueError):
        oracle.keygen_onehot(p4, 4, SEED)
    with pytest.raises(ValueError):
        oracle.keygen_fresh(p8, 8, [50], SEED)
    for fn in (lambda: P.keygen(p8, 8, SEED), lambda: P.keygen_onehot(p4, 4, SEED),
               lambda: P.fresh_token_size(p8, 8, [50])):
        with pytest.raises(P.OblivgmError) as e:
            fn()
        assert e.value.status == P.EINVAL
        assert "combine" in str(e.value) or "AND" in str(e.value)


def test_oracle_rejects_tampered_op_fields():
    n = 6
    vals = _grid(n)
    tab = W.table(vals, n, W.rng(44))
    preds = _preds(n)
    toks = oracle.keygen(preds, n, SEED)
    offs = _record_offsets(toks[0], n)
    el = np.arange(10)
    # servers disagree on an op
    t1 = bytearray(toks[1])
    t1[offs[1] + 20] = OR
    with pytest.raises(ValueError):
        oracle.filter_group([toks[0], bytes(t1), toks[2]], 1, PRF, [(tab["shares"], n)], 0, el)
    # an op on a group's first predicate, in all three tokens
    bad = [bytearray(t) for t in toks]
    for t in bad:
        t[offs[4] + 20] = XOR
    with pytest.raises(ValueError):
        oracle.filter_group([bytes(t) for t in bad], 1, PRF, [(tab["shares"], n)], 1, el)
    # a nonzero reserved byte
    bad = [bytearray(t) for t in toks]
    for t in bad:
        t[offs[2] + 22] = 1
    with pytest.raises(ValueError):
        oracle.filter_group([bytes(t) for t in bad], 1, PRF, [(tab["shares"], n)], 0, el)
