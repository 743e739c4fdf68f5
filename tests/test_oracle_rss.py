"""Pins for the oracle's re-share (Sec. III-B), AND fold (Sec. V-D) and full secEval.

* zero-sharing: the three PRF masks F(k_i) - F(k_{i-1}) add up to 0, so a
  re-share keeps the sum of the shares;
* the AND fold reconstructs to the product of the predicate bits;
* the three share sets of a group reconstruct to the plaintext AND of its
  predicates on every element (Eq. predEval + re-share + AND).
"""
import numpy as np
import pytest

import oracle
import workload as W

M32 = 0xFFFFFFFF
PRF = bytes(range(48))


@pytest.mark.parametrize("elem,step,table,query", [(0, 0, 0, 0), (12345, 3, 1, 9), (2**40 + 7, 64 + 5, 2, 2**31)])
def test_zero_sharing_sums_to_zero(elem, step, table, query):
    out = oracle.reshare(PRF, [0, 0, 0], elem, step, table, query)
    assert sum(out) & M32 == 0
    assert len(set(out)) == 3                   # fresh, not all zero
    z = [5, 7, 11]
    out2 = oracle.reshare(PRF, z, elem, step, table, query)
    assert sum(out2) & M32 == 23
    assert out2 != z


def test_reshare_masks_change_with_counter():
    a = oracle.reshare(PRF, [0, 0, 0], 1, 0, 0, 0)
    b = oracle.reshare(PRF, [0, 0, 0], 1, 1, 0, 0)
    c = oracle.reshare(PRF, [0, 0, 0], 2, 0, 0, 0)
    d = oracle.reshare(PRF, [0, 0, 0], 1, 0, 0, 1)
    assert len({tuple(a), tuple(b), tuple(c), tuple(d)}) == 4


def _small_table(g, n_elems, n_attrs, bits):
    vals = W.uniform_attrs(g, n_attrs, n_elems, bits)
    return W.table(vals, bits, g)


def test_filter_single_predicate_reconstructs():
    g = W.rng(5)
    bits = 8
    t = _small_table(g, 300, 2, bits)
    preds = [W.range_pred(0, 1, 0, 40, 180)]
    toks = oracle.keygen(preds, bits, bytes(range(16)))
    out = oracle.filter_group(toks, 3, PRF, [(t["shares"], bits)], 0, np.arange(300))
    assert np.array_equal(oracle.reconstruct(out), oracle.plain_group(preds, 0, t["values"]))


def test_filter_and_fold_reconstructs():
    # values drawn from a tiny domain so every AND outcome occurs
    g = W.rng(6)
    bits = 4
    t = _small_table(g, 400, 3, bits)
    preds = [W.range_pred(0, 0, 0, 2, 12), W.eq_pred(0, 1, 0, 7), W.range_pred(0, 2, 0, 0, 9),
             W.eq_pred(0, 0, 1, 3), W.range_pred(0, 1, 1, 5, 15)]
    toks = oracle.keygen(preds, bits, bytes(range(3, 19)))
    for grp in (0, 1):
        out = oracle.filter_group(toks, 77, PRF, [(t["shares"], bits)], grp, np.arange(400))
        rec = oracle.reconstruct(out)
        want = oracle.plain_group(preds, grp, t["values"])
        assert np.array_equal(rec, want)
        assert 0 < int(want.sum()) < 400


def test_rss_and_matches_product_of_bits():
    # reconstruct each predicate alone and the AND of the pair: AND == product
    g = W.rng(7)
    bits = 3
    t = _small_table(g, 200, 2, bits)
    pa, pb = W.range_pred(0, 0, 0, 1, 5), W.range_pred(0, 1, 0, 3, 7)
    toks = oracle.keygen([pa, pb], bits, bytes(16))
    both = oracle.reconstruct(oracle.filter_group(toks, 1, PRF, [(t["shares"], bits)], 0, np.arange(200)))
    a = oracle.plain_pred(pa, t["values"][0])
    b = oracle.plain_pred(pb, t["values"][1])
    assert np.array_equal(both, a * b)


def test_filter_threads_equal_serial():
    g = W.rng(8)
    t = _small_table(g, 256, 1, 16)
    preds = [W.eq_pred(0, 0, 0, int(t["values"][0, 3])), W.range_pred(0, 0, 0, 100, 40000)]
    toks = oracle.keygen(preds, 16, bytes(range(16)))
    a = oracle.filter_group(toks, 5, PRF, [(t["shares"], 16)], 0, np.arange(256), threads=1)
    b = oracle.filter_group(toks, 5, PRF, [(t["shares"], 16)], 0, np.arange(256), threads=4)
    assert np.array_equal(a, b)


def test_shares_depend_on_query_id_but_not_result():
    g = W.rng(9)
    t = _small_table(g, 64, 1, 8)
    preds = [W.range_pred(0, 0, 0, 10, 100)]
    toks = oracle.keygen(preds, 8, bytes(16))
    a = oracle.filter_group(toks, 1, PRF, [(t["shares"], 8)], 0, np.arange(64))
    b = oracle.filter_group(toks, 2, PRF, [(t["shares"], 8)], 0, np.arange(64))
    assert not np.array_equal(a, b)
    assert np.array_equal(oracle.reconstruct(a), oracle.reconstruct(b))


def test_fetch_unique_reconstructs_the_match():
    # secFetch case I: with exactly one matching element, the fetched shares reconstruct to its
    # index and attribute values; with none, to zero
    g = W.rng(12)
    bits = 16
    vals = W.uniform_attrs(g, 3, 500, bits)
    vals[0] = np.arange(500, dtype=np.uint32) * 7 + 3           # attribute 0 unique per element
    t = W.table(vals, bits, g)
    target = 321
    preds = [W.eq_pred(0, 0, 0, int(vals[0, target]))]
    toks = oracle.keygen(preds, bits, bytes(range(16)))
    x = oracle.filter_group(toks, 6, PRF, [(t["shares"], bits)], 0, np.arange(500))
    got = oracle.fetch_unique(x, [(t["shares"], bits)], 0, [0, 1, 2], 6, 0, PRF)
    rec = oracle.reconstruct(got)
    assert rec[0] == target
    for col, a in enumerate([0, 1, 2]):
        assert rec[1 + col] % (1 << bits) == vals[a, target]
    assert len(set(got[:, 1])) == 3                              # re-shared, not the plain value
    none = oracle.keygen([W.eq_pred(0, 0, 0, 2)], bits, bytes(16))   # 2 is no element's value
    x0 = oracle.filter_group(none, 6, PRF, [(t["shares"], bits)], 0, np.arange(500))
    assert not oracle.reconstruct(oracle.fetch_unique(x0, [(t["shares"], bits)], 0, [1], 6, 0, PRF)).any()
