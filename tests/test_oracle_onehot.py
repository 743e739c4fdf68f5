"""Pins for the oracle's one-hot mode (the paper's secEval as written).

* Z_2 DPF / DCF (beta = 1 in Z_2, Sec. V-C): the two shares XOR to the point /
  comparison function at every input of small domains;
* Eq. predEval on binary-RSS one-hot vectors (Sec. V-B, V-D): the three
  binary share sets reconstruct (XOR) to the plaintext predicate, for
  equality, ranges touching either end of the domain, the full domain, and
  ANDs of several predicates;
* the Fig. 1 worked example gives the paper's g1, g2 through this mode too.
"""
import struct

import numpy as np
import pytest

import oracle
import workload as W

PRF = bytes(range(48))


def _seeds(g):
    return bytes(g.integers(0, 256, 16, dtype=np.uint8)), bytes(g.integers(0, 256, 16, dtype=np.uint8))


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8])
def test_z2_dpf_dcf_brute_force(n):
    g = np.random.default_rng(400 + n)
    xs = np.arange(1 << n)
    top = (1 << n) - 1
    for alpha in sorted({0, top, int(g.integers(0, top + 1)), min(1, top)}):
        d0, d1 = oracle.dpf_gen_z2(n, alpha, *_seeds(g))
        c0, c1 = oracle.dcf_gen_z2(n, alpha, *_seeds(g))
        dp = oracle.eval_many(d0, xs, oracle.KIND_DPF) ^ oracle.eval_many(d1, xs, oracle.KIND_DPF)
        dc = oracle.eval_many(c0, xs, oracle.KIND_DCF) ^ oracle.eval_many(c1, xs, oracle.KIND_DCF)
        assert np.array_equal(dp, (xs == alpha).astype(np.uint32)), alpha
        assert np.array_equal(dc, (xs < alpha).astype(np.uint32)), alpha
        assert d0[3] == 1 and c1[3] == 1                  # group byte: Z_2


def test_onehot_token_has_no_mask_and_z2_keys():
    toks = oracle.keygen_onehot([W.eq_pred(0, 0, 0, 3), W.range_pred(0, 1, 1, 2, 7)], 4, bytes(16))
    for t in toks:
        assert t[7] == 1
        off = 16
        assert struct.unpack_from("<II", t, off + 8) == (0, 0)
    with pytest.raises(ValueError):
        oracle.keygen_onehot([W.eq_pred(0, 0, 0, 3)], 17, bytes(16))   # one-hot domains stop at 2^16


def test_onehot_encoding_reconstructs():
    g = W.rng(1)
    vals = W.uniform_attrs(g, 2, 50, 6)
    s1, s2, s3 = W.onehot_shares(g, vals, 6)
    e = s1 ^ s2 ^ s3
    for a in range(2):
        for c in range(50):
            bits = [(e[a, c, l // 32] >> (l % 32)) & 1 for l in range(64)]
            assert sum(bits) == 1 and bits[vals[a, c]] == 1


@pytest.mark.parametrize("n", [3, 6])
def test_onehot_filter_reconstructs_to_plaintext(n):
    g = W.rng(10 + n)
    top = (1 << n) - 1
    vals = W.uniform_attrs(g, 2, 120, n)
    tab = W.onehot_table(vals, n, g)
    preds = [
        W.eq_pred(0, 0, 0, int(vals[0, 5])),
        W.range_pred(0, 1, 1, 0, top // 2),           # starts at 0
        W.range_pred(0, 0, 2, top // 3, top),         # ends at the domain's end (hi + 1 wraps)
        W.range_pred(0, 1, 3, 0, top),                # the full domain
        W.range_pred(0, 0, 4, 1, top - 1), W.eq_pred(0, 1, 4, int(vals[1, 9])),   # an AND of two
    ]
    toks = oracle.keygen_onehot(preds, n, bytes([n]) * 16)
    for grp in range(5):
        out = oracle.filter_onehot(toks, 9, PRF, [(tab["shares"], n)], grp, np.arange(120))
        assert set(np.unique(out)) <= {0, 1}
        rec = oracle.reconstruct_bits(out)
        assert np.array_equal(rec, oracle.plain_group(preds, grp, vals)), grp


def test_onehot_rejected_by_masked_filter_and_vice_versa():
    g = W.rng(3)
    vals = W.uniform_attrs(g, 1, 8, 4)
    tab1 = W.onehot_table(vals, 4, g)
    tab2 = W.table(vals, 4, g)
    t_onehot = oracle.keygen_onehot([W.eq_pred(0, 0, 0, 1)], 4, bytes(16))
    t_masked = oracle.keygen([W.eq_pred(0, 0, 0, 1)], 4, bytes(16))
    with pytest.raises(ValueError):
        oracle.filter_group(t_onehot, 1, PRF, [(tab2["shares"], 4)], 0, np.arange(8))
    with pytest.raises(ValueError):
        oracle.filter_onehot(t_masked, 1, PRF, [(tab1["shares"], 4)], 0, np.arange(8))


def test_fig1_example_in_onehot_mode():
    from tests.test_oracle_matcher import PAPER_RESULTS, Q_EDGES, Q_PREDS, _fig1_graph
    attrs, edges = _fig1_graph()
    n = 6                       # one-hot length 64 covers the codes 1..50 used by the example
    g = W.rng(12)
    tab = W.onehot_table(attrs, n, g)
    toks = oracle.keygen_onehot(Q_PREDS, n, bytes(range(16)))
    ok = []
    for q in range(5):
        out = oracle.filter_onehot(toks, 4, PRF, [(tab["shares"], n)], q, np.arange(9))
        ok.append(oracle.reconstruct_bits(out).astype(bool))
    assert oracle.match(9, edges, 5, Q_EDGES, ok, [None] * 4) == PAPER_RESULTS
