"""The benchmark's algorithmic work per element, checked against the oracle's own work.

bench.py reports AES blocks per second (and derives its roofline from the same per-element
count).  The count is a formula: 6 DPF walks of n levels (one PRG block per level) per
equality predicate, 12 DCF walks of n levels (two blocks per level: seed / control bit and
value) per range predicate, and 3 PRF blocks per re-share, of which an AND-group of P
predicates has 2P - 1.  Here the oracle, which runs the constructions step by step, counts
the AES-128 blocks it encrypts while filtering one element, and the two must agree.  A
dropped or doubled PRG call on either side changes the number.  The keygen line's count
per key pair is checked the same way against the oracle's Gen.
"""
import numpy as np
import pytest

import bench
import oracle
import workload as W

PRF = bytes(range(48))


def _oracle_blocks(preds, n_bits, shares, elem=0):
    toks = oracle.keygen(preds, n_bits, bytes(range(16)))
    oracle.aes_blocks_reset()
    oracle.filter_group(toks, 3, PRF, [(shares, n_bits)], 0, np.array([elem]), threads=1)
    return oracle.aes_blocks()


def test_bench_workload_blocks_per_element():
    wl = W.bulk_vertex_filter(n_vertices=64, seed=2)       # the headline's predicates, fewer vertices
    preds = wl["preds"]
    got = _oracle_blocks(preds, 32, wl["tables"][0]["shares"])
    assert got == bench.aes_per_element(preds) == 3885


@pytest.mark.parametrize("kinds", [("eq",), ("range",), ("eq", "range"), ("range", "eq", "eq")])
@pytest.mark.parametrize("n_bits", [16, 32])
def test_blocks_per_element_by_predicate_mix(kinds, n_bits):
    g = W.rng(7)
    vals = W.uniform_attrs(g, 2, 16, n_bits)
    tab = W.table(vals, n_bits, g)
    top = (1 << n_bits) - 1
    preds = [W.eq_pred(0, i % 2, 0, int(vals[i % 2, 3])) if k == "eq" else W.range_pred(0, i % 2, 0, 5, top // 3)
             for i, k in enumerate(kinds)]
    assert _oracle_blocks(preds, n_bits, tab["shares"], elem=3) == bench.aes_per_element(preds, n_bits)


def test_counter_counts_blocks():
    oracle.aes_blocks_reset()
    for _ in range(5):
        oracle.aes128(bytes(16), bytes(16))
    assert oracle.aes_blocks() == 5


@pytest.mark.parametrize("n_bits", [5, 16, 32])
@pytest.mark.parametrize("dcf", [False, True])
def test_keygen_blocks_per_pair(n_bits, dcf):
    """bench.py's keygen line counts a pair's Gen as 2 root-seed blocks plus the tree's
    blocks; the oracle's Gen, given the root seeds, encrypts exactly the tree's."""
    gen = oracle.dcf_gen if dcf else oracle.dpf_gen
    oracle.aes_blocks_reset()
    gen(n_bits, 11, 1, bytes(range(16)), bytes(range(16, 32)))
    full, w0 = bench.keygen_blocks_per_pair(dcf, n_bits)
    assert oracle.aes_blocks() + 2 == full + w0
