"""Pins for the oracle's secShuffle (Alg. 5) and secFetch case II (Alg. 4).

* the pseudo-random permutation is a bijection of [0, n) for small, odd,
  power-of-two and one-past-power-of-two n, and depends on its seed;
* the shuffled shares reconstruct to the input rows moved by
  pi23(pi31(pi12(.))) -- for XOR shares (Alg. 5 as written) and for additive
  shares mod 2^32; independently of the permutation's definition, the
  reconstructed rows are the input rows as a multiset;
* no output share set is a permutation of an input share set (fresh masks);
* secFetch case II returns exactly the matched records (by id and attribute
  values), as many as there are matches, none when nothing matches.
"""
import collections

import numpy as np
import pytest

import oracle
import workload as W

SEEDS = bytes(range(48))


@pytest.mark.parametrize("n", [1, 2, 3, 5, 16, 17, 255, 256, 257, 1000, 4097])
def test_prp_is_a_bijection(n):
    img = [oracle.prp(SEEDS[:16], n, x) for x in range(n)]
    assert sorted(img) == list(range(n))


def test_prp_depends_on_seed_and_moves_points():
    n = 1000
    a = [oracle.prp(SEEDS[:16], n, x) for x in range(n)]
    b = [oracle.prp(SEEDS[16:32], n, x) for x in range(n)]
    assert a != b
    assert sum(1 for x in range(n) if a[x] == x) < 20          # about one fixed point expected


def _shares(g, n, w, group):
    d = g.integers(0, 1 << 32, (n, w), dtype=np.uint64).astype(np.uint32)
    s1 = g.integers(0, 1 << 32, (n, w), dtype=np.uint64).astype(np.uint32)
    s2 = g.integers(0, 1 << 32, (n, w), dtype=np.uint64).astype(np.uint32)
    s3 = (d ^ s1 ^ s2) if group == oracle.SHUF_XOR else (d - s1 - s2)
    return d, [s1, s2, s3]


def _rec(s, group):
    return (s[0] ^ s[1] ^ s[2]) if group == oracle.SHUF_XOR else (s[0] + s[1] + s[2])


@pytest.mark.parametrize("group", [oracle.SHUF_XOR, oracle.SHUF_ADD])
@pytest.mark.parametrize("n,w", [(1, 3), (2, 1), (37, 5), (300, 6)])
def test_shuffle_reconstructs_the_permuted_rows(group, n, w):
    g = W.rng(n * 10 + w + group)
    d, sh = _shares(g, n, w, group)
    out = oracle.shuffle(sh, SEEDS, group)
    rec = _rec(out, group)
    # rows as a multiset: holds for any permutation
    assert collections.Counter(map(tuple, rec.tolist())) == collections.Counter(map(tuple, d.tolist()))
    # and the composed permutation pi23(pi31(pi12(i)))
    for i in range(n):
        j = oracle.prp(SEEDS[0:16], n, i)
        k = oracle.prp(SEEDS[32:48], n, j)
        l = oracle.prp(SEEDS[16:32], n, k)
        assert np.array_equal(rec[l], d[i]), i
    if n > 1:
        for j in range(3):                      # re-randomised: not a permutation of an input share
            assert collections.Counter(map(tuple, out[j].tolist())) != collections.Counter(map(tuple, sh[j].tolist()))


def test_shuffle_output_independent_of_input_sharing():
    # two different sharings of the same table give the same outputs: the masks R1, R2 come
    # from the seeds, and R3 = pi(D) - R1 - R2 depends only on D
    g = W.rng(5)
    d, sh = _shares(g, 50, 4, oracle.SHUF_ADD)
    s1 = g.integers(0, 1 << 32, d.shape, dtype=np.uint64).astype(np.uint32)
    sh2 = [s1, sh[1], d - s1 - sh[1]]
    a = oracle.shuffle(sh, SEEDS, oracle.SHUF_ADD)
    b = oracle.shuffle(sh2, SEEDS, oracle.SHUF_ADD)
    for j in range(3):
        assert np.array_equal(a[j], b[j])


def _filter_shares(g, flags):
    x = flags.astype(np.uint32)
    s1 = g.integers(0, 1 << 32, len(x), dtype=np.uint64).astype(np.uint32)
    s2 = g.integers(0, 1 << 32, len(x), dtype=np.uint64).astype(np.uint32)
    return [s1, s2, x - s1 - s2]


def test_fetch_multi_returns_the_matched_records():
    g = W.rng(7)
    n, bits = 400, 16
    vals = W.uniform_attrs(g, 3, n, bits)
    t = W.table(vals, bits, g)
    flags = vals[1] < 9000                          # many matches
    m, rows = oracle.fetch_multi(_filter_shares(g, flags), (t["shares"], bits), [0, 2], SEEDS, cap=n)
    assert m == int(flags.sum())
    rec = (rows[0].astype(np.uint64) + rows[1] + rows[2]) & 0xFFFFFFFF
    rec[:, 1:] &= (1 << bits) - 1                   # attribute shares are additive mod 2^n
    got = sorted(map(tuple, rec.tolist()))
    want = sorted((c, int(vals[0, c]), int(vals[2, c])) for c in np.flatnonzero(flags))
    assert got == want
    # the order is the shuffled one, not the input order
    assert [r[0] for r in rec.tolist()] != sorted(r[0] for r in rec.tolist())


def test_fetch_multi_none_and_cap():
    g = W.rng(8)
    n, bits = 64, 8
    vals = W.uniform_attrs(g, 1, n, bits)
    t = W.table(vals, bits, g)
    m, rows = oracle.fetch_multi(_filter_shares(g, np.zeros(n, dtype=bool)), (t["shares"], bits), [0], SEEDS, cap=n)
    assert m == 0 and len(rows[0]) == 0
    flags = np.zeros(n, dtype=bool)
    flags[[3, 9, 40]] = True
    m, rows = oracle.fetch_multi(_filter_shares(g, flags), (t["shares"], bits), [0], SEEDS, cap=2)
    assert m == 3 and len(rows[0]) == 2
