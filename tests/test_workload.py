"""The seeded input recipe: the generators produce what the design states.

* Chung-Lu graphs: simple (no self-loops, no repeated undirected edge), the requested
  size, and heavy-tailed with the stated exponent: a vertex's degree follows its weight
  (i + 1)^(-1/(gamma - 1)), so log degree against log rank has slope -1/(gamma - 1).
* bounded Zipf(s) attributes: inside the domain, P(0) / P(1) = 2^s.
* additive shares reconstruct mod 2^bits and each share set alone is uniform.
* one-hot shares XOR to e_v.
* same seed, same inputs.
"""
import numpy as np
import pytest

import workload as W


def test_chung_lu_simple_and_sized():
    e = W.chung_lu(2000, 12000, 2.1, seed=5)
    assert e.shape == (12000, 2)
    assert np.all(e[:, 0] < e[:, 1])                       # lo < hi: no self-loops
    keys = e[:, 0].astype(np.int64) * 2000 + e[:, 1]
    assert len(np.unique(keys)) == len(keys)               # no repeated edge
    assert np.array_equal(e, W.chung_lu(2000, 12000, 2.1, seed=5))
    assert not np.array_equal(e, W.chung_lu(2000, 12000, 2.1, seed=6))


def test_chung_lu_power_law_exponent():
    gamma, n, m = 2.1, 50_000, 200_000
    e = W.chung_lu(n, m, gamma, seed=9)
    deg = np.bincount(e.ravel().astype(np.int64), minlength=n).astype(np.float64)
    # expected degree is proportional to the weight (i + 1)^(-1 / (gamma - 1)); away from the
    # few top vertices (capped by the rejection of repeated edges) and the sparse tail, the
    # mean degree over log-spaced rank bins falls with that slope
    edges = np.unique(np.logspace(np.log10(30), np.log10(5000), 12).astype(int))
    ranks, means = [], []
    for lo, hi in zip(edges[:-1], edges[1:]):
        ranks.append(np.sqrt(lo * hi))
        means.append(deg[lo:hi].mean())
    slope = np.polyfit(np.log(ranks), np.log(means), 1)[0]
    assert slope == pytest.approx(-1.0 / (gamma - 1.0), abs=0.12)
    # heavy tail: the top 1 % of vertices carry far more than 1 % of the edge ends
    assert deg[: n // 100].sum() / deg.sum() > 0.2


@pytest.mark.parametrize("s", [1.1, 1.2])
def test_zipf_ratio_and_domain(s):
    bits = 16
    v = W.zipf_attrs(W.rng(3), 1, 400_000, s, bits).ravel()
    assert v.max() < (1 << bits)
    c = np.bincount(v.astype(np.int64), minlength=4)
    assert c[0] / c[1] == pytest.approx(2.0 ** s, rel=0.05)
    assert c[1] / c[3] == pytest.approx(2.0 ** s, rel=0.08)


@pytest.mark.parametrize("bits", [16, 32])
def test_additive_shares(bits):
    g = W.rng(4)
    vals = W.uniform_attrs(g, 2, 100_000, bits)
    s1, s2, s3 = W.share3(g, vals, bits)
    mask = (1 << bits) - 1
    rec = (s1.astype(np.uint64) + s2 + s3) & mask
    assert np.array_equal(rec, vals.astype(np.uint64))
    for s in (s1, s2, s3):       # each share set alone: uniform on [0, 2^bits)
        assert s.max() <= mask
        assert s.astype(np.float64).mean() / (1 << bits) == pytest.approx(0.5, abs=0.01)


def test_onehot_shares_xor_to_the_indicator():
    bits = 6
    g = W.rng(8)
    vals = W.uniform_attrs(g, 1, 500, bits)
    tab = W.onehot_table(vals, bits, g)
    x = tab["shares"][0] ^ tab["shares"][1] ^ tab["shares"][2]       # [attr][elem][word]
    words = x.reshape(500, -1)
    bitsv = ((words[:, :, None] >> np.arange(32, dtype=np.uint32)) & 1).reshape(500, -1)[:, : 1 << bits]
    assert np.array_equal(bitsv.sum(axis=1), np.ones(500))
    assert np.array_equal(bitsv.argmax(axis=1), vals[0].astype(np.int64))
