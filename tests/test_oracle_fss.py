"""Pins for the oracle's DPF and DCF: brute force over whole tiny domains.

FSS correctness (Def. 3): the two Eval shares add up to the function's value at
every input.  For the point function f^=_{alpha,beta} that is beta * [x == alpha],
for the comparison function g^<_{alpha,beta} it is beta * [x < alpha] (Sec. V-C).
"""
import numpy as np
import pytest

import oracle

M32 = 0xFFFFFFFF


def _seeds(g):
    return bytes(g.integers(0, 256, 16, dtype=np.uint8)), bytes(g.integers(0, 256, 16, dtype=np.uint8))


def _alphas(n, g):
    top = (1 << n) - 1
    a = {0, top, top // 2, int(g.integers(0, top + 1))}
    return sorted(a)


@pytest.mark.parametrize("n", list(range(1, 11)))
def test_dpf_brute_force(n):
    g = np.random.default_rng(100 + n)
    xs = np.arange(1 << n)
    for alpha in _alphas(n, g):
        beta = int(g.integers(1, 1 << 32))
        k0, k1 = oracle.dpf_gen(n, alpha, beta, *_seeds(g))
        y = (oracle.eval_many(k0, xs, oracle.KIND_DPF).astype(np.uint64)
             + oracle.eval_many(k1, xs, oracle.KIND_DPF)) & M32
        want = np.where(xs == alpha, beta, 0)
        assert np.array_equal(y, want), (n, alpha)


@pytest.mark.parametrize("n", list(range(1, 11)))
def test_dcf_brute_force(n):
    g = np.random.default_rng(200 + n)
    xs = np.arange(1 << n)
    for alpha in _alphas(n, g) + [1]:
        beta = int(g.integers(1, 1 << 32))
        k0, k1 = oracle.dcf_gen(n, alpha, beta, *_seeds(g))
        y = (oracle.eval_many(k0, xs, oracle.KIND_DCF).astype(np.uint64)
             + oracle.eval_many(k1, xs, oracle.KIND_DCF)) & M32
        want = np.where(xs < alpha, beta, 0)
        assert np.array_equal(y, want), (n, alpha)


@pytest.mark.parametrize("n", [16, 32])
def test_full_width_points(n):
    g = np.random.default_rng(300 + n)
    top = (1 << n) - 1
    for _ in range(4):
        alpha = int(g.integers(0, top + 1))
        beta = int(g.integers(1, 1 << 32))
        pts = [alpha, (alpha + 1) & top, (alpha - 1) & top, 0, top] + [int(v) for v in g.integers(0, top + 1, 8)]
        d0, d1 = oracle.dpf_gen(n, alpha, beta, *_seeds(g))
        c0, c1 = oracle.dcf_gen(n, alpha, beta, *_seeds(g))
        for x in pts:
            assert (oracle.dpf_eval(d0, x) + oracle.dpf_eval(d1, x)) & M32 == (beta if x == alpha else 0)
            assert (oracle.dcf_eval(c0, x) + oracle.dcf_eval(c1, x)) & M32 == (beta if x < alpha else 0)


def test_key_sizes():
    # header 8 + seed 16 + n levels + final word 4
    assert oracle.key_len(oracle.KIND_DPF, 32) == 8 + 16 + 32 * 20 + 4 == 668
    assert oracle.key_len(oracle.KIND_DCF, 32) == 8 + 16 + 32 * 24 + 4 == 796


def test_single_share_hides_the_point():
    # one party's shares over the domain are not an indicator of alpha: they are spread
    # over Z_{2^32} (a Convert that returned a constant would fail here)
    g = np.random.default_rng(7)
    n = 10
    k0, _ = oracle.dpf_gen(n, 77, 1, *_seeds(g))
    y = oracle.eval_many(k0, np.arange(1 << n), oracle.KIND_DPF)
    assert len(np.unique(y)) > (1 << n) - 8
    # top bits roughly balanced
    assert 400 < int(np.sum(y >> 31)) < 624


def test_planted_correction_word_error_is_caught():
    # flipping one byte of a level's seed correction word must break the brute-force identity
    g = np.random.default_rng(8)
    n = 8
    k0, k1 = oracle.dpf_gen(n, 5, 9, *_seeds(g))
    bad = bytearray(k1)
    bad[24 + 2 * 20 + 5] ^= 0x10
    xs = np.arange(1 << n)
    y = (oracle.eval_many(k0, xs, oracle.KIND_DPF).astype(np.uint64)
         + oracle.eval_many(bytes(bad), xs, oracle.KIND_DPF)) & M32
    assert not np.array_equal(y, np.where(xs == 5, 9, 0))
