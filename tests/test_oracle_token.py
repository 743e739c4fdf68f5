"""Pins for the token of Sec. V-C on masked inputs and the range decomposition.

Invariant (Eq. predEval, masked form): the six key-half outputs of the three
servers add up to the predicate's value on the unmasked attribute, i.e.
sum_i z_i = [pred(x)] mod 2^32 with z_i evaluated at x^ = x + r.
"""
import itertools
import struct

import numpy as np
import pytest

import oracle
import workload as W

M32 = 0xFFFFFFFF


def _records(tok, n):
    """(offset of each predicate record, kind) by walking the token layout."""
    n_preds = struct.unpack_from("<H", tok, 8)[0]
    off, out = 16, []
    for _ in range(n_preds):
        kind = tok[off]
        half = oracle.key_len(oracle.KIND_DPF, n) if kind == 1 else 2 * oracle.key_len(oracle.KIND_DCF, n)
        out.append((off, kind, half))
        off += 24 + 2 * half
    assert off == len(tok)
    return out


def _mask(tokens, p, n):
    """r = <r>_1 + <r>_2 + <r>_3 from each server's own share in its record."""
    r = 0
    for t in tokens:
        off, _, _ = _records(t, n)[p]
        r += struct.unpack_from("<I", t, off + 8)[0]
    return r & ((1 << n) - 1)


def test_beta_prime_is_inverse_of_three():
    assert (3 * oracle.BETA_PRIME) & M32 == 1


def test_token_layout_and_server_assignment():
    n = 8
    preds = [W.eq_pred(0, 1, 0, 17), W.range_pred(0, 0, 0, 3, 200)]
    toks = oracle.keygen(preds, n, bytes(range(16)))
    dpf, dcf = oracle.key_len(1, n), oracle.key_len(2, n)
    assert len(toks[0]) == 16 + (24 + 2 * dpf) + (24 + 4 * dcf)
    # key-half parties: CS1 (pair1,b0),(pair2,b0); CS2 (pair2,b1),(pair3,b0); CS3 (pair3,b1),(pair1,b1)
    want_party = [(0, 0), (1, 0), (1, 1)]
    for i, t in enumerate(toks):
        assert struct.unpack_from("<I", t, 0)[0] == 0x544D474F and t[5] == i + 1
        for off, kind, half in _records(t, n):
            for h in range(2):
                key = t[off + 24 + h * half:]
                assert key[2] == want_party[i][h]
    # the mask shares: CS_i holds (<r>_i, <r>_{i+1})
    for off, _, _ in _records(toks[0], n):
        r_own = [struct.unpack_from("<I", toks[i], off + 8)[0] for i in range(3)]
        r_next = [struct.unpack_from("<I", toks[i], off + 12)[0] for i in range(3)]
        assert r_next == [r_own[1], r_own[2], r_own[0]]


def test_pairs_are_complete_key_pairs():
    # pair 1 = CS1 half A + CS3 half B; pair 2 = CS1 half B + CS2 half A; pair 3 = CS2 half B + CS3 half A
    n = 8
    alpha = 99
    toks = oracle.keygen([W.eq_pred(0, 0, 0, alpha)], n, bytes(16))
    r = _mask(toks, 0, n)
    dpf = oracle.key_len(1, n)
    halves = {}
    for i, t in enumerate(toks):
        off = 16
        halves[(i, 0)] = t[off + 24: off + 24 + dpf]
        halves[(i, 1)] = t[off + 24 + dpf: off + 24 + 2 * dpf]
    pairs = [((0, 0), (2, 1)), ((0, 1), (1, 0)), ((1, 1), (2, 0))]
    for a, b in pairs:
        for x in range(1 << n):
            y = (oracle.dpf_eval(halves[a], x) + oracle.dpf_eval(halves[b], x)) & M32
            assert y == (oracle.BETA_PRIME if x == (alpha + r) % (1 << n) else 0)


def _check_all(preds, n, seed, xs):
    toks = oracle.keygen(preds, n, seed)
    for p, pred in enumerate(preds):
        r = _mask(toks, p, n)
        want = oracle.plain_pred(pred, xs)
        for x, w in zip(xs, want):
            z, y = oracle.pred_z(toks, p, (int(x) + r) & ((1 << n) - 1))
            assert sum(z) & M32 == int(w), (pred, int(x))
            assert sum(y) & M32 == int(w)


def test_range_decomposition_exhaustive_n4():
    # every inclusive range [lo, hi] of a 4-bit domain, every x, one fresh mask per range
    n = 4
    xs = np.arange(1 << n)
    for lo, hi in itertools.combinations_with_replacement(range(1 << n), 2):
        _check_all([W.range_pred(0, 0, 0, lo, hi)], n, bytes([lo, hi]) + bytes(14), xs)


def test_equality_exhaustive_n4():
    n = 4
    xs = np.arange(1 << n)
    for a in range(1 << n):
        _check_all([W.eq_pred(0, 0, 0, a)], n, bytes([a, 7]) + bytes(14), xs)


@pytest.mark.parametrize("seed", range(6))
def test_range_wraps_and_full_domain_n8(seed):
    # many masks so that a1 = hi + 1 + r wraps below a0 = lo + r; plus the full domain and single points
    n = 8
    g = np.random.default_rng(seed)
    xs = np.arange(1 << n)
    ranges = [(0, 255), (0, 0), (255, 255), (10, 10)] + [tuple(sorted(g.integers(0, 256, 2))) for _ in range(3)]
    for lo, hi in ranges:
        _check_all([W.range_pred(0, 0, 0, int(lo), int(hi))], n, bytes(g.integers(0, 256, 16, dtype=np.uint8)), xs)


def test_keygen_rejects_bad_predicates():
    with pytest.raises(ValueError):
        oracle.keygen([W.range_pred(0, 0, 0, 9, 3)], 8, bytes(16))        # empty range
    with pytest.raises(ValueError):
        oracle.keygen([W.eq_pred(0, 0, 0, 256)], 8, bytes(16))            # outside the domain
    with pytest.raises(ValueError):
        oracle.keygen([], 8, bytes(16))


def test_keygen_is_deterministic_in_seed():
    preds = [W.eq_pred(0, 0, 0, 5), W.range_pred(0, 1, 0, 1, 9)]
    a = oracle.keygen(preds, 16, bytes(range(16)))
    b = oracle.keygen(preds, 16, bytes(range(16)))
    c = oracle.keygen(preds, 16, bytes(range(1, 17)))
    assert a == b and a != c
