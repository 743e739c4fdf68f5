"""Pins for the one-hot mode's re-share PRF into Z_2 (Sec. III-B re-share, binary RSS).

F(k, ctr) must be a PRF; one AES block serves 128 consecutive elements: the bit of
element e is bit e mod 128 of AES_k(c), c = u64 (e div 128) | 2^63 || u16 step ||
u16 table || u32 query.  Fixed here against the oracle's AES, which the FIPS-197
known-answer tests pin on their own:

* the bit equals that bit of AES_k(c), with c built byte by byte in the test;
* elements of one 128-element block read different bits of one block, elements of
  different blocks read different blocks;
* the bits are balanced over elements, steps and queries, and fail to be with a
  constant F planted in the oracle on purpose.
"""
import math
import struct

import numpy as np
import pytest

import oracle

KEY = bytes(range(16, 32))


def _block(e, step, table, query):
    return struct.pack("<QHHI", (e >> 7) | (1 << 63), step, table, query)


def _bit(block_out, j):
    return (block_out[j // 8] >> (j % 8)) & 1


@pytest.mark.parametrize("e", [0, 1, 7, 8, 127, 128, 129, 255, 4096 + 77, (1 << 40) + 5])
def test_bit_of_aes_under_the_counter_block(e):
    for step, table, query in [(0, 0, 0), (3, 1, 9), (64 + 2, 7, 0xDEADBEEF)]:
        out = oracle.aes128(KEY, _block(e, step, table, query))
        assert oracle.prf_bit(KEY, e, step, table, query) == _bit(out, e % 128)


def test_one_block_per_128_elements():
    out0 = oracle.aes128(KEY, _block(0, 5, 0, 1))
    out1 = oracle.aes128(KEY, _block(128, 5, 0, 1))
    assert out0 != out1
    got = [oracle.prf_bit(KEY, e, 5, 0, 1) for e in range(256)]
    assert got == [_bit(out0, j) for j in range(128)] + [_bit(out1, j) for j in range(128)]


def _balanced(bits):
    b = np.asarray(bits, dtype=np.int64)
    return abs(int(b.sum()) - len(b) / 2) <= 5 * math.sqrt(len(b)) / 2


def _sample():
    return ([oracle.prf_bit(KEY, e, 3, 1, 2) for e in range(4096)]
            + [oracle.prf_bit(KEY, 1000, s, 1, 2) for s in range(512)]
            + [oracle.prf_bit(KEY, 1000, 3, 1, q) for q in range(512)])


def test_bits_balanced():
    assert _balanced(_sample())


def test_balance_fails_on_planted_constant():
    oracle.test_plant(oracle.PLANT_CONST)
    try:
        bits = _sample()
    finally:
        oracle.test_plant(oracle.PLANT_NONE)
    assert not _balanced(bits)
