"""Host-side checks of the C-ABI library (no GPU): it loads, exports every
declared entry point, and its client-side token generation is byte-identical
to the oracle's independent implementation of the same construction."""
import re
import os

import numpy as np
import pytest

import oracle
import paper_2209_03526_gb300 as P
import workload as W
from paper_2209_03526_gb300 import _native as N

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            txt = open(os.path.join(inc, f)).read()
            names |= set(re.findall(r"^\s*(?:oblivgm_status|uint32_t|uint64_t)\s+(oblivgm_\w+)\s*\(", txt, re.M))
    return names


def test_library_exports_every_declared_symbol():
    lib = N.load()
    declared = _declared()
    assert len(declared) >= 19
    for name in declared:
        assert hasattr(lib, name), name
    assert set(N._SIGS) == declared


def test_version():
    assert P.version() == 0x000100


def _random_preds(g, n, k, n_tables=2):
    preds = []
    top = (1 << n) - 1
    for i in range(k):
        t = int(g.integers(0, n_tables))
        if g.random() < 0.5:
            preds.append(W.eq_pred(t, int(g.integers(0, 4)), int(g.integers(0, 3)), int(g.integers(0, top + 1))))
        else:
            lo, hi = sorted(int(v) for v in g.integers(0, top + 1, 2))
            preds.append(W.range_pred(t, int(g.integers(0, 4)), int(g.integers(0, 3)), lo, hi))
    return preds


@pytest.mark.parametrize("n", [1, 5, 16, 31, 32])
def test_keygen_byte_identical_to_oracle(n):
    g = np.random.default_rng(n)
    for trial in range(3):
        preds = _random_preds(g, n, int(g.integers(1, 7)))
        seed = bytes(g.integers(0, 256, 16, dtype=np.uint8))
        assert P.keygen(preds, n, seed) == oracle.keygen(preds, n, seed)


def test_keygen_full_domain_and_wrap_ranges_identical():
    preds = [W.range_pred(0, 0, 0, 0, 0xFFFFFFFF), W.range_pred(0, 1, 0, 5, 5), W.eq_pred(0, 0, 1, 0xFFFFFFFF),
             W.range_pred(1, 0, 2, 0xFFFFFF00, 0xFFFFFFFF)]
    for s in range(4):
        seed = bytes([s]) * 16
        assert P.keygen(preds, 32, seed) == oracle.keygen(preds, 32, seed)


def test_keygen_sizes_and_errors():
    preds = [W.eq_pred(0, 0, 0, 3), W.range_pred(0, 0, 0, 1, 9)]
    assert P.token_len(preds, 32) == 16 + (24 + 2 * 668) + (24 + 4 * 796)
    with pytest.raises(P.OblivgmError) as e:
        P.keygen([W.range_pred(0, 0, 0, 9, 1)], 8, bytes(16))
    assert e.value.status == N.EINVAL
    with pytest.raises(P.OblivgmError):
        P.keygen([W.eq_pred(0, 0, 0, 300)], 8, bytes(16))
    with pytest.raises(P.OblivgmError):
        P.keygen([W.eq_pred(0, 0, 0, 3)], 33, bytes(16))
    with pytest.raises(P.OblivgmError):
        P.keygen([W.eq_pred(0, 0, 0, 3)] * 65, 8, bytes(16))


def test_keygen_buffer_too_small_reports_size():
    import ctypes
    lib = N.load()
    preds = [W.eq_pred(0, 0, 0, 3)]
    arr = P._pred_array(preds)
    bufs = [ctypes.create_string_buffer(10) for _ in range(3)]
    ptrs = (N.c_vp * 3)(*[ctypes.addressof(b) for b in bufs])
    lens = (N.c_size * 3)()
    seed = ctypes.create_string_buffer(16)
    st = lib.oblivgm_keygen(arr, 1, 8, ctypes.addressof(seed), ptrs, 10, lens)
    assert st == N.ERANGE and lens[0] == P.token_len(preds, 8)


@pytest.mark.parametrize("n", [1, 3, 5, 6, 7, 8, 12, 16])
def test_onehot_keygen_byte_identical_to_oracle(n):
    g = np.random.default_rng(50 + n)
    for trial in range(2):
        preds = _random_preds(g, n, int(g.integers(1, 6)))
        seed = bytes(g.integers(0, 256, 16, dtype=np.uint8))
        assert P.keygen_onehot(preds, n, seed) == oracle.keygen_onehot(preds, n, seed)
    with pytest.raises(P.OblivgmError):
        P.keygen_onehot([W.eq_pred(0, 0, 0, 1)], 17, bytes(16))


def test_fresh_token_size_matches_oracle_layout():
    preds = [W.eq_pred(0, 0, 0, 5), W.range_pred(1, 1, 1, 2, 9), W.range_pred(0, 2, 0, 0, 255)]
    for n, elems in ((8, [1, 1]), (8, [1003, 17]), (32, [4096, 5])):
        assert P.fresh_token_size(preds, n, elems) == oracle.fresh_token_len(preds, n, elems)
    with pytest.raises(P.OblivgmError):
        P.fresh_token_size(preds, 8, [10])                 # table 1 has no size
    with pytest.raises(P.OblivgmError):
        P.fresh_token_size([W.range_pred(0, 0, 0, 9, 2)], 8, [10])
    with pytest.raises(P.OblivgmError):
        P.fresh_token_size(preds, 33, [10, 10])


def test_bitsliced_sbox_header_is_the_checked_circuit():
    # the bitsliced layout's S-box is a gate circuit derived from the tower-field inverse; the
    # generator checks it on all 256 inputs against the S-box's definition before emitting it,
    # and the committed header must be exactly what it emits
    import importlib.util
    path = os.path.join(ROOT, "paper_2209_03526_gb300", "csrc", "gen_aes_bitsliced.py")
    spec = importlib.util.spec_from_file_location("gen_aes_bitsliced", path)
    gen = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(gen)
    assert gen.SBOX[0x53] == 0xED and gen.SBOX[0] == 0x63
    assert [gen.SBOX[a] for a in range(256)] == [oracle.sbox(a) for a in range(256)]
    with open(os.path.join(ROOT, "paper_2209_03526_gb300", "csrc", "aes_bitsliced_sbox.cuh")) as f:
        assert f.read() == gen.header_text()
