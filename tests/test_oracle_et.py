"""Pins for the oracle's early-terminated Z_2 keys (the one-hot mode's DPF and DCF).

BGI16, the DPF the paper cites (Sec. IV-B), ends the tree early for small output
groups: over Z_2 a leaf seed expands into 2^m <= 128 output bits (m = min(n, 7)), so a
key has n - m levels.  The DCF does the same over the vector group Z_2^(2^m).  What
fixes these functions, independently of their code:

* brute force over whole domains: the two parties' bits XOR to [x == alpha] (DPF) or
  [x < alpha] (DCF) at every x, for n = 1..10 (no levels up to n = 7, then 1..3) and at
  n = 16, the one-hot mode's largest domain, with alpha at both ends of a leaf and of
  the domain;
* the same functions as the full-depth Z_2 keys, which test_oracle_fss.py pins on
  their own, give on the same domain;
* one party's output bits, the final correction word and the DCF's value corrections
  are balanced across keys (the FSS definition: one key alone looks random);
* each pin fails on a mistake planted in the oracle on purpose (oracle.test_plant):
  a constant leaf conversion, and a leaf conversion that reads the seed itself
  instead of expanding it (its bit 0 is the cleared control bit).
"""
import math

import numpy as np
import pytest

import oracle


def balanced(bits) -> bool:
    b = np.asarray(bits, dtype=np.int64)
    return abs(int(b.sum()) - len(b) / 2) <= 5 * math.sqrt(len(b)) / 2


def _planted(mode, fn):
    oracle.test_plant(mode)
    try:
        return fn()
    finally:
        oracle.test_plant(oracle.PLANT_NONE)


def _seeds(g):
    return bytes(g.integers(0, 256, 16, dtype=np.uint8)), bytes(g.integers(0, 256, 16, dtype=np.uint8))


def _alphas(n, g):
    top = (1 << n) - 1
    al = {0, top, int(g.integers(0, top + 1))}
    if n > 7:
        al |= {128, 127, (int(g.integers(0, 1 << (n - 7))) << 7) | 127}
    return sorted(a for a in al if a <= top)


def _table(k0, k1, n):
    return np.array([oracle.eval_et(k0, x) ^ oracle.eval_et(k1, x) for x in range(1 << n)])


def test_key_lengths_follow_the_layout():
    for n in range(1, 17):
        levels = max(n - 7, 0)
        assert oracle.key_len_et(oracle.KIND_DPF, n) == 24 + 20 * levels + 16
        assert oracle.key_len_et(oracle.KIND_DCF, n) == 24 + 36 * levels + 16


@pytest.mark.parametrize("n", list(range(1, 11)) + [16])
def test_dpf_et_brute_force(n):
    g = np.random.default_rng(100 + n)
    xs = np.arange(1 << n)
    for a in (_alphas(n, g) if n < 16 else [int(g.integers(0, 1 << 16)) | 127]):
        k0, k1 = oracle.dpf_gen_et(n, a, *_seeds(g))
        assert np.array_equal(_table(k0, k1, n), (xs == a).astype(int)), a


@pytest.mark.parametrize("n", list(range(1, 11)) + [16])
def test_dcf_et_brute_force(n):
    g = np.random.default_rng(200 + n)
    xs = np.arange(1 << n)
    for a in (_alphas(n, g) if n < 16 else [(int(g.integers(0, 1 << 9)) << 7) | 5]):
        k0, k1 = oracle.dcf_gen_et(n, a, *_seeds(g))
        assert np.array_equal(_table(k0, k1, n), (xs < a).astype(int)), a


def test_et_keys_agree_with_full_depth_z2_keys():
    n = 10
    g = np.random.default_rng(7)
    for a in (3, 600, 1023):
        s = _seeds(g)
        e0, e1 = oracle.dpf_gen_et(n, a, *s)
        f0, f1 = oracle.dpf_gen_z2(n, a, *s)
        full = [oracle.dpf_eval(f0, x) ^ oracle.dpf_eval(f1, x) for x in range(1 << n)]
        assert list(_table(e0, e1, n)) == full
        e0, e1 = oracle.dcf_gen_et(n, a, *s)
        f0, f1 = oracle.dcf_gen_z2(n, a, *s)
        full = [oracle.dcf_eval(f0, x) ^ oracle.dcf_eval(f1, x) for x in range(1 << n)]
        assert list(_table(e0, e1, n)) == full


def _party0_bits(gen, n=9, keys=256, alpha=300):
    """Party 0's output bits at every x, one row per key (random root seeds, fixed alpha)."""
    g = np.random.default_rng(31)
    rows = []
    for _ in range(keys):
        k0, _k1 = gen(n, alpha, *_seeds(g))
        rows.append([oracle.eval_et(k0, x) for x in range(1 << n)])
    return np.array(rows)


def _each_bit_balanced(rows, n=9):
    """Every bit position j of the leaf vectors balanced over keys and leaves."""
    m = min(n, 7)
    by_j = rows.reshape(rows.shape[0], -1, 1 << m)
    return all(balanced(by_j[:, :, j].ravel()) for j in range(1 << m))


@pytest.mark.parametrize("kind", ["dpf", "dcf"])
def test_one_party_output_bits_balanced(kind):
    gen = oracle.dpf_gen_et if kind == "dpf" else oracle.dcf_gen_et
    assert _each_bit_balanced(_party0_bits(gen))


@pytest.mark.parametrize("mode", [oracle.PLANT_CONST, oracle.PLANT_CLEARED_BIT])
def test_one_party_balance_fails_on_planted_conversion(mode):
    """Shown on the DPF: both kinds convert a leaf seed with the same oracle function.  In a
    DCF party's bits the value terms (and the random control bits times the correction
    vectors) would hide either mistake; its constant value vectors are caught by the
    correction-word pin below."""
    assert not _planted(mode, lambda: _each_bit_balanced(_party0_bits(oracle.dpf_gen_et, keys=64)))


def _words(gen, n=9, keys=1024, alpha=300):
    """Per key: the final correction word (128 bits) and, for a DCF, level 1's V_CW."""
    g = np.random.default_rng(41)
    fin, vcw = [], []
    levels = n - 7
    for _ in range(keys):
        k0, _k1 = gen(n, alpha, *_seeds(g))
        lb = 20 if k0[0] == oracle.KIND_DPF else 36
        fin.append(np.unpackbits(np.frombuffer(k0[24 + levels * lb:24 + levels * lb + 16], np.uint8)))
        if lb == 36:
            vcw.append(np.unpackbits(np.frombuffer(k0[24 + 20:24 + 36], np.uint8)))
    return np.array(fin), (np.array(vcw) if vcw else None)


@pytest.mark.parametrize("kind", ["dpf", "dcf"])
def test_correction_words_balanced(kind):
    gen = oracle.dpf_gen_et if kind == "dpf" else oracle.dcf_gen_et
    fin, vcw = _words(gen)
    assert all(balanced(fin[:, j]) for j in range(128))
    if vcw is not None:
        assert all(balanced(vcw[:, j]) for j in range(128))


@pytest.mark.parametrize("kind", ["dpf", "dcf"])
def test_correction_word_balance_fails_on_constant_conversion(kind):
    gen = oracle.dpf_gen_et if kind == "dpf" else oracle.dcf_gen_et
    fin, _ = _planted(oracle.PLANT_CONST, lambda: _words(gen, keys=256))
    assert not all(balanced(fin[:, j]) for j in range(128))
