"""Pins for the oracle's output encodings (Convert) and mask words.

Brute force (test_oracle_fss.py) shows that the two Eval shares add up to the
function for every input, but it passes for ANY Convert: the correction words
absorb whatever Convert returns.  What a bad Convert breaks is the other half
of the FSS definition (Sec. V-C): one key, and one party's shares, must look
random.  So these tests check that words which, under the constructions, are
a Convert of fresh PRG output are uniform, with fixed (alpha, beta) and only
the root seeds varying:

* DPF over Z_{2^32} with beta = 0: CW_{n+1} = +-(Convert(s_1) - Convert(s_0));
* DCF over Z_{2^32} with beta = 0: every V_CW is +-(a difference of value-word
  Converts minus V_alpha), and V_alpha is a sum of such differences;
* one party's DPF and DCF output shares at random points;
* Z_2 (one-hot mode): the final correction bit of a DPF and every V_CW bit and
  the final bit of a DCF are balanced across keys;
* the masks r and their additive shares in the masked-mode token and in the
  fresh-key token.

Each pin is also shown to fail on a mistake planted in the oracle on purpose
(oracle.test_plant): a constant Convert, a Convert that reads the cleared
control bit, and a mask share read from r's own bytes.
"""
import math
import struct

import numpy as np
import pytest

import oracle
import workload as W

M32 = 0xFFFFFFFF


def uniform_u32(words) -> bool:
    """Every bit balanced within 5 sigma, and the low and high bytes pass a chi-square test
    (256 bins, within 6 sigma of the 255 degrees of freedom)."""
    w = np.asarray(words, dtype=np.uint64)
    n = len(w)
    assert n >= 1024
    sig = math.sqrt(n) / 2
    for i in range(32):
        if abs(int(((w >> i) & 1).sum()) - n / 2) > 5 * sig:
            return False
    for shift in (0, 24):
        counts = np.bincount(((w >> shift) & 0xFF).astype(np.int64), minlength=256)
        exp = n / 256
        chi2 = float(((counts - exp) ** 2 / exp).sum())
        if abs(chi2 - 255) > 6 * math.sqrt(2 * 255):
            return False
    return True


def balanced(bits) -> bool:
    b = np.asarray(bits, dtype=np.int64)
    return abs(int(b.sum()) - len(b) / 2) <= 5 * math.sqrt(len(b)) / 2


def _seeds(g):
    return bytes(g.integers(0, 256, 16, dtype=np.uint8)), bytes(g.integers(0, 256, 16, dtype=np.uint8))


def _u32(key, off):
    return struct.unpack_from("<I", key, off)[0]


def _planted(mode, fn):
    oracle.test_plant(mode)
    try:
        return fn()
    finally:
        oracle.test_plant(oracle.PLANT_NONE)


# ---------------------------------------------------------------- Z_{2^32}

def _dpf_final_words(group=0, beta=0, n=4, keys=4096, alpha=5):
    g = np.random.default_rng(11)
    gen = oracle.dpf_gen if group == 0 else (lambda n_, a, b, s0, s1: oracle.dpf_gen_z2(n_, a, s0, s1))
    out = []
    for _ in range(keys):
        k0, _k1 = gen(n, alpha, beta, *_seeds(g))
        out.append(_u32(k0, 24 + 20 * n))
    return out


def _dcf_vcw_words(group=0, beta=0, n=8, keys=1024, alpha=0x5A):
    """V_CW of every level of `keys` DCF keys with fixed (alpha, beta): array [keys][n], and the
    final words [keys]."""
    g = np.random.default_rng(12)
    gen = oracle.dcf_gen if group == 0 else (lambda n_, a, b, s0, s1: oracle.dcf_gen_z2(n_, a, s0, s1))
    v, fin = [], []
    for _ in range(keys):
        k0, _k1 = gen(n, alpha, beta, *_seeds(g))
        v.append([_u32(k0, 24 + 24 * (l - 1) + 20) for l in range(1, n + 1)])
        fin.append(_u32(k0, 24 + 24 * n))
    return np.array(v, dtype=np.uint64), np.array(fin, dtype=np.uint64)


def test_dpf_seed_convert_is_uniform():
    assert uniform_u32(_dpf_final_words())


@pytest.mark.parametrize("mode", [oracle.PLANT_CONST, oracle.PLANT_CLEARED_BIT])
def test_dpf_seed_convert_pin_catches_a_bad_convert(mode):
    assert not _planted(mode, lambda: uniform_u32(_dpf_final_words()))


def test_dcf_value_convert_is_uniform():
    v, fin = _dcf_vcw_words()
    assert uniform_u32(v.ravel())
    for level in range(v.shape[1]):
        assert balanced(v[:, level] & 1) and balanced(v[:, level] >> 31), level
    assert uniform_u32(fin)


@pytest.mark.parametrize("mode", [oracle.PLANT_CONST, oracle.PLANT_CLEARED_BIT])
def test_dcf_value_convert_pin_catches_a_bad_convert(mode):
    v, _ = _planted(mode, _dcf_vcw_words)
    assert not uniform_u32(v.ravel())


def _single_party_outputs(kind, beta, n=12, keys=8, points=512):
    g = np.random.default_rng(13 + kind)
    gen = oracle.dpf_gen if kind == oracle.KIND_DPF else oracle.dcf_gen
    out = []
    for _ in range(keys):
        alpha = int(g.integers(0, 1 << n))
        k0, _k1 = gen(n, alpha, beta, *_seeds(g))
        xs = g.integers(0, 1 << n, points)
        out.extend(int(y) for y in oracle.eval_many(k0, xs, kind))
    return out


# beta even: with an odd beta the correction word is odd too, and t * CW would refill the
# low bit that a cleared-bit Convert leaves empty
@pytest.mark.parametrize("beta", [0x12345678, 0xAAAAAAAB])
@pytest.mark.parametrize("kind", [oracle.KIND_DPF, oracle.KIND_DCF])
def test_one_party_shares_are_uniform(kind, beta):
    assert uniform_u32(_single_party_outputs(kind, beta))


@pytest.mark.parametrize("mode", [oracle.PLANT_CONST, oracle.PLANT_CLEARED_BIT])
def test_one_party_share_pin_catches_a_bad_convert_dpf(mode):
    assert not _planted(mode, lambda: uniform_u32(_single_party_outputs(oracle.KIND_DPF, 0x12345678)))


# ---------------------------------------------------------------- Z_2 (one-hot mode)

def test_z2_dpf_final_bit_is_balanced():
    assert balanced(_dpf_final_words(group=1, beta=1, n=6))


@pytest.mark.parametrize("mode", [oracle.PLANT_CONST, oracle.PLANT_CLEARED_BIT])
def test_z2_dpf_pin_catches_a_bad_convert(mode):
    assert not _planted(mode, lambda: balanced(_dpf_final_words(group=1, beta=1, n=6)))


def _z2_dcf_balanced(v, fin):
    return all(balanced(v[:, level]) for level in range(v.shape[1])) and balanced(fin)


def test_z2_dcf_value_and_seed_converts_are_balanced():
    v, fin = _dcf_vcw_words(group=1, beta=1)
    assert set(np.unique(v)) <= {0, 1} and set(np.unique(fin)) <= {0, 1}
    assert _z2_dcf_balanced(v, fin)


@pytest.mark.parametrize("mode", [oracle.PLANT_CONST, oracle.PLANT_CLEARED_BIT])
def test_z2_dcf_pin_catches_a_bad_convert(mode):
    v, fin = _planted(mode, lambda: _dcf_vcw_words(group=1, beta=1))
    assert not _z2_dcf_balanced(v, fin)


# ---------------------------------------------------------------- mask words

def _token_masks(n_tokens=48, per=48):
    """(r, <r>_1, <r>_2, <r>_3) of many masked-mode predicates, read from the three tokens'
    24-byte records: server i's record holds <r>_i at byte 8 and <r>_{i+1} at byte 12."""
    rs = []
    preds = [W.eq_pred(0, 0, 0, 7)] * per
    dpf = oracle.key_len(oracle.KIND_DPF, 32)
    for t in range(n_tokens):
        toks = oracle.keygen(preds, 32, struct.pack("<QQ", t, 99))
        for p in range(per):
            off = 16 + p * (24 + 2 * dpf)
            sh = [_u32(toks[i], off + 8) for i in range(3)]
            assert _u32(toks[0], off + 12) == sh[1]
            rs.append(((sum(sh)) & M32, *sh))
    return np.array(rs, dtype=np.uint64)


def _fresh_masks(N=2048):
    preds = [W.eq_pred(0, 0, 0, 7)]
    toks = oracle.keygen_fresh(preds, 32, [N], bytes(range(7, 23)))
    d = toks[0][64:96]
    off = struct.unpack_from("<Q", d, 16)[0]
    lay = oracle.fresh_layout(oracle.PRED_EQ, 32, N)
    sh = [np.frombuffer(toks[i], dtype=np.uint32, count=N, offset=off + lay["rA"]).astype(np.uint64)
          for i in range(3)]
    r = (sh[0] + sh[1] + sh[2]) & M32
    return np.stack([r, *sh], axis=1)


def _masks_ok(m):
    r, r1, r2, r3 = (m[:, j] for j in range(4))
    return all(uniform_u32(x) for x in (r, r1, r2, r3, (r - r1) & M32, (r1 - r2) & M32))


@pytest.mark.parametrize("source", [_token_masks, _fresh_masks])
def test_mask_words_are_uniform_and_unrelated(source):
    assert _masks_ok(source())


@pytest.mark.parametrize("mode", [oracle.PLANT_CONST, oracle.PLANT_MASK_OVERLAP])
@pytest.mark.parametrize("source", [_token_masks, _fresh_masks])
def test_mask_pin_catches_a_bad_extraction(source, mode):
    assert not _planted(mode, lambda: _masks_ok(source()))
