"""Pins for the oracle's AES-128 and PRG against FIPS-197's printed vectors."""
import os

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [l.split() for l in f if l.strip() and not l.startswith("#")]


def test_fips197_known_answers():
    rows = _rows("fips197_aes128.txt")
    assert len(rows) == 2
    for key, pt, ct in rows:
        assert oracle.aes128(bytes.fromhex(key), bytes.fromhex(pt)).hex() == ct


def test_sbox_points_through_one_round_structure():
    # The S-box is derived from GF(2^8) inversion + the affine map.  Pin single entries by
    # encrypting with a key chosen so the first SubBytes sees the wanted byte is impractical;
    # instead check the S-box indirectly: AES is a permutation, and the printed entries are
    # used by FIPS-197's own key-expansion example (Appendix A.1), which the KAT above covers.
    rows = _rows("fips197_sbox_points.txt")
    assert ("53", "ed") in [tuple(r) for r in rows]
    # permutation property on 256 distinct single-byte-varied plaintexts
    key = bytes(range(16))
    outs = {oracle.aes128(key, bytes([b]) + bytes(15)) for b in range(256)}
    assert len(outs) == 256


def test_prg_fixed_key_is_mmo_of_fips_vector():
    # K_L = 00 01 .. 0f is the FIPS-197 Appendix C.1 key, so H_{K_L}(p) = AES(p) xor p
    key, pt, ct = _rows("fips197_aes128.txt")[0]
    want = bytes(a ^ b for a, b in zip(bytes.fromhex(ct), bytes.fromhex(pt)))
    assert oracle.prg(0, bytes.fromhex(pt)) == want


def test_prg_keys_are_distinct():
    s = bytes(range(100, 116))
    outs = {oracle.prg(w, s) for w in range(4)}
    assert len(outs) == 4
