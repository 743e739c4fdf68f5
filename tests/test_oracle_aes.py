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


def test_sbox_entries_printed_in_fips197():
    # the oracle derives its S-box from the GF(2^8) inverse and the affine map; the entries
    # FIPS-197 prints (Sec. 5.1.1's worked example, rows 0 and f of Fig. 7) pin that derivation
    rows = _rows("fips197_sbox_points.txt")
    assert len(rows) == 33
    for x, y in rows:
        assert oracle.sbox(int(x, 16)) == int(y, 16), x


def test_sbox_is_a_permutation_without_fixed_points():
    # properties the AES S-box was designed with (FIPS-197 Sec. 5.1.1: the affine constant
    # makes S(a) != a and S(a) != ~a for every byte a); a wrong affine map or inverse breaks them
    s = [oracle.sbox(a) for a in range(256)]
    assert sorted(s) == list(range(256))
    assert all(s[a] != a and s[a] != a ^ 0xFF for a in range(256))


def test_prg_fixed_key_is_mmo_of_fips_vector():
    # K_L = 00 01 .. 0f is the FIPS-197 Appendix C.1 key, so H_{K_L}(p) = AES(p) xor p
    key, pt, ct = _rows("fips197_aes128.txt")[0]
    want = bytes(a ^ b for a, b in zip(bytes.fromhex(ct), bytes.fromhex(pt)))
    assert oracle.prg(0, bytes.fromhex(pt)) == want


def test_prg_keys_are_distinct():
    s = bytes(range(100, 116))
    outs = {oracle.prg(w, s) for w in range(4)}
    assert len(outs) == 4
