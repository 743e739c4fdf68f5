"""Pins for the oracle's fresh-key mode (Sec. V-C, one mask and one key triple per value).

* the three share sets reconstruct to the plaintext AND of the group's
  predicates on every element (Def. 2), for equality and for ranges whose
  shifted bounds wrap around 2^n (the c * beta' term);
* the token's mask fields and root seeds are the AES blocks of the client
  seed that the definition names (re-derived here with FIPS-197 AES);
* a key pair read back from the token layout by this test (not by the C code)
  reconstructs beta' at the element's shifted point and 0 elsewhere;
* equal attribute values open to different masked values (no shared mask);
* the token-free computation from the seed equals the token path.
"""
import struct

import numpy as np
import pytest

import oracle
import workload as W

PRF = bytes(range(48))
SEED = bytes(range(50, 66))
BETA = 0xAAAAAAAB
M32 = 0xFFFFFFFF


def _block(c, p, tag, j):
    return struct.pack("<QHHI", c, p, tag, j)


def _aes_words(c, p, tag, j):
    return struct.unpack("<4I", oracle.aes128(SEED, _block(c, p, tag, j)))


def _setup(n_elems=240, bits=9, seed=3):
    g = W.rng(seed)
    vals = W.uniform_attrs(g, 3, n_elems, bits)
    vals[2, : n_elems // 2] = 17                       # many equal values on attribute 2
    t = W.table(vals, bits, g)
    return vals, t


def _desc(tok, p):
    d = tok[64 + 32 * p: 96 + 32 * p]
    kind, n, table, attr, group = struct.unpack("<BBHHH", d[:8])
    N, off = struct.unpack("<QQ", d[8:24])
    return kind, n, table, attr, group, N, off


def test_fresh_reconstructs_plaintext_and():
    vals, t = _setup()
    bits = 9
    top = (1 << bits) - 1
    preds = [W.range_pred(0, 0, 0, 100, 400), W.eq_pred(0, 2, 0, 17),        # group 0: range AND eq
             W.range_pred(0, 1, 1, 0, top), W.range_pred(0, 0, 1, 37, 38),    # group 1: full domain AND narrow
             W.eq_pred(0, 1, 2, int(vals[1, 5]))]
    toks = oracle.keygen_fresh(preds, bits, [vals.shape[1]], SEED)
    assert all(len(x) == oracle.fresh_token_len(preds, bits, [vals.shape[1]]) for x in toks)
    for grp in range(3):
        out = oracle.filter_fresh(toks, 4, PRF, [(t["shares"], bits)], grp, np.arange(vals.shape[1]))
        want = oracle.plain_group(preds, grp, t["values"])
        assert np.array_equal(oracle.reconstruct(out), want), grp
    # group 0 has hits and misses
    w0 = oracle.plain_group(preds, 0, t["values"])
    assert 0 < int(w0.sum()) < len(w0)


def test_fresh_wrapping_ranges_use_c_beta():
    # every element's own mask makes a1 = hi + 1 + r wrap below a0 = lo + r for some
    # elements and not others: both branches must give the right bit
    vals, t = _setup(n_elems=300, seed=4)
    bits = 9
    preds = [W.range_pred(0, 0, 0, 50, 460)]
    toks = oracle.keygen_fresh(preds, bits, [300], SEED)
    kind, n, _, _, _, N, off = _desc(toks[0], 0)
    lay = oracle.fresh_layout(kind, n, N)
    cb = np.frombuffer(toks[0], dtype=np.uint32, count=N, offset=off + lay["cb"])
    assert set(np.unique(cb)) == {0, BETA}                     # both cases occur
    out = oracle.filter_fresh(toks, 1, PRF, [(t["shares"], bits)], 0, np.arange(300))
    assert np.array_equal(oracle.reconstruct(out), oracle.plain_group(preds, 0, t["values"]))


def test_fresh_mask_fields_follow_the_client_blocks():
    vals, _ = _setup()
    bits = 9
    m = (1 << bits) - 1
    preds = [W.eq_pred(0, 0, 0, 3), W.range_pred(0, 1, 0, 10, 20)]
    toks = oracle.keygen_fresh(preds, bits, [vals.shape[1]], SEED)
    for p in range(2):
        kind, n, _, _, _, N, off = _desc(toks[0], p)
        lay = oracle.fresh_layout(kind, n, N)
        rA = [np.frombuffer(tk, dtype=np.uint32, count=N, offset=off + lay["rA"]) for tk in toks]
        rB = [np.frombuffer(tk, dtype=np.uint32, count=N, offset=off + lay["rB"]) for tk in toks]
        for c in (0, 1, 77, N - 1):
            w = _aes_words(c, p, 1, 0)
            assert rA[0][c] == w[1] & m and rA[1][c] == w[2] & m
            assert (int(rA[0][c]) + int(rA[1][c]) + int(rA[2][c])) & m == w[0] & m
            for i in range(3):
                assert rB[i][c] == rA[(i + 1) % 3][c]


def _key_from_layout(tok, p, half, sub, c, party):
    """Rebuild the wire-format key of element c from the token bytes (test-side reader)."""
    kind, n, _, _, _, N, off = _desc(tok, p)
    lay = oracle.fresh_layout(kind, n, N)
    nsub = 1 if kind == oracle.PRED_EQ else 2
    kkind = oracle.KIND_DPF if kind == oracle.PRED_EQ else oracle.KIND_DCF
    base = off + lay["keys_at"] + (half * nsub + sub) * lay["key_block"]
    N4 = lay["N4"]
    seed = tok[base + 16 * c: base + 16 * c + 16]
    scw0 = base + 16 * N
    tl0 = scw0 + 16 * n * N
    tr0 = tl0 + 4 * N4
    vcw0 = tr0 + 4 * N4
    cw0 = vcw0 + (4 * n * N4 if kkind == oracle.KIND_DCF else 0)
    tl = struct.unpack_from("<I", tok, tl0 + 4 * c)[0]
    tr = struct.unpack_from("<I", tok, tr0 + 4 * c)[0]
    key = bytearray(struct.pack("<BBBB4x", kkind, n, party, 0) + seed)
    for lv in range(n):
        key += tok[scw0 + 16 * (lv * N + c): scw0 + 16 * (lv * N + c) + 16]
        key += bytes([(tl >> lv) & 1, (tr >> lv) & 1, 0, 0])
        if kkind == oracle.KIND_DCF:
            key += tok[vcw0 + 4 * (lv * N4 + c): vcw0 + 4 * (lv * N4 + c) + 4]
    key += tok[cw0 + 4 * c: cw0 + 4 * c + 4]
    return bytes(key), kkind, seed


@pytest.mark.parametrize("kind", ["eq", "range"])
def test_fresh_key_pair_from_layout_reconstructs(kind):
    vals, _ = _setup()
    bits = 9
    m = (1 << bits) - 1
    pred = W.eq_pred(0, 0, 0, 300) if kind == "eq" else W.range_pred(0, 0, 0, 40, 90)
    toks = oracle.keygen_fresh([pred], bits, [vals.shape[1]], SEED)
    pts = np.arange(1 << bits, dtype=np.uint32)
    for c in (0, 5, 239):
        r = _aes_words(c, 0, 1, 0)[0] & m
        # pair 1 (index 0): party 0 is CS1's half A, party 1 is CS3's half B
        for sub in range(1 if kind == "eq" else 2):
            k0, kk, s0 = _key_from_layout(toks[0], 0, 0, sub, c, 0)
            k1, _, s1 = _key_from_layout(toks[2], 0, 1, sub, c, 1)
            assert s0 == oracle.aes128(SEED, _block(c, 0, 2, 0 + 2 * sub))      # root seeds per definition
            assert s1 == oracle.aes128(SEED, _block(c, 0, 2, 1 + 2 * sub))
            rec = (oracle.eval_many(k0, pts, kk).astype(np.uint64) + oracle.eval_many(k1, pts, kk)) & M32
            if kind == "eq":
                want = np.where(pts == ((300 + r) & m), BETA, 0)
            else:
                a = ((91 + r) & m) if sub == 0 else ((40 + r) & m)
                b = BETA if sub == 0 else (-BETA) & M32
                want = np.where(pts < a, b, 0)
            assert np.array_equal(rec, want), (c, sub)


def test_fresh_masks_hide_equal_values():
    vals, t = _setup()
    bits = 9
    m = (1 << bits) - 1
    preds = [W.eq_pred(0, 2, 0, 17)]
    toks = oracle.keygen_fresh(preds, bits, [vals.shape[1]], SEED)
    kind, n, _, _, _, N, off = _desc(toks[0], 0)
    lay = oracle.fresh_layout(kind, n, N)
    rA = [np.frombuffer(tk, dtype=np.uint32, count=N, offset=off + lay["rA"]).astype(np.uint64)
          for tk in toks]
    xs = [s[2].astype(np.uint64) for s in t["shares"]]
    xhat = (xs[0] + xs[1] + xs[2] + rA[0] + rA[1] + rA[2]) & m
    same = np.flatnonzero(vals[2] == 17)
    assert len(same) >= 100
    assert len(np.unique(xhat[same])) > 0.5 * len(same)     # masks differ per element
    # and the masked values still open to x + r
    r = np.array([_aes_words(int(c), 0, 1, 0)[0] & m for c in same], dtype=np.uint64)
    assert np.array_equal(xhat[same], (17 + r) & m)


def test_fresh_direct_equals_token_path():
    vals, t = _setup(n_elems=120, seed=8)
    bits = 9
    preds = [W.range_pred(0, 0, 0, 3, 300), W.eq_pred(0, 2, 0, 17), W.range_pred(0, 1, 1, 200, 511)]
    toks = oracle.keygen_fresh(preds, bits, [120], SEED)
    for grp in (0, 1):
        a = oracle.filter_fresh(toks, 9, PRF, [(t["shares"], bits)], grp, np.arange(120))
        b = oracle.fresh_direct(preds, bits, SEED, 9, PRF, [(t["shares"], bits)], grp, np.arange(120), threads=2)
        assert np.array_equal(a, b)


def test_fresh_rejects_bad_predicates():
    with pytest.raises(ValueError):
        oracle.fresh_token_len([W.range_pred(0, 0, 0, 5, 4)], 8, [10])
    with pytest.raises(ValueError):
        oracle.fresh_token_len([W.eq_pred(1, 0, 0, 5)], 8, [10])        # table 1 of 1
