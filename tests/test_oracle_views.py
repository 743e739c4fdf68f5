"""Per-server views (Sec. V-C half assignment, Sec. III-B re-share): what each server's
output depends on.

CS_i holds key halves of its own token only, share sets i and i+1, and PRF keys
k_i and k_{i-1}.  The oracle's per-server results must not move when anything
outside that view changes:
* z_i (Eq. predEval, masked form) is unchanged when the other two servers' key
  halves are corrupted, and changes when its own are;
* the re-shared r_i is unchanged when k_{i+1} (the key CS_i does not hold)
  changes;
* one-hot mode: for a one-predicate group, CS_i's output share is unchanged when
  share set i+2 and the other servers' key halves are replaced.
The masked open of x^ reads every share by design (it is the protocol's open
step), so the masked-mode checks fix x^ and vary the keys.
"""
import numpy as np
import pytest

import oracle
import workload as W

PRF = bytes(range(48))


def _key_spans(tok, n):
    """(start, length) of every key in a token, after its 8-byte header (a one-hot token,
    group byte 1, holds early-terminated keys)."""
    spans = []
    off = 16
    klen = oracle.key_len_et if tok[7] == 1 else oracle.key_len
    dpf, dcf = klen(oracle.KIND_DPF, n), klen(oracle.KIND_DCF, n)
    while off < len(tok):
        kind = tok[off]
        keys = [dpf, dpf] if kind == oracle.PRED_EQ else [dcf] * 4
        k = off + 24
        for L in keys:
            spans.append((k + 8, L - 8))
            k += L
        off = k
    return spans


def _corrupt(tok, n, g):
    b = bytearray(tok)
    for s, L in _key_spans(tok, n):
        b[s:s + L] = bytes(g.integers(0, 256, L, dtype=np.uint8))
    return bytes(b)


@pytest.mark.parametrize("pred", [W.eq_pred(0, 0, 0, 77), W.range_pred(0, 0, 0, 10, 200)])
def test_z_i_reads_only_its_own_key_halves(pred):
    n = 8
    g = np.random.default_rng(3)
    toks = oracle.keygen([pred], n, bytes(range(16)))
    for xhat in (0, 77, 150, 255):
        z, _ = oracle.pred_z(toks, 0, xhat)
        for i in range(3):
            mixed = [toks[j] if j == i else _corrupt(toks[j], n, g) for j in range(3)]
            zi, _ = oracle.pred_z(mixed, 0, xhat)
            assert zi[i] == z[i], (i, xhat)
            own = [_corrupt(toks[j], n, g) if j == i else toks[j] for j in range(3)]
            zo, _ = oracle.pred_z(own, 0, xhat)
            assert zo[i] != z[i], (i, xhat)   # its own halves matter


def test_reshare_r_i_does_not_read_k_next():
    z = [11, 22, 33]
    base = oracle.reshare(PRF, z, 5, 3, 1, 9)
    for i in range(3):
        keys = bytearray(PRF)
        nxt = (i + 1) % 3
        keys[16 * nxt:16 * nxt + 16] = bytes(range(200, 216))
        out = oracle.reshare(bytes(keys), z, 5, 3, 1, 9)
        assert out[i] == base[i]
        assert out[nxt] != base[nxt] or out[(i + 2) % 3] != base[(i + 2) % 3]


def test_onehot_output_share_reads_only_its_view():
    n, N = 5, 40
    g = W.rng(11)
    vals = W.uniform_attrs(g, 1, N, n)
    tab = W.onehot_table(vals, n, g)
    preds = [W.range_pred(0, 0, 0, 3, 20)]
    toks = oracle.keygen_onehot(preds, n, bytes(range(16)))
    base = oracle.filter_onehot(toks, 2, PRF, [(tab["shares"], n)], 0, np.arange(N))
    gg = np.random.default_rng(4)
    for i in range(3):
        other = (i + 2) % 3
        shares = [s.copy() for s in tab["shares"]]
        shares[other] = gg.integers(0, 1 << 32, shares[other].shape, dtype=np.uint64).astype(np.uint32)
        mixed = [toks[j] if j == i else _corrupt(toks[j], n, gg) for j in range(3)]
        got = oracle.filter_onehot(mixed, 2, PRF, [(shares, n)], 0, np.arange(N))
        assert np.array_equal(got[i], base[i]), i
