"""The three secEval modes on the GPU answer the same question.

One plaintext table, loaded as additive shares (masked and fresh-key modes) and
as binary-RSS one-hot vectors (one-hot mode); one predicate list with equality,
ranges (including one touching the top of the domain and one wrapping the
shifted bounds), and ANDs.  The reconstructed bits of the per-predicate-mask
mode, the fresh-key mode and the one-hot mode (the paper's secEval as written)
are equal to each other and to the plaintext, on every element.
"""
import numpy as np
import pytest

import oracle
import workload as W
from tests._helpers import PRF, from_dev, to_dev

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2209_03526_gb300")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = P.Context(0, prf_keys=PRF)
    yield c
    c.close()


def _unpack(words, n):
    w = np.asarray(words, dtype=np.uint32)
    return ((w[:, None] >> np.arange(32, dtype=np.uint32)) & 1).reshape(-1)[:n]


@pytest.mark.parametrize("n,n_elems", [(8, 5000), (12, 2049)])
def test_masked_fresh_and_onehot_modes_agree(ctx, n, n_elems):
    g = W.rng(500 + n)
    top = (1 << n) - 1
    vals = W.uniform_attrs(g, 2, n_elems, n)
    vals[0, ::7] = 5
    preds = [W.eq_pred(0, 0, 0, 5), W.range_pred(0, 1, 0, top // 3, top),
             W.range_pred(0, 1, 1, 1, top - 1), W.range_pred(0, 0, 1, top // 8, top // 2),
             W.eq_pred(0, 1, 2, int(vals[1, 11]))]
    n_groups = 3
    plain = [oracle.plain_group(preds, grp, vals) for grp in range(n_groups)]

    add = W.table(vals, n, g)
    ctx.load_shares(0, [to_dev(s) for s in add["shares"]], n)
    outs = [[torch.empty(n_elems, dtype=torch.int32, device="cuda") for _ in range(3)] for _ in range(n_groups)]
    ctx.filter_and_combine(3, P.keygen(preds, n, bytes(range(16))), outs)
    ctx.sync()
    masked = [oracle.reconstruct(np.stack([from_dev(t) for t in grp])) for grp in outs]

    L = P.fresh_token_size(preds, n, [n_elems])
    toks = [torch.zeros(L, dtype=torch.uint8, device="cuda") for _ in range(3)]
    ctx.keygen_fresh(preds, n, [n_elems], bytes(range(1, 17)), toks)
    fouts = [[torch.empty(n_elems, dtype=torch.int32, device="cuda") for _ in range(3)] for _ in range(n_groups)]
    ctx.filter_fresh(4, toks, fouts)
    ctx.sync()
    fresh = [oracle.reconstruct(np.stack([from_dev(t) for t in grp])) for grp in fouts]

    hot = W.onehot_table(vals, n, g)
    ctx.load_onehot(0, [to_dev(s) for s in hot["shares"]], n)
    words = (n_elems + 31) // 32
    houts = [[torch.empty(words, dtype=torch.int32, device="cuda") for _ in range(3)] for _ in range(n_groups)]
    ctx.filter_onehot(5, P.keygen_onehot(preds, n, bytes(range(2, 18))), houts)
    ctx.sync()
    onehot = [oracle.reconstruct_bits(np.stack([_unpack(from_dev(t), n_elems) for t in grp])) for grp in houts]

    for grp in range(n_groups):
        assert np.array_equal(masked[grp], plain[grp]), grp
        assert np.array_equal(fresh[grp], plain[grp]), grp
        assert np.array_equal(onehot[grp], plain[grp]), grp
        assert 0 < int(plain[grp].sum()) < n_elems
