"""GPU parity of secShuffle (Alg. 5) and secFetch case II (Alg. 4).

* the three output share sets equal the oracle's bit for bit, for XOR and
  additive shares, 1 to 13 words per row, 1 to 4,099 rows;
* at 1,048,576 rows x 6 words: the reconstruction is the input moved by the
  composed permutation (sampled rows, permutation from the oracle) and, for
  every row, the same multiset of rows;
* secFetch case II equals the oracle's records and count, in the same order;
  a GPU filter followed by the GPU fetch returns exactly the plaintext matches;
  no match, a cap below the count, one row.
"""
import numpy as np
import pytest

import oracle
import workload as W
from tests._helpers import PRF, from_dev, to_dev

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2209_03526_gb300")

SEEDS = bytes(range(100, 148))


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = P.Context(0, prf_keys=PRF)
    yield c
    c.close()


def _dev2(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).cuda()


def _host(t):
    return t.cpu().numpy().view(np.uint32)


def _shares(g, n, w, group):
    d = g.integers(0, 1 << 32, (n, w), dtype=np.uint64).astype(np.uint32)
    s1 = g.integers(0, 1 << 32, (n, w), dtype=np.uint64).astype(np.uint32)
    s2 = g.integers(0, 1 << 32, (n, w), dtype=np.uint64).astype(np.uint32)
    s3 = (d ^ s1 ^ s2) if group == oracle.SHUF_XOR else (d - s1 - s2)
    return d, [s1, s2, s3]


def _gpu_shuffle(ctx, sh, group):
    ins = [_dev2(s) for s in sh]
    outs = [torch.empty_like(ins[0]) for _ in range(3)]
    ctx.shuffle(ins, SEEDS, outs, group=group)
    ctx.sync()
    return [_host(o) for o in outs]


@pytest.mark.parametrize("group", [oracle.SHUF_ADD, oracle.SHUF_XOR])
@pytest.mark.parametrize("n,w", [(1, 1), (2, 5), (1000, 6), (4099, 13), (513, 4)])
def test_shuffle_equals_oracle(ctx, group, n, w):
    g = W.rng(n + 7 * w + group)
    _, sh = _shares(g, n, w, group)
    got = _gpu_shuffle(ctx, sh, group)
    want = oracle.shuffle(sh, SEEDS, group)
    for j in range(3):
        assert np.array_equal(got[j], want[j]), j


def test_shuffle_full_size_properties(ctx):
    g = W.rng(31)
    n, w = 1 << 20, 6
    d, sh = _shares(g, n, w, oracle.SHUF_ADD)
    got = _gpu_shuffle(ctx, sh, oracle.SHUF_ADD)
    rec = got[0] + got[1] + got[2]
    for i in list(g.choice(n, 200, replace=False)) + [0, n - 1]:
        i = int(i)
        j = oracle.prp(SEEDS[0:16], n, i)
        k = oracle.prp(SEEDS[32:48], n, j)
        l = oracle.prp(SEEDS[16:32], n, k)
        assert np.array_equal(rec[l], d[i]), i
    # all rows: the same multiset (sort rows lexicographically)
    key = lambda a: a[np.lexsort(a.T[::-1])]
    assert np.array_equal(key(rec), key(d))


def _filter_shares(g, flags):
    x = flags.astype(np.uint32)
    s1 = g.integers(0, 1 << 32, len(x), dtype=np.uint64).astype(np.uint32)
    s2 = g.integers(0, 1 << 32, len(x), dtype=np.uint64).astype(np.uint32)
    return [s1, s2, x - s1 - s2]


def _gpu_fetch(ctx, xs, attrs, cap):
    outs = [torch.zeros((max(cap, 1), 1 + len(attrs)), dtype=torch.int32, device="cuda") for _ in range(3)]
    m = ctx.fetch_multi(0, [to_dev(x) for x in xs], attrs, SEEDS, [o[:cap] for o in outs])
    return m, [_host(o[:min(m, cap)]) for o in outs]


def test_fetch_multi_equals_oracle(ctx):
    g = W.rng(32)
    n, bits = 5003, 16
    vals = W.uniform_attrs(g, 4, n, bits)
    t = W.table(vals, bits, g)
    ctx.load_shares(0, [to_dev(s) for s in t["shares"]], bits)
    flags = vals[2] < 6000
    xs = _filter_shares(g, flags)
    m, rows = _gpu_fetch(ctx, xs, [3, 0, 2], cap=n)
    wm, wrows = oracle.fetch_multi(xs, (t["shares"], bits), [3, 0, 2], SEEDS, cap=n)
    assert m == wm == int(flags.sum())
    for j in range(3):
        assert np.array_equal(rows[j], wrows[j]), j


def test_filter_then_fetch_returns_the_plaintext_matches(ctx):
    g = W.rng(33)
    n, bits = 200_000, 32
    vals = W.uniform_attrs(g, 3, n, bits)
    vals[1, ::1000] = 4242
    t = W.table(vals, bits, g)
    ctx.load_shares(0, [to_dev(s) for s in t["shares"]], bits)
    preds = [W.eq_pred(0, 1, 0, 4242)]
    toks = P.keygen(preds, bits, bytes(range(16)))
    x = [torch.empty(n, dtype=torch.int32, device="cuda") for _ in range(3)]
    ctx.filter_and_combine(5, toks, [x])
    ctx.sync()
    m, rows = _gpu_fetch(ctx, [from_dev(v) for v in x], [0, 2], cap=1000)
    match = np.flatnonzero(vals[1] == 4242)
    assert m == len(match)
    rec = (rows[0].astype(np.uint64) + rows[1] + rows[2]) & 0xFFFFFFFF
    got = sorted(map(tuple, rec.tolist()))
    assert got == sorted((int(c), int(vals[0, c]), int(vals[2, c])) for c in match)


def test_fetch_multi_edges(ctx):
    g = W.rng(34)
    n, bits = 777, 8
    vals = W.uniform_attrs(g, 1, n, bits)
    t = W.table(vals, bits, g)
    ctx.load_shares(0, [to_dev(s) for s in t["shares"]], bits)
    m, _ = _gpu_fetch(ctx, _filter_shares(g, np.zeros(n, dtype=bool)), [0], cap=10)
    assert m == 0
    flags = np.zeros(n, dtype=bool)
    flags[[0, 5, 300, 776]] = True
    xs = _filter_shares(g, flags)
    m, rows = _gpu_fetch(ctx, xs, [0], cap=2)
    wm, wrows = oracle.fetch_multi(xs, (t["shares"], bits), [0], SEEDS, cap=2)
    assert m == wm == 4
    for j in range(3):
        assert np.array_equal(rows[j], wrows[j])
    one = W.table(np.array([[9]], dtype=np.uint32), bits, g)
    ctx.load_shares(0, [to_dev(s) for s in one["shares"]], bits)
    m, rows = _gpu_fetch(ctx, _filter_shares(g, np.ones(1, dtype=bool)), [0], cap=1)
    assert m == 1
    rec = (rows[0].astype(np.uint64) + rows[1] + rows[2]) & 0xFFFFFFFF
    assert int(rec[0, 0]) == 0 and int(rec[0, 1]) % 256 == 9


def test_shuffle_rejects_bad_arguments(ctx):
    a = _dev2(np.zeros((4, 3), dtype=np.uint32))
    with pytest.raises(P.OblivgmError):
        ctx.shuffle([a, a, a], SEEDS, [torch.empty_like(a) for _ in range(3)], group=7)
    big = _dev2(np.zeros((2, 65), dtype=np.uint32))
    with pytest.raises(P.OblivgmError):
        ctx.shuffle([big, big, big], SEEDS, [torch.empty_like(big) for _ in range(3)])
