"""GPU parity on a table past 2^32 elements: 64-bit element indices end to end.

4,294,967,309 elements (2^32 + 13, a ragged tail past the 32-bit boundary) of one 16-bit
attribute; one group of two equality predicates joined by OR (Sec. V-D), so every element
runs the predicate's re-share and the fold's re-share, whose PRF counter carries the 64-bit
element index (its high word is 1 past 2^32).  Every element must reconstruct to the
plaintext predicate (Def. 2), and sampled elements -- both sides of 2^31 and 2^32 and of the
tile boundaries there, the ends, the planted matches and random ones -- must equal the oracle
share for share (integer work: bit-exact).

The shares are drawn on the device from a seeded generator (the sizes are the point; the
values are uniform); the oracle reads the sampled elements from host arrays that hold only
those elements (the rest of each array is never touched).
"""
import numpy as np
import pytest

import oracle
import workload as W
from tests._helpers import PRF

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2209_03526_gb300")

N = (1 << 32) + 13
BITS = 16
CHUNK = 1 << 28
# x, three share sets, the library's resident copy of them, three outputs: 4 bytes each,
# plus room for the chunked int64 temporaries
NEED_BYTES = 10 * N * 4 + (8 << 30)


def _u32(t):
    return t.cpu().numpy().view(np.uint32)


def test_table_past_2_pow_32_elements():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    free, _ = torch.cuda.mem_get_info()
    if free < NEED_BYTES:
        pytest.skip(f"needs {NEED_BYTES / 2**30:.0f} GiB of free device memory, {free / 2**30:.0f} GiB free")
    dev = torch.device("cuda", 0)
    gen = torch.Generator(device=dev)
    gen.manual_seed(97)
    x = torch.randint(0, 1 << BITS, (N,), dtype=torch.int32, device=dev, generator=gen)
    s0 = torch.randint(-(1 << 31), 1 << 31, (N,), dtype=torch.int32, device=dev, generator=gen)
    s1 = torch.randint(-(1 << 31), 1 << 31, (N,), dtype=torch.int32, device=dev, generator=gen)
    s2 = torch.empty_like(x)
    for lo in range(0, N, CHUNK):
        hi = min(N, lo + CHUNK)
        t = (x[lo:hi].long() - s0[lo:hi].long() - s1[lo:hi].long()) & 0xFFFFFFFF
        s2[lo:hi] = (t - ((t >> 31) << 32)).to(torch.int32)
        del t

    # one match planted past 2^32 and one just past 2^31 (uniform 16-bit values give about
    # 2^16 matches each besides)
    a1, a2 = int(x[N - 3]), int(x[(1 << 31) + 5])
    preds = [W.eq_pred(0, 0, 0, a1), W.eq_pred(0, 0, 0, a2, combine=P.COMBINE_OR)]
    toks = P.keygen(preds, BITS, bytes(range(40, 56)))

    rng = W.rng(98)
    tile = 768
    edges = [b + d for b in (1 << 31, 1 << 32, (1 << 32) // tile * tile) for d in (-tile - 1, -tile, -1, 0, 1, tile)]
    fixed = np.array([0, 1, N - 3, N - 2, N - 1, (1 << 31) + 5] + edges, dtype=np.int64)
    sample = np.unique(np.concatenate([fixed, rng.integers(0, N, 160, dtype=np.int64)]))
    sample = sample[sample < N].astype(np.uint64)
    idx = torch.from_numpy(sample.astype(np.int64)).to(dev)
    host = [np.zeros((1, N), dtype=np.uint32) for _ in range(3)]   # pages of untouched elements stay unmapped
    for j, sj in enumerate((s0, s1, s2)):
        host[j][0, sample] = _u32(sj[idx])
    del sj

    with P.Context(0, prf_keys=PRF) as ctx:
        ctx.load_shares(0, [s0.view(1, N), s1.view(1, N), s2.view(1, N)], BITS)
        torch.cuda.synchronize()
        ctx.sync()
        del s0, s1, s2
        outs = [[torch.empty(N, dtype=torch.int32, device=dev) for _ in range(3)]]
        ctx.filter_and_combine(1, toks, outs)
        torch.cuda.synchronize()
        ctx.sync()

    o = outs[0]
    positives = 0
    for lo in range(0, N, CHUNK):
        hi = min(N, lo + CHUNK)
        rec = (o[0][lo:hi].long() + o[1][lo:hi].long() + o[2][lo:hi].long()) & 0xFFFFFFFF
        want = ((x[lo:hi] == a1) | (x[lo:hi] == a2)).long()
        assert torch.equal(rec, want), lo
        positives += int(want.sum())
    assert positives >= 2
    for e in (N - 3, (1 << 31) + 5):
        assert int((o[0][e].long() + o[1][e].long() + o[2][e].long()) & 0xFFFFFFFF) == 1

    got = np.stack([_u32(t[idx]) for t in o])
    want = oracle.filter_group(toks, 1, PRF, [(host, BITS)], 0, sample, threads=16)
    assert np.array_equal(got, want)
