"""The fixed-key PRG H_K(s) = AES-128_K(s) xor s in both AES layouts, against the oracle.

oblivgm_prg_batch computes the PRG of the DPF / DCF constructions (Sec. V-C) on counter
blocks in the T-table layout the walks use and in a bitsliced layout (32 blocks per thread,
SubBytes as a gate circuit); the autotuner times the two.  Both must equal the oracle's
byte-wise FIPS-197 AES word for word, for all four fixed keys, at counters with high bits
set (the bitsliced layout builds them as bit planes), and the parity words must be the
parity of those blocks."""
import struct

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2209_03526_gb300")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = P.Context(0)
    yield c
    c.close()


def _want(key, first, n):
    out = np.zeros((n, 4), dtype=np.uint32)
    for i in range(n):
        out[i] = np.frombuffer(oracle.prg(key, struct.pack("<QQ", first + i, 0)), dtype="<u4")
    return out


@pytest.mark.parametrize("layout", [P.AES_TTABLE, P.AES_BITSLICED])
@pytest.mark.parametrize("key,first", [(0, 0), (1, (1 << 40) + 96), (2, (1 << 63) - 4096), (3, 0xDEADBEEF00)])
def test_prg_layout_equals_oracle(ctx, layout, key, first):
    n = 2048
    out = torch.zeros(4 * n, dtype=torch.int32, device="cuda")
    ctx.prg_batch(layout, key, first, n, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy().view(np.uint32).reshape(n, 4)
    assert np.array_equal(got, _want(key, first, n))


@pytest.mark.parametrize("layout", [P.AES_TTABLE, P.AES_BITSLICED])
def test_prg_parity_words(ctx, layout):
    n, first = 4096, 1 << 33
    full = torch.zeros(4 * n, dtype=torch.int32, device="cuda")
    par = torch.zeros(n // 32, dtype=torch.int32, device="cuda")
    ctx.prg_batch(P.AES_TTABLE, 0, first, n, full)
    ctx.prg_batch(layout, 0, first, n, par, parity=True)
    torch.cuda.synchronize()
    blocks = full.cpu().numpy().view(np.uint32).reshape(n, 4)
    x = np.bitwise_xor.reduce(blocks, axis=1)
    bits = np.array([bin(int(v)).count("1") & 1 for v in x], dtype=np.uint64).reshape(-1, 32)
    want = (bits << np.arange(32, dtype=np.uint64)).sum(axis=1).astype(np.uint32)
    assert np.array_equal(par.cpu().numpy().view(np.uint32), want)


def test_prg_rejects_bad_arguments(ctx):
    out = torch.zeros(128, dtype=torch.int32, device="cuda")
    for args in [(2, 0, 0, 32), (0, 4, 0, 32), (0, 0, 5, 32), (0, 0, 0, 33)]:
        with pytest.raises(P.OblivgmError) as e:
            ctx.prg_batch(*args, out)
        assert e.value.status == P.EINVAL
    with pytest.raises(P.OblivgmError) as e:
        ctx.prg_batch(0, 0, 0, 64, out)           # needs 256 words
    assert e.value.status == P.ERANGE


def test_aes_layout_autotune_reports_both_rates(ctx):
    lay, tt, bs = ctx.autotune_aes_layout()
    assert tt > 0 and bs > 0
    assert lay == (P.AES_BITSLICED if bs > tt else P.AES_TTABLE)
