"""GPU key generation (the client's genToken, Sec. V-C, batched) against the oracle's Gen.

Pair i comes from the root seeds AES_seed(2 i) and AES_seed(2 i + 1); the test
derives those two seeds with the oracle's FIPS-197 AES and runs the oracle's
DPF / DCF Gen on them, so every generated key must match byte for byte.  The
keys are then evaluated on the device (OBLIVGM_KEYS_DEVICE) with one key pair
per element -- the per-value keys of the masked-input approach -- and the two
parties' outputs must reconstruct the point / comparison function.
"""
import struct

import numpy as np
import pytest

import oracle
from tests._helpers import from_dev, to_dev

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2209_03526_gb300")

SEED = bytes(range(100, 116))


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = P.Context(0, prf_keys=bytes(range(48)))
    yield c
    c.close()


def _root(seed, c):
    return oracle.aes128(seed, struct.pack("<Q", c) + bytes(8))


def _oracle_pair(kind, n, seed, i, alpha, beta):
    gen = oracle.dpf_gen if kind == P.KEY_DPF else oracle.dcf_gen
    return gen(n, alpha, beta, _root(seed, 2 * i), _root(seed, 2 * i + 1))


def _gen(ctx, kind, n, alpha, beta, seed=SEED):
    L = oracle.key_len(kind, n)
    out = torch.zeros(2 * len(alpha) * L, dtype=torch.uint8, device="cuda")
    ctx.keygen_device(kind, n, to_dev(alpha), to_dev(beta), seed, out)
    torch.cuda.synchronize()
    return out, L


@pytest.mark.parametrize("kind", [P.KEY_DPF, P.KEY_DCF])
@pytest.mark.parametrize("n", [1, 9, 32])
def test_keys_match_oracle_gen(ctx, kind, n):
    g = np.random.default_rng(1000 + 10 * n + kind)
    top = (1 << n) - 1
    m = 700                                   # several 256-thread blocks and a ragged tail
    alpha = g.integers(0, top + 1, m, dtype=np.uint64).astype(np.uint32)
    alpha[:2] = [0, top]
    beta = g.integers(0, 1 << 32, m, dtype=np.uint64).astype(np.uint32)
    beta[2] = 0
    out, L = _gen(ctx, kind, n, alpha, beta)
    got = out.cpu().numpy().tobytes()
    for i in range(m):
        k0, k1 = _oracle_pair(kind, n, SEED, i, int(alpha[i]), int(beta[i]))
        assert got[2 * i * L:(2 * i + 1) * L] == k0, i
        assert got[(2 * i + 1) * L:(2 * i + 2) * L] == k1, i


@pytest.mark.parametrize("kind", [P.KEY_DPF, P.KEY_DCF])
def test_keys_grid_stride_sampled(ctx, kind):
    # more pairs than resident threads: the grid-stride loop wraps; sampled pairs vs the oracle
    g = np.random.default_rng(77 + kind)
    n, m = 32, 100_003
    alpha = g.integers(0, 1 << 32, m, dtype=np.uint64).astype(np.uint32)
    beta = g.integers(0, 1 << 32, m, dtype=np.uint64).astype(np.uint32)
    out, L = _gen(ctx, kind, n, alpha, beta)
    host = out.cpu().numpy()
    for i in list(g.choice(m, 150, replace=False)) + [0, m - 1, 38911, 38912]:
        i = int(i)
        k0, k1 = _oracle_pair(kind, n, SEED, i, int(alpha[i]), int(beta[i]))
        assert host[2 * i * L:(2 * i + 1) * L].tobytes() == k0, i
        assert host[(2 * i + 1) * L:(2 * i + 2) * L].tobytes() == k1, i


@pytest.mark.parametrize("kind", [P.KEY_DPF, P.KEY_DCF])
def test_per_element_keys_reconstruct(ctx, kind):
    # one fresh key pair per element, evaluated on that element's (masked) value
    g = np.random.default_rng(5 + kind)
    n, m = 32, 20_000
    alpha = g.integers(0, 1 << 32, m, dtype=np.uint64).astype(np.uint32)
    beta = g.integers(1, 1 << 32, m, dtype=np.uint64).astype(np.uint32)
    x = g.integers(0, 1 << 32, m, dtype=np.uint64).astype(np.uint32)
    x[::3] = alpha[::3]                       # hits of the point function
    x[1::7] = alpha[1::7] - 1                 # just below the threshold
    keys, L = _gen(ctx, kind, n, alpha, beta)
    pts = to_dev(np.repeat(x, 2))
    kop = to_dev(np.arange(2 * m, dtype=np.uint32))      # point 2c+b -> key b of pair c
    out = torch.empty(2 * m, dtype=torch.int32, device="cuda")
    ctx.eval_device_keys(kind, n, keys, 2 * m, pts, out, key_of_point=kop)
    ctx.sync()
    got = from_dev(out).reshape(m, 2)
    rec = (got[:, 0].astype(np.uint64) + got[:, 1]) & 0xFFFFFFFF
    hit = (x == alpha) if kind == P.KEY_DPF else (x < alpha)
    assert np.array_equal(rec, np.where(hit, beta, 0))
    host = keys.cpu().numpy()
    for c in g.choice(m, 40, replace=False):
        c = int(c)
        for b in range(2):
            key = host[(2 * c + b) * L:(2 * c + b + 1) * L].tobytes()
            assert got[c, b] == oracle.eval_many(key, [int(x[c])], kind)[0]


def test_device_keys_all_pairs_match_host_keys(ctx):
    # the same keys through the host-key and the device-key paths give the same outputs
    g = np.random.default_rng(9)
    n = 20
    alpha = g.integers(0, 1 << n, 6, dtype=np.uint64).astype(np.uint32)
    beta = g.integers(0, 1 << 32, 6, dtype=np.uint64).astype(np.uint32)
    pts = to_dev(g.integers(0, 1 << n, 777, dtype=np.uint64).astype(np.uint32))
    for kind in (P.KEY_DPF, P.KEY_DCF):
        keys, L = _gen(ctx, kind, n, alpha, beta)
        a = torch.empty(12 * 777, dtype=torch.int32, device="cuda")
        b = torch.empty_like(a)
        ctx.eval_device_keys(kind, n, keys, 12, pts, a, all_pairs=True)
        fn = ctx.eval_dpf_batch if kind == P.KEY_DPF else ctx.eval_dcf_batch
        fn(keys.cpu().numpy().tobytes(), 12, pts, b, all_pairs=True)
        ctx.sync()
        assert torch.equal(a, b)


def test_device_key_header_mismatch_reports_fault(ctx):
    # keys of n = 20 evaluated as n = 8: every header disagrees, the outputs are those of
    # zero keys, and the next sync reports the device-side error (no fault, context usable)
    alpha = np.array([5, 6], dtype=np.uint32)
    beta = np.array([1, 1], dtype=np.uint32)
    keys, _ = _gen(ctx, P.KEY_DPF, 20, alpha, beta)
    pts = to_dev(np.arange(16, dtype=np.uint32))
    out = torch.empty(4 * 16, dtype=torch.int32, device="cuda")
    ctx.eval_device_keys(P.KEY_DPF, 8, keys, 4, pts, out, all_pairs=True)
    with pytest.raises(P.OblivgmError) as e:
        ctx.sync()
    assert e.value.status == P.EFAULT_DEVICE
    ctx.sync()                                # flag cleared, context still usable
    ok = torch.empty(4 * 16, dtype=torch.int32, device="cuda")
    ctx.eval_device_keys(P.KEY_DPF, 20, keys, 4, pts, ok, all_pairs=True)
    ctx.sync()
    rec = (from_dev(ok).reshape(2, 2, 16).astype(np.uint64).sum(axis=1)) & 0xFFFFFFFF
    assert np.array_equal(rec[0], (np.arange(16) == 5).astype(np.uint64))
    assert np.array_equal(rec[1], (np.arange(16) == 6).astype(np.uint64))


def test_keygen_rejects_bad_arguments(ctx):
    a = to_dev(np.zeros(4, dtype=np.uint32))
    small = torch.zeros(10, dtype=torch.uint8, device="cuda")
    with pytest.raises(P.OblivgmError) as e:
        ctx.keygen_device(P.KEY_DPF, 8, a, a, SEED, small)
    assert e.value.status == P.ERANGE
    big = torch.zeros(1 << 16, dtype=torch.uint8, device="cuda")
    for kind, n in ((7, 8), (P.KEY_DPF, 0), (P.KEY_DCF, 33)):
        with pytest.raises(P.OblivgmError) as e:
            ctx.keygen_device(kind, n, a, a, SEED, big)
        assert e.value.status == P.EINVAL
    with pytest.raises(P.OblivgmError) as e:     # misaligned key buffer
        ctx.keygen_device(P.KEY_DPF, 8, a, a, SEED, big[1:])
    assert e.value.status == P.EINVAL
