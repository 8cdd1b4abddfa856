"""Block floating-point codec kernels (rcf_bfp_encode / rcf_bfp_decode, Section III-C-3)
against the oracle.

Byte and integer work: the compressed stream must equal the oracle's byte for byte and the
decoded values must equal the oracle's bit for bit, at every rate, on ragged lengths, on
unaligned pointers (the scalar load/store paths), and, at the size of one residual block
of the 20^3 p = 5 workload (256 vectors x 4,000,000 reals), on sampled blocks plus the
exponent definition and the error bound over every value.
"""
import numpy as np
import pytest

import workloads
from oracle.bfp import bfp_decode, bfp_decode_block, bfp_encode, bfp_encode_block, bfp_layout, bfp_stream_bytes

pytestmark = pytest.mark.gpu

RATES = (16, 12, 10)
F32_MAX = float(np.finfo(np.float32).max)
SPECIAL = np.float32([
    [0.0, 0.0, 0.0, 0.0], [-0.0, 0.0, -0.0, 0.0],
    [1.0, 2.5 * 2.0 ** -12, 3.5 * 2.0 ** -12, -2.5 * 2.0 ** -12],      # ties at 16 bits
    [1.0, 2.5 * 2.0 ** -8, -0.5 * 2.0 ** -8, 126.5 * 2.0 ** -8],       # ties at 12 bits
    [1.0, 0.5 * 2.0 ** -6, 1.5 * 2.0 ** -6, -2.5 * 2.0 ** -6],         # ties at 10 bits
    [F32_MAX, -F32_MAX, 1.0, 0.0], [-F32_MAX, -F32_MAX, -F32_MAX, -F32_MAX],
    [2.0 ** -149, -(2.0 ** -149), 0.0, 0.0], [5 * 2.0 ** -139, -3 * 2.0 ** -139, 2.0 ** -130, 0.0],
    [np.nextafter(np.float32(1), np.float32(0)), -0.75, 0.0, 0.0],
    [-np.nextafter(np.float32(1), np.float32(0)), 0.75, 0.0, 0.0],
    [2.0 ** -126, -(2.0 ** -127), 0.0, 1e-45],
]).ravel()


@pytest.fixture(scope="module")
def ctx():
    import torch
    from paper_2605_30128_gb300 import rchfsi as R
    torch.cuda.set_device(0)
    c = R.rcf_create(0)
    yield c
    R.rcf_destroy(c)


def gpu_codec(ctx, x_host, nbits, x_offset=0, s_offset=0, y_offset=0):
    """(stream bytes, decoded float32) from the kernels, with the tensors placed at the given
    element offsets inside larger allocations."""
    import torch
    from paper_2605_30128_gb300 import rchfsi as R
    n = x_host.size
    nbytes = R.rcf_bfp_stream_bytes(n, nbits)
    xb = torch.zeros(n + x_offset, dtype=torch.float32, device="cuda")
    x = xb[x_offset:]
    x.copy_(torch.from_numpy(x_host))
    sb = torch.zeros(nbytes + s_offset, dtype=torch.uint8, device="cuda")
    s = sb[s_offset:]
    yb = torch.full((n + y_offset,), float("nan"), dtype=torch.float32, device="cuda")
    y = yb[y_offset:]
    R.rcf_bfp_encode(ctx, x, nbits, s)
    R.rcf_bfp_decode(ctx, s, nbits, y)
    torch.cuda.synchronize()
    return s.cpu().numpy(), y.cpu().numpy()


def assert_bits_equal(a, b):
    assert a.shape == b.shape
    bad = np.flatnonzero(a.view(np.uint32) != b.view(np.uint32))
    assert bad.size == 0, (bad[:5], a[bad[:5]], b[bad[:5]])


@pytest.mark.parametrize("nbits", RATES)
@pytest.mark.parametrize("n", [1, 3, 4, 5, 1030, 262147])
def test_stream_and_values_match_oracle(ctx, nbits, n):
    x = workloads.bfp_values(1000 + n, n)
    k = min(n, SPECIAL.size)
    x[:k] = SPECIAL[:k]
    s, y = gpu_codec(ctx, x, nbits)
    ref = bfp_encode(x, nbits)
    assert s.size == bfp_stream_bytes(n, nbits)
    bad = np.flatnonzero(s != ref)
    assert bad.size == 0, bad[:8]
    assert_bits_equal(y, bfp_decode(ref, n, nbits))


@pytest.mark.parametrize("nbits", RATES)
def test_decode_of_the_oracle_stream(ctx, nbits):
    import torch
    from paper_2605_30128_gb300 import rchfsi as R
    n = 40001
    x = workloads.bfp_values(7, n)
    ref = bfp_encode(x, nbits)
    s = torch.from_numpy(ref).cuda()
    y = torch.empty(n, dtype=torch.float32, device="cuda")
    R.rcf_bfp_decode(ctx, s, nbits, y)
    torch.cuda.synchronize()
    assert_bits_equal(y.cpu().numpy(), bfp_decode(ref, n, nbits))


@pytest.mark.parametrize("nbits", RATES)
def test_unaligned_pointers_take_the_scalar_paths(ctx, nbits):
    n = 4099
    x = workloads.bfp_values(5, n)
    s0, y0 = gpu_codec(ctx, x, nbits)
    soff = {16: 8, 12: 2, 10: 1}[nbits]       # the smallest offset the rate allows
    s1, y1 = gpu_codec(ctx, x, nbits, x_offset=1, s_offset=soff, y_offset=3)
    assert np.array_equal(s0, s1)
    assert_bits_equal(y0, y1)
    assert np.array_equal(s0, bfp_encode(x, nbits))


def test_empty_and_invalid_arguments(ctx):
    import torch
    from paper_2605_30128_gb300 import rchfsi as R
    l0 = R.rcf_launch_count(ctx)
    R.rcf_bfp_encode(ctx, torch.empty(0, device="cuda"), 16, torch.empty(0, dtype=torch.uint8, device="cuda"))
    R.rcf_bfp_decode(ctx, torch.empty(0, dtype=torch.uint8, device="cuda"), 16, torch.empty(0, device="cuda"))
    assert R.rcf_launch_count(ctx) == l0
    x = torch.ones(64, device="cuda")
    s = torch.empty(64, dtype=torch.uint8, device="cuda")
    for bad_nbits in (8, 14, 32):
        with pytest.raises(R.RcfError) as e:
            R.rcf_bfp_encode(ctx, x, bad_nbits, s)
        assert e.value.status == R.RCF_EINVAL
    with pytest.raises(R.RcfError) as e:            # 16 bits needs an 8-byte aligned stream
        R.rcf_bfp_encode(ctx, x[:8], 16, s[4:])
    assert e.value.status == R.RCF_EINVAL
    with pytest.raises(R.RcfError) as e:            # 12 bits needs a 2-byte aligned stream
        R.rcf_bfp_decode(ctx, s[1:], 12, x[:8])
    assert e.value.status == R.RCF_EINVAL
    with pytest.raises(R.RcfError) as e:            # values and stream overlap
        R.rcf_bfp_encode(ctx, x, 16, x.view(torch.uint8)[128:])
    assert e.value.status == R.RCF_EINVAL
    with pytest.raises(ValueError):
        R.rcf_bfp_encode(ctx, x, 16, s[:8])           # too small for 64 values
    assert R.rcf_launch_count(ctx) == l0


def test_full_residual_block_size(ctx):
    """One residual block of the 20^3 p = 5 workload: 256 vectors x 2,000,000 complex entries,
    as 1,024,000,000 FP32 values, at 16 bits (the launch configuration the benchmark times)."""
    import torch
    from paper_2605_30128_gb300 import rchfsi as R
    nbits, v = 16, 14
    n = 256 * 4_000_000
    g = torch.Generator(device="cuda")
    g.manual_seed(123)
    nblk = n // 4
    x = torch.exp2(torch.rand(nblk, 1, generator=g, device="cuda") * 276.0 - 149.0)
    x = x * torch.exp2(-24.0 * torch.rand(nblk, 4, generator=g, device="cuda"))
    x = torch.where(torch.rand(nblk, 4, generator=g, device="cuda") < 0.5, -x, x).reshape(-1)
    s = torch.empty(R.rcf_bfp_stream_bytes(n, nbits), dtype=torch.uint8, device="cuda")
    y = torch.empty_like(x)
    R.rcf_bfp_encode(ctx, x, nbits, s)
    R.rcf_bfp_decode(ctx, s, nbits, y)
    torch.cuda.synchronize()
    # sampled blocks (and the first and last) against the oracle, byte and bit exact
    rng = np.random.default_rng(9)
    idx = np.concatenate([[0, nblk - 1], rng.integers(0, nblk, 4000)])
    it = torch.from_numpy(idx).cuda()
    xs = x.view(nblk, 4)[it].cpu().numpy()
    ss = s.view(nblk, 8)[it].cpu().numpy()
    ys = y.view(nblk, 4)[it].cpu().numpy()
    for j in range(idx.size):
        ref = bfp_encode_block(xs[j], nbits)
        assert ss[j].tobytes() == ref, (idx[j], xs[j])
        assert_bits_equal(ys[j], bfp_decode_block(ref, nbits))
    # every block: the exponent definition and the error bound (FP64 on the GPU, in chunks)
    e_all = s.view(nblk, 8)[:, 0]
    chunk = 1 << 24
    for b0 in range(0, nblk, chunk):
        xb = x.view(nblk, 4)[b0:b0 + chunk].double()
        yb = y.view(nblk, 4)[b0:b0 + chunk].double()
        e = e_all[b0:b0 + chunk].long()
        m = xb.abs().amax(dim=1)
        emax = (e - 127).double()
        normal = m >= 2.0 ** -126
        assert bool(((e == 0) == (m == 0)).all())
        assert bool((torch.exp2(emax - 1) <= m)[normal].all()) and bool((m < torch.exp2(emax))[m > 0].all())
        assert bool((e[(m > 0) & ~normal] == 1).all())
        quantum = torch.exp2(emax - v + 1).unsqueeze(1)
        err = (yb - xb).abs()
        assert bool((err <= quantum).all())
        unclamped = xb.abs() / quantum <= 2 ** (v - 1) - 1
        assert bool((err[unclamped] <= (quantum / 2).expand_as(err)[unclamped]).all())
