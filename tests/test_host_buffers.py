"""Host-buffer entry points (hz_compress_host / hz_decompress_host): streams equal
the oracle's and the device-buffer path's, round trips are exact, and the
pipelined decompression of large indexed streams (groups of blocks copied in,
decoded and copied out concurrently) agrees with the plain path, including on
corrupt input and on streams without an index."""
import numpy as np
import pytest
import torch

import datagen
import oracle

pytestmark = pytest.mark.gpu
MiB = 1 << 20


@pytest.fixture(scope="module")
def hz():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1107_1525_gb300 import build
    build.build()
    import paper_1107_1525_gb300.hz as hzmod
    return hzmod


def _pinned(x):
    h = torch.empty(x.numel(), dtype=torch.uint8, pin_memory=True)
    h.copy_(x.cpu() if x.is_cuda else x)
    return h


def _host_round_trip(hz, ctx, x, B):
    h_in = _pinned(x)
    cap = hz.hz_compress_bound(x.numel(), B)
    h_s = torch.empty(cap, dtype=torch.uint8, pin_memory=True)
    st, slen = hz.hz_compress_host(ctx, h_in, x.numel(), B, h_s, cap)
    assert st == 0
    h_y = torch.empty(max(x.numel(), 1), dtype=torch.uint8, pin_memory=True)
    st2, ylen = hz.hz_decompress_host(ctx, h_s, slen, h_y, x.numel())
    return st2, h_s[:slen], h_y[:ylen], h_in


def test_small_host_round_trip_matches_oracle(hz):
    ctx = hz.Context(0)
    x = datagen.zipf_buffer(3 * MiB + 17, s=1.2, seed=40)
    st, s, y, h_in = _host_round_trip(hz, ctx, x, 4096)
    assert st == 0 and torch.equal(y, h_in)
    assert np.array_equal(s.numpy(), oracle.compress(x.numpy(), 4096))
    ctx.close()


@pytest.mark.parametrize("B", [65536, 16384])
def test_pipelined_host_decompress(hz, B):
    ctx = hz.Context(0)
    x = datagen.mixed_buffer(n=96 * MiB, segment=16 * MiB, seed=2, device="cuda:0")
    st, s, y, h_in = _host_round_trip(hz, ctx, x, B)
    assert st == 0 and torch.equal(y, h_in)
    # the same stream from the device-buffer path
    assert torch.equal(hz.compress(x, B, ctx=ctx).cpu(), s)
    ctx.close()


def test_pipelined_host_decompress_rejects_a_corrupt_record(hz):
    ctx = hz.Context(0)
    x = datagen.mixed_buffer(n=64 * MiB, segment=16 * MiB, seed=3, device="cuda:0")
    s = hz.compress(x, 65536, ctx=ctx).cpu()
    hdr = oracle.parse_header(s[:280].numpy())
    nb = hdr["nb"]
    idx = np.frombuffer(s[280:280 + 4 * nb].numpy().tobytes(), dtype="<u4")
    k = nb // 2 + 3  # a record in a middle group
    at = 280 + 4 * nb + 4 * int(idx[k])
    bad = s.clone()
    bad[at] ^= 0x01  # its delimiter no longer matches the index
    h_bad = _pinned(bad)
    h_y = torch.empty(x.numel(), dtype=torch.uint8, pin_memory=True)
    st, _ = hz.hz_decompress_host(ctx, h_bad, bad.numel(), h_y, x.numel())
    assert st == hz.HZ_ERR_CORRUPT
    # the context stays usable
    st, ylen = hz.hz_decompress_host(ctx, _pinned(s), s.numel(), h_y, x.numel())
    assert st == 0 and ylen == x.numel() and torch.equal(h_y, x.cpu())
    ctx.close()


def test_host_decompress_without_index_takes_the_plain_path(hz):
    ctx = hz.Context(0)
    ctx.set_option(hz.HZ_OPT_INDEX, 0)
    x = datagen.mixed_buffer(n=48 * MiB, segment=16 * MiB, seed=4, device="cuda:0")
    st, s, y, h_in = _host_round_trip(hz, ctx, x, 65536)
    assert st == 0 and torch.equal(y, h_in)
    assert oracle.parse_header(s[:280].numpy())["flags"] & 1 == 0
    ctx.close()


def test_host_decompress_capacity(hz):
    ctx = hz.Context(0)
    x = datagen.mixed_buffer(n=40 * MiB, segment=8 * MiB, seed=5, device="cuda:0")
    s = hz.compress(x, 65536, ctx=ctx).cpu()
    h_y = torch.empty(x.numel() - 1, dtype=torch.uint8, pin_memory=True)
    st, _ = hz.hz_decompress_host(ctx, _pinned(s), s.numel(), h_y, x.numel() - 1)
    assert st == hz.HZ_ERR_CAPACITY
    ctx.close()


def test_pipelined_host_compress_capacity(hz):
    """The pipelined host compression (inputs of 32 MiB and more) checks the
    stream size against the caller's capacity before copying anything out."""
    ctx = hz.Context(0)
    x = datagen.mixed_buffer(n=40 * MiB, segment=8 * MiB, seed=6, device="cuda:0")
    exact = hz.compress(x, 65536, ctx=ctx).cpu()
    h_in = _pinned(x)
    h_s = torch.empty(exact.numel(), dtype=torch.uint8, pin_memory=True)
    st, _ = hz.hz_compress_host(ctx, h_in, x.numel(), 65536, h_s, exact.numel() - 1)
    assert st == hz.HZ_ERR_CAPACITY
    st, slen = hz.hz_compress_host(ctx, h_in, x.numel(), 65536, h_s, exact.numel())
    assert st == 0 and slen == exact.numel() and torch.equal(h_s, exact)
    ctx.close()


@pytest.mark.parametrize("B", [4096, 10000, 65536])
def test_pipelined_host_compress_ragged(hz, B):
    """The pipelined host compression on a size that is no multiple of the
    input chunks or the tiles, with blocks whose tiles hold record starts
    (4096: the chunked packer; 10000: the general one): its stream equals the
    device-buffer path's and the oracle's."""
    ctx = hz.Context(0)
    n = 33 * MiB + 12345
    x = datagen.mixed_buffer(n=n, segment=4 * MiB, seed=11, device="cuda:0")
    st, s, y, h_in = _host_round_trip(hz, ctx, x, B)
    assert st == 0 and torch.equal(y, h_in)
    assert torch.equal(hz.compress(x, B, ctx=ctx).cpu(), s)
    xs = x[: 3 * MiB].cpu().numpy()  # and the oracle agrees with the device path
    assert np.array_equal(hz.compress(x[: 3 * MiB], B, ctx=ctx).cpu().numpy(),
                          oracle.compress(xs, B))
    ctx.close()
