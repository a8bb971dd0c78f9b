"""Streams without a stored index (the paper's own layout): the decoder rebuilds
the record offsets -- by walking the delimiters the first time a context meets
such a stream, and by the parallel chase after that.  Both must decode exactly,
reject corrupt streams, and survive data whose payload words look like record
starts."""
import numpy as np
import pytest
import torch

import datagen
import oracle

pytestmark = pytest.mark.gpu
MiB = 1 << 20
DEV = "cuda:0"


@pytest.fixture(scope="module")
def hz():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1107_1525_gb300 import build
    build.build()
    import paper_1107_1525_gb300.hz as hzmod
    return hzmod


def _compress_no_index(hz, ctx, x, B):
    ctx.set_option(hz.HZ_OPT_INDEX, 0)
    s = hz.compress(x, B, ctx=ctx)
    ctx.set_option(hz.HZ_OPT_INDEX, 1)
    assert oracle.parse_header(s[:280].cpu().numpy())["flags"] & 1 == 0
    return s


def _decompress(hz, ctx, s, n):
    y = torch.empty(n, dtype=torch.uint8, device=DEV)
    ol = torch.zeros(1, dtype=torch.int64, device=DEV)
    ctx.profile_read()
    ctx.set_option(hz.HZ_OPT_PROFILE, 1)
    hz.hz_decompress(ctx, s, s.numel(), y, n, ol)
    st = hz.hz_sync(ctx)
    names = [k for k, _ in ctx.profile_read()]
    ctx.set_option(hz.HZ_OPT_PROFILE, 0)
    return st, y, names


def test_walk_then_parallel_chase(hz):
    ctx = hz.Context(0)
    x = datagen.mixed_buffer(n=64 * MiB, segment=16 * MiB, seed=6, device=DEV)
    s = _compress_no_index(hz, ctx, x, 16384)
    st, y, names = _decompress(hz, ctx, s, x.numel())
    assert st == 0 and torch.equal(x, y) and "decode_chase" not in names  # the walk
    for _ in range(2):
        st, y, names = _decompress(hz, ctx, s, x.numel())
        assert st == 0 and torch.equal(x, y) and "decode_chase" in names
    # the stream with an index decodes alike, and differs only by the index
    s_idx = hz.compress(x, 16384, ctx=ctx)
    assert s_idx.numel() == s.numel() + 4 * (x.numel() // 16384)
    ctx.close()


def test_parallel_chase_rejects_corrupt_streams(hz):
    ctx = hz.Context(0)
    x = datagen.mixed_buffer(n=32 * MiB, segment=8 * MiB, seed=7, device=DEV)
    s = _compress_no_index(hz, ctx, x, 65536)
    st, y, _ = _decompress(hz, ctx, s, x.numel())  # the walk; the context now chases
    assert st == 0 and torch.equal(x, y)
    bad = s.clone()
    bad[280] ^= 0x40  # the first record's delimiter: 64 bits more or fewer
    st, _, names = _decompress(hz, ctx, bad, x.numel())
    assert st == hz.HZ_ERR_CORRUPT and "decode_chase" in names
    short = s[:-4].clone()
    st, _, _ = _decompress(hz, ctx, short, x.numel())
    assert st == hz.HZ_ERR_CORRUPT
    st, y, _ = _decompress(hz, ctx, s, x.numel())  # still usable
    assert st == 0 and torch.equal(x, y)
    ctx.close()


def test_parallel_chase_with_payload_that_looks_like_delimiters(hz):
    """With the given code "symbol s -> the 4 bits of s" (s < 16) every
    1024-symbol block has exactly 4096 payload bits, and bytes 0,0,0,0,1,0,0,0
    repeated make every payload word equal 4096: in the first half of the stream
    every word is a candidate record start, and the false chains run beside the
    true one until they die in the random second half."""
    ctx = hz.Context(0)
    n = 16 * MiB
    rng = np.random.default_rng(8)
    x = rng.integers(0, 16, size=n, dtype=np.uint8)
    x[: n // 2] = np.tile(np.array([0, 0, 0, 0, 1, 0, 0, 0], dtype=np.uint8), n // 16)
    lengths = np.zeros(256, dtype=np.uint8)
    lengths[:16] = 4
    codes = hz.make_codes(lengths, oracle.canonical_codes(lengths))
    xd = torch.from_numpy(x).to(DEV)
    ctx.set_option(hz.HZ_OPT_INDEX, 0)
    s = hz.compress(xd, 1024, ctx=ctx, codes=codes)
    ctx.set_option(hz.HZ_OPT_INDEX, 1)
    assert np.array_equal(s.cpu().numpy(), oracle.compress(x, 1024, lengths=lengths, index=False))
    for k in range(2):  # the walk, then the chase
        st, y, names = _decompress(hz, ctx, s, n)
        assert st == 0 and torch.equal(xd, y)
        assert ("decode_chase" in names) == (k == 1)
    ctx.close()
