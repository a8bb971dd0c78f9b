"""Streams with sub-block offsets (flags bit 1): the compressor must write the
oracle's stream for the same S byte for byte, and the single-pass decoder -- one
lane per S-symbol sub-block, started at its stored offset and writing straight
into its place in the output -- must return the input exactly: in every decoder
table mode, for block sizes with ragged tails (blocks over 64 KiB included), for
both CTA widths, in batches and through host buffers.  Corrupt offsets must be
reported as corrupt.  Integer work: no tolerance."""
import numpy as np
import pytest
import torch

import datagen
import oracle
from tests import format_reader
from tests.test_decode_modes import CODES, _chain, _flat, _sample

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
MiB = 1 << 20


@pytest.fixture(scope="module")
def hz():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1107_1525_gb300 import build
    build.build()
    import paper_1107_1525_gb300.hz as hzmod
    return hzmod


def _ctx(hz, S, **opts):
    ctx = hz.Context(0)
    ctx.set_option(hz.HZ_OPT_SUB_BLOCK, S)
    for k, v in opts.items():
        ctx.set_option(getattr(hz, k), v)
    return ctx


def _decode(hz, ctx, s, n):
    y = torch.empty(max(n, 1), dtype=torch.uint8, device=DEV)
    ol = torch.zeros(1, dtype=torch.int64, device=DEV)
    hz.hz_decompress(ctx, s, s.numel(), y, n, ol)
    return hz.hz_sync(ctx), y[:n]


@pytest.mark.parametrize("n,B,S", [(MiB + 123, 4096, 2048), (5 * MiB + 7, 16384, 2048),
                                   (3 * 65536 + 4321, 65536, 2048), (70_001, 65536, 1024),
                                   (100, 64, 32), (10_000, 96, 32), (4096 * 33, 4096, 4096),
                                   (2 * MiB + 5, 262144, 2048), (0, 4096, 2048), (1, 64, 32)])
def test_sub_block_streams_match_the_oracle(hz, n, B, S):
    ctx = _ctx(hz, S)
    for kind, x in (("zipf", datagen.zipf_buffer(n, s=1.1, seed=n + B, device=DEV)),
                    ("mix", datagen.mixed_buffer(n=n, segment=max(64, n // 4 // 64 * 64 or 64),
                                                 seed=3, device=DEV) if n >= 256 else None)):
        if x is None:
            continue
        s = hz.compress(x, B, ctx=ctx)
        x_np = x.cpu().numpy()
        want = oracle.compress(x_np, B, sub=S)
        assert np.array_equal(s.cpu().numpy(), want), (kind, n, B, S)
        st, y = _decode(hz, ctx, s, n)
        assert st == 0 and torch.equal(y, x), (kind, n, B, S)
        st, y = _decode(hz, ctx, torch.from_numpy(want).to(DEV), n)
        assert st == 0 and torch.equal(y, x)
        if n <= 20_000:
            assert format_reader.decode(want.tobytes()) == x_np.tobytes()
    ctx.close()


@pytest.mark.parametrize("name", ["chain8", "chain10", "chain12", "chain14", "chain40",
                                  "incomplete", "flat8x256", "flat4x16"])
@pytest.mark.parametrize("W", [12, 10, 9])
def test_sub_block_decoder_modes(hz, name, W):
    """Mode 0 with the replicated 10-bit table (codes of at most 10 bits), with
    the W-bit table (11-12 bits, or W = 9), and the general table for codes
    longer than the table or incomplete codes (second level, or codes over 32
    bits read from memory)."""
    lengths = _chain(40) if name == "chain40" else CODES[name]
    longest = np.nonzero(lengths == lengths.max())[0]
    codes = hz.make_codes(lengths, oracle.canonical_codes(lengths))
    ctx = _ctx(hz, 2048, HZ_OPT_DECODE_LUT_BITS=W)
    for B, n, seed in ((65536, 3 * 65536 + 4321, 1), (16384, 40 * 16384 + 77, 2),
                       (262144, 2 * 262144 + 999, 3), (2048, 2048 * 9 + 1, 4)):
        x = _sample(lengths, n, seed + 10 * W)
        x[::4999] = longest[np.arange(len(x[::4999])) % len(longest)]
        xd = torch.from_numpy(x).to(DEV)
        s = hz.compress(xd, B, ctx=ctx, codes=codes)
        assert np.array_equal(s.cpu().numpy(), oracle.compress(x, B, lengths=lengths, sub=2048))
        st, y = _decode(hz, ctx, s, n)
        assert st == 0 and torch.equal(y, xd), (name, W, B)
    ctx.close()


@pytest.mark.parametrize("maxlen", [11, 20, 28, 32])
@pytest.mark.parametrize("B,S", [(65536, 2048), (16384, 512)])
def test_sub_block_runs_of_long_codes(hz, maxlen, B, S):
    """Complete codes with rare codes of over 10 bits (up to 32), in runs:
    hundreds of the longest codes in a row, across refill points and
    sub-block boundaries, at a sub-block's start and at the stream's end, so
    that a lane's steps read far ahead in its ring."""
    lengths = _chain(maxlen)
    syms = np.nonzero(lengths)[0]
    longest = syms[lengths[syms] == maxlen]
    long_ish = syms[lengths[syms] > 10]
    codes = hz.make_codes(lengths, oracle.canonical_codes(lengths))
    ctx = _ctx(hz, S)
    n = 5 * B + 3 * S + 777
    x = _sample(lengths, n, maxlen + B)
    rng = np.random.default_rng(maxlen)
    for at, run in ((0, 300), (S - 100, 400), (2 * B + S, 2 * S), (n - 500, 500),
                    (3 * B + 17, 33)):
        x[at:at + run] = longest[rng.integers(0, len(longest), len(x[at:at + run]))]
    x[rng.integers(0, n, 3000)] = long_ish[rng.integers(0, len(long_ish), 3000)]
    xd = torch.from_numpy(x).to(DEV)
    s = hz.compress(xd, B, ctx=ctx, codes=codes)
    want = oracle.compress(x, B, lengths=lengths, sub=S)
    assert np.array_equal(s.cpu().numpy(), want), (maxlen, B, S)
    st, y = _decode(hz, ctx, s, n)
    assert st == 0 and torch.equal(y, xd), (maxlen, B, S)
    st, y = _decode(hz, ctx, torch.from_numpy(want).to(DEV), n)
    assert st == 0 and torch.equal(y, xd)
    ctx.close()


def _mixed5() -> np.ndarray:
    """A complete code of 1- to 5-bit lengths over 8 symbols spread over the
    byte range (1/2 + 1/4 + 2/16 + 4/32 = 1)."""
    lengths = np.zeros(256, dtype=np.uint8)
    for s, l in zip((9, 200, 31, 32, 120, 121, 122, 255), (1, 2, 4, 4, 5, 5, 5, 5)):
        lengths[s] = l
    return lengths


@pytest.mark.parametrize("name", ["chain5", "flat4x16", "flat5x32", "mixed5", "chain2"])
@pytest.mark.parametrize("B,S", [(65536, 2048), (16384, 512), (4096, 32)])
def test_sub_block_two_codes_a_lookup(hz, name, B, S):
    """No code longer than 5 bits: every 10-bit window holds two whole codes,
    and the sub-block decoder takes two symbols a lookup (in 32-symbol groups;
    one a step before a lane's first 32-byte boundary and after its last
    group).  Ragged lengths, uniform and skewed symbols, runs of the longest
    codes across sub-block boundaries, and the oracle's stream decoded too."""
    lengths = {"chain5": _chain(5), "flat4x16": _flat(4, 16), "flat5x32": _flat(5, 32),
               "mixed5": _mixed5(), "chain2": _chain(2)}[name]
    codes = hz.make_codes(lengths, oracle.canonical_codes(lengths))
    ctx = _ctx(hz, S)
    syms = np.nonzero(lengths)[0]
    longest = syms[lengths[syms] == lengths.max()]
    rng = np.random.default_rng(B + S)
    for n in (3 * B + 5 * S + 29, 2 * B, S + 1, 31):
        x = _sample(lengths, n, n + S)
        for at in (0, S - 7, n - 40):
            if 0 <= at < n:
                x[at:at + 40] = longest[rng.integers(0, len(longest), len(x[at:at + 40]))]
        xd = torch.from_numpy(x).to(DEV)
        s = hz.compress(xd, B, ctx=ctx, codes=codes)
        want = oracle.compress(x, B, lengths=lengths, sub=S)
        assert np.array_equal(s.cpu().numpy(), want), (name, B, S, n)
        st, y = _decode(hz, ctx, s, n)
        assert st == 0 and torch.equal(y, xd), (name, B, S, n)
        # the output at an offset that is not 32-byte aligned (one code a step
        # up to the first boundary)
        out = torch.empty(n + 5, dtype=torch.uint8, device=DEV)
        ol = torch.zeros(1, dtype=torch.int64, device=DEV)
        hz.hz_decompress(ctx, s, s.numel(), out[5:], n, ol)
        assert hz.hz_sync(ctx) == 0 and torch.equal(out[5:], xd), (name, B, S, n)
    # a flipped payload bit is caught by the sub-block's end check or decodes to
    # other bytes (never the input)
    x = _sample(lengths, 4 * B, 7)
    xd = torch.from_numpy(x).to(DEV)
    s = hz.compress(xd, B, ctx=ctx, codes=codes)
    bad = s.clone()
    at = s.numel() - 100
    bad[at] ^= 0x10
    st, y = _decode(hz, ctx, bad, x.size)
    assert st == hz.HZ_ERR_CORRUPT or not torch.equal(y, xd)
    st, y = _decode(hz, ctx, s, x.size)
    assert st == 0 and torch.equal(y, xd)
    ctx.close()


def test_sub_block_two_codes_a_lookup_in_batches(hz):
    """The same streams through the batched decoder (which takes them one code
    a lookup, from the plain mode-0 tables)."""
    ctx = hz.Context(0)
    ctx_sub = _ctx(hz, 512)
    streams, bufs = [], []
    for i, name in enumerate(["chain5", "flat4x16", "mixed5", "chain2"] * 3):
        lengths = {"chain5": _chain(5), "flat4x16": _flat(4, 16), "mixed5": _mixed5(),
                   "chain2": _chain(2)}[name]
        codes = hz.make_codes(lengths, oracle.canonical_codes(lengths))
        x = torch.from_numpy(_sample(lengths, 50_000 + 7919 * i, i)).to(DEV)
        streams.append(hz.compress(x, 16384, ctx=ctx_sub, codes=codes).clone())
        bufs.append(x)
    outs = [torch.empty(x.numel(), dtype=torch.uint8, device=DEV) for x in bufs]
    reqs = [(hz.HZ_OP_DECOMPRESS, 0, s, s.numel(), o, o.numel()) for s, o in zip(streams, outs)]
    t = hz.hz_submit(ctx, reqs)
    st, per, lens = hz.hz_poll(ctx, t, len(reqs), -1)
    assert st == 0 and (per == 0).all()
    for x, o in zip(bufs, outs):
        assert torch.equal(x, o)
    ctx.close()
    ctx_sub.close()


@pytest.mark.parametrize("threads", [128, 256])
def test_sub_block_cta_widths(hz, threads):
    ctx = _ctx(hz, 1024, HZ_OPT_DECODE_THREADS=threads)
    x = datagen.mixed_buffer(n=24 * MiB + 1000, segment=6 * MiB, seed=4, device=DEV)
    s = hz.compress(x, 65536, ctx=ctx)
    st, y = _decode(hz, ctx, s, x.numel())
    assert st == 0 and torch.equal(y, x)
    ctx.close()


def test_sub_block_option_values(hz):
    ctx = hz.Context(0)
    assert ctx.get_option(hz.HZ_OPT_SUB_BLOCK) == 0
    for bad in (2, 16, 48, 100, (1 << 24) + 32):
        with pytest.raises(hz.HzError):
            ctx.set_option(hz.HZ_OPT_SUB_BLOCK, bad)
    # an S that does not divide B leaves the stream in the paper's layout
    ctx.set_option(hz.HZ_OPT_SUB_BLOCK, 3072)
    x = datagen.zipf_buffer(300_000, s=1.1, seed=9, device=DEV)
    s = hz.compress(x, 4096, ctx=ctx)
    assert np.array_equal(s.cpu().numpy(), oracle.compress(x.cpu().numpy(), 4096))
    # and the index off means no sub-block offsets either
    ctx.set_option(hz.HZ_OPT_SUB_BLOCK, 2048)
    ctx.set_option(hz.HZ_OPT_INDEX, 0)
    cap = hz.hz_compress_bound_ctx(ctx, x.numel(), 4096)
    out = torch.empty(cap, dtype=torch.uint8, device=DEV)
    ol = torch.zeros(1, dtype=torch.int64, device=DEV)
    hz.hz_compress(ctx, x, x.numel(), 4096, None, out, cap, ol)
    assert hz.hz_sync(ctx) == 0
    got = out[: int(ol.item())].cpu().numpy()
    assert np.array_equal(got, oracle.compress(x.cpu().numpy(), 4096, index=False))
    ctx.close()


def test_sub_block_automatic_size(hz):
    """HZ_SUB_BLOCK_AUTO: the largest S of 4096 .. 512 dividing B that leaves
    four sub-blocks for each of the decoder's resident lanes (SMs x 768), else
    512 when that leaves at least one, else none.  The choice is read back
    from the capacity bound (which counts the offsets) and from a stream,
    which must be the oracle's for that S."""
    ctx = _ctx(hz, hz.HZ_SUB_BLOCK_AUTO)
    assert ctx.get_option(hz.HZ_OPT_SUB_BLOCK) == hz.HZ_SUB_BLOCK_AUTO
    lanes = torch.cuda.get_device_properties(0).multi_processor_count * 768

    def want(n, B):
        for S in (4096, 2048, 1024, 512):
            if B % S == 0 and n // S >= 4 * lanes:
                return S
        return 512 if B % 512 == 0 and n // 512 >= lanes else 0

    def chosen(n, B):
        extra = hz.hz_compress_bound_ctx(ctx, n, B) - hz.hz_compress_bound(n, B)
        if extra == 0:
            return 0
        nb = -(-n // B)
        per_block = (extra - 4) // (4 * nb)  # B / S - 1
        return B // (per_block + 1)

    for n, B in ((MiB, 4096), (lanes * 512, 4096), (lanes * 512 - 1, 4096),
                 (2 * lanes * 512, 256), (4 * lanes * 512, 65536),
                 (4 * lanes * 1024 + 5, 65536), (4 * lanes * 2048, 16384),
                 (4 * lanes * 4096 - 1, 65536), (4 * lanes * 2048, 65536 * 3)):
        assert chosen(n, B) == want(n, B), (n, B)
    # a stream at the smallest size that gets S = 512, and one just below it
    for n, S in ((lanes * 512, 512), (MiB, 0)):
        x = datagen.zipf_buffer(n, s=1.1, seed=12, device=DEV)
        s = hz.compress(x, 4096, ctx=ctx)
        assert np.array_equal(s.cpu().numpy(), oracle.compress(x.cpu().numpy(), 4096, sub=S))
        st, y = _decode(hz, ctx, s, n)
        assert st == 0 and torch.equal(y, x)
    ctx.close()


def test_sub_block_bound_and_capacity(hz):
    ctx = _ctx(hz, 1024)
    x = datagen.sample_iid(datagen.uniform_pmf(256), 2 * MiB, 12, DEV)  # incompressible
    cap = hz.hz_compress_bound_ctx(ctx, x.numel(), 16384)
    want = oracle.compress(x.cpu().numpy(), 16384, sub=1024)
    assert want.size <= cap
    out = torch.empty(cap, dtype=torch.uint8, device=DEV)
    ol = torch.zeros(1, dtype=torch.int64, device=DEV)
    hz.hz_compress(ctx, x, x.numel(), 16384, None, out, want.size - 1, ol)
    assert hz.hz_sync(ctx) == hz.HZ_ERR_CAPACITY and int(ol.item()) == want.size
    hz.hz_compress(ctx, x, x.numel(), 16384, None, out, want.size, ol)
    assert hz.hz_sync(ctx) == 0
    assert np.array_equal(out[: want.size].cpu().numpy(), want)
    ctx.close()


def test_corrupt_sub_block_offsets_are_reported(hz):
    ctx = _ctx(hz, 256)
    x = datagen.zipf_buffer(9000 * 8, s=1.2, seed=4, device=DEV)
    B = 1024
    s = hz.compress(x, B, ctx=ctx)
    s_np = s.cpu().numpy()
    nb = oracle.parse_header(s_np)["nb"]
    sec = 280 + 4 * nb                      # S, then 3 entries per block
    cases = {"S": (sec, 64), "first entry": (sec + 4, None), "a middle entry": (sec + 4 + 4 * 37, None),
             "last block past its end": (sec + 4 + 4 * 3 * (nb - 1) + 8, None)}
    for what, (at, value) in cases.items():
        bad = s.clone()
        if value is None:
            bad[at] ^= 1
        else:
            bad[at] = value
        st, _ = _decode(hz, ctx, bad, x.numel())
        assert st == hz.HZ_ERR_CORRUPT, what
        with pytest.raises(oracle.OracleError):
            oracle.decompress(bad.cpu().numpy())
    # the stream itself still decodes, and the context is usable
    st, y = _decode(hz, ctx, s, x.numel())
    assert st == 0 and torch.equal(y, x)
    ctx.close()


def test_sub_block_streams_in_batches(hz):
    """Decompression requests for streams with and without sub-block offsets in
    one submission, through the batched kernels."""
    ctx = hz.Context(0)
    ctx_sub = _ctx(hz, 2048)
    rng = np.random.default_rng(2)
    bufs, streams = [], []
    for i in range(40):
        n = int(np.exp(rng.uniform(np.log(3000), np.log(6 * MiB))))
        x = datagen.zipf_buffer(n, s=float(rng.uniform(0.6, 1.6)), seed=100 + i, device=DEV)
        B = [4096, 16384, 65536][i % 3]
        c = ctx_sub if i % 2 == 0 else ctx
        streams.append(hz.compress(x, B, ctx=c).clone())
        bufs.append(x)
        if i % 2 == 0:
            assert np.array_equal(streams[-1].cpu().numpy(), oracle.compress(x.cpu().numpy(), B, sub=2048))
    outs = [torch.empty(x.numel(), dtype=torch.uint8, device=DEV) for x in bufs]
    reqs = [(hz.HZ_OP_DECOMPRESS, 0, s, s.numel(), o, o.numel()) for s, o in zip(streams, outs)]
    t = hz.hz_submit(ctx, reqs)
    st, per, lens = hz.hz_poll(ctx, t, len(reqs), -1)
    assert st == 0 and (per == 0).all()
    for x, o in zip(bufs, outs):
        assert torch.equal(x, o)
    ctx.close()
    ctx_sub.close()


def test_sub_block_host_buffers(hz):
    """hz_compress_host / hz_decompress_host with the option on, above the size
    where both run as copy/compute pipelines."""
    ctx = _ctx(hz, 2048)
    x = datagen.mixed_buffer(n=48 * MiB + 4097, segment=12 * MiB, seed=6, device="cpu")
    h_in = torch.empty(x.numel(), dtype=torch.uint8, pin_memory=True)
    h_in.copy_(x)
    cap = hz.hz_compress_bound_ctx(ctx, x.numel(), 65536)
    h_s = torch.empty(cap, dtype=torch.uint8, pin_memory=True)
    st, slen = hz.hz_compress_host(ctx, h_in, x.numel(), 65536, h_s, cap)
    assert st == 0
    want = oracle.compress_omp(x.numpy(), 65536, sub=2048)
    assert slen == want.size and np.array_equal(h_s[:slen].numpy(), want)
    h_y = torch.empty(x.numel(), dtype=torch.uint8, pin_memory=True)
    st, ylen = hz.hz_decompress_host(ctx, h_s, slen, h_y, x.numel())
    assert st == 0 and ylen == x.numel() and torch.equal(h_y, h_in)
    ctx.close()
