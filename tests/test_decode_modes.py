"""The block decoder's table modes, driven by given codes: complete codes whose
longest code fits the table take the multi-code counting steps with a buffer
fill every 2, 3 or 4 steps (longest code 11 or 12, at most 10, at most 8 bits);
codes longer than the table, or incomplete codes, take the escape paths.  Every case
must reproduce the oracle's stream and decode back to the input, on several
block sizes (with ragged last blocks) and table widths."""
import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def hz():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1107_1525_gb300 import build
    build.build()
    import paper_1107_1525_gb300.hz as hzmod
    return hzmod


def _chain(maxlen: int) -> np.ndarray:
    """Complete code: symbol i (i < maxlen - 1) gets length i + 1, the last two
    symbols length maxlen (Kraft sum exactly 1); symbols 7 apart to spread them
    over the byte range."""
    lengths = np.zeros(256, dtype=np.uint8)
    syms = [(7 * i + 3) % 256 for i in range(maxlen + 1)]
    for i in range(maxlen - 1):
        lengths[syms[i]] = i + 1
    lengths[syms[maxlen - 1]] = maxlen
    lengths[syms[maxlen]] = maxlen
    return lengths


def _flat(bits: int, count: int) -> np.ndarray:
    lengths = np.zeros(256, dtype=np.uint8)
    lengths[np.arange(count) * (256 // count)] = bits
    return lengths


CODES = {
    "chain12": _chain(12),      # complete, longest code 12: fill every 2 steps at W = 12
    "chain11": _chain(11),      # every 2 steps
    "chain10": _chain(10),      # every 3 steps
    "chain9": _chain(9),        # every 3 steps
    "chain8": _chain(8),        # every 4 steps
    "flat4x16": _flat(4, 16),   # complete, 4-bit codes only
    "flat8x256": _flat(8, 256), # complete, incompressible
    "chain14": _chain(14),      # longer than the table: escapes
    "incomplete": _flat(5, 20), # Kraft sum below 1
}


def _sample(lengths: np.ndarray, n: int, seed: int) -> np.ndarray:
    """Symbols with the code's own probabilities 2^-length (so that the
    lengths are near-optimal and every length occurs)."""
    syms = np.nonzero(lengths)[0]
    p = np.exp2(-lengths[syms].astype(np.float64))
    p /= p.sum()
    rng = np.random.default_rng(seed)
    return syms[rng.choice(len(syms), size=n, p=p)].astype(np.uint8)


@pytest.mark.parametrize("name", sorted(CODES))
@pytest.mark.parametrize("W", [12, 11, 10, 9, 8])
def test_given_code_round_trip(hz, name, W):
    """W >= 10 with codes of at most 10 bits: the replicated 10-bit table; W of 8
    or 9 with codes that fit: the W-bit table of the same layout; longer codes
    or incomplete codes: the general table with its second level."""
    lengths = CODES[name]
    codes = hz.make_codes(lengths, oracle.canonical_codes(lengths))
    ctx = hz.Context(0)
    ctx.set_option(hz.HZ_OPT_DECODE_LUT_BITS, W)
    for B, n, seed in ((65536, 3 * 65536 + 4321, 1), (16384, 40 * 16384 + 77, 2), (4096, 4096 * 5 + 1, 3)):
        x = _sample(lengths, n, seed + 10 * W)
        xd = torch.from_numpy(x).to(DEV)
        s = hz.compress(xd, B, ctx=ctx, codes=codes)
        assert np.array_equal(s.cpu().numpy(), oracle.compress(x, B, lengths=lengths)), (name, B)
        y = hz.decompress(s, ctx=ctx)
        assert torch.equal(y, xd), (name, W, B)
    ctx.close()


@pytest.mark.parametrize("name", ["chain12", "chain10", "chain8"])
def test_corrupt_record_is_reported(hz, name):
    """A flipped payload bit inside a block of a complete code still decodes to
    some symbols, but the count or the end position no longer matches."""
    lengths = CODES[name]
    codes = hz.make_codes(lengths, oracle.canonical_codes(lengths))
    ctx = hz.Context(0)
    B, n = 65536, 4 * 65536
    x = _sample(lengths, n, 5)
    s = hz.compress(torch.from_numpy(x).to(DEV), B, ctx=ctx, codes=codes)
    hdr = oracle.parse_header(s[:280].cpu().numpy())
    nb = hdr["nb"]
    idx = np.frombuffer(s[280:280 + 4 * nb].cpu().numpy().tobytes(), dtype="<u4")
    rec = 280 + 4 * nb + 4 * int(idx[2])
    bad = s.clone()
    bad[rec + 4 + 100] ^= 0x10  # a payload bit of record 2
    y = torch.empty(n, dtype=torch.uint8, device=DEV)
    ol = torch.zeros(1, dtype=torch.int64, device=DEV)
    hz.hz_decompress(ctx, bad, bad.numel(), y, n, ol)
    st = hz.hz_sync(ctx)
    # a flip either changes the symbol count or the end of the record, or
    # (rarely) swaps symbols of equal total length: then the output differs
    if st == 0:
        assert not torch.equal(y.cpu(), torch.from_numpy(x))
    else:
        assert st == hz.HZ_ERR_CORRUPT
    assert torch.equal(hz.decompress(s, ctx=ctx).cpu(), torch.from_numpy(x))
    ctx.close()


@pytest.mark.parametrize("name", ["chain10", "chain8", "chain12", "chain14"])
@pytest.mark.parametrize("B", [1, 7, 33, 1000])
def test_small_blocks(hz, name, B):
    """Blocks of a few symbols: fewer bit ranges than lanes, ranges shorter than
    one refill period, records of one or two words."""
    lengths = CODES[name]
    codes = hz.make_codes(lengths, oracle.canonical_codes(lengths))
    ctx = hz.Context(0)
    x = _sample(lengths, 20_000 + B, 7 + B)
    xd = torch.from_numpy(x).to(DEV)
    s = hz.compress(xd, B, ctx=ctx, codes=codes)
    assert np.array_equal(s.cpu().numpy(), oracle.compress(x, B, lengths=lengths))
    assert torch.equal(hz.decompress(s, ctx=ctx), xd)
    ctx.close()


@pytest.mark.parametrize("threads", [128, 256])
@pytest.mark.parametrize("name", ["chain10", "chain12", "chain14", "chain40", "incomplete"])
def test_decode_cta_width(hz, threads, name):
    """Both decoder CTA widths give the oracle's data: streams of a few blocks
    (spread one per CTA), many blocks (several per warp), ragged tails, and
    blocks over 64 KiB (one CTA per block).  chain40 (longest code 40 bits)
    takes the decoder that reads codes over 32 bits from memory; every code
    length occurs."""
    lengths = _chain(40) if name == "chain40" else CODES[name]
    longest = np.nonzero(lengths == lengths.max())[0]
    codes = hz.make_codes(lengths, oracle.canonical_codes(lengths))
    ctx = hz.Context(0)
    ctx.set_option(hz.HZ_OPT_DECODE_THREADS, threads)
    assert ctx.get_option(hz.HZ_OPT_DECODE_THREADS) == threads
    for B, n, seed in ((4096, 5 * 4096 + 17, 1), (65536, 300 * 65536 + 5, 2),
                       (1000, 3_000_001, 3), (131072, 5 * 131072 + 999, 4)):
        x = _sample(lengths, n, seed + threads)
        x[::9973] = longest[np.arange(len(x[::9973])) % len(longest)]
        xd = torch.from_numpy(x).to(DEV)
        s = hz.compress(xd, B, ctx=ctx, codes=codes)
        if n < 4_000_000:
            assert np.array_equal(s.cpu().numpy(), oracle.compress(x, B, lengths=lengths)), B
        assert torch.equal(hz.decompress(s, ctx=ctx), xd), (name, threads, B)
    ctx.close()


def test_decode_threads_option_values(hz):
    ctx = hz.Context(0)
    for bad in (0, 64, 512, 1024):
        with pytest.raises(hz.HzError):
            ctx.set_option(hz.HZ_OPT_DECODE_THREADS, bad)
    assert ctx.get_option(hz.HZ_OPT_DECODE_THREADS) == 256
    ctx.close()
