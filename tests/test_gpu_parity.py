"""GPU parity: every stream the CUDA library writes must be byte-identical to the
CPU oracle's stream for the same input, block size and code, and every decode must
return the input exactly (integer work: no tolerance).  All calls go through the
C ABI (paper_1107_1525_gb300.hz is a ctypes binding)."""
import numpy as np
import pytest
import torch

import datagen
import oracle
from tests import format_reader

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


@pytest.fixture(scope="module")
def ctx(hz):
    c = hz.Context(0)
    yield c
    c.close()


DEV = "cuda:0"


def _gpu_compress(hz, ctx, x_dev, B, codes=None, cap=None, index=True):
    ctx.set_option(hz.HZ_OPT_INDEX, 1 if index else 0)
    n = x_dev.numel()
    cap = cap if cap is not None else (hz.hz_compress_bound(n, B) if codes is None
                                       else 280 + 16 * n + 64 * (n // B + 1))
    out = torch.empty(max(cap, 1), dtype=torch.uint8, device=DEV)
    out_len = torch.zeros(1, dtype=torch.int64, device=DEV)
    hz.hz_compress(ctx, x_dev, n, B, codes, out, cap, out_len)
    st = hz.hz_sync(ctx)
    ctx.set_option(hz.HZ_OPT_INDEX, 1)
    return st, out[: int(out_len.item())] if st == 0 else out, int(out_len.item())


def _gpu_decompress(hz, ctx, s_dev, cap=None):
    if cap is None:  # n, from the header bytes themselves
        cap = int(np.frombuffer(s_dev[8:16].cpu().numpy().tobytes(), dtype="<u8")[0])
    out = torch.empty(max(cap, 1), dtype=torch.uint8, device=DEV)
    out_len = torch.zeros(1, dtype=torch.int64, device=DEV)
    hz.hz_decompress(ctx, s_dev, s_dev.numel(), out, cap, out_len)
    st = hz.hz_sync(ctx)
    return st, out[: int(out_len.item())]


def _check_round_trip(hz, ctx, x_np, B, lengths=None, index=True):
    x_dev = torch.from_numpy(x_np).to(DEV) if x_np.size else torch.empty(0, dtype=torch.uint8,
                                                                          device=DEV)
    codes = None
    if lengths is not None:
        codes = hz.make_codes(lengths, oracle.canonical_codes(lengths))
    st, s, _ = _gpu_compress(hz, ctx, x_dev, B, codes=codes, index=index)
    assert st == 0, hz.STATUS_NAMES.get(st)
    want = oracle.compress(x_np, B, lengths=lengths, index=index)
    got = s.cpu().numpy()
    assert got.size == want.size
    if not np.array_equal(got, want):
        bad = np.flatnonzero(got != want)
        pytest.fail(f"stream differs at {bad.size} bytes, first at {bad[:8]}")
    # GPU decode of its own stream and of the oracle's, oracle decode of the GPU stream
    st, y = _gpu_decompress(hz, ctx, s)
    assert st == 0 and np.array_equal(y.cpu().numpy(), x_np)
    assert np.array_equal(oracle.decompress(got), x_np)
    return got


def _zipf(n, s, seed):
    return datagen.zipf_buffer(n, s=s, seed=seed, device="cpu").numpy()


# ------------------------------------------------------------ the 1 MiB round trip
def test_zipf_1mib_4k_blocks_round_trip(hz, ctx):
    x = datagen.zipf_buffer(MiB, s=1.1, seed=0, device=DEV)
    _check_round_trip(hz, ctx, x.cpu().numpy(), 4096)


def test_build_codes_matches_oracle(hz, ctx):
    x = datagen.zipf_buffer(3 * MiB + 17, s=1.3, seed=4, device=DEV)
    lens, codes = hz.hz_build_codes(ctx, x, x.numel())
    freq = oracle.histogram(x.cpu().numpy())
    assert np.array_equal(lens, oracle.code_lengths(freq))
    assert np.array_equal(codes, oracle.canonical_codes(lens))


# ------------------------------------------------------------ edge cases
@pytest.mark.parametrize("n,B", [(1, 1), (1, 4096), (2, 1), (3, 3), (31, 1), (100, 7),
                                 (8191, 4096), (8192, 8192), (8193, 8192), (20_000, 1),
                                 (50_001, 33), (100_000, 100_000), (100_000, 1 << 24),
                                 (262_147, 65_536), (300_000, 8191), (600_000, 131_072),
                                 (1_000_000, 262_144), (196_608, 65_536), (196_611, 65_537)])
def test_sizes_and_block_sizes(hz, ctx, n, B):
    _check_round_trip(hz, ctx, _zipf(n, 1.1, n ^ B), B)


def test_empty_input(hz, ctx):
    s = _check_round_trip(hz, ctx, np.zeros(0, dtype=np.uint8), 4096)
    assert s.size == 280


@pytest.mark.parametrize("B", [1, 64, 4096])
def test_single_symbol(hz, ctx, B):
    _check_round_trip(hz, ctx, np.full(70_000, 200, dtype=np.uint8), B)


def test_two_symbols_and_all_256_uniform(hz, ctx):
    rng = np.random.default_rng(1)
    _check_round_trip(hz, ctx, rng.integers(0, 2, 100_000, dtype=np.uint8), 1000)
    _check_round_trip(hz, ctx, rng.integers(0, 256, 500_000, dtype=np.uint8), 4096)


def test_sixteen_symbol_and_geometric(hz, ctx):
    x = datagen.sample_iid(datagen.uniform_pmf(16), 400_000, 3).numpy()
    _check_round_trip(hz, ctx, x, 16384)
    x = datagen.sample_iid(datagen.geometric_pmf(0.3), 400_000, 5).numpy()
    _check_round_trip(hz, ctx, x, 4096)


def test_fibonacci_frequencies_long_codes(hz, ctx):
    # Fibonacci counts give the deepest Huffman tree a buffer of this size allows
    fib = [1, 1]
    while sum(fib) < 2_000_000:
        fib.append(fib[-1] + fib[-2])
    fib = fib[:-1]
    x = np.concatenate([np.full(f, i, dtype=np.uint8) for i, f in enumerate(fib)])
    np.random.default_rng(2).shuffle(x)
    s = _check_round_trip(hz, ctx, x, 65_536)
    assert max(format_reader.read_container(s.tobytes())["lengths"]) >= 28


@pytest.mark.parametrize("maxlen", [26, 27, 31, 32, 33, 47, 64])
def test_given_codes_beyond_26_and_32_bits(hz, ctx, maxlen):
    # the Kraft-complete chain 1, 2, ..., maxlen, maxlen exercises the long-code paths
    lens = np.zeros(256, dtype=np.uint8)
    lens[:maxlen] = np.arange(1, maxlen + 1)
    lens[maxlen] = maxlen
    rng = np.random.default_rng(maxlen)
    x = rng.integers(0, maxlen + 1, 60_000).astype(np.uint8)
    x[rng.integers(0, x.size, 2000)] = maxlen
    x[rng.integers(0, x.size, 2000)] = maxlen - 1
    _check_round_trip(hz, ctx, x, 1000, lengths=lens)
    _check_round_trip(hz, ctx, x, 7, lengths=lens)
    # blocks of whole 8192-symbol tiles: the summing kernel of the warp-parallel
    # path, which falls back to per-tile summaries for codes over 32 bits
    _check_round_trip(hz, ctx, x, 16384, lengths=lens)


def test_tile_start_inside_a_code_longer_than_26_bits(hz, ctx):
    """A tile that starts 29 bits into a word whose first bits belong to a
    30-bit code of the tile before: the packer rebuilds those bits from the
    previous tile's input, and codes of more than 26 bits must come from its
    full code table (its packed entry table keeps only 26).  One 27-bit code,
    then 30-bit codes: 27 + 8191 * 30 = 29 (mod 32) bits end tile 0."""
    maxlen = 30
    lens = np.zeros(256, dtype=np.uint8)
    lens[:maxlen] = np.arange(1, maxlen + 1)
    lens[maxlen] = maxlen  # the chain 1, 2, ..., 30, 30 is complete
    x = np.full(4 * 8192 + 100, maxlen - 1, dtype=np.uint8)  # symbol 29: 30 bits
    x[0] = 26  # symbol 26: 27 bits
    for B in (8192, 16384):
        _check_round_trip(hz, ctx, x, B, lengths=lens)


@pytest.mark.parametrize("maxlen", [17, 24, 32])
@pytest.mark.parametrize("B,sub", [(8192, 0), (65536, 0), (65536, 2048)])
def test_warp_path_codes_of_17_to_32_bits(hz, maxlen, B, sub):
    """Blocks that are whole tiles and codes of 17 to 32 bits take the warp
    packer one code a step.  A run of the longest codes overflows a warp's
    staging area (2048 codes of more than 16 bits), so those items are
    written straight to the output; the other runs (short codes, a mix) go
    through the staging area.  Streams equal the oracle's byte for byte, with
    and without sub-block offsets."""
    lens = np.zeros(256, dtype=np.uint8)
    lens[:maxlen] = np.arange(1, maxlen + 1)
    lens[maxlen] = maxlen  # the chain 1, 2, ..., maxlen, maxlen is complete
    rng = np.random.default_rng(maxlen * 7 + B)
    parts = [rng.integers(0, 4, 3 * 8192 + 111),                   # short codes
             rng.integers(maxlen - 1, maxlen + 1, 5 * 8192 + 5),   # the longest codes
             rng.integers(maxlen // 2, maxlen + 1, 4 * 8192 + 77)]  # a mix
    x = np.concatenate(parts).astype(np.uint8)
    xd = torch.from_numpy(x).to(DEV)
    codes = hz.make_codes(lens, oracle.canonical_codes(lens))
    c = hz.Context(0)
    c.set_option(hz.HZ_OPT_SUB_BLOCK, sub)
    s = hz.compress(xd, B, ctx=c, codes=codes)
    want = oracle.compress(x, B, lengths=lens, sub=sub)
    got = s.cpu().numpy()
    assert got.size == want.size and np.array_equal(got, want), (maxlen, B, sub)
    st, y = _gpu_decompress(hz, c, s)
    assert st == 0 and np.array_equal(y.cpu().numpy(), x)
    c.close()


def test_no_index_mode(hz, ctx):
    x = _zipf(500_000, 1.2, 9)
    _check_round_trip(hz, ctx, x, 4096, index=False)


def test_misaligned_input_pointer(hz, ctx):
    x = datagen.zipf_buffer(200_003, s=1.1, seed=6, device=DEV)
    for off in (1, 3, 7, 13):
        xs = x[off:]
        st, s, _ = _gpu_compress(hz, ctx, xs, 4096)
        assert st == 0
        assert np.array_equal(s.cpu().numpy(), oracle.compress(xs.cpu().numpy(), 4096))


def test_repeated_calls_are_deterministic(hz, ctx):
    x = datagen.zipf_buffer(5 * MiB, s=0.9, seed=8, device=DEV)
    first = None
    for _ in range(5):
        st, s, _ = _gpu_compress(hz, ctx, x, 65_536)
        assert st == 0
        if first is None:
            first = s.clone()
        assert torch.equal(s, first)


# ------------------------------------------------------------ errors
def test_capacity_errors(hz, ctx):
    x = datagen.zipf_buffer(100_000, s=1.1, seed=1, device=DEV)
    want = oracle.compress(x.cpu().numpy(), 4096).size
    st, _, need = _gpu_compress(hz, ctx, x, 4096, cap=want - 1)
    assert st == hz.HZ_ERR_CAPACITY and need == want
    st, s, _ = _gpu_compress(hz, ctx, x, 4096, cap=want)
    assert st == 0
    st, _ = _gpu_decompress(hz, ctx, s, cap=x.numel() - 1)
    assert st == hz.HZ_ERR_CAPACITY
    # the context stays usable
    st, y = _gpu_decompress(hz, ctx, s)
    assert st == 0 and torch.equal(y, x)


def test_corrupt_streams_are_rejected(hz, ctx):
    x = _zipf(50_000, 1.1, 2)
    s = oracle.compress(x, 512)
    c = format_reader.read_container(s.tobytes())
    blocks_at = 280 + 4 * c["nb"]
    bad = []
    b = s.copy(); b[0] ^= 1; bad.append(b)                      # magic
    bad.append(s[:-4].copy())                                   # truncated
    bad.append(np.concatenate([s, np.zeros(4, np.uint8)]))      # trailing bytes
    b = s.copy(); b[284] ^= 1; bad.append(b)                    # index entry
    b = s.copy(); b[blocks_at] ^= 1; bad.append(b)              # first delimiter
    b = s.copy(); b[4] = 2; bad.append(b)                       # unknown flag
    b = s.copy(); b[24:280] = 0; bad.append(b)                  # no code
    b = s.copy(); b[24 + 5] = 1; bad.append(b)                  # Kraft sum above 1
    r0 = c["records"][0]
    if r0["bits"] % 32:
        last = blocks_at + 4 * (r0["word_offset"] + (r0["bits"] + 31) // 32)
        b = s.copy(); b[last] |= 1; bad.append(b)               # padding bit
    for i, b in enumerate(bad):
        with pytest.raises(oracle.OracleError):
            oracle.decompress(b)
        st, _ = _gpu_decompress(hz, ctx, torch.from_numpy(b).to(DEV), cap=x.size)
        assert st == hz.HZ_ERR_CORRUPT, (i, hz.STATUS_NAMES.get(st))
    st, y = _gpu_decompress(hz, ctx, torch.from_numpy(s).to(DEV))
    assert st == 0 and np.array_equal(y.cpu().numpy(), x)


@pytest.mark.parametrize("n,B", [(5, 4), (20_000, 8192)])
def test_given_code_missing_a_symbol_is_an_error(hz, ctx, n, B):
    lens = np.zeros(256, dtype=np.uint8)
    lens[:2] = 1
    codes = hz.make_codes(lens, oracle.canonical_codes(lens))
    x = torch.tensor([0, 1, 2, 1, 0] * (n // 5), dtype=torch.uint8, device=DEV)
    st, _, _ = _gpu_compress(hz, ctx, x, B, codes=codes)
    assert st == hz.HZ_ERR_ARG


# ------------------------------------------------------------ workload-sized cases
def test_mixed_64mib_segments_small(hz, ctx):
    # the four segment kinds of the 1 GiB workload, at 4 x 4 MiB
    x = datagen.mixed_buffer(n=16 * MiB, segment=4 * MiB, seed=2, device=DEV)
    _check_round_trip(hz, ctx, x.cpu().numpy(), 65_536)


def test_gaussian_field_residuals_small(hz, ctx):
    x = datagen.gaussian_field_residuals(shape=(64, 64, 256), seed=1, device=DEV)
    _check_round_trip(hz, ctx, x.cpu().numpy(), 16_384)


@pytest.mark.slow
@pytest.mark.parametrize("sub", [0, 2048])
def test_mixed_1gib_full_size(hz, ctx, sub):
    """The 1 GiB workload at full size, in the paper's layout and with sub-block
    offsets: the whole stream against the oracle's (its OpenMP driver, whose
    streams equal the sequential oracle's), and exact decode of the whole buffer,
    by the GPU and by the oracle."""
    x = datagen.mixed_buffer(n=1 << 30, segment=64 * MiB, seed=2, device=DEV)
    B = 65_536
    ctx.set_option(hz.HZ_OPT_SUB_BLOCK, sub)
    try:
        s = hz.compress(x, B, ctx=ctx)
    finally:
        ctx.set_option(hz.HZ_OPT_SUB_BLOCK, 0)
    x_np = x.cpu().numpy()
    want = oracle.compress_omp(x_np, B, sub=sub)
    s_np = s.cpu().numpy()
    assert s_np.size == want.size and np.array_equal(s_np, want)
    st, y = _gpu_decompress(hz, ctx, s)
    assert st == 0 and torch.equal(y, x)
    del y
    assert np.array_equal(oracle.decompress_omp(s_np), x_np)


@pytest.mark.slow
def test_gaussian_field_full_size_byte_identical(hz, ctx):
    """The 2^28-value scientific-data stream, whole stream against the oracle."""
    x = datagen.gaussian_field_residuals(shape=(512, 512, 1024), seed=1, device=DEV)
    _check_round_trip(hz, ctx, x.cpu().numpy(), 16_384)
