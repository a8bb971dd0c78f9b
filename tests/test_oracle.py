"""Pins for the CPU oracle: each test ties it to something other than itself --
hand-derived streams, brute force, closed forms, textbook special cases, an
independent reader, and the overhead bounds stated in Sec. 2.1 of the paper."""
import itertools
import os
import random
import struct
from fractions import Fraction

import numpy as np
import pytest

import oracle
from tests import format_reader

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load_golden(name):
    spec, fields = {}, []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip() if not line.startswith("#") else ""
            if not line:
                continue
            key, val = (t.strip() for t in line.split(":", 1))
            if key.isdigit():
                fields.append((int(key), bytes.fromhex(val)))
            else:
                spec[key] = val
    return spec, fields


@pytest.mark.parametrize("name", ["abracadabra_b3.txt", "ties_b4.txt", "sub_offsets_b64.txt"])
def test_hand_derived_streams(name):
    spec, fields = _load_golden(name)
    x = np.frombuffer(spec["input_ascii"].encode(), dtype=np.uint8)
    s = oracle.compress(x, int(spec["block_size"]), sub=int(spec.get("sub_block", 0))).tobytes()
    assert len(s) == int(spec["stream_length"])
    want = bytearray(len(s))
    for off, b in fields:
        want[off:off + len(b)] = b
    assert s == bytes(want)
    assert oracle.decompress(s).tobytes() == spec["input_ascii"].encode()


# ------------------------------------------------------------ histogram
def test_histogram_matches_bincount():
    rng = np.random.default_rng(11)
    for n in (0, 1, 7, 4096, 100_003):
        x = rng.integers(0, 256, size=n, dtype=np.uint8)
        assert np.array_equal(oracle.histogram(x), np.bincount(x, minlength=256).astype(np.uint64))


# ------------------------------------------------------------ lengths
def _kraft(lengths):
    return sum(Fraction(1, 2 ** int(l)) for l in lengths if l > 0)


def _brute_min_cost(freqs):
    """Minimum sum f*l over complete prefix codes: every multiset of lengths with
    Kraft sum exactly 1, paired shortest-with-most-frequent (rearrangement inequality)."""
    m = len(freqs)
    fs = sorted(freqs, reverse=True)
    best = None
    for ls in itertools.combinations_with_replacement(range(1, m), m):
        if sum(Fraction(1, 2 ** l) for l in ls) != 1:
            continue
        cost = sum(f * l for f, l in zip(fs, ls))
        best = cost if best is None else min(best, cost)
    return best


def _brute_min_cost_all_vectors(freqs):
    m = len(freqs)
    best = None
    for ls in itertools.product(range(1, m), repeat=m):
        if sum(Fraction(1, 2 ** l) for l in ls) == 1:
            cost = sum(f * l for f, l in zip(freqs, ls))
            best = cost if best is None else min(best, cost)
    return best


def test_optimal_cost_brute_force_small_alphabets():
    rng = random.Random(5)
    for trial in range(300):
        m = rng.randint(2, 8)
        syms = rng.sample(range(256), m)
        freq = np.zeros(256, dtype=np.uint64)
        for s in syms:
            freq[s] = rng.choice([1, 1, 2, 3, 5, 8, rng.randint(1, 1000)])
        lens = oracle.code_lengths(freq)
        cost = int(sum(int(freq[s]) * int(lens[s]) for s in syms))
        assert cost == _brute_min_cost([int(freq[s]) for s in syms]), (trial, freq[syms])
        if m <= 5:
            assert cost == _brute_min_cost_all_vectors([int(freq[s]) for s in syms])
        assert all(lens[s] > 0 for s in syms) and lens.sum() == sum(lens[s] for s in syms)


def test_kraft_sum_is_one():
    rng = np.random.default_rng(3)
    for _ in range(200):
        m = int(rng.integers(2, 257))
        freq = np.zeros(256, dtype=np.uint64)
        syms = rng.choice(256, size=m, replace=False)
        freq[syms] = rng.integers(1, 10**9, size=m).astype(np.uint64)
        assert _kraft(oracle.code_lengths(freq)) == 1


def test_dyadic_frequencies_give_exact_lengths():
    # p_k = 2^-k (k = 1..m-1) plus a second 2^-(m-1) symbol: Huffman gives len = k exactly
    for m in range(2, 40):
        freq = np.zeros(256, dtype=np.uint64)
        for k in range(1, m):
            freq[k] = 2 ** (m - 1 - k)
        freq[m] = 1
        lens = oracle.code_lengths(freq)
        want = [k for k in range(1, m)] + [m - 1]
        assert list(lens[1:m + 1]) == want


@pytest.mark.parametrize("m", [1, 2, 3, 4, 5, 6, 7, 8])
def test_uniform_power_of_two_alphabet(m):
    freq = np.zeros(256, dtype=np.uint64)
    freq[: 2 ** m] = 7
    lens = oracle.code_lengths(freq)
    assert set(lens[: 2 ** m].tolist()) == {m}
    assert lens[2 ** m:].sum() == 0


def test_fibonacci_weights_give_the_maximal_chain():
    # weights F1..Fm force a degenerate tree: one leaf per depth 1..m-2, two at m-1
    fib = [1, 1]
    while len(fib) < 60:
        fib.append(fib[-1] + fib[-2])
    for m in (3, 10, 33, 45, 60):
        freq = np.zeros(256, dtype=np.uint64)
        freq[:m] = fib[:m]
        lens = oracle.code_lengths(freq)
        assert sorted(lens[:m].tolist()) == sorted(list(range(1, m - 1)) + [m - 1, m - 1])
        assert _kraft(lens) == 1


def test_two_queue_form_equals_direct_form():
    rng = np.random.default_rng(17)
    for _ in range(400):
        m = int(rng.integers(0, 257))
        freq = np.zeros(256, dtype=np.uint64)
        syms = rng.choice(256, size=m, replace=False)
        # small weights make many ties, large ones few
        hi = int(rng.choice([3, 20, 10**6]))
        freq[syms] = rng.integers(1, hi, size=m).astype(np.uint64)
        assert np.array_equal(oracle.code_lengths(freq), oracle.code_lengths_two_queue(freq))


def test_special_cases_of_lengths():
    freq = np.zeros(256, dtype=np.uint64)
    assert oracle.code_lengths(freq).sum() == 0
    freq[200] = 5
    lens = oracle.code_lengths(freq)
    assert lens[200] == 1 and lens.sum() == 1
    freq[3] = 1
    lens = oracle.code_lengths(freq)
    assert lens[200] == 1 and lens[3] == 1


# ------------------------------------------------------------ canonical codes
def _check_canonical(lengths):
    codes = oracle.canonical_codes(lengths)
    present = [(int(lengths[s]), s) for s in range(256) if lengths[s] > 0]
    strs = {s: format(int(codes[s]), f"0{l}b") for l, s in present}
    for l, s in present:
        assert int(codes[s]) < 2 ** l
    # prefix-free
    items = sorted(strs.values())
    for a, b in zip(items, items[1:]):
        assert not b.startswith(a)
    # ordered: left-justified values increase in (length, symbol) order, consecutive within a length
    order = sorted(present)
    lj = [int(codes[s]) << (64 - l) for l, s in order]
    assert lj == sorted(lj) and len(set(lj)) == len(lj)
    for (l1, s1), (l2, s2) in zip(order, order[1:]):
        if l1 == l2:
            assert int(codes[s2]) == int(codes[s1]) + 1
    return codes


def test_canonical_codes_properties():
    rng = np.random.default_rng(23)
    for _ in range(100):
        m = int(rng.integers(2, 257))
        freq = np.zeros(256, dtype=np.uint64)
        freq[rng.choice(256, size=m, replace=False)] = rng.integers(1, 10**6, size=m).astype(np.uint64)
        _check_canonical(oracle.code_lengths(freq))


def test_canonical_codes_rfc1951_example():
    # RFC 1951 3.2.2 example: lengths (3,3,3,3,3,2,4,4) for A..H give
    # 010 011 100 101 110 00 1110 1111.
    lens = np.zeros(256, dtype=np.uint8)
    lens[65:73] = [3, 3, 3, 3, 3, 2, 4, 4]
    codes = _check_canonical(lens)
    want = ["010", "011", "100", "101", "110", "00", "1110", "1111"]
    assert [format(int(codes[65 + i]), f"0{int(lens[65 + i])}b") for i in range(8)] == want


def test_canonical_rejects_kraft_violation():
    lens = np.zeros(256, dtype=np.uint8)
    lens[:3] = 1
    with pytest.raises(oracle.OracleError):
        oracle.canonical_codes(lens)


# ------------------------------------------------------------ stream format
def _zipf_bytes(n, s, seed):
    rng = np.random.default_rng(seed)
    p = np.arange(1, 257, dtype=np.float64) ** -s
    return rng.choice(256, size=n, p=p / p.sum()).astype(np.uint8)


def _format_invariants(x, B, s):
    c = format_reader.read_container(s.tobytes())
    n = x.size
    assert c["n"] == n and c["B"] == B and c["nb"] == -(-n // B)
    assert c["end"] == s.size
    lengths = np.array(c["lengths"], dtype=np.uint8)
    freq = np.bincount(x, minlength=256)
    # Sec. 2.1: each delimiter is the sum of its block's code lengths
    total_bits = 0
    for k, rec in enumerate(c["records"]):
        blk = x[k * B:(k + 1) * B]
        assert rec["bits"] == int(lengths[blk].astype(np.int64).sum())
        overhead = 32 + (-rec["bits"]) % 32
        assert 32 <= overhead <= 63                         # Sec. 2.1: 32-63 bits per block
        total_bits += rec["bits"]
        if c["index"] is not None:
            assert c["index"][k] == rec["word_offset"]
    # sum of delimiters == sum over symbols of freq * len
    assert total_bits == int((freq * lengths.astype(np.int64)).sum())
    # closed-form size
    size = 280 + (4 * c["nb"] if c["index"] is not None else 0) + sum(
        4 * (1 + (r["bits"] + 31) // 32) for r in c["records"])
    assert size == s.size
    return c


@pytest.mark.parametrize("n,B", [(0, 1), (0, 4096), (1, 1), (1, 4096), (5, 1), (17, 3),
                                 (1000, 7), (4096, 4096), (4097, 4096), (10_000, 64),
                                 (3000, 1 << 24), (65_537, 65_536)])
def test_round_trip_and_invariants(n, B):
    x = _zipf_bytes(n, 1.1, n + B)
    s = oracle.compress(x, B)
    _format_invariants(x, B, s)
    assert np.array_equal(oracle.decompress(s), x)
    if n <= 20_000:
        assert format_reader.decode(s.tobytes()) == x.tobytes()


def test_empty_input_is_header_only():
    s = oracle.compress(np.zeros(0, dtype=np.uint8), 4096)
    assert s.size == 280
    assert s[:4].tobytes() == b"HZB1" and s[24:280].sum() == 0


def test_single_symbol_and_two_symbols():
    x = np.full(1000, 42, dtype=np.uint8)
    s = oracle.compress(x, 100)
    c = _format_invariants(x, 100, s)
    assert c["lengths"][42] == 1 and sum(c["lengths"]) == 1
    assert all(r["bits"] == 100 and r["words"] == [0] * 4 for r in c["records"])
    assert np.array_equal(oracle.decompress(s), x)
    x2 = np.array([1, 2] * 50 + [2], dtype=np.uint8)
    s2 = oracle.compress(x2, 8)
    assert np.array_equal(oracle.decompress(s2), x2)
    assert format_reader.decode(s2.tobytes()) == x2.tobytes()


def test_all_256_uniform_gives_eight_bit_codes():
    x = np.tile(np.arange(256, dtype=np.uint8), 64)
    s = oracle.compress(x, 1024)
    c = _format_invariants(x, 1024, s)
    assert set(c["lengths"]) == {8}
    # 8-bit canonical codes are the identity: each payload is the raw bytes, big-endian per word
    rec = c["records"][0]
    assert rec["bits"] == 8192 and rec["words"][0] == 0x00010203


def test_no_index_mode_round_trips():
    x = _zipf_bytes(20_000, 1.3, 9)
    s = oracle.compress(x, 1000, index=False)
    c = _format_invariants(x, 1000, s)
    assert c["index"] is None and c["flags"] == 0
    assert np.array_equal(oracle.decompress(s), x)
    assert s.size == oracle.compress(x, 1000).size - 4 * 20


def test_long_codes_beyond_32_and_48_bits():
    # Kraft-complete chain 1,2,...,62,63,63 over 64 symbols: codes up to 63 bits
    lens = np.zeros(256, dtype=np.uint8)
    lens[:62] = np.arange(1, 63)
    lens[62] = 63
    lens[63] = 63
    assert _kraft(lens) == 1
    rng = np.random.default_rng(4)
    x = rng.integers(0, 64, size=3000, dtype=np.uint8)
    x[:10] = [63, 62, 61, 40, 33, 32, 31, 0, 1, 63]
    s = oracle.compress(x, 37, lengths=lens)
    c = _format_invariants(x, 37, s)
    assert max(c["lengths"]) == 63
    assert np.array_equal(oracle.decompress(s), x)
    assert format_reader.decode(s.tobytes()) == x.tobytes()


def test_given_lengths_must_cover_the_data():
    lens = np.zeros(256, dtype=np.uint8)
    lens[:2] = 1
    with pytest.raises(oracle.OracleError):
        oracle.compress(np.array([0, 1, 2], dtype=np.uint8), 4, lengths=lens)


def test_encode_block_equals_stream_records():
    x = _zipf_bytes(50_000, 0.9, 1)
    B = 4096
    s = oracle.compress(x, B)
    c = format_reader.read_container(s.tobytes())
    lengths = np.array(c["lengths"], dtype=np.uint8)
    for k in (0, 3, len(c["records"]) - 1):
        words = oracle.encode_block(x[k * B:(k + 1) * B], lengths)
        rec = c["records"][k]
        assert words.tolist() == [rec["bits"]] + rec["words"]


def test_overhead_below_one_percent_for_large_blocks():
    # Sec. 2.1 / Fig. 5: constant bytes per block, so the share shrinks with block size
    x = _zipf_bytes(1 << 20, 1.1, 0)
    shares = []
    for B in (256, 4096, 65536):
        c = format_reader.read_container(oracle.compress(x, B).tobytes())
        payload = sum(r["bits"] for r in c["records"])
        over = sum(32 + (-r["bits"]) % 32 for r in c["records"])
        shares.append(over / payload)
    assert shares[0] > shares[1] > shares[2]
    assert shares[2] < 0.01


# ------------------------------------------------------------ corrupt streams
def test_corrupt_streams_are_rejected():
    x = _zipf_bytes(5000, 1.1, 2)
    s = oracle.compress(x, 512)
    bad = []
    b = s.copy(); b[0] ^= 1; bad.append(b)                          # magic
    bad.append(s[:-4].copy())                                       # truncated
    bad.append(np.concatenate([s, np.zeros(4, np.uint8)]))          # trailing bytes
    b = s.copy(); b[280] ^= 1; bad.append(b)                        # index entry
    c = format_reader.read_container(s.tobytes())
    blocks_at = 280 + 4 * c["nb"]
    b = s.copy(); b[blocks_at] ^= 1; bad.append(b)                  # first delimiter
    b = s.copy(); b[4] = 2; bad.append(b)                           # unknown flag
    b = s.copy(); b[24:280] = 0; bad.append(b)                      # no code at all
    b = s.copy(); b[16] = 0; b[17] = 0; bad.append(b)               # B inconsistent with nb
    # a nonzero padding bit in the first record
    r0 = c["records"][0]
    if r0["bits"] % 32:
        last = blocks_at + 4 * (r0["word_offset"] + (r0["bits"] + 31) // 32)
        b = s.copy(); b[last] |= 1; bad.append(b)
    for b in bad:
        with pytest.raises(oracle.OracleError) as e:
            oracle.decompress(b)
        assert e.value.status == oracle.ERR_CORRUPT


# ------------------------------------------------------------ sub-block offsets (R14)
@pytest.mark.parametrize("n,B,S", [(0, 64, 32), (1, 64, 32), (100, 64, 32), (4096, 4096, 2048),
                                   (4097, 4096, 1024), (70_001, 65_536, 2048),
                                   (10_000, 96, 32), (5000, 2048, 2048), (3000, 64, 64)])
def test_sub_block_offsets_round_trip_and_invariants(n, B, S):
    x = _zipf_bytes(n, 1.1, n + 3 * B + S)
    s = oracle.compress(x, B, sub=S)
    c = format_reader.read_container(s.tobytes())
    assert c["flags"] == 3 and c["S"] == S and c["end"] == s.size
    lengths = np.array(c["lengths"], dtype=np.int64)
    M = B // S
    for k, rec in enumerate(c["records"]):
        blk = x[k * B:(k + 1) * B]
        # entry j: the sum of the code lengths of the block's first j*S symbols
        want = [int(lengths[blk[:j * S]].sum()) for j in range(1, M)]
        assert c["sub"][k] == want
        assert all(0 < e <= rec["bits"] for e in want)
    # the records are those of the stream without the section
    plain = format_reader.read_container(oracle.compress(x, B).tobytes())
    assert [r["words"] for r in plain["records"]] == [r["words"] for r in c["records"]]
    assert s.size == oracle.compress(x, B).size + 4 + 4 * c["nb"] * (M - 1)
    assert np.array_equal(oracle.decompress(s), x)
    if n <= 20_000:
        assert format_reader.decode(s.tobytes()) == x.tobytes()


def test_sub_block_layout_is_checked():
    x = _zipf_bytes(1000, 1.1, 1)
    for B, S in ((64, 48), (64, 16), (96, 64), (32, 64)):  # S not a multiple of 32 dividing B
        with pytest.raises(oracle.OracleError):
            oracle.compress(x, B, sub=S)
    with pytest.raises(oracle.OracleError):  # bit 1 needs bit 0
        oracle.compress(x, 64, index=False, sub=32)


def test_corrupt_sub_block_offsets_are_rejected():
    x = _zipf_bytes(9000, 1.2, 4)
    s = oracle.compress(x, 1024, sub=256)
    c = format_reader.read_container(s.tobytes())
    sec = 280 + 4 * c["nb"]          # the section: S, then 3 entries per block
    bad = []
    b = s.copy(); b[sec] = 64; bad.append(b)                      # S that does not match
    b = s.copy(); b[sec + 4] ^= 1; bad.append(b)                  # first entry off by one
    last = sec + 4 + 4 * 3 * (c["nb"] - 1) + 8                    # the last block's last entry
    b = s.copy(); b[last] ^= 2; bad.append(b)                     # past its end: must be bits_k
    b = s.copy(); b[4] = 2; bad.append(b)                         # bit 1 without bit 0
    for b in bad:
        with pytest.raises(oracle.OracleError) as e:
            oracle.decompress(b)
        assert e.value.status == oracle.ERR_CORRUPT
        with pytest.raises((ValueError, struct.error)):  # the naive reader fails too
            format_reader.decode(b.tobytes())


# ------------------------------------------------------------ OpenMP driver
@pytest.mark.parametrize("threads", [1, 3, 0])
def test_openmp_driver_writes_the_oracle_stream(threads):
    rng = np.random.default_rng(8)
    cases = [(0, 4096, 0), (1, 1, 0), (17, 3, 0), (100_003, 1000, 0), (300_000, 65_536, 2048),
             (50_000, 4096, 1024), (65_537, 65_536, 0)]
    for n, B, S in cases:
        x = _zipf_bytes(n, float(rng.uniform(0.7, 1.6)), n + B)
        for index in (True, False):
            if S and not index:
                continue
            want = oracle.compress(x, B, index=index, sub=S)
            got = oracle.compress_omp(x, B, index=index, sub=S, threads=threads)
            assert np.array_equal(got, want), (n, B, S, index)
            assert np.array_equal(oracle.decompress_omp(want, threads=threads), x)
    # a given code, as for the sequential form
    lens = np.zeros(256, dtype=np.uint8)
    lens[:62] = np.arange(1, 63)
    lens[62:64] = 63
    x = rng.integers(0, 64, size=5000, dtype=np.uint8)
    assert np.array_equal(oracle.compress_omp(x, 37, lengths=lens, threads=threads),
                          oracle.compress(x, 37, lengths=lens))
    assert oracle.omp_threads(threads) == (threads if threads else oracle.omp_threads(0))


def test_openmp_driver_rejects_what_the_oracle_rejects():
    x = _zipf_bytes(5000, 1.1, 2)
    s = oracle.compress(x, 512, sub=256)
    for b in (s[:-4].copy(), np.concatenate([s, np.zeros(4, np.uint8)])):
        with pytest.raises(oracle.OracleError) as e:
            oracle.decompress_omp(b)
        assert e.value.status == oracle.ERR_CORRUPT
    b = s.copy(); b[280 + 4 * 10 + 8] ^= 1
    with pytest.raises(oracle.OracleError):
        oracle.decompress_omp(b)
    with pytest.raises(oracle.OracleError):
        oracle.compress_omp(x, 64, sub=48)
