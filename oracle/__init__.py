"""CPU oracle for the block-decomposed Huffman coder (test infrastructure).

This package is the checker, not the product.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
it.  It wraps ``hz_oracle.c`` (plain C, standard library only) and
``hz_oracle_omp.c`` (the same functions called for independent blocks from
OpenMP loops: the paper's parallel CPU coder, Sec. 3.1-3.2), which it builds
with gcc on first use, and shares nothing with the CUDA library.

Every function cites the part of Cloud et al. (arXiv 1107.1525) it follows;
the C source states the readings taken where the paper is silent.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hz_oracle.c")
_SRC_OMP = os.path.join(_HERE, "hz_oracle_omp.c")
_HDR = os.path.join(_HERE, "hz_oracle.h")
_LIB_PATH = os.path.join(_HERE, "libhz_oracle.so")
_lock = threading.Lock()
_lib = None

OK, ERR_ARG, ERR_CAPACITY, ERR_CORRUPT, ERR_NOMEM = 0, -1, -2, -3, -4
HEADER_BYTES = 280
FLAG_INDEX = 1
FLAG_SUB = 2
_NAMES = {ERR_ARG: "ERR_ARG", ERR_CAPACITY: "ERR_CAPACITY", ERR_CORRUPT: "ERR_CORRUPT",
          ERR_NOMEM: "ERR_NOMEM"}


class OracleError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {_NAMES.get(status, status)}")
        self.status = status


def build(force: bool = False) -> str:
    """Compile hz_oracle.c (plain) and hz_oracle_omp.c (with -fopenmp) into
    libhz_oracle.so with gcc (no CUDA involved)."""
    with _lock:
        newest = max(os.path.getmtime(f) for f in (_SRC, _SRC_OMP, _HDR))
        stale = not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < newest
        if force or stale:
            tmp = _LIB_PATH + f".{os.getpid()}.tmp"
            objs = [tmp + ".a.o", tmp + ".b.o"]
            common = ["gcc", "-O2", "-std=c11", "-Wall", "-Wextra", "-fPIC", "-c"]
            subprocess.run(common + ["-o", objs[0], _SRC], check=True)
            subprocess.run(common + ["-fopenmp", "-o", objs[1], _SRC_OMP], check=True)
            subprocess.run(["gcc", "-shared", "-fopenmp", "-o", tmp] + objs, check=True)
            for o in objs:
                os.remove(o)
            os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB_PATH)
    P, U8P, U32P, U64P = ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p
    u64, u32, i32 = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int
    lib.oracle_histogram.argtypes = [U8P, u64, U64P]
    lib.oracle_histogram.restype = None
    lib.oracle_code_lengths.argtypes = [U64P, U8P]
    lib.oracle_code_lengths.restype = i32
    lib.oracle_code_lengths_two_queue.argtypes = [U64P, U8P]
    lib.oracle_code_lengths_two_queue.restype = i32
    lib.oracle_canonical_codes.argtypes = [U8P, U64P]
    lib.oracle_canonical_codes.restype = i32
    lib.oracle_block_bits.argtypes = [U8P, u64, U8P]
    lib.oracle_block_bits.restype = u64
    lib.oracle_encode_block.argtypes = [U8P, u64, U8P, U64P, U32P, u64]
    lib.oracle_encode_block.restype = u64
    lib.oracle_stream_size.argtypes = [U8P, u64, u32, U8P, u32, u32, ctypes.POINTER(u64)]
    lib.oracle_stream_size.restype = i32
    lib.oracle_sub_offsets.argtypes = [U8P, u64, U8P, u32, u32, U32P]
    lib.oracle_sub_offsets.restype = None
    lib.oracle_compress.argtypes = [U8P, u64, u32, U8P, u32, u32, U8P, u64, ctypes.POINTER(u64)]
    lib.oracle_compress.restype = i32
    lib.oracle_decompress.argtypes = [U8P, u64, U8P, u64, ctypes.POINTER(u64)]
    lib.oracle_decompress.restype = i32
    lib.oracle_compress_omp.argtypes = [U8P, u64, u32, U8P, u32, u32, U8P, u64,
                                        ctypes.POINTER(u64), i32]
    lib.oracle_compress_omp.restype = i32
    lib.oracle_decompress_omp.argtypes = [U8P, u64, U8P, u64, ctypes.POINTER(u64), i32]
    lib.oracle_decompress_omp.restype = i32
    lib.oracle_omp_threads.argtypes = [i32]
    lib.oracle_omp_threads.restype = i32
    lib.oracle_parse_header.argtypes = [U8P, u64, ctypes.POINTER(u64), ctypes.POINTER(u32),
                                        ctypes.POINTER(u32), ctypes.POINTER(u32),
                                        ctypes.POINTER(u32), U8P]
    lib.oracle_parse_header.restype = i32
    del P
    _lib = lib
    return lib


def _u8(a) -> np.ndarray:
    a = np.ascontiguousarray(np.frombuffer(a, dtype=np.uint8) if isinstance(a, (bytes, bytearray))
                             else a)
    if a.dtype != np.uint8:
        raise TypeError("expected uint8 data")
    return a.reshape(-1)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def histogram(x) -> np.ndarray:
    """Sec. 2: occurrences of every byte value in the uncompressed data (uint64[256])."""
    x = _u8(x)
    freq = np.zeros(256, dtype=np.uint64)
    _load().oracle_histogram(_ptr(x), x.size, _ptr(freq))
    return freq


def code_lengths(freq) -> np.ndarray:
    """Sec. 2 / Fig. 2: Huffman code lengths (leaf depths), direct form, tie-break R1."""
    freq = np.ascontiguousarray(freq, dtype=np.uint64)
    out = np.zeros(256, dtype=np.uint8)
    st = _load().oracle_code_lengths(_ptr(freq), _ptr(out))
    if st != OK:
        raise OracleError(st, "code_lengths")
    return out


def code_lengths_two_queue(freq) -> np.ndarray:
    """Same lengths by the two-queue construction (must equal code_lengths)."""
    freq = np.ascontiguousarray(freq, dtype=np.uint64)
    out = np.zeros(256, dtype=np.uint8)
    st = _load().oracle_code_lengths_two_queue(_ptr(freq), _ptr(out))
    if st != OK:
        raise OracleError(st, "code_lengths_two_queue")
    return out


def canonical_codes(lengths) -> np.ndarray:
    """Reading R2: canonical code values (uint64[256]) for a length table."""
    lengths = np.ascontiguousarray(lengths, dtype=np.uint8)
    out = np.zeros(256, dtype=np.uint64)
    st = _load().oracle_canonical_codes(_ptr(lengths), _ptr(out))
    if st != OK:
        raise OracleError(st, "canonical_codes")
    return out


def block_bits(x, lengths) -> int:
    """Sec. 2.1: the extra pass -- sum of the code lengths of one block's symbols."""
    x = _u8(x)
    lengths = np.ascontiguousarray(lengths, dtype=np.uint8)
    return int(_load().oracle_block_bits(_ptr(x), x.size, _ptr(lengths)))


def encode_block(x, lengths) -> np.ndarray:
    """Sec. 2.1 / Fig. 4: one block record as uint32 words (delimiter, payload)."""
    x = _u8(x)
    lengths = np.ascontiguousarray(lengths, dtype=np.uint8)
    codes = canonical_codes(lengths)
    cap = 1 + (block_bits(x, lengths) + 31) // 32
    words = np.zeros(cap, dtype=np.uint32)
    got = _load().oracle_encode_block(_ptr(x), x.size, _ptr(lengths), _ptr(codes), _ptr(words),
                                      cap)
    if got != cap:
        raise OracleError(ERR_CAPACITY, "encode_block")
    return words


def _flags(index: bool, sub: int) -> int:
    return (FLAG_INDEX if index else 0) | (FLAG_SUB if sub else 0)


def stream_size(x, block_size: int, lengths, index: bool = True, sub: int = 0) -> int:
    """Exact stream size in bytes for x under a length table."""
    x = _u8(x)
    lengths = np.ascontiguousarray(lengths, dtype=np.uint8)
    size = ctypes.c_uint64(0)
    st = _load().oracle_stream_size(_ptr(x), x.size, block_size, _ptr(lengths),
                                    _flags(index, sub), sub, ctypes.byref(size))
    if st != OK:
        raise OracleError(st, "stream_size")
    return int(size.value)


def sub_offsets(x, lengths, S: int, M: int) -> np.ndarray:
    """Reading R14: payload bit of the code of symbol j*S of one block, j = 1..M-1."""
    x = _u8(x)
    lengths = np.ascontiguousarray(lengths, dtype=np.uint8)
    out = np.zeros(max(M - 1, 1), dtype=np.uint32)
    _load().oracle_sub_offsets(_ptr(x), x.size, _ptr(lengths), S, M, _ptr(out))
    return out[: max(M - 1, 0)]


def _compress_with(fn, x, block_size, lengths, index, sub, *extra):
    x = _u8(x)
    given = None
    if lengths is not None:
        given = np.ascontiguousarray(lengths, dtype=np.uint8)
    out_len = ctypes.c_uint64(0)
    flags = _flags(index, sub)
    gp = _ptr(given) if given is not None else None
    st = fn(_ptr(x), x.size, block_size, gp, flags, sub, None, 0, ctypes.byref(out_len), *extra)
    if st not in (OK, ERR_CAPACITY):
        raise OracleError(st, "compress")
    out = np.zeros(max(int(out_len.value), 1), dtype=np.uint8)
    st = fn(_ptr(x), x.size, block_size, gp, flags, sub, _ptr(out), out.size,
            ctypes.byref(out_len), *extra)
    if st != OK:
        raise OracleError(st, "compress")
    return out[: int(out_len.value)]


def compress(x, block_size: int, lengths=None, index: bool = True, sub: int = 0) -> np.ndarray:
    """Sec. 2-2.1: the whole compressed stream (uint8 array) for x.  sub = S > 0
    adds the sub-block offsets of every S symbols (reading R14)."""
    return _compress_with(_load().oracle_compress, x, block_size, lengths, index, sub)


def compress_omp(x, block_size: int, lengths=None, index: bool = True, sub: int = 0,
                 threads: int = 0) -> np.ndarray:
    """compress() with the oracle's block steps spread over host threads (OpenMP,
    Sec. 3.1's parallel CPU encoder); the stream is the same byte for byte."""
    return _compress_with(_load().oracle_compress_omp, x, block_size, lengths, index, sub,
                          threads)


def _decompress_with(fn, stream, *extra):
    s = _u8(stream)
    hdr = parse_header(s)
    out = np.zeros(max(hdr["n"], 1), dtype=np.uint8)
    n_out = ctypes.c_uint64(0)
    st = fn(_ptr(s), s.size, _ptr(out), out.size, ctypes.byref(n_out), *extra)
    if st != OK:
        raise OracleError(st, "decompress")
    return out[: int(n_out.value)]


def decompress(stream) -> np.ndarray:
    """Sec. 2.1: decode every block of a stream; raises OracleError on corrupt input."""
    return _decompress_with(_load().oracle_decompress, stream)


def decompress_omp(stream, threads: int = 0) -> np.ndarray:
    """decompress() with the blocks decoded on host threads (OpenMP, Sec. 3.2)."""
    return _decompress_with(_load().oracle_decompress_omp, stream, threads)


def omp_threads(threads: int = 0) -> int:
    """Host threads the OpenMP driver uses for `threads` (0 = all it is offered)."""
    return int(_load().oracle_omp_threads(threads))


def parse_header(stream) -> dict:
    """Container header fields: n, flags, B, nb, the sub-block size S (0 without
    the sub-block section) and the 256 code lengths."""
    s = _u8(stream)
    n = ctypes.c_uint64(0)
    flags, B, nb, S = (ctypes.c_uint32(0) for _ in range(4))
    lengths = np.zeros(256, dtype=np.uint8)
    st = _load().oracle_parse_header(_ptr(s) if s.size else None, s.size, ctypes.byref(n),
                                     ctypes.byref(flags), ctypes.byref(B), ctypes.byref(nb),
                                     ctypes.byref(S), _ptr(lengths))
    if st != OK:
        raise OracleError(st, "parse_header")
    return {"n": int(n.value), "flags": int(flags.value), "B": int(B.value),
            "nb": int(nb.value), "S": int(S.value), "lengths": lengths}
