"""Thin ctypes binding over libhz's C ABI (include/hz.h).

Argument marshalling only: every function here forwards to the C entry point of
the same name, turning torch tensors into device pointers and torch streams
into cudaStream_t handles.  All work runs in libhz's CUDA kernels.  There is no
CPU fallback: importing this module without a built libhz.so raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhz.so")

HZ_OK, HZ_PENDING = 0, 1
HZ_ERR_ARG, HZ_ERR_CAPACITY, HZ_ERR_CORRUPT, HZ_ERR_NOMEM = -1, -2, -3, -4
HZ_ERR_BUSY, HZ_ERR_TIMEOUT, HZ_ERR_CUDA = -5, -6, -7
STATUS_NAMES = {0: "HZ_OK", 1: "HZ_PENDING", -1: "HZ_ERR_ARG", -2: "HZ_ERR_CAPACITY",
                -3: "HZ_ERR_CORRUPT", -4: "HZ_ERR_NOMEM", -5: "HZ_ERR_BUSY",
                -6: "HZ_ERR_TIMEOUT", -7: "HZ_ERR_CUDA"}
HEADER_BYTES = 280
HZ_OPT_INDEX, HZ_OPT_PROFILE, HZ_OPT_DECODE_LUT_BITS = 1, 2, 3
HZ_OPT_DECODE_THREADS, HZ_OPT_AUTOTUNE, HZ_OPT_BATCH_PLAIN = 4, 5, 6
HZ_OPT_BATCH_MAX_REQS, HZ_OPT_SUB_BLOCK = 7, 8
HZ_OPT_SPIN_LIMIT, HZ_OPT_INJECT_SCAN_STALL, HZ_OPT_TUNE_BATCHED = 9, 10, 11
HZ_SUB_BLOCK_AUTO = 1  # HZ_OPT_SUB_BLOCK value: S picked per call
HZ_OP_COMPRESS, HZ_OP_DECOMPRESS = 0, 1

# the C symbols include/hz.h declares (checked by the test suite)
EXPORTS = ("hz_create", "hz_destroy", "hz_compress_bound", "hz_compress_bound_ctx",
           "hz_build_codes", "hz_compress",
           "hz_decompress", "hz_sync", "hz_compress_host", "hz_decompress_host",
           "hz_set_option", "hz_get_option", "hz_launch_count", "hz_profile_read",
           "hz_kernel_name", "hz_submit", "hz_poll", "hz_compress_noalloc", "hz_autotune",
           "hz_tuned_block_size", "hz_serve_replay")


class HzError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        super().__init__(f"{what}: {STATUS_NAMES.get(status, status)}")
        self.status = status


class HzCodes(ctypes.Structure):
    _fields_ = [("len", ctypes.c_uint8 * 256), ("code", ctypes.c_uint64 * 256)]


class HzRequest(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int32), ("block_size", ctypes.c_uint32),
                ("d_src", ctypes.c_void_p), ("src_len", ctypes.c_uint64),
                ("d_dst", ctypes.c_void_p), ("dst_cap", ctypes.c_uint64)]


# hz_serve_item / hz_serve_record as numpy record types (same layout as the C structs)
SERVE_ITEM = np.dtype([("arrival_s", "<f8"), ("op", "<i4"), ("block_size", "<u4"),
                       ("d_src", "<u8"), ("src_len", "<u8"), ("d_dst", "<u8"),
                       ("dst_cap", "<u8")])
SERVE_RECORD = np.dtype([("submit_s", "<f8"), ("done_s", "<f8"), ("out_len", "<u8"),
                         ("launch", "<u8"), ("dst_offset", "<u8"), ("status", "<i4"),
                         ("pad", "<u4")])

_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libhz.so (raises OSError when it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError(f"libhz.so not built at {path}: run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    vp, u64, u32, i32, i64 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int32, \
        ctypes.c_int64
    sig = {
        "hz_create": (i32, [ctypes.POINTER(vp), ctypes.c_int, u64]),
        "hz_destroy": (None, [vp]),
        "hz_compress_bound": (u64, [u64, u32]),
        "hz_compress_bound_ctx": (u64, [vp, u64, u32]),
        "hz_build_codes": (i32, [vp, vp, u64, ctypes.POINTER(HzCodes), vp]),
        "hz_compress": (i32, [vp, vp, u64, u32, ctypes.POINTER(HzCodes), vp, u64, vp, vp]),
        "hz_decompress": (i32, [vp, vp, u64, vp, u64, vp, vp]),
        "hz_sync": (i32, [vp, vp]),
        "hz_compress_host": (i32, [vp, vp, u64, u32, vp, u64, ctypes.POINTER(u64), vp]),
        "hz_decompress_host": (i32, [vp, vp, u64, vp, u64, ctypes.POINTER(u64), vp]),
        "hz_set_option": (i32, [vp, ctypes.c_int, i64]),
        "hz_get_option": (i64, [vp, ctypes.c_int]),
        "hz_launch_count": (u64, [vp]),
        "hz_profile_read": (ctypes.c_int, [vp, vp, vp, ctypes.c_int]),
        "hz_kernel_name": (ctypes.c_char_p, [i32]),
        "hz_submit": (i32, [vp, ctypes.POINTER(HzRequest), u32, ctypes.POINTER(u64), vp]),
        "hz_poll": (i32, [vp, u64, i64, vp, vp]),
        "hz_compress_noalloc": (i32, [vp, u64, u32, vp, u64, vp, vp, vp]),
        "hz_autotune": (i32, [vp, vp, u64, vp]),
        "hz_tuned_block_size": (u32, [vp, u64]),
        "hz_serve_replay": (i32, [vp, vp, u64, vp, u64, vp, ctypes.POINTER(ctypes.c_double)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _ptr(x) -> int | None:
    """Device/host address of a tensor / ndarray, or an int / None as given."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)}")


def _stream(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _check(st: int, what: str) -> int:
    if st < 0:
        raise HzError(st, what)
    return st


class Context:
    """Owns an hz_ctx*; every call below goes straight to the C ABI."""

    def __init__(self, device: int = 0, mem_budget: int = 0):
        self._lib = load_library()
        h = ctypes.c_void_p()
        _check(self._lib.hz_create(ctypes.byref(h), device, mem_budget), "hz_create")
        self.handle = h
        self.device = device

    def close(self):
        if getattr(self, "handle", None):
            self._lib.hz_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_option(self, key: int, value: int):
        _check(self._lib.hz_set_option(self.handle, key, value), "hz_set_option")

    def get_option(self, key: int) -> int:
        return int(self._lib.hz_get_option(self.handle, key))

    def launch_count(self) -> int:
        return int(self._lib.hz_launch_count(self.handle))

    def profile_read(self, max_records: int = 1 << 16):
        ids = np.zeros(max_records, dtype=np.int32)
        ms = np.zeros(max_records, dtype=np.float32)
        k = self._lib.hz_profile_read(self.handle, ids.ctypes.data, ms.ctypes.data, max_records)
        return [(self._lib.hz_kernel_name(int(i)).decode(), float(t)) for i, t in
                zip(ids[:k], ms[:k])]


# ------------------------------------------------------- the C entry points
def hz_create(device: int = 0, mem_budget: int = 0) -> Context:
    return Context(device, mem_budget)


def hz_destroy(ctx: Context):
    ctx.close()


def hz_compress_bound(n: int, block_size: int) -> int:
    return int(load_library().hz_compress_bound(n, block_size))


def hz_compress_bound_ctx(ctx: Context, n: int, block_size: int) -> int:
    return int(ctx._lib.hz_compress_bound_ctx(ctx.handle, n, block_size))


def hz_build_codes(ctx: Context, d_in, n: int, stream=None):
    """Returns (lengths uint8[256], codes uint64[256])."""
    c = HzCodes()
    _check(ctx._lib.hz_build_codes(ctx.handle, _ptr(d_in), n, ctypes.byref(c), _stream(stream)),
           "hz_build_codes")
    return (np.frombuffer(bytes(c.len), dtype=np.uint8).copy(),
            np.array(list(c.code), dtype=np.uint64))


def make_codes(lengths, codes) -> HzCodes:
    c = HzCodes()
    for s in range(256):
        c.len[s] = int(lengths[s])
        c.code[s] = int(codes[s])
    return c


def hz_compress(ctx: Context, d_in, n: int, block_size: int, codes, d_out, out_cap: int,
                d_out_len, stream=None) -> int:
    cp = ctypes.byref(codes) if codes is not None else None
    return _check(ctx._lib.hz_compress(ctx.handle, _ptr(d_in), n, block_size, cp, _ptr(d_out),
                                       out_cap, _ptr(d_out_len), _stream(stream)), "hz_compress")


def hz_decompress(ctx: Context, d_in, in_len: int, d_out, out_cap: int, d_out_len,
                  stream=None) -> int:
    return _check(ctx._lib.hz_decompress(ctx.handle, _ptr(d_in), in_len, _ptr(d_out), out_cap,
                                         _ptr(d_out_len), _stream(stream)), "hz_decompress")


def hz_compress_noalloc(d_in, n: int, block_size: int, d_out, out_cap: int, d_out_len,
                        d_status, stream=None) -> int:
    """No context, no device allocation (scratch is a fixed device array; n <= 2^28)."""
    return _check(load_library().hz_compress_noalloc(_ptr(d_in), n, block_size, _ptr(d_out),
                                                     out_cap, _ptr(d_out_len), _ptr(d_status),
                                                     _stream(stream)), "hz_compress_noalloc")


def hz_autotune(ctx: Context, d_sample, n: int, stream=None) -> int:
    return _check(ctx._lib.hz_autotune(ctx.handle, _ptr(d_sample), n, _stream(stream)),
                  "hz_autotune")


def hz_tuned_block_size(ctx: Context, n: int) -> int:
    return int(ctx._lib.hz_tuned_block_size(ctx.handle, n))


def hz_sync(ctx: Context, stream=None) -> int:
    """Returns the device status (0 or a negative HZ_ERR_*); does not raise."""
    return int(ctx._lib.hz_sync(ctx.handle, _stream(stream)))


def hz_compress_host(ctx: Context, h_in, n: int, block_size: int, h_out, out_cap: int,
                     stream=None):
    """Returns (status, out_len)."""
    out_len = ctypes.c_uint64(0)
    st = ctx._lib.hz_compress_host(ctx.handle, _ptr(h_in), n, block_size, _ptr(h_out), out_cap,
                                   ctypes.byref(out_len), _stream(stream))
    return int(st), int(out_len.value)


def hz_decompress_host(ctx: Context, h_in, in_len: int, h_out, out_cap: int, stream=None):
    out_len = ctypes.c_uint64(0)
    st = ctx._lib.hz_decompress_host(ctx.handle, _ptr(h_in), in_len, _ptr(h_out), out_cap,
                                     ctypes.byref(out_len), _stream(stream))
    return int(st), int(out_len.value)


def hz_submit(ctx: Context, requests, stream=None) -> int:
    """requests: sequence of (op, block_size, d_src, src_len, d_dst, dst_cap); the
    batch runs after the work queued on `stream` (default: torch's current stream)."""
    arr = (HzRequest * max(1, len(requests)))()
    for i, (op, bs, src, src_len, dst, cap) in enumerate(requests):
        arr[i] = HzRequest(op, bs, _ptr(src), src_len, _ptr(dst), cap)
    ticket = ctypes.c_uint64(0)
    _check(ctx._lib.hz_submit(ctx.handle, arr, len(requests), ctypes.byref(ticket),
                              _stream(stream)), "hz_submit")
    return int(ticket.value)


def hz_poll(ctx: Context, ticket: int, count: int, timeout_ns: int = -1):
    """Returns (status, per-request statuses, per-request output sizes)."""
    per = np.zeros(max(1, count), dtype=np.int32)
    lens = np.zeros(max(1, count), dtype=np.uint64)
    st = ctx._lib.hz_poll(ctx.handle, ticket, timeout_ns, per.ctypes.data, lens.ctypes.data)
    return int(st), per[:count], lens[:count]


def hz_serve_replay(ctx: Context, items: np.ndarray, ring=None, ring_bytes: int | None = None):
    """Replay `items` (a SERVE_ITEM array sorted by arrival_s; d_dst 0 = use the
    ring) open-loop; returns (SERVE_RECORD array, wall seconds)."""
    items = np.ascontiguousarray(items, dtype=SERVE_ITEM)
    rec = np.zeros(len(items), dtype=SERVE_RECORD)
    wall = ctypes.c_double(0.0)
    if ring_bytes is None:
        ring_bytes = ring.numel() if ring is not None else 0
    _check(ctx._lib.hz_serve_replay(ctx.handle, items.ctypes.data if len(items) else None,
                                    len(items), _ptr(ring), ring_bytes,
                                    rec.ctypes.data if len(items) else None, ctypes.byref(wall)),
           "hz_serve_replay")
    return rec, float(wall.value)


# ------------------------------------------------ tensor-level conveniences
def compress(x, block_size: int = 0, ctx: Context | None = None, codes=None, stream=None):
    """Compress a CUDA uint8 tensor; returns the stream as a CUDA uint8 tensor."""
    import torch
    ctx = ctx or default_context(x.device.index or 0)
    n = x.numel()
    cap = hz_compress_bound_ctx(ctx, n, block_size) if codes is None else 280 + 16 * n + 4096
    out = torch.empty(cap, dtype=torch.uint8, device=x.device)
    out_len = torch.zeros(1, dtype=torch.int64, device=x.device)
    hz_compress(ctx, x, n, block_size, codes, out, cap, out_len, stream)
    st = hz_sync(ctx, stream)
    if st != HZ_OK:
        raise HzError(st, "compress")
    return out[: int(out_len.item())]


def decompress(s, ctx: Context | None = None, out=None, stream=None):
    """Decompress a CUDA uint8 stream tensor; returns the data as a CUDA uint8 tensor."""
    import torch
    ctx = ctx or default_context(s.device.index or 0)
    if out is None:
        hdr = s[:24].cpu().numpy().tobytes()
        n = int.from_bytes(hdr[8:16], "little") if len(hdr) >= 16 else 0
        out = torch.empty(max(n, 1), dtype=torch.uint8, device=s.device)
    out_len = torch.zeros(1, dtype=torch.int64, device=s.device)
    hz_decompress(ctx, s, s.numel(), out, out.numel(), out_len, stream)
    st = hz_sync(ctx, stream)
    if st != HZ_OK:
        raise HzError(st, "decompress")
    return out[: int(out_len.item())]


_default = {}


def default_context(device: int = 0) -> Context:
    if device not in _default:
        _default[device] = Context(device)
    return _default[device]
