"""Host-side checks of the C ABI library (no GPU needed): it loads, exports every
entry point include/hz.h declares, and its pure host functions behave."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1107_1525_gb300 import build
    build.build()
    import paper_1107_1525_gb300.hz as hz
    return hz.load_library()


def _declared():
    text = open(os.path.join(ROOT, "include", "hz.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hz_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = _declared()
    for want in ("hz_build_codes", "hz_compress", "hz_decompress", "hz_submit", "hz_poll",
                 "hz_create", "hz_destroy", "hz_sync", "hz_compress_bound"):
        assert want in names


def test_every_declared_symbol_is_exported(lib):
    import paper_1107_1525_gb300.hz as hz
    for name in _declared():
        assert hasattr(lib, name), name
    assert set(hz.EXPORTS) <= set(_declared())


def test_compress_bound_closed_form(lib):
    import paper_1107_1525_gb300.hz as hz
    assert hz.hz_compress_bound(0, 4096) == 280
    for n, B in ((1, 1), (1000, 7), (1 << 20, 4096), (1 << 30, 65536), (12345, 1 << 24)):
        nb = -(-n // B)
        assert hz.hz_compress_bound(n, B) == 280 + 16 * nb + 4 * (-(-n // 4))
    assert hz.hz_compress_bound(1 << 32, 4096) == 0


def test_bound_covers_oracle_streams(lib):
    import numpy as np
    import oracle
    import paper_1107_1525_gb300.hz as hz
    rng = np.random.default_rng(0)
    for n, B in ((0, 5), (1, 1), (100, 3), (5000, 64), (20000, 4096)):
        for x in (rng.integers(0, 256, n, dtype=np.uint8), np.full(n, 9, np.uint8)):
            assert oracle.compress(x, B).size <= hz.hz_compress_bound(n, B)


def test_create_without_a_gpu_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    st = lib.hz_create(ctypes.byref(h), 0, 0)
    assert st in (-7, -1) and not h.value


def test_null_arguments_are_rejected_without_a_gpu(lib):
    assert lib.hz_compress(None, None, 0, 0, None, None, 0, None, None) == -1
    assert lib.hz_decompress(None, None, 0, None, 0, None, None) == -1
    assert lib.hz_sync(None, None) == -1
    assert lib.hz_set_option(None, 1, 1) == -1
    assert lib.hz_submit(None, None, 0, None, None) == -1
    assert lib.hz_poll(None, 1, 0, None, None) == -1
    assert lib.hz_launch_count(None) == 0
    assert lib.hz_kernel_name(4) == b"encode_pack"
