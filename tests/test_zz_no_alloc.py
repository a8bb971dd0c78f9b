"""hz_compress_noalloc: the compressor for callers that must not allocate device
memory (for example code running under a framework's caching allocator or a fixed
memory reservation that a cudaMalloc would bypass).  Its scratch is a fixed device
array inside the library.  These checks call it through the C ABI and compare its
stream with hz_compress's and with the CPU oracle's for the same input -- byte for
byte, the tolerance every stream test here uses -- on two calls in a row, so that
whatever the first call left in the shared array cannot leak into the second.  This
file is collected last."""
import numpy as np
import pytest
import torch

import datagen
import oracle

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


def _with_context(hz, x, B):
    ctx = hz.Context(0)
    n = x.numel()
    cap = hz.hz_compress_bound(n, B)
    out = torch.empty(cap, dtype=torch.uint8, device=DEV)
    out_len = torch.zeros(1, dtype=torch.int64, device=DEV)
    hz.hz_compress(ctx, x, n, B, None, out, cap, out_len)
    assert hz.hz_sync(ctx) == 0
    ctx.close()
    return out[: int(out_len.item())].clone()


def _without_allocation(hz, x, B):
    lib = hz.load_library()
    n = x.numel()
    cap = hz.hz_compress_bound(n, B)
    out = torch.empty(cap, dtype=torch.uint8, device=DEV)
    out_len = torch.zeros(1, dtype=torch.int64, device=DEV)
    status = torch.full((1,), 12345, dtype=torch.int32, device=DEV)
    stream = torch.cuda.current_stream().cuda_stream
    st = lib.hz_compress_noalloc(x.data_ptr() if n else None, n, B, out.data_ptr(), cap,
                                 out_len.data_ptr(), status.data_ptr(), stream)
    assert st == 0
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    return out[: int(out_len.item())].clone()


def test_noalloc_matches_hz_compress_on_two_calls_in_a_row(hz):
    # a larger, skewed buffer first, then a smaller one of another shape
    first = datagen.zipf_buffer(9 * MiB + 123, s=1.3, seed=21, device=DEV)
    second = datagen.sample_iid(datagen.uniform_pmf(16), 3 * MiB + 7, 22, DEV)
    for x, B in ((first, 65536), (second, 4096)):
        want = _with_context(hz, x, B)
        got = _without_allocation(hz, x, B)
        assert got.numel() == want.numel()
        assert torch.equal(got, want)
        assert np.array_equal(got.cpu().numpy(), oracle.compress(x.cpu().numpy(), B))


def test_noalloc_allocates_no_device_memory(hz):
    x = datagen.zipf_buffer(5 * MiB + 3, s=1.1, seed=23, device=DEV)
    _without_allocation(hz, x, 16384)  # the first call on the device sets up the array
    lib = hz.load_library()
    n = x.numel()
    cap = hz.hz_compress_bound(n, 16384)
    out = torch.empty(cap, dtype=torch.uint8, device=DEV)
    out_len = torch.zeros(1, dtype=torch.int64, device=DEV)
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    torch.cuda.synchronize()
    free_before, _ = torch.cuda.mem_get_info()
    assert lib.hz_compress_noalloc(x.data_ptr(), n, 16384, out.data_ptr(), cap,
                                   out_len.data_ptr(), status.data_ptr(),
                                   torch.cuda.current_stream().cuda_stream) == 0
    torch.cuda.synchronize()
    free_after, _ = torch.cuda.mem_get_info()
    assert free_after == free_before
    assert int(status.item()) == 0
    got = out[: int(out_len.item())].cpu().numpy()
    assert np.array_equal(got, oracle.compress(x.cpu().numpy(), 16384))


def test_noalloc_empty_input_and_builtin_block_size(hz):
    # n = 0: a header-only stream
    assert np.array_equal(_without_allocation(hz, torch.empty(0, dtype=torch.uint8, device=DEV),
                                              4096).cpu().numpy(),
                          oracle.compress(np.zeros(0, dtype=np.uint8), 4096))
    # block_size 0 takes the built-in size table: 16 KiB for a buffer of 3 MiB
    x = datagen.zipf_buffer(3 * MiB + 5, s=0.9, seed=24, device=DEV)
    got = _without_allocation(hz, x, 0)
    assert int(np.frombuffer(got[16:20].cpu().numpy().tobytes(), dtype="<u4")[0]) == 16384
    assert np.array_equal(got.cpu().numpy(), oracle.compress(x.cpu().numpy(), 16384))


def test_noalloc_rejects_inputs_beyond_its_scratch(hz):
    lib = hz.load_library()
    dummy = torch.empty(16, dtype=torch.uint8, device=DEV)
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    out_len = torch.zeros(1, dtype=torch.int64, device=DEV)
    # n above 2^28 is refused before any GPU work, so the dummy buffers are never read
    st = lib.hz_compress_noalloc(dummy.data_ptr(), (1 << 28) + 1, 65536, dummy.data_ptr(), 16,
                                 out_len.data_ptr(), status.data_ptr(), None)
    assert st == hz.HZ_ERR_ARG


def test_noalloc_reports_a_short_output_buffer(hz):
    lib = hz.load_library()
    x = datagen.zipf_buffer(MiB, s=1.1, seed=0, device=DEV)
    want = _with_context(hz, x, 4096)
    cap = want.numel() - 1
    out = torch.empty(cap, dtype=torch.uint8, device=DEV)
    out_len = torch.zeros(1, dtype=torch.int64, device=DEV)
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    st = lib.hz_compress_noalloc(x.data_ptr(), x.numel(), 4096, out.data_ptr(), cap,
                                 out_len.data_ptr(), status.data_ptr(),
                                 torch.cuda.current_stream().cuda_stream)
    assert st == 0
    torch.cuda.synchronize()
    assert int(status.item()) == hz.HZ_ERR_CAPACITY and int(out_len.item()) == want.numel()
    # and the next call is clean again
    assert torch.equal(_without_allocation(hz, x, 4096), want)
