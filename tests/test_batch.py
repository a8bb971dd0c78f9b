"""Batched path (hz_submit / hz_poll): every request's result must equal what the
oracle produces for it alone and what the single-buffer calls produce, in any mix,
in any number of concurrent batches; the plain (one launch sequence per buffer)
mode must give the same bytes; admission must respect the device-memory budget."""
import ctypes
import concurrent.futures
import os

import numpy as np
import pytest
import torch

import datagen
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


def _buffers(sizes, seed=0):
    rng = np.random.default_rng(seed)
    out = []
    for i, n in enumerate(sizes):
        s = float(rng.uniform(0.6, 1.6))
        out.append(datagen.zipf_buffer(int(n), s=s, seed=seed * 1000 + i, device=DEV))
    return out


def _run(hz, ctx, reqs, timeout_ns=-1):
    t = hz.hz_submit(ctx, reqs)
    st, per, lens = hz.hz_poll(ctx, t, len(reqs), timeout_ns)
    assert st == 0
    return per, lens


def _compress_reqs(hz, bufs, B):
    reqs, outs = [], []
    for x in bufs:
        cap = hz.hz_compress_bound(x.numel(), B or 1)
        o = torch.empty(max(cap, 16), dtype=torch.uint8, device=DEV)
        outs.append(o)
        reqs.append((hz.HZ_OP_COMPRESS, B, x if x.numel() else o, x.numel(), o, cap))
    return reqs, outs


SIZES = [1, 7, 3000, 4096, 4097, 65_536, 100_000, 1 << 20, 3 * (1 << 20) + 5, 9_000_000]


@pytest.mark.parametrize("B", [4096, 65536, 0, 131072, 1 << 20])
def test_batched_compress_matches_oracle_and_single_calls(hz, B):
    ctx = hz.Context(0)
    bufs = _buffers(SIZES, seed=1)
    reqs, outs = _compress_reqs(hz, bufs, B)
    per, lens = _run(hz, ctx, reqs)
    assert list(per) == [0] * len(bufs)
    for x, o, n in zip(bufs, outs, lens):
        Bx = B or hz.load_library().hz_tuned_block_size(ctx.handle, x.numel())
        want = oracle.compress(x.cpu().numpy(), Bx)
        got = o[: int(n)].cpu().numpy()
        assert got.size == want.size and np.array_equal(got, want)
        assert torch.equal(hz.compress(x, Bx, ctx=ctx), o[: int(n)])
    ctx.close()


def test_batched_decompress_and_mixed_batch(hz):
    ctx = hz.Context(0)
    bufs = _buffers(SIZES, seed=2)
    streams = [hz.compress(x, 16384, ctx=ctx) for x in bufs]
    # decompress-only batch
    dsts = [torch.empty(max(x.numel(), 1), dtype=torch.uint8, device=DEV) for x in bufs]
    reqs = [(hz.HZ_OP_DECOMPRESS, 0, s, s.numel(), d, x.numel()) for s, d, x in
            zip(streams, dsts, bufs)]
    per, lens = _run(hz, ctx, reqs)
    assert list(per) == [0] * len(bufs)
    for x, d, n in zip(bufs, dsts, lens):
        assert int(n) == x.numel() and torch.equal(d[: x.numel()], x)
    # mixed: interleave compress of new buffers with decompress of the streams
    new = _buffers(SIZES[::-1], seed=3)
    creqs, couts = _compress_reqs(hz, new, 65536)
    dsts2 = [torch.empty(max(x.numel(), 1), dtype=torch.uint8, device=DEV) for x in bufs]
    dreqs = [(hz.HZ_OP_DECOMPRESS, 0, s, s.numel(), d, x.numel()) for s, d, x in
             zip(streams, dsts2, bufs)]
    mixed = [r for pair in zip(creqs, dreqs) for r in pair]
    per, lens = _run(hz, ctx, mixed)
    assert list(per) == [0] * len(mixed)
    for i, (x, o) in enumerate(zip(new, couts)):
        n = int(lens[2 * i])
        assert np.array_equal(o[:n].cpu().numpy(), oracle.compress(x.cpu().numpy(), 65536))
    for i, (x, d) in enumerate(zip(bufs, dsts2)):
        assert torch.equal(d[: x.numel()], x)
    ctx.close()


@pytest.mark.parametrize("B", [65536, 131072, 1 << 20])
def test_batched_decompress_of_large_blocks(hz, B):
    """Streams whose blocks are longer than 64 KiB (the single-buffer decoder
    gives them a CTA each; the batched one decodes them a warp per block)."""
    ctx = hz.Context(0)
    bufs = _buffers([100_000, 1 << 20, 3 * (1 << 20) + 5, 9_000_000], seed=4)
    streams = [hz.compress(x, B, ctx=ctx) for x in bufs]
    for x, s in zip(bufs[:2], streams[:2]):
        assert np.array_equal(s.cpu().numpy(), oracle.compress(x.cpu().numpy(), B))
    dsts = [torch.empty(x.numel(), dtype=torch.uint8, device=DEV) for x in bufs]
    reqs = [(hz.HZ_OP_DECOMPRESS, 0, s, s.numel(), d, x.numel()) for s, d, x in
            zip(streams, dsts, bufs)]
    per, lens = _run(hz, ctx, reqs)
    assert list(per) == [0] * len(bufs)
    for x, d, n in zip(bufs, dsts, lens):
        assert int(n) == x.numel() and torch.equal(d, x)
    ctx.close()


@pytest.mark.parametrize("plain", [0, 1])
def test_submission_waits_for_the_callers_stream(hz, plain):
    """The sources are written on a side stream behind a ~20 ms GPU spin and the
    requests submitted at once, without a host wait: the batch must see the
    written data, not the zeros that were there before."""
    ctx = hz.Context(0)
    ctx.set_option(hz.HZ_OPT_BATCH_PLAIN, plain)
    src = _buffers([1 << 20, 3 * (1 << 20) + 5, 100_000], seed=21)
    xs = [torch.zeros_like(x) for x in src]
    reqs, outs = _compress_reqs(hz, xs, 65536)
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        torch.cuda._sleep(40_000_000)  # about 20 ms at 2 GHz
        for x, y in zip(xs, src):
            x.copy_(y)
        t = hz.hz_submit(ctx, reqs, stream=side)
    st, per, lens = hz.hz_poll(ctx, t, len(reqs), -1)
    assert st == 0 and list(per) == [0] * len(reqs)
    for x, o, n in zip(src, outs, lens):
        assert np.array_equal(o[: int(n)].cpu().numpy(), oracle.compress(x.cpu().numpy(), 65536))
    ctx.close()


def test_plain_mode_gives_the_same_bytes(hz):
    ctx = hz.Context(0)
    bufs = _buffers(SIZES[:8], seed=4)
    reqs, outs = _compress_reqs(hz, bufs, 16384)
    per, lens = _run(hz, ctx, reqs)
    ctx.set_option(hz.HZ_OPT_BATCH_PLAIN, 1)
    reqs2, outs2 = _compress_reqs(hz, bufs, 16384)
    per2, lens2 = _run(hz, ctx, reqs2)
    assert list(per) == list(per2) == [0] * len(bufs)
    assert list(lens) == list(lens2)
    for o, o2, n in zip(outs, outs2, lens):
        assert torch.equal(o[: int(n)], o2[: int(n)])
    ctx.close()


def test_concurrent_batches_and_a_corrupt_request(hz):
    ctx = hz.Context(0)
    tickets, expect = [], []
    for b in range(5):
        bufs = _buffers([50_000 * (b + 1), 1 << 20, 12345], seed=10 + b)
        reqs, outs = _compress_reqs(hz, bufs, 4096)
        tickets.append((hz.hz_submit(ctx, reqs), len(reqs)))
        expect.append((bufs, outs))
    for (t, k), (bufs, outs) in zip(tickets, expect):
        st, per, lens = hz.hz_poll(ctx, t, k, -1)
        assert st == 0 and list(per) == [0] * k
        for x, o, n in zip(bufs, outs, lens):
            assert np.array_equal(o[: int(n)].cpu().numpy(), oracle.compress(x.cpu().numpy(), 4096))
    # a batch with one corrupt stream: only that request fails
    x = _buffers([200_000], seed=20)[0]
    good = hz.compress(x, 4096, ctx=ctx)
    bad = good.clone()
    bad[0] ^= 1
    d1 = torch.empty(x.numel(), dtype=torch.uint8, device=DEV)
    d2 = torch.empty(x.numel(), dtype=torch.uint8, device=DEV)
    per, lens = _run(hz, ctx, [(hz.HZ_OP_DECOMPRESS, 0, bad, bad.numel(), d1, x.numel()),
                               (hz.HZ_OP_DECOMPRESS, 0, good, good.numel(), d2, x.numel())])
    assert per[0] == hz.HZ_ERR_CORRUPT and per[1] == 0 and torch.equal(d2, x)
    ctx.close()


def test_admission_budget(hz):
    x = _buffers([1 << 20], seed=30)[0]
    ctx = hz.Context(0, mem_budget=3 << 20)
    o = torch.empty(2 << 20, dtype=torch.uint8, device=DEV)
    big = [(hz.HZ_OP_COMPRESS, 4096, x, x.numel(), o, 4 << 20)]
    with pytest.raises(hz.HzError) as e:
        hz.hz_submit(ctx, big)  # 1 MiB in + 4 MiB out: more than the whole budget
    assert e.value.status == hz.HZ_ERR_BUSY
    reqs, outs = _compress_reqs(hz, [x], 4096)
    t1 = hz.hz_submit(ctx, reqs)
    reqs2, outs2 = _compress_reqs(hz, [x], 4096)
    t2 = hz.hz_submit(ctx, reqs2)  # waits for the first one's memory
    st, _, _ = hz.hz_poll(ctx, t2, 1, 0)
    assert st in (0, hz.HZ_PENDING)
    st1, per1, l1 = hz.hz_poll(ctx, t1, 1, -1)
    st2, per2, l2 = hz.hz_poll(ctx, t2, 1, -1)
    assert st1 == st2 == 0 and per1[0] == per2[0] == 0 and l1[0] == l2[0]
    assert torch.equal(outs[0][: int(l1[0])], outs2[0][: int(l2[0])])
    st, _, _ = hz.hz_poll(ctx, t1, 1, 0)  # a ticket is polled once
    assert st == hz.HZ_ERR_ARG
    ctx.close()


def test_batched_workload_full_size(hz):
    """The bench's batched workload at full size, in the bench's launch shape:
    4096 buffers, lengths log-uniform in [4 KiB, 16 MiB] (about 8.2 GB), Zipf(s_i)
    bytes, tuned block sizes, all in one submission out of one arena.  Every
    buffer must come back from the batched decompression, and every one of the
    4096 streams must be the oracle's, byte for byte."""
    lens, s = datagen.batch_sizes(count=4096, seed=3)
    offs = np.zeros(len(lens) + 1, dtype=np.int64)
    offs[1:] = np.cumsum((lens + 255) // 256 * 256)
    arena = torch.empty(int(offs[-1]), dtype=torch.uint8, device=DEV)
    for i in range(len(lens)):
        arena[offs[i]:offs[i] + lens[i]] = datagen.sample_iid(
            datagen.zipf_pmf(float(s[i])), int(lens[i]), (3 << 20) + i, DEV)
    ctx = hz.Context(0)
    lib = hz.load_library()
    Bs = [lib.hz_tuned_block_size(ctx.handle, int(n)) for n in lens]
    caps = np.array([hz.hz_compress_bound(int(n), int(b)) for n, b in zip(lens, Bs)])
    coffs = np.zeros(len(lens) + 1, dtype=np.int64)
    coffs[1:] = np.cumsum((caps + 255) // 256 * 256)
    out = torch.empty(int(coffs[-1]), dtype=torch.uint8, device=DEV)
    back = torch.zeros_like(arena)
    creqs = [(hz.HZ_OP_COMPRESS, 0, arena.data_ptr() + int(offs[i]), int(lens[i]),
              out.data_ptr() + int(coffs[i]), int(caps[i])) for i in range(len(lens))]
    per, slen = _run(hz, ctx, creqs)
    assert (per == 0).all()
    dreqs = [(hz.HZ_OP_DECOMPRESS, 0, out.data_ptr() + int(coffs[i]), int(slen[i]),
              back.data_ptr() + int(offs[i]), int(lens[i])) for i in range(len(lens))]
    per, dl = _run(hz, ctx, dreqs)
    assert (per == 0).all() and (dl.astype(np.int64) == lens).all()
    assert torch.equal(back, arena)
    # every stream against the oracle's, byte for byte (the oracle's calls run
    # on host threads: its ctypes calls release the GIL)
    a_np, o_np = arena.cpu().numpy(), out.cpu().numpy()

    def check(i):
        x = a_np[int(offs[i]):int(offs[i]) + int(lens[i])]
        got = o_np[int(coffs[i]):int(coffs[i]) + int(slen[i])]
        return bool(np.array_equal(got, oracle.compress_omp(x, int(Bs[i]), threads=1)))

    with concurrent.futures.ThreadPoolExecutor(max_workers=os.cpu_count() or 8) as ex:
        same = list(ex.map(check, range(len(lens))))
    assert all(same), [i for i, v in enumerate(same) if not v][:10]
    ctx.close()


def test_batched_workload_sample(hz):
    """The 4096-buffer workload's size and skew mix, at 128 buffers of up to 1 MiB."""
    lens, s = datagen.batch_sizes(count=128, lo=4096, hi=1 << 20, seed=3)
    bufs = [datagen.zipf_buffer(int(n), s=float(v), seed=(3 << 20) + i, device=DEV)
            for i, (n, v) in enumerate(zip(lens, s))]
    ctx = hz.Context(0)
    reqs, outs = _compress_reqs(hz, bufs, 0)
    per, slen = _run(hz, ctx, reqs)
    assert list(per) == [0] * len(bufs)
    dsts = [torch.empty(x.numel(), dtype=torch.uint8, device=DEV) for x in bufs]
    dreqs = [(hz.HZ_OP_DECOMPRESS, 0, o, int(n), d, x.numel()) for o, n, d, x in
             zip(outs, slen, dsts, bufs)]
    per, dl = _run(hz, ctx, dreqs)
    assert list(per) == [0] * len(bufs)
    rng = np.random.default_rng(0)
    for i in range(len(bufs)):
        assert torch.equal(dsts[i], bufs[i])
    for i in rng.choice(len(bufs), 12, replace=False):
        B = hz.load_library().hz_tuned_block_size(ctx.handle, bufs[i].numel())
        want = oracle.compress(bufs[i].cpu().numpy(), B)
        assert np.array_equal(outs[i][: int(slen[i])].cpu().numpy(), want)
    ctx.close()


def test_autotune_and_cache(hz, tmp_path):
    path = str(tmp_path / "tune.json")
    os.environ["HZ_TUNE_CACHE"] = path
    try:
        x = datagen.mixed_buffer(n=64 << 20, segment=16 << 20, seed=2, device=DEV)
        ctx = hz.Context(0)
        lib = hz.load_library()
        st = lib.hz_autotune(ctx.handle, x.data_ptr(), x.numel(),
                             torch.cuda.current_stream().cuda_stream)
        assert st == 0
        chosen = [lib.hz_tuned_block_size(ctx.handle, n) for n in (1 << 16, 1 << 20, 16 << 20,
                                                                    64 << 20)]
        assert all(b in (4096, 8192, 16384, 32768, 65536) for b in chosen)
        W = ctx.get_option(hz.HZ_OPT_DECODE_LUT_BITS)
        assert W in (10, 11, 12)
        T = ctx.get_option(hz.HZ_OPT_DECODE_THREADS)
        assert T in (128, 256)
        assert os.path.exists(path)
        ctx.close()
        # a new context picks the choice up from the cache
        ctx2 = hz.Context(0)
        assert [lib.hz_tuned_block_size(ctx2.handle, n) for n in (1 << 16, 1 << 20, 16 << 20,
                                                                  64 << 20)] == chosen
        assert ctx2.get_option(hz.HZ_OPT_DECODE_LUT_BITS) == W
        assert ctx2.get_option(hz.HZ_OPT_DECODE_THREADS) == T
        # block_size 0 uses it, and the stream is the oracle's for that block size
        y = x[: 3 << 20]
        s = hz.compress(y, 0, ctx=ctx2)
        assert np.array_equal(s.cpu().numpy(), oracle.compress(y.cpu().numpy(), chosen[2]))
        ctx2.close()
    finally:
        del os.environ["HZ_TUNE_CACHE"]
