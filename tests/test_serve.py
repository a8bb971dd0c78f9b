"""Request replay (hz_serve_replay): mixed compress / decompress requests that
arrive while others are on the GPU are merged into shared device batches, and
every result must be the same as the same request run alone -- for results in
caller buffers, in the replay's device ring, with a ring small enough that
requests wait for room, and in plain (one launch sequence per request) mode."""
import concurrent.futures
import os

import numpy as np
import pytest
import torch

import datagen
import oracle

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
ARENA = 8 << 20


@pytest.fixture(scope="module")
def hz():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1107_1525_gb300 import build
    build.build()
    import paper_1107_1525_gb300.hz as hzmod
    return hzmod


@pytest.fixture(scope="module")
def workload(hz):
    """Arenas of Zipf(s_j) bytes, a pool of streams compressed alone, and a trace."""
    ctx = hz.Context(0)
    arenas = [datagen.zipf_buffer(ARENA, s=0.6 + j / 7, seed=(5 << 20) + j, device=DEV)
              for j in range(8)]
    rng = np.random.default_rng(7)
    pool = []
    for k in range(24):
        n = int(np.exp(rng.uniform(np.log(1024), np.log(4 << 20))))
        j, off = int(rng.integers(8)), int(rng.integers(0, ARENA - n + 1))
        x = arenas[j][off:off + n]
        pool.append((x, hz.compress(x, 0, ctx=ctx)))
    t, is_c, size, s = datagen.arrivals(rate=50000.0, duration=0.008, lo=1024, hi=4 << 20,
                                        seed=5)
    reqs = []
    for i in range(t.size):
        if is_c[i]:
            j = int(round((s[i] - 0.6) * 7))
            off = int(rng.integers(0, ARENA - int(size[i]) + 1))
            reqs.append(("c", arenas[j][off:off + int(size[i])]))
        else:
            reqs.append(("d", pool[int(rng.integers(len(pool)))]))
    # the result of each request run alone
    alone = []
    for kind, r in reqs:
        alone.append(hz.compress(r, 0, ctx=ctx) if kind == "c" else r[0])
    ctx.close()
    return arenas, pool, t, reqs, alone


def _items(hz, reqs, t, own_dst):
    items = np.zeros(len(reqs), dtype=hz.SERVE_ITEM)
    dsts = []
    for i, (kind, r) in enumerate(reqs):
        items[i]["arrival_s"] = t[i]
        if kind == "c":
            cap = hz.hz_compress_bound(r.numel(), 4096)
            items[i]["op"], items[i]["d_src"], items[i]["src_len"] = 0, r.data_ptr(), r.numel()
        else:
            x, st = r
            cap = x.numel()
            items[i]["op"], items[i]["d_src"], items[i]["src_len"] = 1, st.data_ptr(), st.numel()
        items[i]["dst_cap"] = cap
        if own_dst:
            d = torch.empty(cap, dtype=torch.uint8, device=DEV)
            dsts.append(d)
            items[i]["d_dst"] = d.data_ptr()
        else:
            dsts.append(None)
    return items, dsts


def _check(rec, dsts, alone, ring=None):
    assert (rec["status"] == 0).all(), rec["status"]
    for i, want in enumerate(alone):
        n = int(rec[i]["out_len"])
        assert n == want.numel(), i
        if dsts[i] is not None:
            got = dsts[i][:n]
        elif ring is not None:
            off = int(rec[i]["dst_offset"])
            got = ring[off:off + n]
        else:
            continue
        assert torch.equal(got, want), i


@pytest.mark.parametrize("burst", [True, False])
def test_replay_results_equal_alone(hz, workload, burst):
    arenas, pool, t, reqs, alone = workload
    ctx = hz.Context(0, mem_budget=40 << 30)
    tt = np.zeros_like(t) if burst else t
    items, dsts = _items(hz, reqs, tt, own_dst=True)
    rec, wall = hz.hz_serve_replay(ctx, items)
    _check(rec, dsts, alone)
    assert wall > 0 and (rec["done_s"] >= rec["submit_s"]).all()
    launches = np.unique(rec["launch"]).size
    if burst:
        assert launches < len(reqs) // 4  # queued requests went out together
    # every compress result against the oracle, with the tuned block size
    lib = hz.load_library()
    comp = [k for k, (kind, _) in enumerate(reqs) if kind == "c"]
    assert len(comp) > 100

    def check(i):
        x = reqs[i][1].cpu().numpy()
        B = lib.hz_tuned_block_size(ctx.handle, x.size)
        got = dsts[i][: int(rec[i]["out_len"])].cpu().numpy()
        return bool(np.array_equal(got, oracle.compress_omp(x, B, threads=1)))

    with concurrent.futures.ThreadPoolExecutor(max_workers=os.cpu_count() or 8) as ex:
        same = list(ex.map(check, comp))
    assert all(same)
    ctx.close()


def test_replay_into_ring(hz, workload):
    arenas, pool, t, reqs, alone = workload
    ctx = hz.Context(0)
    items, dsts = _items(hz, reqs, t, own_dst=False)
    total = int(sum((int(c) + 255) // 256 * 256 for c in items["dst_cap"]))
    ring = torch.empty(total, dtype=torch.uint8, device=DEV)  # every result keeps its place
    rec, _ = hz.hz_serve_replay(ctx, items, ring)
    _check(rec, dsts, alone, ring)
    # a ring that holds only a few results at once: requests wait for room
    small = torch.empty(3 * int(items["dst_cap"].max()) + 1024, dtype=torch.uint8, device=DEV)
    rec2, _ = hz.hz_serve_replay(ctx, items.copy(), small)
    assert (rec2["status"] == 0).all()
    assert np.array_equal(rec2["out_len"], rec["out_len"])
    ctx.close()


def test_replay_plain_mode(hz, workload):
    arenas, pool, t, reqs, alone = workload
    ctx = hz.Context(0)
    ctx.set_option(hz.HZ_OPT_BATCH_PLAIN, 1)
    items, dsts = _items(hz, reqs[:60], np.zeros(60), own_dst=True)
    rec, _ = hz.hz_serve_replay(ctx, items)
    _check(rec, dsts, alone[:60])
    ctx.close()


def test_replay_rejects_bad_input(hz):
    ctx = hz.Context(0)
    x = torch.zeros(4096, dtype=torch.uint8, device=DEV)
    items = np.zeros(2, dtype=hz.SERVE_ITEM)
    items["arrival_s"] = [0.5, 0.1]  # unsorted
    items["d_src"], items["src_len"], items["dst_cap"] = x.data_ptr(), 4096, 8192
    items["d_dst"] = x.data_ptr()
    with pytest.raises(hz.HzError):
        hz.hz_serve_replay(ctx, items)
    items["arrival_s"] = [0.0, 0.0]
    items["d_dst"] = 0  # no ring given
    with pytest.raises(hz.HzError):
        hz.hz_serve_replay(ctx, items)
    ctx.close()
