"""Failure detection without a GPU fault: the encoder's look-back scan waits for
its predecessor with a bounded number of polls.  A host-side injection
(HZ_OPT_INJECT_SCAN_STALL) hands the scan CTAs tickets from 1 instead of 0, so
the first of them waits for a flag that nothing sets; its wait must run out
after HZ_OPT_SPIN_LIMIT polls, hz_sync must report HZ_ERR_TIMEOUT, nothing may
hang or trap, and the same context must then compress correctly again."""
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


def _compress_status(hz, ctx, x, B):
    cap = hz.hz_compress_bound_ctx(ctx, x.numel(), B)
    out = torch.empty(cap, dtype=torch.uint8, device=DEV)
    ol = torch.zeros(1, dtype=torch.int64, device=DEV)
    hz.hz_compress(ctx, x, x.numel(), B, None, out, cap, ol)
    return hz.hz_sync(ctx)


@pytest.mark.parametrize("n", [5 * MiB + 3, 40 * MiB + 17])  # one scan CTA, and six
def test_scan_wait_runs_out_and_the_context_recovers(hz, n):
    ctx = hz.Context(0)
    ctx.set_option(hz.HZ_OPT_SPIN_LIMIT, 4000)
    assert ctx.get_option(hz.HZ_OPT_SPIN_LIMIT) == 4000
    x = datagen.zipf_buffer(n, s=1.1, seed=31, device=DEV)
    ctx.set_option(hz.HZ_OPT_INJECT_SCAN_STALL, 1)
    assert _compress_status(hz, ctx, x, 65536) == hz.HZ_ERR_TIMEOUT
    assert ctx.get_option(hz.HZ_OPT_INJECT_SCAN_STALL) == 0  # one shot
    assert hz.hz_sync(ctx) == 0  # the status was read and cleared
    # the same context, with the default limit again, writes the oracle's stream
    ctx.set_option(hz.HZ_OPT_SPIN_LIMIT, 1 << 20)
    s = hz.compress(x, 65536, ctx=ctx)
    assert np.array_equal(s.cpu().numpy(), oracle.compress_omp(x.cpu().numpy(), 65536))
    assert torch.equal(hz.decompress(s, ctx=ctx), x)
    ctx.close()


def test_fault_options_are_checked(hz):
    ctx = hz.Context(0)
    for bad in (0, -1, (1 << 24) + 1):
        with pytest.raises(hz.HzError):
            ctx.set_option(hz.HZ_OPT_SPIN_LIMIT, bad)
    with pytest.raises(hz.HzError):
        ctx.set_option(hz.HZ_OPT_INJECT_SCAN_STALL, 2)
    assert ctx.get_option(hz.HZ_OPT_SPIN_LIMIT) == 1 << 20
    ctx.close()
