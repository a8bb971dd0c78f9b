"""The bench's workload table and its host samples (CPU): every workload's
sub-block size suits its block size, the oracle arm's bounded samples have the
workload's block size and value range, and the DRAM-traffic stamps name a
workload, a sub-block size and the kernels the bench reports."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_workload_block_and_sub_block_sizes():
    for name, w in bench.WORKLOADS.items():
        B, S = w["block"], w["sub"]
        assert B > 0 and w["n"] > 0, name
        if S:
            assert S >= 32 and S % 32 == 0 and B % S == 0, name
        assert bench.sub_block_of(type("A", (), {"sub_block": None, "workload": name})()) == S


def test_oracle_samples():
    x, B = bench.oracle_sample("uniform16-1GiB", 1 << 16)
    assert x.dtype == np.uint8 and x.size == 1 << 16 and B == 65536
    assert x.max() < 16 and len(np.unique(x)) == 16
    x, B = bench.oracle_sample("mixed-1GiB", 1 << 16)
    assert x.size == 1 << 16 and B == 65536
    # equal slices of the four segment kinds: the uniform-256 slice reaches 255
    assert x.max() == 255
    x, B = bench.oracle_sample("zipf-1MiB", 0)
    assert x.size == 1 << 20 and B == 4096


def test_traffic_stamps_are_well_formed():
    for wname, stamp in bench.NCU_TRAFFIC.items():
        assert wname in bench.WORKLOADS
        assert stamp["sub_block"] == bench.WORKLOADS[wname]["sub"]
        for kernel, k in stamp.items():
            if kernel == "sub_block":
                continue
            assert kernel in bench.KERNEL_SOURCES
            assert len(k["digest"]) == 16 and int(k["digest"], 16) >= 0
            # per 1 GiB launch: about the input plus the stream, read and written once
            assert 1.0e9 < k["bytes"] < 4.0e9


def test_kernel_digest_covers_each_kernels_sources():
    for kernel, files in bench.KERNEL_SOURCES.items():
        for f in files:
            assert os.path.exists(os.path.join(ROOT, "paper_1107_1525_gb300", "csrc", f)), f
        d = bench.kernel_digest(kernel)
        assert len(d) == 16 and d == bench.kernel_digest(kernel)
    assert bench.kernel_digest("decode") != bench.kernel_digest("encode_pack")


def test_digest_ignores_comments_only():
    a = "int f(int x) {  // one\n  return x + 1; /* two\n three */\n}\n"
    b = "int f(int x) {\n\n  return x + 1;\n}  // other words\n"
    c = "int f(int x) {\n  return x + 2;\n}\n"
    assert bench.source_code_only(a) == bench.source_code_only(b)
    assert bench.source_code_only(a) != bench.source_code_only(c)
    assert "return x + 1;" in bench.source_code_only(a)
