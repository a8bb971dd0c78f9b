"""Benchmark: block-decomposed Huffman encode + decode on one GB300 (or N
independent replicas under torchrun).

One step = compress (histogram, code construction, encode) + decompress
(setup, block decode) of the workload buffer, through the C ABI.  The default
workload is the 1 GiB buffer of 64 MiB segments cycling Zipf(1.1),
geometric(0.3), uniform-256 and uniform-16 bytes, in 64 KiB blocks.  Inputs
(1 GiB) are larger than the 129 MB L2, so no flush is needed between steps.

Prints ONE JSON line (rank 0).  --impl reference times the CPU oracle instead,
on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

MiB = 1 << 20
GiB = 1 << 30
METRIC = "Huffman enc/dec GB/s of input, % of HBM peak; batch p50/p99 latency vs plain"
WORKLOADS = {
    "mixed-1GiB": dict(n=GiB, segment=64 * MiB, block=65536,
                       desc="1 GiB uint8 in 64 MiB segments cycling Zipf(1.1) / geometric(0.3) "
                            "clipped to 255 / uniform-256 / uniform-16, 64 KiB blocks"),
    "mixed-256MiB": dict(n=256 * MiB, segment=64 * MiB, block=65536,
                         desc="256 MiB: one 64 MiB segment of each kind of the 1 GiB mix, "
                              "64 KiB blocks (profiling case)"),
    "zipf-1MiB": dict(n=MiB, block=4096, desc="1 MiB i.i.d. Zipf(1.1) bytes, 4 KiB blocks"),
    "field-256MiB": dict(n=1 << 28, block=16384,
                         desc="2^28 int8 residuals of a smooth 512x512x1024 Gaussian field, "
                              "16 KiB blocks"),
}
# DRAM traffic per launch from an ncu capture of the same kernel revision
# (dram__bytes_read.sum + dram__bytes_write.sum); None until captured.
NCU_TRAFFIC = {}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def make_input(name, device):
    import datagen
    w = WORKLOADS[name]
    if name.startswith("mixed"):
        return datagen.mixed_buffer(n=w["n"], segment=w["segment"], seed=2, device=device)
    if name == "zipf-1MiB":
        return datagen.zipf_buffer(w["n"], s=1.1, seed=0, device=device)
    return datagen.gaussian_field_residuals(shape=(512, 512, 1024), seed=1, device=device)


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled while the timed region runs."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except FileNotFoundError:
            self.proc = None
        time.sleep(0.3)
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 8:
                self.rows.append(parts)

    def __exit__(self, *exc):
        if self.proc:
            time.sleep(0.1)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return None
        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[0]) for r in self.rows if num(r[0]) is not None]
        mx = [num(r[1]) for r in self.rows if num(r[1]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4)
                          if r[4 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if (args.impl != "reference" and torch.cuda.is_available()) else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
        pg = dist
    return world, rank, local, pg


def barrier(pg):
    if pg is not None:
        pg.barrier()


def max_over_ranks(pg, v: float, device=None) -> float:
    if pg is None:
        return v
    import torch
    t = torch.tensor([v], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(pg, v: float, device=None) -> float:
    if pg is None:
        return v
    import torch
    t = torch.tensor([v], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.SUM)
    return float(t.item())


# ------------------------------------------------------------------ oracle arm
def oracle_sample(name: str, sample_bytes: int):
    """A bounded host sample of the workload: equal slices of each segment kind."""
    import datagen
    import torch
    w = WORKLOADS[name]
    if name.startswith("mixed"):
        per = sample_bytes // 4
        parts = [datagen.sample_iid(datagen.segment_pmf(k), per, (2 << 16) + j, "cpu")
                 for j, k in enumerate(datagen.SEGMENT_KINDS)]
        return torch.cat(parts).numpy(), w["block"]
    if name == "zipf-1MiB":
        return datagen.zipf_buffer(w["n"], s=1.1, seed=0).numpy(), w["block"]
    x = datagen.gaussian_field_residuals(shape=(64, 512, 1024), seed=1).numpy()
    return x[:sample_bytes], w["block"]


def time_oracle(x, B, steps: int):
    import oracle
    t_enc = t_dec = 0.0
    for _ in range(steps):
        t0 = time.perf_counter()
        s = oracle.compress(x, B)
        t1 = time.perf_counter()
        y = oracle.decompress(s)
        t2 = time.perf_counter()
        t_enc += t1 - t0
        t_dec += t2 - t1
        assert y.size == x.size
    return t_enc / steps, t_dec / steps, s.size


def run_reference(args, world, rank, pg):
    if rank != 0:
        return
    sample = args.ref_sample_mib * MiB
    x, B = oracle_sample(args.workload, sample)
    for _ in range(args.warmup):
        time_oracle(x, B, 1)
    t_enc, t_dec, slen = time_oracle(x, B, args.steps)
    gbs = x.size / (t_enc + t_dec) / 1e9
    desc = f"{x.size // MiB} MiB host sample of the workload, CPU oracle (single thread)"
    line = {"impl": "reference", "metric": METRIC, "value": gbs, "unit": "GB/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": (t_enc + t_dec) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
            "data": "synthetic",
            "config": {"workload": args.workload, "block_size": B, "sample_bytes": int(x.size),
                       "note": "CPU oracle on the host cores, as it stands"},
            "encode_gbs": x.size / t_enc / 1e9, "decode_gbs": x.size / t_dec / 1e9,
            "cpu_baseline": {"value": gbs, "unit": "GB/s", "cores": 1, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": gbs, "unit": "GB/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU arm
def run_gpu(args, world, rank, local, pg):
    import torch

    import paper_1107_1525_gb300.hz as hz
    from paper_1107_1525_gb300 import build
    build.build()
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    w = WORKLOADS[args.workload]
    B = w["block"]
    x = make_input(args.workload, dev)
    n = x.numel()
    ctx = hz.Context(local)
    stream = torch.cuda.Stream(device=dev)
    cap = hz.hz_compress_bound(n, B)
    s_buf = torch.empty(cap, dtype=torch.uint8, device=dev)
    y = torch.empty(n, dtype=torch.uint8, device=dev)
    lens = torch.zeros(2, dtype=torch.int64, device=dev)

    def step():
        hz.hz_compress(ctx, x, n, B, None, s_buf, cap, lens[0:1], stream)
        hz.hz_decompress(ctx, s_buf, stream_len, y, n, lens[1:2], stream)

    # first call sizes the stream; check it round-trips before timing anything
    with torch.cuda.stream(stream):
        hz.hz_compress(ctx, x, n, B, None, s_buf, cap, lens[0:1], stream)
        st = hz.hz_sync(ctx, stream)
        if st:
            raise hz.HzError(st, "compress")
        stream_len = int(lens[0].item())
        hz.hz_decompress(ctx, s_buf, stream_len, y, n, lens[1:2], stream)
        st = hz.hz_sync(ctx, stream)
        if st or not torch.equal(x, y):
            raise RuntimeError("round trip failed")
    for _ in range(max(3, args.warmup)):
        step()
    stream.synchronize()
    ctx.profile_read()

    # ---- timed region: K steps, events on the launch stream, profile on
    ctx.set_option(hz.HZ_OPT_PROFILE, 1)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    l0 = ctx.launch_count()
    barrier(pg)
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clocks:
        ev[0].record(stream)
        for _ in range(args.steps):
            step()
        ev[1].record(stream)
        ev[1].synchronize()
    torch.cuda.synchronize(dev)
    barrier(pg)
    launches = ctx.launch_count() - l0
    ms_total = ev[0].elapsed_time(ev[1])
    prof = ctx.profile_read()
    ctx.set_option(hz.HZ_OPT_PROFILE, 0)
    st = hz.hz_sync(ctx, stream)
    if st:
        raise hz.HzError(st, "timed region")
    ms_step = max_over_ranks(pg, ms_total / args.steps, dev)

    per_kernel = {}
    for name, t in prof:
        d = per_kernel.setdefault(name, [0.0, 0])
        d[0] += t
        d[1] += 1
    enc_kernels = ("histogram", "build_codes", "encode_summary", "encode_scan", "encode_pack")
    enc_ms = sum(per_kernel.get(k, [0, 0])[0] for k in enc_kernels) / args.steps
    dec_ms = sum(per_kernel.get(k, [0, 0])[0] for k in ("decode_setup", "decode")) / args.steps
    # algorithmic bytes per launch of each kernel
    ntiles = (n + 8191) // 8192
    algo = {"histogram": n, "encode_summary": n, "encode_scan": 32 * ntiles,
            "encode_pack": n + stream_len, "decode": stream_len + n,
            "build_codes": 1024, "decode_setup": 8192}
    dom = max(per_kernel, key=lambda k: per_kernel[k][0])
    dom_avg_ms = per_kernel[dom][0] / per_kernel[dom][1]
    peak, peak_kind = load_peaks()
    achieved = algo[dom] / (dom_avg_ms * 1e-3) / 1e9
    kernels = {k: {"launches": v[1], "avg_ms": v[0] / v[1],
                   "gbs": algo.get(k, 0) / (v[0] / v[1] * 1e-3) / 1e9,
                   "share": v[0] / sum(u[0] for u in per_kernel.values())}
               for k, v in per_kernel.items()}

    # ---- end to end: host (pinned) buffers through the C ABI, copies inside the timing
    h_in = torch.empty(n, dtype=torch.uint8, pin_memory=True)
    h_in.copy_(x.cpu())
    h_s = torch.empty(cap, dtype=torch.uint8, pin_memory=True)
    h_y = torch.empty(n, dtype=torch.uint8, pin_memory=True)
    e2e_steps = max(1, min(args.steps, args.e2e_steps))
    for _ in range(2):
        st, slen = hz.hz_compress_host(ctx, h_in, n, B, h_s, cap, stream)
        st2, ylen = hz.hz_decompress_host(ctx, h_s, slen, h_y, n, stream)
    barrier(pg)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        st, slen = hz.hz_compress_host(ctx, h_in, n, B, h_s, cap, stream)
        st2, ylen = hz.hz_decompress_host(ctx, h_s, slen, h_y, n, stream)
    t_e2e = (time.perf_counter() - t0) / e2e_steps
    barrier(pg)
    if st or st2 or ylen != n or not torch.equal(h_y, h_in):
        raise RuntimeError("end-to-end round trip failed")
    t_e2e = max_over_ranks(pg, t_e2e, dev)

    total_bytes = sum_over_ranks(pg, float(n), dev)
    value = total_bytes / (ms_step * 1e-3) / 1e9
    if rank != 0:
        return
    # CPU oracle baseline, rank 0 only, bounded sample
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        xs, Bs = oracle_sample(args.workload, args.cpu_sample_mib * MiB)
        te, td, _ = time_oracle(xs, Bs, 1)
        cpu = {"value": xs.size / (te + td) / 1e9, "unit": "GB/s", "cores": 1, "kind": "oracle",
               "sample": f"{xs.size // MiB} MiB host sample of the workload (equal slices of each "
                         f"segment kind), one compress + decompress, single thread"}
    traffic = NCU_TRAFFIC.get(dom)
    line = {
        "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8",
        "data": "synthetic (seeded generators, see datagen)",
        "config": {"workload": args.workload, "desc": w["desc"], "n_bytes": n, "block_size": B,
                   "stream_bytes": stream_len, "ratio": stream_len / n,
                   "l2": "inputs larger than L2 (no flush needed)",
                   "step": "compress + decompress", "parallelism": f"replicas x{world}"},
        "encode_gbs": n / (enc_ms * 1e-3) / 1e9, "decode_gbs": n / (dec_ms * 1e-3) / 1e9,
        "encode_ms": enc_ms, "decode_ms": dec_ms,
        "kernels": kernels,
        "roofline": {"kernel": dom, "bound": "hbm", "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": achieved / peak, "peak_kind": peak_kind,
                     "traffic": traffic, "algorithmic_bytes": algo[dom]},
        "cpu_baseline": cpu,
        "e2e": {"value": total_bytes / t_e2e / 1e9, "unit": "GB/s",
                "h2d_bytes_per_step": n + stream_len, "d2h_bytes_per_step": stream_len + n,
                "ms_per_step": t_e2e * 1e3},
        "gpu_launches": launches,
        "clocks": clocks.summary(),
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="hz", choices=["hz", "reference"])
    ap.add_argument("--workload", default="mixed-1GiB", choices=sorted(WORKLOADS))
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--ref-sample-mib", type=int, default=16,
                    help="per-step host sample of the reference (oracle) arm")
    ap.add_argument("--cpu-sample-mib", type=int, default=192,
                    help="host sample for the cpu_baseline key of the GPU arm")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    world, rank, local, pg = dist_setup(args)
    try:
        if args.impl == "reference":
            run_reference(args, world, rank, pg)
        else:
            run_gpu(args, world, rank, local, pg)
    finally:
        if pg is not None:
            pg.destroy_process_group()


if __name__ == "__main__":
    main()
