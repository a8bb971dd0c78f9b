"""Seeded synthetic inputs for the Huffman coder's workloads.

This module holds no coding arithmetic: it only draws bytes.  Both the CUDA
path's tests and benchmark and the CPU oracle's tests take their inputs from
here, so it is the one module the two sides share.  Inputs are drawn with
torch's seeded generators on the requested device; a given (seed, device)
always yields the same bytes, and a test that compares the two sides draws the
bytes once and hands the same array to both.

The paper (arXiv 1107.1525) names no data set, so every workload here is a
synthetic stand-in with the distribution stated in its docstring.
"""
from __future__ import annotations

import math

import numpy as np
import torch

MiB = 1 << 20
GiB = 1 << 30


# ----------------------------------------------------------------- pmfs
def zipf_pmf(s: float, k: int = 256) -> np.ndarray:
    """p[v] proportional to (v+1)^-s for byte value v < k (rank v -> byte v)."""
    p = np.zeros(256, dtype=np.float64)
    p[:k] = (np.arange(1, k + 1, dtype=np.float64)) ** (-s)
    return p / p.sum()


def geometric_pmf(p: float) -> np.ndarray:
    """v = min(G - 1, 255) with G ~ Geometric(p) on {1, 2, ...}."""
    v = np.arange(256, dtype=np.float64)
    pm = p * (1.0 - p) ** v
    pm[255] = (1.0 - p) ** 255
    return pm / pm.sum()


def uniform_pmf(m: int = 256) -> np.ndarray:
    """Uniform over byte values 0..m-1."""
    pm = np.zeros(256, dtype=np.float64)
    pm[:m] = 1.0 / m
    return pm


def _gen(seed: int, device) -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return g


def sample_iid(pmf: np.ndarray, n: int, seed: int, device="cpu",
               chunk: int = 64 * MiB) -> torch.Tensor:
    """n i.i.d. bytes with probabilities pmf, by inverse CDF on uniform doubles."""
    device = torch.device(device)
    cdf = torch.tensor(np.cumsum(pmf / pmf.sum()), dtype=torch.float64, device=device)
    cdf[-1] = 1.0
    out = torch.empty(n, dtype=torch.uint8, device=device)
    g = _gen(seed, device)
    for lo in range(0, n, chunk):
        hi = min(n, lo + chunk)
        u = torch.rand(hi - lo, generator=g, dtype=torch.float64, device=device)
        idx = torch.searchsorted(cdf, u, right=True).clamp_(max=255)
        out[lo:hi] = idx.to(torch.uint8)
    return out


# ------------------------------------------------------------ workloads
def zipf_buffer(n: int, s: float = 1.1, seed: int = 0, device="cpu") -> torch.Tensor:
    """i.i.d. Zipf(s) bytes over 256 symbols (the 1 MiB round-trip case uses s=1.1, seed 0)."""
    return sample_iid(zipf_pmf(s), n, seed, device)


SEGMENT_KINDS = ("zipf1.1", "geometric0.3", "uniform256", "uniform16")


def segment_pmf(kind: str) -> np.ndarray:
    return {"zipf1.1": lambda: zipf_pmf(1.1), "geometric0.3": lambda: geometric_pmf(0.3),
            "uniform256": lambda: uniform_pmf(256), "uniform16": lambda: uniform_pmf(16)}[kind]()


def mixed_buffer(n: int = GiB, segment: int = 64 * MiB, seed: int = 2,
                 device="cpu") -> torch.Tensor:
    """Segments of `segment` bytes cycling Zipf(1.1), geometric(0.3) clipped to 255,
    uniform bytes (incompressible) and a 16-symbol uniform alphabet; segment j is
    drawn with seed (seed << 16) + j."""
    out = torch.empty(n, dtype=torch.uint8, device=device)
    for j, lo in enumerate(range(0, n, segment)):
        hi = min(n, lo + segment)
        kind = SEGMENT_KINDS[j % 4]
        out[lo:hi] = sample_iid(segment_pmf(kind), hi - lo, (seed << 16) + j, device)
    return out


def gaussian_field_residuals(shape=(512, 512, 1024), sigma: float = 4.0, scale: float = 4.0,
                             seed: int = 1, device="cpu") -> torch.Tensor:
    """Scientific-data stand-in: white N(0,1) float32 on a periodic (z, y, x) grid,
    Gaussian low-pass (std `sigma` voxels) in Fourier space, scaled to unit variance,
    first-differenced along x (d[0] = f[0]), quantised as
    clip(rint(d * scale / mean|d|), -128, 127) and returned as the int8 bytes (uint8 view)."""
    device = torch.device(device)
    g = _gen(seed, device)
    f = torch.randn(shape, generator=g, dtype=torch.float32, device=device)
    F = torch.fft.rfftn(f)
    del f
    kz = torch.fft.fftfreq(shape[0], device=device).view(-1, 1, 1)
    ky = torch.fft.fftfreq(shape[1], device=device).view(1, -1, 1)
    kx = torch.fft.rfftfreq(shape[2], device=device).view(1, 1, -1)
    k2 = (kz * kz + ky * ky + kx * kx) * (2.0 * math.pi) ** 2
    F *= torch.exp(-0.5 * sigma * sigma * k2).to(F.dtype)
    del k2
    f = torch.fft.irfftn(F, s=shape)
    del F
    f = (f - f.mean()) / f.std()
    d = torch.empty_like(f)
    d[..., 0] = f[..., 0]
    d[..., 1:] = f[..., 1:] - f[..., :-1]
    del f
    q = torch.clamp(torch.round(d * (scale / d.abs().mean())), -128, 127).to(torch.int8)
    return q.reshape(-1).view(torch.uint8)


def batch_sizes(count: int = 4096, lo: int = 4096, hi: int = 16 * MiB, seed: int = 3):
    """Buffer lengths log-uniform in [lo, hi] and per-buffer Zipf exponents U[0.6, 1.6]."""
    rng = np.random.default_rng(seed)
    lens = np.floor(np.exp(rng.uniform(math.log(lo), math.log(hi), size=count))).astype(np.int64)
    lens = np.clip(lens, lo, hi)
    s = rng.uniform(0.6, 1.6, size=count)
    return lens, s


def batch_buffers(count: int = 4096, lo: int = 4096, hi: int = 16 * MiB, seed: int = 3,
                  device="cpu"):
    """Independent buffers for the batched workload: buffer i holds Zipf(s_i) bytes."""
    lens, s = batch_sizes(count, lo, hi, seed)
    return [sample_iid(zipf_pmf(float(s[i])), int(lens[i]), (seed << 20) + i, device)
            for i in range(count)], lens, s


def arrivals(rate: float = 20000.0, duration: float = 60.0, frac_compress: float = 0.6,
             lo: int = 1024, hi: int = 64 * MiB, seed: int = 5):
    """Open-loop request trace: Poisson arrivals at `rate`/s for `duration` s; each
    request is compress with probability frac_compress (else decompress), its size is
    log-uniform in [lo, hi] and its data Zipf with s uniform in [0.6, 1.6].
    Returns arrays (t_arrival_s, is_compress, size, s)."""
    rng = np.random.default_rng(seed)
    n_est = int(rate * duration * 1.2) + 16
    t = np.cumsum(rng.exponential(1.0 / rate, size=n_est))
    t = t[t < duration]
    m = t.size
    is_c = rng.uniform(size=m) < frac_compress
    size = np.floor(np.exp(rng.uniform(math.log(lo), math.log(hi), size=m))).astype(np.int64)
    size = np.clip(size, lo, hi)
    s = rng.uniform(0.6, 1.6, size=m)
    return t, is_c, size, s
