"""Seeded synthetic inputs shared by the oracle tests, the CUDA tests and the benchmark.

This module holds no arithmetic of the least-squares method: it only draws the data
pair (A, b) of the problem x* = argmin 1/2 <x, A^T A x> - <b, x>.  The recipe follows
the workloads of the randomized-preconditioning literature the paper builds on (the
paper itself does not state its data):

    A = G diag(sigma),  G iid N(0,1),  sigma_j = sigma_max^(j/(d-1))  (log-spaced 1..sigma_max)
    optionally a fraction of rows scaled x100 (high-leverage outliers)
    x_true ~ N(0, I),  y = A x_true + noise * N(0, I),  b = A^T y

Draws use numpy's Philox bit generator, keyed by (seed, stream, chunk) so that the
result does not depend on the number of threads that fill it.
"""
from __future__ import annotations

import concurrent.futures as _cf
import math
import os

import numpy as np

_ROW_CHUNK = 1 << 16


def sigma(d: int, sigma_max: float) -> np.ndarray:
    if d == 1:
        return np.ones(1)
    return sigma_max ** (np.arange(d) / (d - 1))


def _gen(seed: int, stream: int, chunk: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=[(seed << 20) ^ (stream << 12) ^ 0x5EED, chunk]))


def _fill_normal(out: np.ndarray, seed: int, stream: int, threads: int) -> None:
    n = out.shape[0]
    chunks = [(c, min(c + _ROW_CHUNK, n)) for c in range(0, n, _ROW_CHUNK)]

    def work(k):
        lo, hi = chunks[k]
        g = _gen(seed, stream, k)
        if out.dtype == np.float64:
            g.standard_normal(out=out[lo:hi])
        else:
            out[lo:hi] = g.standard_normal(size=out[lo:hi].shape)

    if threads <= 1 or len(chunks) == 1:
        for k in range(len(chunks)):
            work(k)
    else:
        with _cf.ThreadPoolExecutor(threads) as ex:
            list(ex.map(work, range(len(chunks))))


def make_problem(n: int, d: int, sigma_max: float, seed: int = 1, noise: float = 0.1,
                 dtype=np.float64, outlier_frac: float = 0.0, outlier_scale: float = 100.0,
                 threads: int | None = None):
    """Returns dict(A (n x d, row-major, `dtype`), b (d, FP64), x_true, y).

    For FP32 A, b is formed from the FP32 values (upcast), so that (A, b) is an exact
    FP64 problem whose matrix is representable in FP32."""
    threads = threads or min(16, os.cpu_count() or 1)
    A = np.empty((n, d), dtype=dtype)
    _fill_normal(A, seed, 0, threads)
    A *= sigma(d, sigma_max).astype(dtype)
    if outlier_frac > 0:
        u = _gen(seed, 3).random(n)
        A[u < outlier_frac] *= dtype(outlier_scale) if dtype != np.float64 else outlier_scale
    x_true = _gen(seed, 1).standard_normal(d)
    eps = np.empty(n)
    _fill_normal(eps, seed, 2, threads)
    A64 = A if A.dtype == np.float64 else A.astype(np.float64)
    y = A64 @ x_true + noise * eps
    b = A64.T @ y
    return {"A": A, "b": np.ascontiguousarray(b), "x_true": x_true, "y": y}


def make_problem_cuda(n: int, d: int, sigma_max: float, seed: int = 1, noise: float = 0.1, dtype=None,
                      outlier_frac: float = 0.0, outlier_scale: float = 100.0, device="cuda", chunk: int = 1 << 18):
    """The same recipe drawn directly in device memory with torch's CUDA generator (for
    workloads too large to draw on the host; the draws differ from make_problem's).
    y and b = A^T y are accumulated in FP64 over row chunks.  Returns dict(A, b) on device."""
    import torch

    dtype = dtype or torch.float32
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    A = torch.empty((n, d), dtype=dtype, device=device)
    sig = torch.tensor(sigma(d, sigma_max), dtype=torch.float64, device=device)
    for r0 in range(0, n, chunk):
        r1 = min(n, r0 + chunk)
        blk = torch.randn((r1 - r0, d), generator=g, dtype=torch.float64, device=device) * sig
        A[r0:r1] = blk.to(dtype)
    if outlier_frac > 0:
        u = torch.rand(n, generator=g, device=device)
        A[u < outlier_frac] *= outlier_scale
    x_true = torch.randn(d, generator=g, dtype=torch.float64, device=device)
    b = torch.zeros(d, dtype=torch.float64, device=device)
    for r0 in range(0, n, chunk):
        r1 = min(n, r0 + chunk)
        blk = A[r0:r1].to(torch.float64)
        y = blk @ x_true + noise * torch.randn(r1 - r0, generator=g, dtype=torch.float64, device=device)
        b += blk.T @ y
    return {"A": A, "b": b}


def batch_shapes(nprob: int, seed: int, n_range=(1 << 12, 1 << 18), d_range=(32, 512), k_range=(1, 16)):
    """Shapes of an uneven batch: n and d log-uniform in their ranges, k uniform in k_range."""
    g = _gen(seed, 10)
    u = g.random((nprob, 2))
    n = np.floor(np.exp(np.log(n_range[0]) + u[:, 0] * (np.log(n_range[1]) - np.log(n_range[0])))).astype(np.int64)
    d = np.floor(np.exp(np.log(d_range[0]) + u[:, 1] * (np.log(d_range[1]) - np.log(d_range[0])))).astype(np.int64)
    k = g.integers(k_range[0], k_range[1] + 1, size=nprob)
    return [(int(a), int(b), int(c)) for a, b, c in zip(n, d, k)]


def make_batch(shapes, seed: int = 1, scale_max: float = 1e4, dtype=np.float32, noise: float = 0.1):
    """One problem per (n, d, k): A = G diag(sigma) (sigma log-spaced 1..scale_max), rounded to
    `dtype`; k right-hand sides b_j = A^T (A x_j + noise eps_j) formed from the rounded A in FP64.
    Returns a list of dicts (A (n x d), B (k x d FP64), X_true (k x d))."""
    out = []
    for p, (n, d, k) in enumerate(shapes):
        A = np.empty((n, d), dtype=np.float64)
        _fill_normal(A, seed * 1000003 + p, 0, 1)
        A = (A * sigma(d, scale_max)).astype(dtype)
        A64 = A.astype(np.float64)
        g = _gen(seed * 1000003 + p, 4)
        Xt = g.standard_normal((k, d))
        E = g.standard_normal((k, n))
        Y = Xt @ A64.T + noise * E
        B = np.ascontiguousarray(Y @ A64)
        out.append({"A": A, "B": B, "X_true": Xt})
    return out


def make_batch_cuda(shapes, seed: int = 1, scale_max: float = 1e4, dtype=None, noise: float = 0.1, device="cuda"):
    """The same recipe drawn in device memory with torch's CUDA generator (draws differ from
    make_batch's).  Returns a list of (A, B) CUDA tensors."""
    import torch

    dtype = dtype or torch.float32
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    out = []
    for n, d, k in shapes:
        sig = torch.tensor(sigma(d, scale_max), dtype=torch.float64, device=device)
        A = (torch.randn((n, d), generator=g, dtype=torch.float64, device=device) * sig).to(dtype)
        A64 = A.to(torch.float64)
        Xt = torch.randn((k, d), generator=g, dtype=torch.float64, device=device)
        Y = Xt @ A64.T + noise * torch.randn((k, n), generator=g, dtype=torch.float64, device=device)
        B = (Y @ A64).contiguous()
        del A64, Y
        out.append((A, B))
    return out


def small_problem(n: int, d: int, kappa: float = 1e2, seed: int = 7):
    """Small dense test problem with column scales log-spaced 1..kappa."""
    return make_problem(n, d, kappa, seed=seed)


# Workloads, named by what they are.  Each entry: shape, conditioning, sketch, target.
WORKLOADS = {
    # Gaussian embedding, FP64, the small case the oracle finishes in seconds.
    "gauss_4096x64_m256": dict(n=4096, d=64, sigma_max=1e4, dtype="f64", sketch="gauss", m=256,
                               seed_data=1, seed_sketch=0, tol=1e-12),
    # FP64 at scale: SRHT / SJLT(s=8) sketches, m in {1024, 2048, 4096}.
    "fp64_1048576x512": dict(n=1 << 20, d=512, sigma_max=1e6, dtype="f64", sketch="srht", m=4096,
                             ms=(1024, 2048, 4096), s=8, seed_data=1, seed_sketch=0, tol=1e-10),
    # FP32-stored A with outliers, Gaussian m=4096.
    "fp32_4194304x1024": dict(n=1 << 22, d=1024, sigma_max=1e5, dtype="f32", sketch="gauss", m=4096,
                              outlier_frac=0.05, seed_data=1, seed_sketch=0, tol=1e-10),
    # Batch: 256 problems, n in [2^12, 2^18], d in [32, 512] (log-uniform), k in 1..16 right-hand
    # sides, A FP32 with column scales 1..1e4; SJLT (s = 8), m = 4d; PCG per right-hand side.
    "batch256_fp32": dict(nprob=256, n_range=(1 << 12, 1 << 18), d_range=(32, 512), k_range=(1, 16),
                          scale_max=1e4, dtype="f32", sketch="sjlt", s=8, m_factor=4.0, seed_data=1,
                          seed_sketch=0, tol=1e-10),
}


def log_spaced_count(lo: float, hi: float, k: int, seed: int) -> np.ndarray:
    """k integers log-uniform in [lo, hi] (for uneven problem batches)."""
    u = _gen(seed, 9).random(k)
    return np.floor(np.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))).astype(np.int64)
