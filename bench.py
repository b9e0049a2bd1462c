"""Benchmark: time-to-1e-10 (relative H-norm error) of the randomized-preconditioned
least-squares solve on one GB300, sketch + factor + iterations, A resident in HBM.

Default workload (fp32_4194304x1024_gauss4096_pcg): A 2^22 x 1024 stored in FP32,
A = G diag(sigma) with sigma log-spaced 1..1e5 and 5 % of the rows scaled x100 (high-leverage
outliers), b = A^T (A x_true + 0.1 eps) formed in FP64 from the FP32 values; Gaussian sketch
m = 4096 (seed 0) generated on the fly in BF16 on the tensor cores with FP32 accumulation;
double-FP32 Gram, FP64 Cholesky and triangular products; mixed-precision PCG (FP32 passes over
A, FP64 residual replacement and update) from x0 = 0 to 1e-10.  A (16 GiB) is larger than L2
(~129 MB), so no flush is needed between steps.

The line also carries, under "secondary", the FP64 workload fp64_1048576x512_srht4096_pcg
(A 2^20 x 512 FP64, sigma 1..1e6, FP32 SRHT m = 4096 that writes the FP32 copy of A, mixed PCG).

Prints one JSON line (see the repository's design notes for every key).
    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload NAME] [--precision f64|mixed] [--sketch srht|sjlt|gauss] [--m 4096]
                    [--n-log2 22] [--d 1024] [--a-dtype f32|f64] [--no-secondary] ...
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import tempfile
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as WL  # noqa: E402

SOLVE_KERNEL = "solve_kernel"

# The timed workloads, named by what they are.  Explicit shape options override a preset.
PRESETS = {
    # FP32-stored A with outliers, BF16 Gaussian sketch on the tensor cores, mixed PCG
    "fp32_4194304x1024_gauss4096_pcg": dict(n_log2=22, d=1024, sigma_max=1e5, a_dtype="f32", outlier_frac=0.05,
                                            sketch="gauss", sketch_precision="bf16", m=4096),
    # FP64 A, FP32 SRHT writing the FP32 copy of A, mixed PCG
    "fp64_1048576x512_srht4096_pcg": dict(n_log2=20, d=512, sigma_max=1e6, a_dtype="f64", outlier_frac=0.0,
                                          sketch="srht", sketch_precision="f32", m=4096),
}
DEFAULT_WORKLOAD = "fp32_4194304x1024_gauss4096_pcg"
SECONDARY = {"fp32_4194304x1024_gauss4096_pcg": "fp64_1048576x512_srht4096_pcg"}

# DRAM traffic of solve_kernel over its algorithmic bytes, from one ncu capture per instance
# (dram__bytes_read.sum + dram__bytes_write.sum of the kernel / the algorithmic bytes of that
# launch), keyed by (A dtype, d, FP32 copy of A): scaled to a launch of the bench by its
# algorithmic bytes (units processed: passes x rows), and reported only while the solve
# sources hash to the captured ones.
#   ("f32", 1024, 0): A 2^18 x 1024 FP32, Gaussian BF16 m = 4096, 36 passes of which 2 exact
#   (profiles/solve_kernel_fp32_262144x1024_gauss4096.md);
#   ("f64", 512, 2): A 2^18 x 512 FP64, SRHT m = 4096, 25 passes of which 2 exact, the FP32 copy
#   supplied by the sketch (profiles/solve_kernel_mixed_262144x512_srht4096.md); ("f64", 512, 1)
#   adds the solve's own narrow_copy_kernel<16> (1.554 GB, from a full capture of that kernel).
SOLVE_TRAFFIC = {
    "sources_sha256": "087cd550b9f9303f7f15ab8132e1f017e5b9befc536eae6e8c89f9d918b62795",
    "ratios": {
        ("f32", 1024, 0): (38971788544 + 48382720) / 38654705664,
        ("f64", 512, 2): (14553791744 + 34407936) / 14495514624,
        ("f64", 512, 1): (1553537240 + 14553791744 + 34407936) / 16106127360,
    },
}


# The same for the batched ring pass (bpass_ring_kernel): one FP32 pass of iteration 0 over every
# problem of the 64-problem batch (ncu --metrics gpu__time_duration.sum,dram__bytes_read.sum,
# dram__bytes_write.sum -k regex:bpass_ring -s 1 -c 1, python bench.py --batch 64 --steps 1
# --warmup 1 --no-cpu --no-e2e): reads of A plus the chunk partials written, over A's bytes.  The
# exact passes stream A through the same ring.
BATCH_TRAFFIC = {
    "sources_sha256": "24f75dc8026795c2dccf6d3c67aa4f6b483408194d47cf2c6680f9ac32380ad6",
    "ratio": (2664949504 + 27429888) / 2663123140,
}


def batch_sources_sha256() -> str:
    import hashlib

    h = hashlib.sha256()
    for f in ("bring.cuh", "batch.cu", "common.cuh", "apass.cuh"):
        with open(os.path.join(ROOT, "paper_1911_02675_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def solve_sources_sha256() -> str:
    import hashlib

    h = hashlib.sha256()
    for f in ("solve.cu", "apass.cuh", "common.cuh"):
        with open(os.path.join(ROOT, "paper_1911_02675_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(PRESETS),
                    help="preset workload; the shape options below override its fields")
    ap.add_argument("--precision", default=os.environ.get("LSQ_BENCH_PRECISION", "mixed"), choices=["f64", "mixed"])
    ap.add_argument("--sketch", default=None, choices=["srht", "sjlt", "gauss"])
    ap.add_argument("--sketch-precision", default=None, choices=["f64", "f32", "bf16"],
                    help="sketch arithmetic (default: the preset's; bf16 for the batched SJLT)")
    ap.add_argument("--a-dtype", default=None, choices=["f64", "f32"])
    ap.add_argument("--outlier-frac", type=float, default=None)
    ap.add_argument("--m", "--sketch-rows", dest="m", type=int, default=None)
    ap.add_argument("--n-log2", type=int, default=None)
    ap.add_argument("--d", "--dim", dest="d", type=int, default=None)
    ap.add_argument("--sigma-max", type=float, default=None)
    ap.add_argument("--tol", type=float, default=1e-10)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle legs (cpu_baseline and the accuracy check)")
    ap.add_argument("--no-plain", action="store_true", help="skip timing plain FP64 PCG beside the build")
    ap.add_argument("--no-secondary", action="store_true", help="skip the secondary workload")
    ap.add_argument("--m-sweep", default="", help="comma-separated sketch sizes: time the solve at each "
                    "(time against m, beside Section 6's advised m*) instead of the bench line")
    ap.add_argument("--sketch-sweep", default="",
                    help="comma-separated kind:precision[:m] (e.g. sjlt:f32:4096,sjlt:bf16:4096): time lsq_sketch "
                    "alone for each on the workload instead of the bench line")
    ap.add_argument("--batch", type=int, default=0,
                    help="time the batched solve of this many uneven problems instead (k right-hand sides each)")
    ap.add_argument("--batch-seed", type=int, default=1)
    args = ap.parse_args(argv)
    apply_preset(args, args.workload)
    if args.batch > 0 and args.sketch_precision_given is False:
        args.sketch_precision = "bf16"  # the batched workload's SJLT over BF16-rounded A
    return args


def apply_preset(args, name):
    """Fills every shape option left unset from the preset `name`."""
    args.sketch_precision_given = args.sketch_precision is not None
    for k, v in PRESETS[name].items():
        if getattr(args, k, None) is None:
            setattr(args, k, v)
    return args


def preset_args(base, name, steps):
    """A copy of `base` on the preset workload `name` (for the secondary line)."""
    a = argparse.Namespace(**vars(base))
    for k, v in PRESETS[name].items():
        setattr(a, k, v)
    a.workload, a.steps = name, steps
    return a


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), float(p["bf16_tflops"]), float(p.get("bf16_tflops_sustained", p["bf16_tflops"])), \
            "measured"
    except Exception:
        return 6800.0, 1900.0, 1700.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        # the raw samples go to LSQ_CLOCKS_DIR (default: the system temporary directory); the
        # bench line carries their summary
        out_dir = os.environ.get("LSQ_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out_dir, f"lsq_clocks_gpu{gpu_index}_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        try:
            rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
        except Exception:
            return out
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if sm:
            out.update(sm_mhz=statistics.median(sm), sm_max_mhz=max(mx), reasons=sorted(reasons), samples=len(sm))
        return out


def max_over_ranks(value: float, world: int, device=None) -> float:
    """The largest of the ranks' values (the job's time is its slowest rank's); the value itself
    when there is one rank.  Uses the initialised process group (NCCL on GPUs, gloo on CPU)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(value)], dtype=torch.float64, device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def make_inputs(args, seed):
    """The workload's (A, b) on the host (FP32 or FP64 A; b formed in FP64 from A's values)."""
    return WL.make_problem(1 << args.n_log2, args.d, args.sigma_max, seed=seed,
                           dtype=np.float32 if args.a_dtype == "f32" else np.float64,
                           outlier_frac=args.outlier_frac)


def workload_config(args, parallelism):
    n = 1 << args.n_log2
    elem = 8 if args.a_dtype == "f64" else 4
    cfg = {"workload": f"{args.a_dtype[:1]}p{args.a_dtype[1:]}_{n}x{args.d}_{args.sketch}{args.m}_pcg",
           "n": n, "d": args.d, "sigma_max": args.sigma_max, "outlier_frac": args.outlier_frac,
           "sketch": args.sketch, "m": args.m, "sketch_precision": args.sketch_precision,
           "precision": args.precision, "method": "pcg", "tol": args.tol, "A_dtype": args.a_dtype,
           "l2": f"inputs larger than L2 (A = {n * args.d * elem / 2**30:.1f} GiB), no flush",
           "parallelism": parallelism}
    return cfg


# ------------------------------------------------------------------------------ oracle legs
# (the only places the bench runs the oracle: the cpu_baseline leg, its accuracy check, and the
# reference arm)
GAUSS_ORACLE_FULL_LIMIT = 2e10  # m n d multiply-adds the oracle's Gaussian sketch runs in whole


def _as_f64(A):
    return A if A.dtype == np.float64 else A.astype(np.float64)


def oracle_estimate(args, P, A64=None, sketch_rows=None):
    """Oracle time (ms) per solve of the workload: sketch + factor + PCG on the host cores.

    * up to 2^20 rows, a Gaussian sketch within GAUSS_ORACLE_FULL_LIMIT multiply-adds, or another
      sketch: the whole workload (above 2^20 rows: the first 2^20 rows, the O(n) phases scaled);
    * a larger Gaussian sketch: `sketch_rows` rows of S (default: one per oracle thread, so every
      core works as in the whole sketch) timed over all n rows and scaled by m / sketch_rows (the
      oracle's sketch is a plain triple loop, parallel over rows of S); the factor timed on an m x d
      matrix; the iterations as (T + 1) passes over all of A, T = ceil(log(4/tol^2)/log(m/d)) the
      iteration count Section 6 predicts, one pass timed as the mean of two."""
    import oracle as O

    n, d, m = P["A"].shape[0], args.d, args.m
    A64 = _as_f64(P["A"]) if A64 is None else A64
    b = P["b"]
    if args.sketch == "gauss" and float(m) * n * d > GAUSS_ORACLE_FULL_LIMIT:
        sketch_rows = min(m, sketch_rows or max(16, O.num_threads()))
        rows = np.linspace(0, m - 1, sketch_rows).astype(np.int64)
        t0 = time.perf_counter()
        O.sketch_gauss_rows(A64, m, 0, rows)
        t_sketch = (time.perf_counter() - t0) * m / sketch_rows
        M = np.random.default_rng(0).standard_normal((m, d))
        t0 = time.perf_counter()
        O.factor(M)
        t_factor = time.perf_counter() - t0
        p = np.random.default_rng(1).standard_normal(d)
        t0 = time.perf_counter()
        for _ in range(2):
            O.hmatvec(A64, p)
        t_pass = (time.perf_counter() - t0) / 2
        T = O.pcg_iterations_bound(args.tol ** 2, d / m)
        est = t_sketch + t_factor + (T + 1) * t_pass
        sample = (f"oracle (FP64 on the FP64 upcast of A): Gaussian SA on {sketch_rows} of {m} rows of S over all "
                  f"{n} rows, scaled by {m / sketch_rows:g} ({t_sketch * sketch_rows / m:.2f} s measured); factor of "
                  f"an {m} x {d} matrix ({t_factor:.2f} s); {T} + 1 passes over A for PCG to {args.tol:g} "
                  f"(T = Section 6's predicted count at rho = d/m), one pass {t_pass:.3f} s measured")
        return est * 1e3, sample, O.num_threads()
    n_sample = min(n, 1 << 20)
    As, bs = A64[:n_sample], b
    if n_sample < n:
        Ps = WL.make_problem(n_sample, d, args.sigma_max, seed=1, outlier_frac=args.outlier_frac,
                             dtype=P["A"].dtype)
        As, bs = _as_f64(Ps["A"]), Ps["b"]
    ms = min(m, O.next_pow2(n_sample))
    t0 = time.perf_counter()
    SA = O.sketch(As, args.sketch, ms, 0)
    t1 = time.perf_counter()
    R = O.factor(SA)
    t2 = time.perf_counter()
    _, it, _, _ = O.pcg(As, bs, R, tol=args.tol, maxit=1000, rho_hat=d / ms)
    t3 = time.perf_counter()
    scale = n / n_sample
    est = (t1 - t0) * scale + (t2 - t1) + (t3 - t2) * scale
    what = "the whole workload" if scale == 1 else f"the first {n_sample} rows of the same recipe"
    sample = (f"oracle on {what} (d={d}, {args.sketch} m={ms}, PCG to {args.tol:g}, {it} iterations)"
              + ("" if scale == 1 else f"; sketch and passes scaled by {scale:g}, factor unscaled")
              + f"; measured {t3 - t0:.2f} s")
    return est * 1e3, sample, O.num_threads()


def oracle_accuracy(A64, b, x):
    """Relative H-norm error ||x - x*||_H / ||x*||_H of the GPU's x, by the oracle: x* - x = H^{-1} r
    with r = b - H x (the oracle's double-double residual), so ||x - x*||_H^2 = r^T H^{-1} r, with
    H^{-1} r from the oracle's PCG to 1e-3 (an error of 1e-6 relative in r^T H^{-1} r), and
    ||x*||_H^2 = <b, x*> estimated by <b, x>.  The PCG's preconditioner is numpy's Cholesky factor
    of the Gram matrix of the first max(64 d, 4096) rows (any preconditioner gives the same H^{-1} r; enough rows that the
    5 % high-leverage rows of the FP32 workload are well represented)."""
    import oracle as O

    n, d = A64.shape
    k = min(n, max(64 * d, 4096))
    t0 = time.perf_counter()
    Ak = A64[:k]
    R = np.linalg.cholesky(Ak.T @ Ak).T  # (library Cholesky: only a preconditioner, not part of the result)
    r = O.residual_dd(A64, b, x)
    z, it, st, _ = O.pcg(A64, r, R, tol=1e-3, maxit=500, rho_hat=d / k)
    err = float(np.sqrt(max(float(r @ z), 0.0) / float(b @ x)))
    return {"rel_h_err_vs_oracle": err, "oracle_s": time.perf_counter() - t0, "oracle_pcg_iters": it,
            "oracle": "sqrt(r^T H^-1 r / <b, x>), r = b - H x in double-double, H^-1 r by the oracle's PCG"}


def run_reference(args):
    rank, world, _ = dist_info()
    if rank != 0:
        return
    P = make_inputs(args, seed=1)
    A64 = _as_f64(P["A"])
    times = []
    for _ in range(args.warmup):
        oracle_estimate(args, P, A64)
    sample, cores = "", 0
    for _ in range(args.steps):
        ms, sample, cores = oracle_estimate(args, P, A64)
        times.append(ms)
    value = statistics.median(times)
    line = {
        "impl": "reference", "metric": "time-to-1e-10 H-norm error per solve", "value": value, "unit": "ms",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": value,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args, "oracle"),
        "cpu_baseline": {"value": value, "unit": "ms", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------ our arm
def _events(torch):
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def _time_calls(torch, dev, stream, fn, reps):
    out = []
    for _ in range(reps):
        e0, e1 = _events(torch)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        r = fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        out.append((e0.elapsed_time(e1), r))
    return out


def measure_workload(args, rank, world, local, secondary=False):
    """Times the workload `args` on this rank's GPU; returns the fields of its bench line."""
    import torch

    dev = torch.device("cuda", local)
    import paper_1911_02675_gb300 as L

    hbm, bf16_burst, bf16_sust, peak_kind = peaks()
    P = make_inputs(args, seed=1 + rank)
    A_host = torch.from_numpy(P["A"])
    b_host = torch.from_numpy(P["b"])
    A = A_host.to(dev)
    b = b_host.to(dev)
    n, d = A.shape
    ctx = L.Context(dev)
    # the sketch and the factor do not wait for their own work; their errors surface at the solve
    ctx.set_deferred_checks(True)
    stream = torch.cuda.current_stream(dev)

    # mixed precision over FP64 A: the sketch also writes the FP32 narrowing of A that the solve's
    # FP32 passes stream (a caller-owned buffer, like SA, W and x)
    a32 = L.narrow_buffer(A) if (args.precision == "mixed" and A.dtype == torch.float64) else None

    def solve_once(Ad, bd, A_from=None):
        # A_from: pinned host rows that lsq_upload_sketch copies into Ad while sketching them
        if A_from is None:
            SA = L.lsq_sketch(ctx, Ad, args.sketch, args.m, 0, precision=args.sketch_precision, a32=a32)
        else:
            SA = L.lsq_upload_sketch(ctx, A_from, Ad, args.sketch, args.m, 0, precision=args.sketch_precision, a32=a32)
        _, Wm = L.lsq_factor(ctx, SA, precision=args.precision)
        x, info = L.lsq_solve(ctx, Ad, bd, "pcg", Wm, tol=args.tol, maxit=1000, m=args.m,
                              precision=args.precision, a32=a32)
        return x, info

    if args.sketch_sweep:
        # each sketch alone (CUDA events), its bytes of A read per unit time and whether two calls agree bit for bit
        rows = []
        for spec in args.sketch_sweep.split(","):
            parts = spec.split(":")
            kind, prec = parts[0], parts[1]
            m = int(parts[2]) if len(parts) > 2 else args.m
            fn = lambda: L.lsq_sketch(ctx, A, kind, m, 0, precision=prec)  # noqa: E731
            first = fn()
            L.lsq_sync(ctx)
            for _ in range(max(1, args.warmup)):
                fn()
            res = _time_calls(torch, dev, stream, fn, max(3, args.steps))
            L.lsq_sync(ctx)
            ms = statistics.median(t for t, _ in res)
            rows.append({"sketch": kind, "precision": prec, "m": m, "ms": ms,
                         "A_GBps": n * d * A.element_size() / (ms * 1e-3) / 1e9,
                         "repeats_bitwise": bool(torch.equal(first, res[-1][1]))})
        ctx.close()
        return {"metric": "sketch time", "unit": "ms", "higher_is_better": False, "sketches": rows,
                "config": workload_config(args, f"replicas{world}")}

    if args.m_sweep:
        # time to tolerance against the sketch size (the paper's trade-off of Section 6: a larger m
        # costs more sketch and factor but fewer passes), beside the advised m*
        sweep = []
        for m in (int(v) for v in args.m_sweep.split(",")):
            args.m = m
            for _ in range(max(1, args.warmup)):
                solve_once(A, b)
            res = _time_calls(torch, dev, stream, lambda: solve_once(A, b)[1], max(1, args.steps))
            total = statistics.median(t for t, _ in res)
            inf = res[-1][1]
            sweep.append({"m": m, "ms": total, "solve_ms": inf["ms_total"], "sketch_factor_ms": total - inf["ms_total"],
                          "iters": inf["iters"], "passes": inf["passes"], "est_err": inf["est_err"],
                          "status": inf["status"]})
        try:
            adv = L.lsq_advise_sketch_size(n, d, args.tol, args.sketch)
        except L.LsqError:
            adv = None
        ctx.close()
        return {"metric": "time-to-1e-10 H-norm error per solve against sketch size", "unit": "ms",
                "higher_is_better": False, "sweep": sweep, "advised": adv,
                "config": workload_config(args, f"replicas{world}")}

    for _ in range(args.warmup):
        x, info = solve_once(A, b)
    torch.cuda.synchronize(dev)

    # device-timed steps (inputs resident), kernel-level split of the solve phase
    ev = [_events(torch) for _ in range(args.steps)]
    infos = []
    launches0 = L.lsq_launch_count()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            ev[k][0].record(stream)
            x, info = solve_once(A, b)
            ev[k][1].record(stream)
            infos.append(info)
        torch.cuda.synchronize(dev)
    launches = L.lsq_launch_count() - launches0
    step_ms = [a.elapsed_time(b_) for a, b_ in ev]
    total_ms = max_over_ranks(sum(step_ms), world, dev)
    ms_per_solve = total_ms / (args.steps * world)
    x_last = x.cpu().numpy()

    solve_ms = statistics.median(i["ms_total"] for i in infos)
    passes = statistics.median(i["passes"] for i in infos)
    exact_passes = statistics.median(i["exact_passes"] for i in infos)
    iters = statistics.median(i["iters"] for i in infos)
    pass_bytes = n * d * A.element_size()
    a32_copy = int(infos[-1]["a32_copy"])
    if a32_copy:
        # FP32 passes over the FP32 copy of A, exact residual passes over A, plus (when the solve
        # made the copy itself) one read of A and one write of the copy
        solve_bytes = (passes - exact_passes) * n * d * 4 + exact_passes * pass_bytes
        if a32_copy == 1:
            solve_bytes += n * d * 12
    else:
        solve_bytes = passes * pass_bytes
    achieved = solve_bytes / (solve_ms * 1e-3) / 1e9
    traffic = None
    key = (args.a_dtype, d, a32_copy)
    if (args.precision == "mixed" and key in SOLVE_TRAFFIC["ratios"]
            and solve_sources_sha256() == SOLVE_TRAFFIC["sources_sha256"]):
        traffic = SOLVE_TRAFFIC["ratios"][key] * solve_bytes

    # the sketch phase alone (the tensor-core kernel for the BF16 Gaussian sketch), after the timed steps
    sk = _time_calls(torch, dev, stream, lambda: L.lsq_sketch(ctx, A, args.sketch, args.m, 0,
                                                              precision=args.sketch_precision, a32=a32), 3)
    L.lsq_sync(ctx)
    sketch_ms = statistics.median(t for t, _ in sk)
    roofline_sketch = None
    if args.sketch == "gauss" and args.sketch_precision == "bf16":
        flops = 2.0 * args.m * n * d
        roofline_sketch = {"bound": "tensor", "kernel": "gauss_tc_kernel (with pack_kernel and the split sum)",
                           "achieved": flops / (sketch_ms * 1e-3) / 1e12, "peak": bf16_sust, "unit": "TFLOP/s",
                           "frac": flops / (sketch_ms * 1e-3) / 1e12 / bf16_sust,
                           "peak_kind": f"{peak_kind} (sustained bf16)", "algorithmic_flops": flops,
                           "sketch_ms": sketch_ms}
    elif args.sketch == "srht":
        sbytes = n * d * A.element_size() + (n * d * 4 if a32 is not None else 0)
        roofline_sketch = {"bound": "hbm", "kernel": "srht_tma_kernel (with the row selection and the split sum)",
                           "achieved": sbytes / (sketch_ms * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
                           "frac": sbytes / (sketch_ms * 1e-3) / 1e9 / hbm, "peak_kind": f"{peak_kind} (burst copy)",
                           "algorithmic_bytes": sbytes, "sketch_ms": sketch_ms}

    # end to end: pinned host A and b -> device, solve, x -> host, every step (before the plain FP64
    # leg, whose minute of FP64 work would otherwise precede it)
    e2e = None
    if not args.no_e2e:
        A_pin = A_host.pin_memory()
        b_pin = b_host.pin_memory()
        x_pin = torch.empty(d, dtype=torch.float64).pin_memory()
        A_dev2 = torch.empty_like(A)
        b_dev2 = torch.empty_like(b)

        def e2e_once():
            b_dev2.copy_(b_pin, non_blocking=True)
            xx, _ = solve_once(A_dev2, b_dev2, A_from=A_pin)
            x_pin.copy_(xx, non_blocking=True)

        e2e_once()  # warm-up
        e_ms = [t for t, _ in _time_calls(torch, dev, stream, e2e_once, max(1, min(args.steps, 3)))]
        del A_dev2, A_pin
        e2e = {"value": statistics.median(e_ms), "unit": "ms",
               "h2d_bytes_per_step": n * d * A.element_size() + d * 8, "d2h_bytes_per_step": d * 8,
               "path": "lsq_upload_sketch (host A copied into HBM inside the call), factor, solve, x to host"}

    # plain FP64 PCG on the same GPU: the same sketch type in FP64 arithmetic, FP64 factor and FP64
    # passes over FP64 data (the FP64 upcast of an FP32 A)
    plain = None
    if not args.no_plain and (args.precision != "f64" or args.sketch_precision != "f64"):
        A64d = A if A.dtype == torch.float64 else A.to(torch.float64)

        def plain_sketch(kind):
            return L.lsq_sketch(ctx, A64d, kind, args.m, 0, precision="f64")

        def plain_rest(SA):
            _, Wm = L.lsq_factor(ctx, SA)
            return L.lsq_solve(ctx, A64d, b, "pcg", Wm, tol=args.tol, maxit=1000, m=args.m, precision="f64")

        slow_sketch = args.sketch == "gauss" and float(args.m) * n * d > 1e12
        entries = {}
        for kind in [args.sketch] + (["srht"] if args.sketch != "srht" else []):
            # the FP64 SIMT Gaussian sketch of a large A takes about a minute: timed once
            reps = 1 if (slow_sketch and kind == "gauss") else 3
            if reps > 1:
                plain_rest(plain_sketch(kind))  # warm-up (context scratch for the FP64 shapes)
            s_ms = statistics.median(t for t, _ in _time_calls(torch, dev, stream, lambda: plain_sketch(kind), reps))
            SA64 = plain_sketch(kind)
            L.lsq_sync(ctx)
            plain_rest(SA64)
            rest = _time_calls(torch, dev, stream, lambda: plain_rest(SA64), 3)
            r_ms = statistics.median(t for t, _ in rest)
            inf = rest[-1][1][1]
            entries[kind] = {"ms": s_ms + r_ms, "sketch_ms": s_ms, "factor_solve_ms": r_ms, "iters": inf["iters"],
                             "est_err": inf["est_err"], "status": inf["status"], "sketch": f"{kind} f64",
                             "sketch_reps": reps, "speedup": (s_ms + r_ms) / statistics.median(step_ms)}
        plain = dict(entries[args.sketch])
        if args.sketch != "srht":
            plain["srht_f64"] = entries["srht"]
        if A64d is not A:
            del A64d
        torch.cuda.empty_cache()

    cpu, accuracy = None, None
    if rank == 0 and world == 1 and not args.no_cpu:
        A64 = _as_f64(P["A"])
        ms, sample, cores = oracle_estimate(args, P, A64)
        cpu = {"value": ms, "unit": "ms", "cores": cores, "kind": "oracle", "sample": sample}
        accuracy = oracle_accuracy(A64, P["b"], x_last)
        accuracy["tol"] = args.tol
        accuracy["met"] = bool(accuracy["rel_h_err_vs_oracle"] <= args.tol)
        del A64

    out = {
        "metric": "time-to-1e-10 H-norm error per solve", "value": ms_per_solve, "unit": "ms",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.precision == "f64" else ("bf16+f32+f64" if args.sketch_precision == "bf16" else "f32+f64"),
        "data": "synthetic (seeded; A = G diag(sigma), replicas on distinct seeds)",
        "config": workload_config(args, f"replicas{world}"),
        "phases": {"solve_ms": solve_ms, "iters": iters, "passes": passes, "exact_passes": exact_passes,
                   "a32_copy": a32_copy, "sketch_factor_ms": statistics.median(step_ms) - solve_ms,
                   "sketch_ms": sketch_ms, "status": infos[-1]["status"], "est_err": infos[-1]["est_err"]},
        "accuracy": accuracy,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "traffic": traffic,
                     "kernel": SOLVE_KERNEL, "peak_kind": f"{peak_kind} (burst copy)",
                     "algorithmic_bytes_per_launch": solve_bytes},
        "roofline_sketch": roofline_sketch,
        "plain_fp64_pcg": plain,
        "cpu_baseline": cpu, "e2e": e2e, "clocks": clk.summary(), "gpu_launches": launches,
    }
    ctx.close()
    del A
    torch.cuda.empty_cache()
    return out


def run_ours(args):
    import torch

    rank, world, local = dist_info()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    line = measure_workload(args, rank, world, local)
    if not args.m_sweep and not args.sketch_sweep and not args.no_secondary and args.workload in SECONDARY and \
            world == 1 and \
            all(getattr(args, k) == v for k, v in PRESETS[args.workload].items()):
        sec = preset_args(args, SECONDARY[args.workload], steps=min(args.steps, 10))
        s = measure_workload(sec, rank, world, local, secondary=True)
        line["secondary"] = {s["config"]["workload"]: {k: s[k] for k in (
            "value", "unit", "steps", "phases", "accuracy", "roofline", "roofline_sketch", "plain_fp64_pcg",
            "cpu_baseline", "e2e", "clocks", "gpu_launches", "config")}}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


# ------------------------------------------------------------------------------ batched workload
def batch_config(args, parallelism):
    return {"workload": f"batch{args.batch}_fp32_sjlt_m4d_pcg", "nprob": args.batch,
            "n_range": [1 << 12, 1 << 18], "d_range": [32, 512], "k_range": [1, 16], "scale_max": 1e4,
            "sketch": "sjlt", "s": 8, "m_factor": 4.0, "sketch_precision": args.sketch_precision,
            "precision": args.precision, "method": "pcg (per right-hand side)", "tol": args.tol, "A_dtype": "f32",
            "l2": "inputs larger than L2", "parallelism": parallelism}


def oracle_batch_estimate(args, shapes):
    """Oracle time for the whole batch from the problems of a bounded prefix (about 10 s of CPU
    work), scaled by the share of sum(n d k) they carry."""
    import oracle as O

    total = sum(n * d * k for n, d, k in shapes)
    done, t_acc, used = 0, 0.0, 0
    for p, (n, d, k) in enumerate(shapes):
        q = WL.make_batch([(n, d, k)], seed=args.batch_seed * 7919 + p, scale_max=1e4, dtype=np.float32)[0]
        t0 = time.perf_counter()
        O.solve_batched([(q["A"], q["B"])], kind="sjlt", s=8, m_factor=4.0, seed=0, tol=args.tol)
        t_acc += time.perf_counter() - t0
        done += n * d * k
        used += 1
        if t_acc > 10.0:
            break
    est = t_acc * total / done
    sample = (f"oracle on the first {used} of {len(shapes)} problems ({100.0 * done / total:.1f} % of sum n d k), "
              f"scaled by sum n d k; measured {t_acc:.2f} s")
    return est * 1e3, sample, O.num_threads()


def run_batch(args):
    import torch

    rank, world, local = dist_info()
    if args.impl == "reference":
        if rank != 0:
            return
        shapes = WL.batch_shapes(args.batch, seed=args.batch_seed)
        times, sample, cores = [], "", 0
        for _ in range(max(1, args.steps)):
            ms, sample, cores = oracle_batch_estimate(args, shapes)
            times.append(ms)
        value = statistics.median(times)
        print(json.dumps({
            "impl": "reference", "metric": "time-to-1e-10 H-norm error per batch", "value": value, "unit": "ms",
            "n_gpus": world, "steps": args.steps, "warmup": 0, "ms_per_step": value, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": batch_config(args, "oracle"),
            "cpu_baseline": {"value": value, "unit": "ms", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}), flush=True)
        return
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import paper_1911_02675_gb300 as L

    hbm, _, _, peak_kind = peaks()
    shapes = WL.batch_shapes(args.batch, seed=args.batch_seed + rank)
    probs = WL.make_batch_cuda(shapes, seed=args.batch_seed + rank, device=dev)
    a_bytes = [n * d * 4 for n, d, _ in shapes]
    ctx = L.Context(dev)
    stream = torch.cuda.current_stream(dev)

    def solve_once():
        return L.lsq_solve_batched(ctx, probs, tol=args.tol, maxit=1000, precision=args.precision,
                                   sketch_precision=args.sketch_precision, seed=0)

    for _ in range(args.warmup):
        solve_once()
    torch.cuda.synchronize(dev)
    launches0 = L.lsq_launch_count()
    if world > 1:
        torch.distributed.barrier()
    infos, step_ms, pers = [], [], []
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            e0, e1 = _events(torch)
            e0.record(stream)
            X, per, info = solve_once()
            e1.record(stream)
            torch.cuda.synchronize(dev)
            step_ms.append(e0.elapsed_time(e1))
            infos.append(info)
            pers.append(per)
    launches = L.lsq_launch_count() - launches0
    total_ms = max_over_ranks(sum(step_ms), world, dev)
    ms_per_batch = total_ms / (args.steps * world)
    info = infos[-1]
    per = pers[-1]
    solve_ms = statistics.median(i["ms_solve"] for i in infos)
    # algorithmic bytes of the persistent launch: one read of A_p per iteration the problem took
    pass_bytes = sum(b * it for b, (it, _) in zip(a_bytes, per))
    achieved = pass_bytes / (solve_ms * 1e-3) / 1e9
    statuses = sorted(set(st for _, st in per))
    # DRAM bytes of the passes from the calibrated ratio (the ring pass: FP32 A, mixed precision)
    batch_traffic = None
    if args.precision == "mixed" and batch_sources_sha256() == BATCH_TRAFFIC["sources_sha256"]:
        batch_traffic = BATCH_TRAFFIC["ratio"] * pass_bytes
    # end to end: every problem's A and B copied from pinned host memory into HBM, the batched
    # solve, every X read back to pinned host memory, all inside the timed region
    e2e = None
    if not args.no_e2e:
        pins = [(A.cpu().pin_memory(), B.cpu().pin_memory()) for A, B in probs]
        x_pins = [torch.empty(B.shape, dtype=torch.float64).pin_memory() for _, B in probs]

        def e2e_once():
            for (A, B), (Ah, Bh) in zip(probs, pins):
                A.copy_(Ah, non_blocking=True)
                B.copy_(Bh, non_blocking=True)
            Xs, _, _ = solve_once()
            for Xd, Xh in zip(Xs, x_pins):
                Xh.copy_(Xd, non_blocking=True)

        e2e_once()  # warm-up
        e_ms = [t for t, _ in _time_calls(torch, dev, stream, e2e_once, max(1, min(args.steps, 3)))]
        h2d = sum(A.numel() * A.element_size() + B.numel() * 8 for A, B in probs)
        d2h = sum(B.numel() * 8 for _, B in probs)
        del pins, x_pins
        e2e = {"value": statistics.median(e_ms), "unit": "ms", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "path": "every A_p and B_p from pinned host memory, lsq_solve_batched, every X_p to host"}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        ms, sample, cores = oracle_batch_estimate(args, shapes)
        cpu = {"value": ms, "unit": "ms", "cores": cores, "kind": "oracle", "sample": sample}
    if rank == 0:
        print(json.dumps({
            "metric": "time-to-1e-10 H-norm error per batch", "value": ms_per_batch, "unit": "ms", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if args.precision == "f64" else "f32+f64",
            "data": "synthetic (seeded shapes; A drawn on the device, column scales 1..1e4)",
            "config": batch_config(args, f"replicas{world}"),
            "phases": {"sketch_ms": info["ms_sketch"], "factor_ms": info["ms_factor"], "solve_ms": solve_ms,
                       "iters_max": info["iters_max"], "passes": info["passes"], "exact_passes": info["exact_passes"],
                       "statuses": statuses, "rhs": sum(k for _, _, k in shapes),
                       "launch_phases_ms": info["ms_phase"],
                       "pass_chunk_elems": info["pass_chunk_elems"], "pass_grid": info["pass_grid"],
                       "A_GiB": sum(a_bytes) / 2 ** 30},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                         "traffic": batch_traffic, "peak_kind": f"{peak_kind} (burst copy)",
                         "kernel": "the batched iterations (bpass_ring_kernel for FP32 A: the passes, about 90 % of "
                                   "the solve phase; A bytes over the whole solve phase's time)",
                         "algorithmic_bytes_per_launch": pass_bytes},
            "cpu_baseline": cpu, "e2e": e2e, "clocks": clk.summary(), "gpu_launches": launches}), flush=True)
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    args = parse()
    if args.batch > 0:
        run_batch(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
