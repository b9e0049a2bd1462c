"""Host logic of bench.py (no GPU): argument defaults per mode, the workload name, and the
solve-traffic calibration it reports only while the solve sources are the captured ones."""
import importlib.util
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _parse(mod, argv, monkeypatch):
    monkeypatch.setattr(sys, "argv", ["bench.py"] + argv)
    return mod.parse()


def test_sketch_precision_defaults_per_mode(monkeypatch):
    mod = _bench()
    a = _parse(mod, [], monkeypatch)
    # the default workload: FP32 A 2^22 x 1024 with outliers, BF16 Gaussian sketch on the tensor cores
    assert (a.sketch, a.sketch_precision, a.m, a.n_log2, a.d, a.a_dtype) == ("gauss", "bf16", 4096, 22, 1024, "f32")
    assert a.outlier_frac == 0.05 and a.sigma_max == 1e5 and a.precision == "mixed"
    f = _parse(mod, ["--workload", "fp64_1048576x512_srht4096_pcg"], monkeypatch)
    assert (f.sketch, f.sketch_precision, f.m, f.n_log2, f.d, f.a_dtype) == ("srht", "f32", 4096, 20, 512, "f64")
    o = _parse(mod, ["--workload", "fp64_1048576x512_srht4096_pcg", "--m", "2048", "--n-log2", "18"], monkeypatch)
    assert (o.m, o.n_log2, o.d) == (2048, 18, 512)
    b = _parse(mod, ["--batch", "256"], monkeypatch)
    assert b.sketch_precision == "bf16"  # the batched workload's SJLT over BF16-rounded A
    c = _parse(mod, ["--batch", "256", "--sketch-precision", "f32"], monkeypatch)
    assert c.sketch_precision == "f32"
    d = _parse(mod, ["--m-sweep", "1024,2048"], monkeypatch)
    assert d.m_sweep == "1024,2048"


def test_workload_name_and_config(monkeypatch):
    mod = _bench()
    a = _parse(mod, [], monkeypatch)
    cfg = mod.workload_config(a, "replicas1")
    assert cfg["workload"] == "fp32_4194304x1024_gauss4096_pcg" == mod.DEFAULT_WORKLOAD
    assert cfg["n"] == 2**22 and cfg["d"] == 1024 and cfg["m"] == 4096 and cfg["tol"] == 1e-10
    assert "model" not in cfg
    for name in mod.PRESETS:
        assert mod.workload_config(_parse(mod, ["--workload", name], monkeypatch), "x")["workload"] == name
    sec = mod.preset_args(a, mod.SECONDARY[mod.DEFAULT_WORKLOAD], steps=5)
    assert mod.workload_config(sec, "x")["workload"] == "fp64_1048576x512_srht4096_pcg" and sec.steps == 5


def test_traffic_calibration_is_sane():
    """The committed DRAM-traffic ratios (measured over algorithmic bytes) say nothing is
    re-read, and they are tied to a hash of the solve sources (bench.py reports
    roofline.traffic only while the sources still hash to it)."""
    mod = _bench()
    for key, ratio in mod.SOLVE_TRAFFIC["ratios"].items():
        assert 1.0 <= ratio < 1.02, key
    h = mod.SOLVE_TRAFFIC["sources_sha256"]
    assert len(h) == 64 and int(h, 16) >= 0
    assert len(mod.solve_sources_sha256()) == 64
    assert 1.0 <= mod.BATCH_TRAFFIC["ratio"] < 1.02
    assert len(mod.BATCH_TRAFFIC["sources_sha256"]) == 64 and len(mod.batch_sources_sha256()) == 64


def test_oracle_accuracy_matches_the_error_against_xstar():
    """The bench's accuracy check (sqrt(r^T H^-1 r / <b, x>) with the oracle's double-double residual
    and PCG) equals the relative H-norm error against the oracle's x* on a perturbed solution."""
    import numpy as np

    import oracle as O
    import workloads as W

    mod = _bench()
    P = W.make_problem(6000, 40, 1e5, seed=3, dtype=np.float32, outlier_frac=0.05)
    A64, b = P["A"].astype(np.float64), P["b"]
    xs = O.solve_direct(A64, b)
    e = np.random.default_rng(1).standard_normal(40)
    for size in (1e-6, 1e-10):
        x = xs + e * size * np.sqrt(O.hmatvec(A64, xs)[1] / O.hmatvec(A64, e)[1])
        acc = mod.oracle_accuracy(A64, b, x)
        assert acc["rel_h_err_vs_oracle"] == pytest.approx(O.rel_h_err(A64, x, xs), rel=1e-3)
