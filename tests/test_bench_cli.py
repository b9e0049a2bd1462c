"""Host logic of bench.py (no GPU): argument defaults per mode, the workload name, and the
solve-traffic calibration it reports only while the solve sources are the captured ones."""
import importlib.util
import os
import sys

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
    assert a.sketch_precision == "f32" and a.sketch == "srht" and a.m == 4096 and a.n_log2 == 20 and a.d == 512
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
    assert cfg["workload"] == "fp64_1048576x512_srht4096_pcg"
    assert cfg["n"] == 2**20 and cfg["d"] == 512 and cfg["m"] == 4096 and cfg["tol"] == 1e-10
    assert "model" not in cfg


def test_traffic_calibration_is_sane():
    """The committed DRAM-traffic ratios (measured over algorithmic bytes) say nothing is
    re-read, and they are tied to a hash of the solve sources (bench.py reports
    roofline.traffic only while the sources still hash to it)."""
    mod = _bench()
    assert 1.0 <= mod.SOLVE_TRAFFIC["ratio_solve"] < 1.01
    assert 1.0 <= mod.SOLVE_TRAFFIC["ratio_with_copy"] < 1.01
    h = mod.SOLVE_TRAFFIC["sources_sha256"]
    assert len(h) == 64 and int(h, 16) >= 0
    assert len(mod.solve_sources_sha256()) == 64
