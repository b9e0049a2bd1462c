"""Sketch-size advisor (Section 6) against the values the paper prints for its worked
example (tests/golden/paper_cost_ratios.txt), for both the oracle and the library's host
entry point (no GPU needed), and against the first-order condition of the Gaussian cost."""
import ctypes
import math
import os

import pytest

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_cost_ratios.txt")


def cases():
    for line in open(GOLDEN):
        if line.strip() and not line.startswith("#"):
            kind, n, d, _, ratio = line.split()
            yield kind, int(n), int(d), float(ratio)


@pytest.mark.parametrize("kind,n,d,printed", list(cases()))
def test_oracle_reproduces_printed_ratio(kind, n, d, printed):
    m_star, ratio = O.optimal_sketch_size(n, d, d / n, kind)
    assert round(ratio, 2) == printed
    assert m_star > d


def test_gaussian_optimum_is_stationary():
    n, d, eps = 10**7, 50, 50 / 10**7
    m_star, _ = O.optimal_sketch_size(n, d, eps, "gauss")
    a = m_star / d
    assert a * math.log(a) == pytest.approx(n / d**2 * math.log(1 / eps), rel=1e-12)


@pytest.fixture(scope="module")
def lib():
    import importlib.util

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    spec = importlib.util.spec_from_file_location("_b", os.path.join(root, "paper_1911_02675_gb300", "build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    L = ctypes.CDLL(mod.build())

    class Advice(ctypes.Structure):
        _fields_ = [("m_star", ctypes.c_double), ("cost_ratio", ctypes.c_double),
                    ("predicted_iters", ctypes.c_double), ("regime", ctypes.c_int32)]

    L.lsq_advise_sketch_size.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_double, ctypes.c_int32,
                                         ctypes.POINTER(Advice)]
    L.lsq_advise_sketch_size.restype = ctypes.c_int
    return L, Advice


@pytest.mark.parametrize("kind,n,d,printed", list(cases()))
def test_library_advisor_matches_paper_and_oracle(lib, kind, n, d, printed):
    L, Advice = lib
    out = Advice()
    assert L.lsq_advise_sketch_size(n, d, d / n, {"gauss": 0, "srht": 1}[kind], ctypes.byref(out)) == 0
    assert round(out.cost_ratio, 2) == printed
    m_star, ratio = O.optimal_sketch_size(n, d, d / n, kind)
    assert out.m_star == pytest.approx(m_star, rel=1e-12)
    assert out.cost_ratio == pytest.approx(ratio, rel=1e-12)
    assert out.predicted_iters >= 1


def test_library_advisor_rejects(lib):
    L, Advice = lib
    out = Advice()
    assert L.lsq_advise_sketch_size(1000, 50, 1e-6, 1, ctypes.byref(out)) == 1   # n <= d^2
    assert L.lsq_advise_sketch_size(10**7, 50, 1e-6, 2, ctypes.byref(out)) == 1  # SJLT
