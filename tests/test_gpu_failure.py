"""Failure detection on the GPU without a fault: every cooperative kernel of the library waits
on bounded grid barriers, and a wait that runs out must end the launch with LSQ_ERR_TIMEOUT
and leave the context usable.  lsq_selftest_wait runs such a barrier waiting for arrivals that
never come (more than its grid has), with a short limit, so the wait runs out on purpose; the
kernel itself always returns."""
import time

import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_util import rel_fro, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import paper_1911_02675_gb300 as lib
    return lib


@pytest.mark.parametrize("kind", [0, 1])
def test_bounded_wait_times_out_and_context_stays_usable(L, kind):
    ctx = L.Context(0)
    try:
        assert L.lsq_selftest_wait(ctx, kind=kind, missing=0, wait_ns=200_000_000) == L.LSQ_OK
        t0 = time.perf_counter()
        st = L.lsq_selftest_wait(ctx, kind=kind, missing=1, wait_ns=50_000_000)
        elapsed = time.perf_counter() - t0
        assert st == L.LSQ_ERR_TIMEOUT
        assert elapsed < 3.0  # the 50 ms limit, or the spin-count limit, ended the wait
        # the same context: a normal barrier, a fused pass and a solve still work
        assert L.lsq_selftest_wait(ctx, kind=kind, missing=0, wait_ns=200_000_000) == L.LSQ_OK
        P = W.make_problem(3000, 24, 1e2, seed=5)
        A, b = P["A"], P["b"]
        Ad, bd = to_dev(A), to_dev(b)
        p = np.random.default_rng(0).standard_normal(24)
        v, q = L.lsq_hmatvec(ctx, Ad, to_dev(p))
        vr, qr = O.hmatvec(A, p)
        assert rel_fro(v.cpu().numpy(), vr) < 1e-13
        _, Wm = L.lsq_factor(ctx, L.lsq_sketch(ctx, Ad, "gauss", 128, 0))
        x, info = L.lsq_solve(ctx, Ad, bd, "pcg", Wm, tol=1e-10, maxit=200, m=128)
        assert info["status"] == 0 and O.rel_h_err(A, x.cpu().numpy(), O.solve_direct(A, b)) <= 1e-10
    finally:
        ctx.close()


def test_bounded_wait_rejects_bad_arguments(L):
    ctx = L.Context(0)
    try:
        for kind, missing, ns in [(2, 1, 1000), (0, -1, 1000), (0, 2000, 1000), (1, 1, 5_000_000_000)]:
            assert L.lsq_selftest_wait(ctx, kind=kind, missing=missing, wait_ns=ns) == L.LSQ_ERR_ARG
    finally:
        ctx.close()
