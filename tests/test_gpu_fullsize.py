"""Parity at the sizes and kernel instances the benchmark times.

* The timed pipeline itself: A 2^20 x 512 FP64 (column scales 1..1e6), FP32 SRHT m = 4096 that
  also writes the FP32 copy of A, double-FP32 Gram + FP64 Cholesky, mixed-precision PCG over
  that copy (the solve kernel's 16-column-per-lane instance), deferred checks on -- checked
  against the oracle's x* (iterative refinement with double-double residuals) to 1e-10 in
  relative H-norm error (Section 1, eq. (PCG)), and its sketch against the oracle's SRHT.
* The wide instance (d = 1024): FP32 A with 5 % outlier rows (x100), BF16 Gaussian sketch on the
  tensor cores, mixed PCG; its sketch checked row by row against the oracle's S on 32 rows.
* The plain FP64 solve at d = 512 and d = 1024 against the oracle's PCG iterates.
"""
import numpy as np
import pytest
import oracle as O
import workloads as W
from gpu_util import rel_fro, to_dev

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def L():
    import paper_1911_02675_gb300 as lib
    return lib


def _xstar(A, b, m):
    """x* of the oracle: refinement with double-double residuals around the oracle's PCG,
    preconditioned by the oracle's own SRHT factor (any preconditioner gives the same x*)."""
    R = O.factor(O.sketch_srht(A, m, 12345))
    return O.solve_refined(A, b, R, A.shape[1] / m, outer=2)


def test_headline_pipeline_reaches_tolerance_against_oracle(L):
    n, d, m, tol = 1 << 20, 512, 4096, 1e-10
    P = W.make_problem(n, d, 1e6, seed=1)
    A, b = P["A"], P["b"]
    ctx = L.Context(0)
    try:
        ctx.set_deferred_checks(True)
        Ad, bd = to_dev(A), to_dev(b)
        a32 = L.narrow_buffer(Ad)
        SA = L.lsq_sketch(ctx, Ad, "srht", m, 0, precision="f32", a32=a32)
        _, Wm = L.lsq_factor(ctx, SA, precision="mixed")
        x, info = L.lsq_solve(ctx, Ad, bd, "pcg", Wm, tol=tol, maxit=1000, m=m, precision="mixed", a32=a32)
        L.lsq_sync(ctx)
        assert info["status"] == 0 and info["a32_copy"] == 2, info
        SA_h = SA.cpu().numpy()
        x_h = x.cpu().numpy()
    finally:
        ctx.close()
    # the FP32 SRHT (staged transform over 2048-row blocks) against the FP64 oracle sketch
    assert rel_fro(SA_h, O.sketch_srht(A, m, 0)) < 5e-6
    xs = _xstar(A, b, m)
    err = O.rel_h_err(A, x_h, xs)
    assert err <= tol, (err, info)


def test_wide_fp32_bf16_gaussian_pipeline_against_oracle(L):
    n, d, m, tol = 1 << 18, 1024, 4096, 1e-10
    P = W.make_problem(n, d, 1e5, seed=2, dtype=np.float32, outlier_frac=0.05)
    A32 = P["A"]
    A64 = A32.astype(np.float64)
    b = P["b"]
    ctx = L.Context(0)
    try:
        Ad = to_dev(A32)
        SA = L.lsq_sketch(ctx, Ad, "gauss", m, 0, precision="bf16")
        _, Wm = L.lsq_factor(ctx, SA, precision="mixed")
        x, info = L.lsq_solve(ctx, Ad, to_dev(b), "pcg", Wm, tol=tol, maxit=1000, m=m, precision="mixed")
        assert info["status"] == 0, info
        SA_h = SA.cpu().numpy()
        x_h = x.cpu().numpy()
    finally:
        ctx.close()
    # 32 rows of the sketch, spread over it, from the oracle's generator (S[j, i] = z(j, i) / sqrt(m))
    rows = np.linspace(0, m - 1, 32).astype(np.int64)
    ref = O.sketch_gauss_rows(A64, m, 0, rows)
    assert rel_fro(SA_h[rows], ref) < 1e-2  # BF16 operands, FP32 accumulation
    xs = _xstar(A64, b, m)
    err = O.rel_h_err(A64, x_h, xs)
    assert err <= tol, (err, info)


@pytest.mark.parametrize("n,d,m", [(1 << 16, 512, 4096), (1 << 15, 1024, 4096)])
def test_plain_fp64_wide_solve_follows_oracle_iterates(L, n, d, m):
    P = W.make_problem(n, d, 1e4, seed=3)
    A, b = P["A"], P["b"]
    ctx = L.Context(0)
    try:
        Ad, bd = to_dev(A), to_dev(b)
        SA = L.lsq_sketch(ctx, Ad, "srht", m, 0)
        _, Wm = L.lsq_factor(ctx, SA)
        xk = {}
        for k in (1, 3, 8):
            x, info = L.lsq_solve(ctx, Ad, bd, "pcg", Wm, tol=0.0, maxit=k, m=m)
            assert info["iters"] == k and info["status"] == L.LSQ_ERR_MAXIT
            xk[k] = x.cpu().numpy()
        x, info = L.lsq_solve(ctx, Ad, bd, "pcg", Wm, tol=1e-10, maxit=500, m=m)
        assert info["status"] == 0, info
        x_final = x.cpu().numpy()
    finally:
        ctx.close()
    R = O.factor(O.sketch_srht(A, m, 0))
    for k, xg in xk.items():
        xr, it, _, _ = O.pcg(A, b, R, tol=0.0, maxit=k, rho_hat=d / m)
        assert it == k
        assert O.rel_h_err(A, xg, xr) < 1e-9 * max(1.0, O.rel_h_err(A, np.zeros(d), xr)), k
    _, it_ref, st_ref, _ = O.pcg(A, b, R, tol=1e-10, maxit=500, rho_hat=d / m)
    assert st_ref == 0 and abs(info["iters"] - it_ref) <= 1
    xs = _xstar(A, b, m)
    assert O.rel_h_err(A, x_final, xs) <= 1e-10
