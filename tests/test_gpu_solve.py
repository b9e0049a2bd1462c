"""Parity of the fused pass and of lsq_solve (PCG, IHS, Polyak-IHS) with the FP64 oracle.

Bar: the fused pass to FP64 rounding; every solve reaches its tolerance in relative
H-norm error ||x - x*||_H / ||x*||_H against the oracle's x*, with iteration counts
close to the oracle's; refreshed iterations follow the oracle's iterates (same sketches)."""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as W
from gpu_util import rel_fro, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import paper_1911_02675_gb300 as lib
    return lib


@pytest.fixture(scope="module")
def ctx(L):
    c = L.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("n,d,dtype", [(1, 1, np.float64), (1000, 37, np.float64), (4096, 64, np.float64),
                                       (20001, 512, np.float64), (5000, 1024, np.float64), (3000, 100, np.float32),
                                       (777, 300, np.float64)])
def test_hmatvec(L, ctx, n, d, dtype):
    A = W.make_problem(n, d, 1e3, seed=n % 7)["A"].astype(dtype)
    p = np.random.default_rng(1).standard_normal(d)
    v, q = L.lsq_hmatvec(ctx, to_dev(A), to_dev(p))
    vr, qr = O.hmatvec(A.astype(np.float64), p)
    assert rel_fro(v.cpu().numpy(), vr) < 1e-13
    assert abs(q.item() - qr) <= 1e-13 * qr


def _setup(L, ctx, n, d, kappa, kind, m, seed=1, s=8):
    P = W.make_problem(n, d, kappa, seed=seed)
    A, b = P["A"], P["b"]
    xs = O.solve_direct(A, b)
    Ad, bd = to_dev(A), to_dev(b)
    SA = L.lsq_sketch(ctx, Ad, kind, m, 0, s=s)
    R, Wm = L.lsq_factor(ctx, SA)
    return A, b, xs, Ad, bd, Wm


@pytest.mark.parametrize("kind", ["gauss", "srht", "sjlt"])
@pytest.mark.parametrize("tol", [1e-6, 1e-10, 1e-12])
def test_pcg_reaches_tolerance(L, ctx, kind, tol):
    n, d, m = 4096, 64, 256
    A, b, xs, Ad, bd, Wm = _setup(L, ctx, n, d, 1e4, kind, m)
    x, info = L.lsq_solve(ctx, Ad, bd, "pcg", Wm, tol=tol, maxit=300, m=m)
    assert info["status"] == 0
    err = O.rel_h_err(A, x.cpu().numpy(), xs)
    assert err <= tol, (err, info)
    Rref = O.factor(O.sketch(A, kind, m, 0))
    _, it_ref, st_ref, _ = O.pcg(A, b, Rref, tol=tol, maxit=300, rho_hat=d / m)
    assert abs(info["iters"] - it_ref) <= 1


def test_pcg_cfg_small_gaussian(L, ctx):
    """Gaussian 4096 x 64 (column scales 1..1e4), m = 256, to 1e-12."""
    A, b, xs, Ad, bd, Wm = _setup(L, ctx, 4096, 64, 1e4, "gauss", 256)
    x, info = L.lsq_solve(ctx, Ad, bd, "pcg", Wm, tol=1e-12, maxit=300, m=256)
    assert info["status"] == 0 and O.rel_h_err(A, x.cpu().numpy(), xs) <= 1e-12
    assert info["iters"] <= O.pcg_iterations_bound(1e-24, 64 / 256) + 2


def test_pcg_nonzero_start_and_fp32_storage(L, ctx):
    P = W.make_problem(6000, 50, 1e3, seed=4)
    A32 = P["A"].astype(np.float32)
    A64 = A32.astype(np.float64)
    b = A64.T @ P["y"]
    xs = O.solve_direct(A64, b)
    Ad = to_dev(A32)
    _, Wm = L.lsq_factor(ctx, L.lsq_sketch(ctx, Ad, "srht", 400, 3))
    x0 = to_dev(np.random.default_rng(2).standard_normal(50))
    x, info = L.lsq_solve(ctx, Ad, to_dev(b), "pcg", Wm, x0=x0, tol=1e-11, maxit=300, m=400)
    assert info["status"] == 0 and O.rel_h_err(A64, x.cpu().numpy(), xs) <= 1e-11
    assert info["passes"] == info["iters"] + 1


def test_pcg_ragged_sizes(L, ctx):
    for n, d, m, s in [(333, 17, 60, 8), (10007, 200, 800, 8), (257, 1, 4, 2)]:
        A, b, xs, Ad, bd, Wm = _setup(L, ctx, n, d, 1e2, "sjlt", m, s=s)
        x, info = L.lsq_solve(ctx, Ad, bd, "pcg", Wm, tol=1e-10, maxit=500, m=m)
        assert info["status"] == 0 and O.rel_h_err(A, x.cpu().numpy(), xs) <= 1e-10, (n, d, info)


@pytest.mark.parametrize("method", ["ihs", "polyak"])
def test_fixed_ihs_follows_oracle(L, ctx, method):
    n, d, m = 3000, 40, 400
    A, b, xs, Ad, bd, Wm = _setup(L, ctx, n, d, 1e3, "gauss", m)
    rho = d / m
    mu, beta = O.ihs_fixed_params(rho)[0], 0.0
    if method == "polyak":
        mu, beta = O.polyak_fixed_params(rho)
    Rref = O.factor(O.sketch_gauss(A, m, 0))
    for k in (1, 5, 20):
        x, info = L.lsq_solve(ctx, Ad, bd, method, Wm, tol=0.0, maxit=k, m=m)
        xr, _, _, _ = O.ihs(A, b, R=Rref, mu=mu, beta=beta, tol=0.0, maxit=k, rho_hat=rho)
        assert info["iters"] == k and info["status"] == L.LSQ_ERR_MAXIT
        assert O.rel_h_err(A, x.cpu().numpy(), xr) < 1e-9 * max(1.0, O.rel_h_err(A, np.zeros(d), xr))
    x, info = L.lsq_solve(ctx, Ad, bd, method, Wm, tol=1e-10, maxit=500, m=m)
    assert info["status"] == 0 and O.rel_h_err(A, x.cpu().numpy(), xs) <= 1e-10


@pytest.mark.parametrize("method,kind", [("ihs", "gauss"), ("polyak", "gauss"), ("ihs", "srht"), ("ihs", "sjlt")])
def test_refreshed_follows_oracle(L, ctx, method, kind):
    n, d, m = 2048, 16, 128
    P = W.make_problem(n, d, 1e2, seed=5)
    A, b = P["A"], P["b"]
    Ad, bd = to_dev(A), to_dev(b)
    N = O.next_pow2(n)
    t1, t2 = O.theta_srht(m, d, N) if kind == "srht" else O.theta_gaussian(m, d)
    mu = t1 / t2
    beta = 0.1 if method == "polyak" else 0.0
    for k in (1, 4):
        x, info = L.lsq_solve(ctx, Ad, bd, method, None, tol=0.0, maxit=k, m=m, refresh=1, sketch_type=kind, seed=9, s=8)
        xr, _, _, _ = O.ihs(A, b, kind=kind, m=m, s=8, seed=9, mu=mu, beta=beta, tol=0.0, maxit=k, rho_hat=d / m)
        assert info["iters"] == k
        assert rel_fro(x.cpu().numpy(), xr) < 1e-10
    xs = O.solve_direct(A, b)
    x, info = L.lsq_solve(ctx, Ad, bd, method, None, tol=1e-10, maxit=200, m=m, refresh=1, sketch_type=kind, seed=9)
    assert info["status"] == 0 and O.rel_h_err(A, x.cpu().numpy(), xs) <= 1e-10


def test_maxit_and_breakdown_status(L, ctx):
    A, b, xs, Ad, bd, Wm = _setup(L, ctx, 2000, 30, 1e3, "gauss", 120)
    x, info = L.lsq_solve(ctx, Ad, bd, "pcg", Wm, tol=1e-14, maxit=3, m=120)
    assert info["status"] == L.LSQ_ERR_MAXIT and info["iters"] == 3
    with pytest.raises(L.LsqError):
        L.lsq_solve(ctx, Ad, bd, "pcg", Wm, tol=1e-14, maxit=3, m=120, raise_on_maxit=True)
    Abad = A.copy()
    Abad[17, 3] = np.nan
    with pytest.raises(L.LsqError) as e:
        L.lsq_solve(ctx, to_dev(Abad), bd, "pcg", Wm, tol=1e-10, maxit=50, m=120)
    assert e.value.status == L.LSQ_ERR_BREAKDOWN
    # zero right-hand side: x* = 0, converged at once
    x, info = L.lsq_solve(ctx, Ad, torch.zeros_like(bd), "pcg", Wm, tol=1e-10, maxit=50, m=120)
    assert info["status"] == 0 and info["iters"] == 0 and torch.all(x == 0)


@pytest.mark.parametrize("kind,sketch_precision", [("srht", "f32"), ("sjlt", "f64"), ("gauss", "f32")])
@pytest.mark.parametrize("tol", [1e-8, 1e-10, 1e-12])
def test_mixed_pcg_reaches_tolerance(L, ctx, kind, sketch_precision, tol):
    """FP32 inner passes + exact residual replacement reach the same tolerance as FP64."""
    n, d, m = 20000, 128, 512
    P = W.make_problem(n, d, 1e6, seed=3)
    A, b = P["A"], P["b"]
    xs = O.solve_direct(A, b)
    Ad, bd = to_dev(A), to_dev(b)
    _, Wm = L.lsq_factor(ctx, L.lsq_sketch(ctx, Ad, kind, m, 0, precision=sketch_precision))
    x, info = L.lsq_solve(ctx, Ad, bd, "pcg", Wm, tol=tol, maxit=300, m=m, precision="mixed")
    assert info["status"] == 0, info
    assert O.rel_h_err(A, x.cpu().numpy(), xs) <= tol, info
    assert 1 <= info["exact_passes"] < info["passes"]


def test_mixed_pcg_fp32_storage(L, ctx):
    P = W.make_problem(30000, 256, 1e5, seed=8, outlier_frac=0.05)
    A32 = P["A"].astype(np.float32)
    A64 = A32.astype(np.float64)
    b = A64.T @ P["y"]
    xs = O.solve_direct(A64, b)
    Ad = to_dev(A32)
    _, Wm = L.lsq_factor(ctx, L.lsq_sketch(ctx, Ad, "gauss", 1024, 0, precision="f32"))
    x, info = L.lsq_solve(ctx, Ad, to_dev(b), "pcg", Wm, tol=1e-10, maxit=300, m=1024, precision="mixed")
    assert info["status"] == 0 and O.rel_h_err(A64, x.cpu().numpy(), xs) <= 1e-10, info


@pytest.mark.parametrize("method", ["ihs", "polyak"])
def test_mixed_fixed_ihs(L, ctx, method):
    A, b, xs, Ad, bd, Wm = _setup(L, ctx, 8000, 64, 1e4, "srht", 1024)
    x, info = L.lsq_solve(ctx, Ad, bd, method, Wm, tol=1e-10, maxit=500, m=1024, precision="mixed")
    assert info["status"] == 0 and O.rel_h_err(A, x.cpu().numpy(), xs) <= 1e-10, info
    assert info["exact_passes"] < info["passes"]


def test_mixed_refreshed_ihs(L, ctx):
    P = W.make_problem(4096, 32, 1e3, seed=6)
    A, b = P["A"], P["b"]
    xs = O.solve_direct(A, b)
    x, info = L.lsq_solve(ctx, to_dev(A), to_dev(b), "ihs", None, tol=1e-10, maxit=200, m=256, refresh=1,
                          sketch_type="gauss", seed=3, precision="mixed")
    assert info["status"] == 0 and O.rel_h_err(A, x.cpu().numpy(), xs) <= 1e-10, info


def test_mixed_pcg_with_bf16_gaussian_sketch(L, ctx):
    """FP32-stored A with outliers, tensor-core BF16 Gaussian sketch, mixed-precision PCG."""
    P = W.make_problem(50000, 256, 1e5, seed=9, outlier_frac=0.05)
    A32 = P["A"].astype(np.float32)
    A64 = A32.astype(np.float64)
    b = A64.T @ P["y"]
    xs = O.solve_direct(A64, b)
    Ad = to_dev(A32)
    _, Wm = L.lsq_factor(ctx, L.lsq_sketch(ctx, Ad, "gauss", 1024, 0, precision="bf16"))
    x, info = L.lsq_solve(ctx, Ad, to_dev(b), "pcg", Wm, tol=1e-10, maxit=300, m=1024, precision="mixed")
    assert info["status"] == 0 and O.rel_h_err(A64, x.cpu().numpy(), xs) <= 1e-10, info


@pytest.mark.parametrize("method,refresh,d", [("pcg", 0, 128), ("pcg", 0, 37), ("pcg", 0, 600), ("polyak", 0, 64),
                                              ("ihs", 1, 32)])
def test_mixed_fp32_copy_is_bit_identical(L, ctx, method, refresh, d):
    """The FP32 copy of an FP64 A holds the values the FP32 passes narrow to, so the mixed solve
    over it takes the same steps to the last bit as the one that narrows A in every pass, with a
    ragged d (not a multiple of 32), a nonzero x0 and refreshed single-step launches."""
    n, m = 9001, max(4 * d, 256)
    P = W.make_problem(n, d, 1e5, seed=17)
    A, b = P["A"], P["b"]
    Ad, bd = to_dev(A), to_dev(b)
    x0 = to_dev(np.random.default_rng(2).standard_normal(d))
    if refresh:
        kw = dict(refresh=1, sketch_type="gauss", seed=4)  # (SJLT sums with atomics: not bitwise repeatable)
        Wm = None
    else:
        kw = {}
        _, Wm = L.lsq_factor(ctx, L.lsq_sketch(ctx, Ad, "srht", m, 0, precision="f32"))
    res = []
    for copy in (0, 1, 0):
        x, info = L.lsq_solve(ctx, Ad, bd, method, Wm, x0=x0, tol=1e-10, maxit=400, m=m, precision="mixed",
                              a32_copy=copy, **kw)
        assert info["a32_copy"] == copy
        res.append((x.cpu().numpy(), info))
    (x_0, i_0), (x_1, i_1), (x_2, i_2) = res
    assert np.array_equal(x_0, x_2), "the solve does not repeat bit for bit"
    assert i_0["status"] == i_1["status"] == 0
    assert (i_0["iters"], i_0["passes"], i_0["exact_passes"]) == (i_1["iters"], i_1["passes"], i_1["exact_passes"])
    assert np.array_equal(x_0, x_1), np.abs(x_0 - x_1).max()
    assert i_0["est_err"] == i_1["est_err"]


def test_mixed_solve_with_the_sketch_fp32_copy(L, ctx):
    """The FP32 copy the sketch writes (lsq_sketch(a32=)) replaces the solve's own copy: the same
    iterates to the last bit, and the solve reports it used the caller's copy."""
    n, d, m = 30000, 96, 512
    P = W.make_problem(n, d, 1e5, seed=21)
    Ad, bd = to_dev(P["A"]), to_dev(P["b"])
    a32 = L.narrow_buffer(Ad)
    SA = L.lsq_sketch(ctx, Ad, "srht", m, 0, precision="f32", a32=a32)
    _, Wm = L.lsq_factor(ctx, SA, precision="mixed")
    x1, i1 = L.lsq_solve(ctx, Ad, bd, "pcg", Wm, tol=1e-10, maxit=300, m=m, precision="mixed", a32=a32)
    x0, i0 = L.lsq_solve(ctx, Ad, bd, "pcg", Wm, tol=1e-10, maxit=300, m=m, precision="mixed")
    assert i1["a32_copy"] == 2 and i0["a32_copy"] == 1
    assert i0["status"] == i1["status"] == 0 and i0["passes"] == i1["passes"]
    assert np.array_equal(x0.cpu().numpy(), x1.cpu().numpy())


@pytest.mark.parametrize("sketch", ["srht", "gauss"])
def test_deferred_checks_pipeline_is_identical(L, sketch):
    """With deferred checks (no waits inside the sketch and the factor) the pipeline computes
    the same sketch, factor and iterates to the last bit; lsq_sync then reports no error."""
    n, d, m = 20000, 64, 512
    P = W.make_problem(n, d, 1e4, seed=23)
    out = []
    for defer in (False, True):
        c = L.Context(0)
        try:
            c.set_deferred_checks(defer)
            Ad, bd = to_dev(P["A"]), to_dev(P["b"])
            prec = "bf16" if sketch == "gauss" else "f32"
            SA = L.lsq_sketch(c, Ad, sketch, m, 0, precision=prec)
            _, Wm = L.lsq_factor(c, SA, precision="mixed")
            x, info = L.lsq_solve(c, Ad, bd, "pcg", Wm, tol=1e-10, maxit=300, m=m, precision="mixed")
            L.lsq_sync(c)
            assert info["status"] == 0
            out.append((SA.cpu().numpy(), Wm.cpu().numpy(), x.cpu().numpy()))
        finally:
            c.close()
    for u, v in zip(out[0], out[1]):
        assert np.array_equal(u, v)
