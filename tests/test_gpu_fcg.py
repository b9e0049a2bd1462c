"""Parity of lsq_solve's flexible CG with refreshed embeddings (GCC, FCG(k), IPCG; Section 1,
eqs. eqnconjugatedirectionsrefreshed and eqnflexiblecg) with the FP64 oracle.

The CUDA path draws the same sketches as the oracle (Philox keyed by (seed, t)), so in FP64
the iterates agree to rounding; a ragged d (not a multiple of 32), float32 storage of A, a
nonzero x0, a fixed embedding (which makes GCC plain PCG) and the mixed mode, which must
still reach the tolerance against the oracle's x*, are covered."""
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


@pytest.fixture(scope="module")
def ctx(L):
    c = L.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("kind,k", [("gauss", -1), ("gauss", 1), ("srht", -1), ("sjlt", 2), ("srht", 1)])
def test_fcg_follows_oracle(L, ctx, kind, k):
    n, d, m = 3001, 37, 160
    P = W.make_problem(n, d, 1e3, seed=11)
    A, b = P["A"], P["b"]
    Ad, bd = to_dev(A), to_dev(b)
    for T in (1, 3, 6):
        x, info = L.lsq_solve(ctx, Ad, bd, "fcg", None, tol=0.0, maxit=T, m=m, refresh=1, sketch_type=kind, seed=21,
                              s=8, fcg_k=k)
        xr, it, st, _ = O.fcg(A, b, kind=kind, m=m, s=8, seed=21, kmax=k, tol=0.0, maxit=T, rho_hat=d / m)
        assert info["iters"] == T == it
        assert rel_fro(x.cpu().numpy(), xr) < 1e-10, (T, rel_fro(x.cpu().numpy(), xr))
    xs = O.solve_direct(A, b)
    x, info = L.lsq_solve(ctx, Ad, bd, "fcg", None, tol=1e-10, maxit=200, m=m, refresh=1, sketch_type=kind, seed=21,
                          s=8, fcg_k=k)
    xr, it, st, _ = O.fcg(A, b, kind=kind, m=m, s=8, seed=21, kmax=k, tol=1e-10, maxit=200, rho_hat=d / m)
    assert info["status"] == 0 and st == 0
    assert abs(info["iters"] - it) <= 1
    assert O.rel_h_err(A, x.cpu().numpy(), xs) <= 1e-10


def test_fcg_nonzero_x0_f32_storage(L, ctx):
    n, d, m = 4100, 64, 256
    P = W.make_problem(n, d, 1e2, seed=12)
    A = P["A"].astype(np.float32)
    b = P["b"]
    x0 = np.random.default_rng(4).standard_normal(d)
    x, info = L.lsq_solve(ctx, to_dev(A), to_dev(b), "fcg", None, x0=to_dev(x0), tol=0.0, maxit=4, m=m, refresh=1,
                          sketch_type="gauss", seed=5)
    xr, it, st, _ = O.fcg(A.astype(np.float64), b, kind="gauss", m=m, seed=5, kmax=-1, x0=x0, tol=0.0, maxit=4,
                          rho_hat=d / m)
    assert rel_fro(x.cpu().numpy(), xr) < 1e-10
    assert info["passes"] == 5  # the initial residual + one per iteration


def test_fcg_fixed_embedding_is_pcg(L, ctx):
    """With one embedding for every iteration, GCC's directions are PCG's (Section 1)."""
    n, d, m = 5000, 48, 240
    P = W.make_problem(n, d, 1e4, seed=13)
    A, b = P["A"], P["b"]
    Ad, bd = to_dev(A), to_dev(b)
    SA = L.lsq_sketch(ctx, Ad, "gauss", m, seed=2)
    R, Wm = L.lsq_factor(ctx, SA)
    for T in (2, 5):
        xf, _ = L.lsq_solve(ctx, Ad, bd, "fcg", Wm, tol=0.0, maxit=T, m=m)
        xp, _ = L.lsq_solve(ctx, Ad, bd, "pcg", Wm, tol=0.0, maxit=T, m=m)
        assert rel_fro(xf.cpu().numpy(), xp.cpu().numpy()) < 1e-8


@pytest.mark.parametrize("kind", ["gauss", "srht"])
def test_fcg_mixed_reaches_tolerance(L, ctx, kind):
    n, d, m = 20000, 96, 480
    P = W.make_problem(n, d, 1e6, seed=14)
    A, b = P["A"], P["b"]
    xs = O.solve_direct(A, b)
    x, info = L.lsq_solve(ctx, to_dev(A), to_dev(b), "fcg", None, tol=1e-10, maxit=300, m=m, refresh=1,
                          sketch_type=kind, seed=8, precision="mixed")
    assert info["status"] == 0
    assert O.rel_h_err(A, x.cpu().numpy(), xs) <= 1e-10


def test_fcg_zero_rhs_and_maxit(L, ctx):
    n, d, m = 1000, 20, 100
    P = W.make_problem(n, d, 1e2, seed=15)
    Ad = to_dev(P["A"])
    x, info = L.lsq_solve(ctx, Ad, to_dev(np.zeros(d)), "fcg", None, tol=1e-10, maxit=20, m=m, refresh=1)
    assert info["status"] == 0 and info["iters"] == 0 and not x.abs().sum().item()
    x, info = L.lsq_solve(ctx, Ad, to_dev(P["b"]), "fcg", None, tol=1e-15, maxit=2, m=m, refresh=1)
    assert info["status"] == L.LSQ_ERR_MAXIT and info["iters"] == 2
