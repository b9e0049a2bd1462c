"""lsq_factor_qr (Householder QR with column pivoting of SA) against the oracle's pivoted QR, and
PCG with its dense factor W = P R^{-1} (lsq_solve_opts.w_dense) against the oracle's x*.

The sketches here have well separated column norms (scales log-spaced over decades, shuffled),
so the pivot order is decided by gaps far above rounding and must match the oracle's exactly."""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as W
from gpu_util import to_dev

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


@pytest.mark.parametrize("m,d", [(200, 12), (1024, 64), (2048, 600), (4096, 1024), (40, 40)])
def test_pivoted_qr_matches_oracle(L, ctx, m, d):
    rng = np.random.default_rng(m + d)
    SA = rng.standard_normal((m, d)) * np.logspace(0, 3, d)[rng.permutation(d)]
    R, Wm, perm, rank = L.lsq_factor_qr(ctx, to_dev(SA))
    Rr, pr, rr = O.qr_pivoted(SA)
    assert rank == rr == d
    assert np.array_equal(perm.cpu().numpy(), pr)
    Rg = R.cpu().numpy()
    np.testing.assert_allclose(Rg, Rr, rtol=1e-9, atol=1e-11 * np.abs(Rr).max())
    # W = P R^{-1}: row perm[i] of W is row i of the inverse of the oracle's R, and W W^T H_S = I
    Wg = Wm.cpu().numpy()
    Wr = O.tri_inv_upper(Rr)
    np.testing.assert_allclose(Wg[pr], Wr, rtol=1e-7, atol=1e-9 * np.abs(Wr).max())
    H = SA.T @ SA
    np.testing.assert_allclose(Wg @ (Wg.T @ H), np.eye(d), atol=1e-6)


def test_pivoted_qr_reports_rank(L, ctx):
    rng = np.random.default_rng(2)
    B = rng.standard_normal((300, 10)) * np.logspace(0, 2, 10)
    SA = np.column_stack([B, B[:, :4] @ rng.standard_normal((4, 6))])  # rank 10 of 16 columns
    R, Wm, perm, rank = L.lsq_factor_qr(ctx, to_dev(SA), tol=1e-10, raise_on_rank=False)
    _, pr, rr = O.qr_pivoted(SA, tol=1e-10)
    assert Wm is None and rank == rr == 10
    assert np.array_equal(perm.cpu().numpy()[:10], pr[:10])
    assert np.all(R.cpu().numpy()[10:] == 0)
    with pytest.raises(L.LsqError) as e:
        L.lsq_factor_qr(ctx, to_dev(SA), tol=1e-10)
    assert e.value.status == L.LSQ_ERR_RANK


@pytest.mark.parametrize("precision,kind", [("f64", "srht"), ("mixed", "gauss"), ("f64", "sjlt")])
def test_pcg_with_the_pivoted_qr_factor(L, ctx, precision, kind):
    n, d, m = 30000, 96, 512
    P = W.make_problem(n, d, 1e6, seed=13)
    A, b = P["A"], P["b"]
    Ad, bd = to_dev(A), to_dev(b)
    SA = L.lsq_sketch(ctx, Ad, kind, m, 0)
    _, Wq, _, _ = L.lsq_factor_qr(ctx, SA)
    x, info = L.lsq_solve(ctx, Ad, bd, "pcg", Wq, tol=1e-10, maxit=300, m=m, precision=precision, w_dense=1)
    assert info["status"] == 0, info
    xs = O.solve_direct(A, b)
    assert O.rel_h_err(A, x.cpu().numpy(), xs) <= 1e-10
    # the same preconditioner as the Cholesky factor: the same number of iterations, within one
    _, Wc = L.lsq_factor(ctx, SA)
    _, ic = L.lsq_solve(ctx, Ad, bd, "pcg", Wc, tol=1e-10, maxit=300, m=m, precision=precision)
    assert abs(ic["iters"] - info["iters"]) <= 1
    # fixed-embedding IHS with the dense factor too
    x2, i2 = L.lsq_solve(ctx, Ad, bd, "ihs", Wq, tol=1e-10, maxit=500, m=m, w_dense=1)
    assert i2["status"] == 0 and O.rel_h_err(A, x2.cpu().numpy(), xs) <= 1e-10
