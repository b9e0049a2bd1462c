"""Parity of lsq_factor (H_S = R^T R, W = R^{-1}) with the FP64 oracle."""
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


@pytest.mark.parametrize("m,d,kappa", [(40, 1, 1.0), (70, 37, 1e2), (256, 64, 1e4), (300, 100, 1e3), (1024, 512, 1e6),
                                       (1200, 1024, 1e2), (200, 190, 1e1)])
def test_factor_matches_oracle(L, ctx, m, d, kappa):
    SA = W.make_problem(m, d, kappa, seed=d)["A"]
    R, Wm = L.lsq_factor(ctx, to_dev(SA))
    R, Wm = R.cpu().numpy(), Wm.cpu().numpy()
    Rref = O.factor(SA)
    # columnwise relative error (the factor of a column-scaled matrix is column-scaled)
    colscale = np.abs(Rref).max(axis=0)
    assert np.max(np.abs(R - Rref) / colscale) < 1e-11
    assert np.all(np.tril(R, -1) == 0) and np.all(np.diag(R) > 0)
    assert np.all(np.tril(Wm, -1) == 0)
    np.testing.assert_allclose(Wm @ R, np.eye(d), atol=1e-9)
    Wref = O.tri_inv_upper(Rref)
    rowscale = np.abs(Wref).max(axis=1, keepdims=True)
    assert np.max(np.abs(Wm - Wref) / rowscale) < 1e-9


def test_rank_deficient_is_reported(L, ctx):
    SA = np.random.default_rng(0).standard_normal((50, 8))
    SA[:, 3] = 0.0
    with pytest.raises(L.LsqError) as e:
        L.lsq_factor(ctx, to_dev(SA))
    assert e.value.status == L.LSQ_ERR_RANK
    # the context stays usable
    R, _ = L.lsq_factor(ctx, to_dev(np.eye(8) + 0.1))
    assert np.isfinite(R.cpu().numpy()).all()


def test_rank_deficient_is_reported_when_deferred(L):
    """With deferred checks the factor returns at once; the rank failure is raised by the next
    waiting call (lsq_sync, or lsq_solve in preference to its own status), then cleared."""
    c = L.Context(0)
    try:
        c.set_deferred_checks(True)
        SA = np.random.default_rng(0).standard_normal((50, 8))
        SA[:, 3] = 0.0
        L.lsq_factor(c, to_dev(SA))  # no error yet
        with pytest.raises(L.LsqError) as e:
            L.lsq_sync(c)
        assert e.value.status == L.LSQ_ERR_RANK
        L.lsq_sync(c)  # cleared
        # reported by the solve that follows
        P = W.make_problem(400, 8, 1e2, seed=5)
        A, b = to_dev(P["A"]), to_dev(P["b"])
        _, Wbad = L.lsq_factor(c, to_dev(SA))
        with pytest.raises(L.LsqError) as e:
            L.lsq_solve(c, A, b, "pcg", Wbad, tol=1e-10, maxit=50, m=50)
        assert e.value.status == L.LSQ_ERR_RANK
        # a good factor and solve go through
        _, Wok = L.lsq_factor(c, L.lsq_sketch(c, A, "srht", 64, 0))
        x, info = L.lsq_solve(c, A, b, "pcg", Wok, tol=1e-10, maxit=200, m=64)
        assert info["status"] == 0
        L.lsq_sync(c)
    finally:
        c.close()


@pytest.mark.parametrize("m,d,kappa", [(70, 37, 1e2), (1024, 512, 1e6), (1200, 1024, 1e2), (4096, 300, 1e6)])
def test_factor_double_fp32_gram(L, ctx, m, d, kappa):
    """The Gram matrix in double-FP32 (about 45-bit operands, exact products, TwoSum sums) gives
    the FP64 factor to near FP64 accuracy on column-scaled inputs; the Cholesky stays FP64."""
    SA = W.make_problem(m, d, kappa, seed=d + 1)["A"]
    R, Wm = L.lsq_factor(ctx, to_dev(SA), precision="mixed")
    R, Wm = R.cpu().numpy(), Wm.cpu().numpy()
    Rref = O.factor(SA)
    colscale = np.abs(Rref).max(axis=0)
    assert np.max(np.abs(R - Rref) / colscale) < 1e-9
    assert np.all(np.tril(R, -1) == 0) and np.all(np.diag(R) > 0)
    np.testing.assert_allclose(Wm @ R, np.eye(d), atol=1e-9)
    # an FP32-valued SA (what an FP32 sketch produces) splits exactly: the Gram is the FP64 one
    # up to the order of the sums
    S32 = SA.astype(np.float32).astype(np.float64)
    R32, _ = L.lsq_factor(ctx, to_dev(S32), precision="mixed")
    R64, _ = L.lsq_factor(ctx, to_dev(S32))
    assert np.max(np.abs(R32.cpu().numpy() - R64.cpu().numpy()) / colscale) < 1e-10
