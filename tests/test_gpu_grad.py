"""Differentiation through the solve on the GPU against the oracle's gradients."""
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


@pytest.mark.parametrize("n,d,dtype", [(512, 16, np.float64), (5000, 100, np.float64), (3000, 64, np.float32)])
def test_grad_a_kernel(L, ctx, n, d, dtype):
    A = W.make_problem(n, d, 1e3, seed=n)["A"].astype(dtype)
    rng = np.random.default_rng(3)
    x, lam = rng.standard_normal(d), rng.standard_normal(d)
    gA = L.lsq_grad_a(ctx, to_dev(A), to_dev(x), to_dev(lam)).cpu().numpy()
    ref = O.grad_a(A.astype(np.float64), x, lam)
    assert rel_fro(gA, ref) < (1e-13 if dtype == np.float64 else 1e-6)


@pytest.mark.parametrize("precision", ["f64", "mixed"])
def test_autograd_through_solve(L, ctx, precision):
    """grad_b = lam, grad_A = -(A x*) lam^T - (A lam) x*^T; the dense gradient of the 512 x 16
    finite-difference instance and a larger one."""
    for n, d, m in [(512, 16, 64), (20000, 128, 1024)]:
        P = W.make_problem(n, d, 1e4, seed=d)
        A, b = P["A"], P["b"]
        g = np.random.default_rng(4).standard_normal(d)
        xs, gA_ref, gb_ref = O.solve_grads(A, b, g)
        Ad = to_dev(A).requires_grad_(True)
        bd = to_dev(b).requires_grad_(True)
        x = L.lstsq_solve(Ad, bd, ctx, sketch="srht", m=m, tol=1e-12, precision=precision)
        (x * to_dev(g)).sum().backward()
        assert O.rel_h_err(A, x.detach().cpu().numpy(), xs) <= 1e-12
        assert rel_fro(bd.grad.cpu().numpy(), gb_ref) < 1e-9
        assert rel_fro(Ad.grad.cpu().numpy(), gA_ref) < 1e-9
