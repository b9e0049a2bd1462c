"""Pins for the oracle's gradient of x* = H^{-1} b: central finite differences in FP64 of
L = g^T x*(A, b) on a 512 x 16 instance, entry by entry, against
dL/dA = -(A x*) lam^T - (A lam) x*^T and dL/db = lam, lam = H^{-1} g."""
import numpy as np

import oracle as O
import workloads as W


def test_gradient_matches_central_differences():
    P = W.make_problem(512, 16, 1e2, seed=21)
    A, b = P["A"], P["b"]
    g = np.random.default_rng(0).standard_normal(16)
    xs, gA, gb = O.solve_grads(A, b, g)
    rng = np.random.default_rng(1)
    loss = lambda A_, b_: float(g @ O.solve_direct(A_, b_))
    # a plausible mistake (a sign, a transposed operand, one of the two terms missing)
    # moves these well beyond the tolerance
    for _ in range(12):
        i, j = rng.integers(512), rng.integers(16)
        h = 1e-5 * max(1.0, abs(A[i, j]))
        Ap, Am = A.copy(), A.copy()
        Ap[i, j] += h
        Am[i, j] -= h
        fd = (loss(Ap, b) - loss(Am, b)) / (2 * h)
        assert abs(fd - gA[i, j]) <= 1e-6 * max(1e-3, abs(gA).max()), (i, j, fd, gA[i, j])
    for j in range(16):
        h = 1e-5 * max(1.0, abs(b[j]))
        bp, bm = b.copy(), b.copy()
        bp[j] += h
        bm[j] -= h
        fd = (loss(A, bp) - loss(A, bm)) / (2 * h)
        assert abs(fd - gb[j]) <= 1e-7 * max(1e-3, abs(gb).max())


def test_gradient_matches_dense_formula():
    P = W.make_problem(300, 8, 1e1, seed=22)
    A, b = P["A"], P["b"]
    g = np.random.default_rng(2).standard_normal(8)
    xs, gA, gb = O.solve_grads(A, b, g)
    Hinv = np.linalg.inv(A.T @ A)
    lam = Hinv @ g
    np.testing.assert_allclose(gb, lam, rtol=1e-10)
    np.testing.assert_allclose(gA, -np.outer(A @ xs, lam) - np.outer(A @ lam, xs), rtol=1e-9, atol=1e-12)
