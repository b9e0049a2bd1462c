"""Pins for the oracle's closed-form parameters that no iteration identity fixes.

* ihs_fixed_params / polyak_fixed_params (Section 3, theorem theoremihsfixed and its proof):
  on the event E_rho every eigenvalue lambda of C_S lies in [(1-sqrt rho)^2, (1+sqrt rho)^2].
  The IHS step must minimise the worst contraction max_lambda |1 - mu/lambda| over that
  interval, and the Polyak-IHS pair (mu, beta) must minimise the worst spectral radius of the
  heavy-ball matrix [[1 + beta - mu/lambda, -beta], [1, 0]] (the per-eigenvector block of
  M_{mu,beta}, eq. eqndynamics).  Both optima are found here by brute-force search, which
  knows nothing of the closed forms, and the rates are read off the searched optima.
* theta_srht (Section 2, eqs. eqnsrhtmoments / eqnsrhttrace) below m = N: Monte Carlo over
  Haar embeddings built from their definition (orthonormal rows spanning a uniformly random
  subspace: the Q factor of a Gaussian matrix), rescaled to E[S^T S] = I as every sketch of
  this library is, and over the oracle's own SRHT, whose trace moments the paper equates
  with the Haar ones asymptotically.
"""
import math

import numpy as np
import pytest

import oracle as O


def _lambda_grid(rho, k=4001):
    lo, hi = (1 - math.sqrt(rho)) ** 2, (1 + math.sqrt(rho)) ** 2
    return np.linspace(lo, hi, k)


def _worst_ihs_contraction(mu, lam):
    return np.max(np.abs(1.0 - mu / lam))


def _heavy_ball_radius(mu, beta, lam):
    """Largest modulus of the roots of z^2 - (1 + beta - mu/lambda) z + beta over the grid:
    the eigenvalues of the block [[1 + beta - mu/lambda, -beta], [1, 0]]."""
    a = 1.0 + beta - mu / lam
    disc = a * a - 4.0 * beta
    root = np.sqrt(np.abs(disc))
    real_roots = np.maximum(np.abs(a + root), np.abs(a - root)) / 2.0
    return np.max(np.where(disc >= 0, real_roots, math.sqrt(beta)))


@pytest.mark.parametrize("rho", [0.05, 0.125, 0.25, 0.5, 0.8])
def test_ihs_fixed_step_is_the_minimax_step(rho):
    lam = _lambda_grid(rho)
    # golden-section search of the worst contraction over mu (convex in mu: a max of |affine|)
    lo, hi = 1e-6, 4.0
    g = (math.sqrt(5) - 1) / 2
    for _ in range(200):
        a, b = hi - g * (hi - lo), lo + g * (hi - lo)
        if _worst_ihs_contraction(a, lam) <= _worst_ihs_contraction(b, lam):
            hi = b
        else:
            lo = a
    mu_search = 0.5 * (lo + hi)
    rate_search = _worst_ihs_contraction(mu_search, lam) ** 2
    mu, rate = O.ihs_fixed_params(rho)
    assert mu == pytest.approx(mu_search, rel=1e-6)
    # delta_{t+1} <= ||I - mu C_S^-1||^2 delta_t: the rate is the squared worst contraction
    assert rate == pytest.approx(rate_search, rel=1e-6)
    # and the step equalises the contraction at both ends of the interval
    assert abs(1 - mu / lam[0]) == pytest.approx(abs(1 - mu / lam[-1]), rel=1e-12)


@pytest.mark.parametrize("rho", [0.05, 0.125, 0.25, 0.5])
def test_polyak_fixed_params_minimise_the_heavy_ball_radius(rho):
    lam = _lambda_grid(rho, 1001)
    mu, beta = O.polyak_fixed_params(rho)
    r_closed = _heavy_ball_radius(mu, beta, lam)
    # on E_rho the squared spectral radius (the asymptotic rate of delta_t) is at most rho
    assert r_closed ** 2 <= rho * (1 + 1e-6)  # the discriminant vanishes at both ends: rounding
    # brute force: coarse grid over (mu, beta), then a finer grid around its best point
    best = (np.inf, None, None)
    for mus, betas in [(np.linspace(0.01, 2.0, 200), np.linspace(0.0, 0.99, 100))]:
        for m_ in mus:
            for b_ in betas:
                r = _heavy_ball_radius(m_, b_, lam)
                if r < best[0]:
                    best = (r, m_, b_)
    r0, m0, b0 = best
    for _ in range(3):
        hm, hb = 0.02 * max(m0, 0.05), 0.02 * max(b0, 0.05)
        for m_ in np.linspace(m0 - hm, m0 + hm, 41):
            for b_ in np.linspace(max(0.0, b0 - hb), min(0.999, b0 + hb), 41):
                r = _heavy_ball_radius(m_, b_, lam)
                if r < r0:
                    r0, m0, b0 = r, m_, b_
    # the minimax pair is the closed form, and its radius is sqrt(rho)
    assert r0 == pytest.approx(math.sqrt(rho), rel=2e-3)
    assert r_closed == pytest.approx(r0, rel=2e-3)
    assert mu == pytest.approx(m0, rel=2e-2)
    assert beta == pytest.approx(b0, rel=2e-2, abs=2e-3)


def _trace_moments(C_list, d):
    t1 = np.mean([np.trace(np.linalg.inv(C)) / d for C in C_list])
    t2 = np.mean([np.trace(np.linalg.matrix_power(np.linalg.inv(C), 2)) / d for C in C_list])
    return t1, t2


@pytest.mark.slow
@pytest.mark.parametrize("N,m,d,draws", [(512, 128, 8, 600), (1024, 256, 16, 300), (1024, 64, 4, 600)])
def test_theta_srht_matches_haar_embeddings_below_n(N, m, d, draws):
    """E[C_S^-j] for Haar embeddings scaled to E[S^T S] = I against theta_srht(m, d, N)."""
    rng = np.random.default_rng(N + m + d)
    U, _ = np.linalg.qr(rng.standard_normal((N, d)))
    Cs = []
    for _ in range(draws):
        Q, _ = np.linalg.qr(rng.standard_normal((N, m)))  # N x m, orthonormal columns, uniform span
        S = math.sqrt(N / m) * Q.T  # m x N Haar rows, rescaled: E[S^T S] = I_N
        SU = S @ U
        Cs.append(SU.T @ SU)
    t1, t2 = _trace_moments(Cs, d)
    # the mean of C_S itself is I under this scaling (the convention theta_srht assumes)
    np.testing.assert_allclose(np.mean(Cs, axis=0), np.eye(d), atol=0.05)
    th1, th2 = O.theta_srht(m, d, N)
    # the paper's formulas are finite-sample approximations: exact theta_1 of the scaled Haar
    # embedding is (m/N)(N-d-1)/(m-d-1) (inverse mean of a matrix-variate beta); the Monte Carlo
    # error over these draws is near 1 %; 4 % covers both at these sizes
    assert t1 == pytest.approx(th1, rel=0.04)
    assert t2 == pytest.approx(th2, rel=0.06)
    assert t1 == pytest.approx((m / N) * (N - d - 1) / (m - d - 1), rel=0.015)
    # the rate 1 - theta1^2/theta2 is scale free; it is a difference of close numbers, so a few
    # per cent of approximation error in theta_2 moves it by about as much in absolute terms
    assert 1 - th1 ** 2 / th2 == pytest.approx(1 - t1 ** 2 / t2, abs=0.03)


@pytest.mark.slow
def test_theta_srht_matches_the_srht_trace_moments():
    """eq. eqnsrhttrace: the SRHT's trace moments approach the Haar formulas (here N = 1024,
    m = 256, d = 8, over 400 instances of the oracle's SRHT)."""
    N, m, d = 1024, 256, 8
    rng = np.random.default_rng(7)
    U, _ = np.linalg.qr(rng.standard_normal((N, d)))
    Cs = []
    for t in range(400):
        SU = O.sketch_srht(U, m, seed=11, t=t)
        Cs.append(SU.T @ SU)
    t1, t2 = _trace_moments(Cs, d)
    th1, th2 = O.theta_srht(m, d, N)
    assert t1 == pytest.approx(th1, rel=0.04)
    assert t2 == pytest.approx(th2, rel=0.08)
