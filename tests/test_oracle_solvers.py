"""Pins for the oracle's factorisations, H products, x* and the three methods.

References used here never come from the oracle itself: library factorisations
(numpy / scipy), exact rational arithmetic, the optimality identity of PCG
(Section 3, theorem theoremoptimalitypcg), the per-sketch IHS error identity (proof of
theorem thmexacterrorfixed), the exact expected errors with refreshed embeddings
(Section 4, theorem theoremexacterrorrefreshed and the linear system EqnLDSMomentum),
and the one-step convergence of an orthogonal sketch.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
import workloads as W


def _problem(n, d, kappa, seed):
    P = W.make_problem(n, d, kappa, seed=seed)
    return P["A"], P["b"]


def _half_root(A):
    """H^{1/2} = U^T A (notation of Section 1) and U."""
    U, _, _ = np.linalg.svd(A, full_matrices=False)
    return U.T @ A, U


# ---------------------------------------------------------------------------- factor
def test_cholesky_and_qr_match_library():
    rng = np.random.default_rng(0)
    M = rng.standard_normal((60, 7)) * np.logspace(0, 3, 7)
    G = O.gram(M)
    np.testing.assert_allclose(G, M.T @ M, rtol=1e-13)
    R = O.cholesky_upper(G)
    np.testing.assert_allclose(R, np.linalg.cholesky(G).T, rtol=1e-10, atol=1e-12 * np.abs(R).max())
    np.testing.assert_allclose(R.T @ R, G, rtol=1e-13, atol=1e-14 * np.abs(G).max())
    Rq = O.qr_r(M)
    Rn = np.linalg.qr(M, mode="r")
    Rn = np.sign(np.diag(Rn))[:, None] * Rn
    np.testing.assert_allclose(Rq, Rn, rtol=1e-11, atol=1e-13 * np.abs(Rn).max())
    np.testing.assert_allclose(Rq, R, rtol=1e-9, atol=1e-11 * np.abs(R).max())


def test_cholesky_reports_rank_deficiency():
    M = np.random.default_rng(1).standard_normal((10, 4))
    M[:, 2] = M[:, 0]
    with pytest.raises(np.linalg.LinAlgError):
        O.cholesky_upper(M.T @ M - 1e-9 * np.eye(4))


def test_triangular_inverse_and_precond_solve():
    rng = np.random.default_rng(2)
    M = rng.standard_normal((40, 6))
    R = O.qr_r(M)
    W_ = O.tri_inv_upper(R)
    np.testing.assert_allclose(W_ @ R, np.eye(6), atol=1e-13)
    assert np.all(np.tril(W_, -1) == 0)
    r = rng.standard_normal(6)
    np.testing.assert_allclose(O.precond_solve(R, r), np.linalg.solve(R.T @ R, r), rtol=1e-12)


# ---------------------------------------------------------------------------- H products
def test_hmatvec_matches_numpy():
    A, _ = _problem(500, 9, 1e3, 3)
    p = np.random.default_rng(3).standard_normal(9)
    v, q = O.hmatvec(A, p)
    np.testing.assert_allclose(v, A.T @ (A @ p), rtol=1e-12)
    assert q == pytest.approx(np.sum((A @ p) ** 2), rel=1e-12)
    # strided rows
    big = np.zeros((500, 12))
    big[:, :9] = A
    v2, _ = O.hmatvec(big[:, :9], p)
    np.testing.assert_allclose(v2, v, rtol=1e-14)


def test_residual_double_double_is_exact_to_rounding():
    rng = np.random.default_rng(4)
    A = rng.standard_normal((7, 3))
    x = rng.standard_normal(3)
    b = A.T @ (A @ x)  # the exact residual is tiny: heavy cancellation
    exact = []
    Af = [[Fraction(v) for v in row] for row in A]
    xf = [Fraction(v) for v in x]
    w = [sum(Af[i][k] * xf[k] for k in range(3)) for i in range(7)]
    for c in range(3):
        exact.append(Fraction(b[c]) - sum(Af[i][c] * w[i] for i in range(7)))
    r = O.residual_dd(A, b, x)
    for c in range(3):
        assert abs(Fraction(r[c]) - exact[c]) <= abs(exact[c]) * Fraction(1, 2**50) + Fraction(1, 2**200)


# ---------------------------------------------------------------------------- x*
def test_solve_direct_exact_rational():
    rng = np.random.default_rng(5)
    n, d = 12, 3
    A = np.round(rng.standard_normal((n, d)) * 8) / 8
    b = np.round(rng.standard_normal(d) * 8) / 8
    Af = [[Fraction(v) for v in row] for row in A]
    H = [[sum(Af[i][a] * Af[i][c] for i in range(n)) for c in range(d)] for a in range(d)]
    bf = [Fraction(v) for v in b]
    # Gauss-Jordan in exact arithmetic
    M = [H[a][:] + [bf[a]] for a in range(d)]
    for k in range(d):
        piv = M[k][k]
        M[k] = [v / piv for v in M[k]]
        for a in range(d):
            if a != k:
                f = M[a][k]
                M[a] = [va - f * vk for va, vk in zip(M[a], M[k])]
    xs = np.array([float(M[a][d]) for a in range(d)])
    np.testing.assert_allclose(O.solve_direct(A, b), xs, rtol=1e-15, atol=0)


def test_solve_direct_ill_conditioned_columns():
    A, b = _problem(800, 10, 1e6, 6)
    x = O.solve_direct(A, b)
    xl = np.linalg.lstsq(A.T @ A, b, rcond=None)[0]
    assert O.rel_h_err(A, xl, x) < 1e-7
    r = O.residual_dd(A, b, x)
    # backward-error scale of a column-scaled problem: r_j relative to sigma_j-weighted terms
    scale = np.abs(A).T @ np.abs(A @ x)
    assert np.all(np.abs(r) <= 1e-14 * scale)


# ---------------------------------------------------------------------------- PCG
def _sketch_C(A, kind, m, seed, U, s=8):
    S = O.sketch(np.eye(A.shape[0]), kind, m, seed, s=s)  # explicit S (m x n)
    SU = S @ U
    return SU.T @ SU


@pytest.mark.parametrize("kind", ["gauss", "srht", "sjlt"])
def test_pcg_attains_optimal_polynomial_error(kind):
    """||Delta_t||^2 = min_{Q(0)=1, deg Q<=t} sum_i Q(1/lambda_i)^2 xi_i^2 (theorem theoremoptimalitypcg)."""
    n, d, m = 128, 6, 24
    A, b = _problem(n, d, 1e2, 11)
    xs = O.solve_direct(A, b)
    Hh, U = _half_root(A)
    R = O.factor(O.sketch(A, kind, m, seed=3))
    lam, V = np.linalg.eigh(_sketch_C(A, kind, m, 3, U))
    x0 = np.random.default_rng(0).standard_normal(d)
    xi = V.T @ (Hh @ (x0 - xs))
    _, it, st, hist = O.pcg(A, b, R, x0=x0, tol=0.0, maxit=d - 1, rho_hat=0.5, xstar=xs)
    assert it == d - 1
    inv = 1.0 / lam
    for t in range(1, d):
        Vm = np.stack([inv ** k for k in range(1, t + 1)], axis=1) * np.abs(xi)[:, None]
        c = np.linalg.lstsq(Vm, -np.abs(xi), rcond=None)[0]
        ell = np.sum((np.abs(xi) + Vm @ c) ** 2)
        assert 2 * hist[t] == pytest.approx(ell, rel=1e-7, abs=1e-12 * 2 * hist[0])


def test_pcg_terminates_within_d_steps_and_obeys_bound():
    n, d, m = 400, 8, 40
    A, b = _problem(n, d, 1e3, 12)
    xs = O.solve_direct(A, b)
    _, U = _half_root(A)
    R = O.factor(O.sketch_gauss(A, m, seed=1))
    lam = np.linalg.eigvalsh(_sketch_C(A, "gauss", m, 1, U))
    _, it, st, hist = O.pcg(A, b, R, tol=0.0, maxit=d, rho_hat=0.5, xstar=xs)
    assert hist[d] <= 1e-26 * hist[0]
    k = (np.sqrt(lam[-1]) - np.sqrt(lam[0])) / (np.sqrt(lam[-1]) + np.sqrt(lam[0]))
    for t in range(d):
        assert hist[t] <= 4 * k ** (2 * t) * hist[0] * (1 + 1e-9)


@pytest.mark.parametrize("n", [64, 48])
def test_orthogonal_sketch_converges_in_one_step(n):
    """m = N SRHT: S^T S = I, so H_S = H; PCG and IHS with mu = theta1/theta2 = 1 finish in one step."""
    d = 5
    A, b = _problem(n, d, 1e3, 13)
    xs = O.solve_direct(A, b)
    N = O.next_pow2(n)
    R = O.factor(O.sketch_srht(A, N, seed=2))
    t1, t2 = O.theta_srht(N, d, N)
    assert t1 / t2 == pytest.approx(1.0, rel=1e-12)
    x, it, st, hist = O.pcg(A, b, R, tol=0.0, maxit=1, rho_hat=0.5, xstar=xs)
    assert O.rel_h_err(A, x, xs) < 1e-12
    x, it, st, hist = O.ihs(A, b, R=R, mu=1.0, tol=0.0, maxit=1, rho_hat=0.5, xstar=xs)
    assert O.rel_h_err(A, x, xs) < 1e-12
    x, it, st, hist = O.ihs(A, b, kind="srht", m=N, seed=5, mu=1.0, tol=0.0, maxit=1, rho_hat=0.5, xstar=xs)
    assert O.rel_h_err(A, x, xs) < 1e-12


def test_pcg_stopping_rule_reaches_tolerance():
    A, b = _problem(4096, 64, 1e4, 1)
    xs = O.solve_direct(A, b)
    m = 256
    R = O.factor(O.sketch_gauss(A, m, seed=0))
    for tol in (1e-6, 1e-10, 1e-12):
        x, it, st, _ = O.pcg(A, b, R, tol=tol, maxit=200, rho_hat=64 / m)
        assert st == 0
        assert O.rel_h_err(A, x, xs) <= tol
        assert it <= O.pcg_iterations_bound(tol * tol, 64 / m) + 2


# ---------------------------------------------------------------------------- IHS, fixed sketch
def test_fixed_ihs_per_sketch_error_identity():
    """delta_t = 1/2 sum_i (1 - mu/lambda_i)^{2t} xi_i^2 (proof of theorem thmexacterrorfixed)."""
    n, d, m = 300, 7, 50
    A, b = _problem(n, d, 1e2, 14)
    xs = O.solve_direct(A, b)
    Hh, U = _half_root(A)
    R = O.factor(O.sketch_gauss(A, m, seed=8))
    lam, V = np.linalg.eigh(_sketch_C(A, "gauss", m, 8, U))
    mu, rate = O.ihs_fixed_params(d / m)
    x, it, st, hist = O.ihs(A, b, R=R, mu=mu, tol=0.0, maxit=12, rho_hat=d / m, xstar=xs)
    xi = V.T @ (Hh @ (np.zeros(d) - xs))
    for t in range(13):
        pred = 0.5 * np.sum((1 - mu / lam) ** (2 * t) * xi ** 2)
        assert hist[t] == pytest.approx(pred, rel=1e-9, abs=1e-13 * hist[0])


def test_fixed_polyak_ihs_recursion():
    """Delta_{t+1} = ((1+beta) I - mu C_S^-1) Delta_t - beta Delta_{t-1} (proof of theorem theoremihsfixed)."""
    n, d, m = 300, 7, 50
    A, b = _problem(n, d, 1e2, 15)
    xs = O.solve_direct(A, b)
    Hh, U = _half_root(A)
    R = O.factor(O.sketch_sjlt(A, m, 4, seed=8))
    lam, V = np.linalg.eigh(_sketch_C(A, "sjlt", m, 8, U, s=4))
    mu, beta = O.polyak_fixed_params(d / m)
    _, it, st, hist = O.ihs(A, b, R=R, mu=mu, beta=beta, tol=0.0, maxit=12, rho_hat=d / m, xstar=xs)
    cur = V.T @ (Hh @ (np.zeros(d) - xs))
    prev = cur.copy()
    for t in range(13):
        assert hist[t] == pytest.approx(0.5 * np.sum(cur ** 2), rel=1e-9, abs=1e-13 * hist[0])
        cur, prev = (1 + beta - mu / lam) * cur - beta * prev, cur


# ---------------------------------------------------------------------------- refreshed sketches
def _mc_refreshed(mu, beta, trials, T, n=64, d=4, m=16, kind="gauss"):
    A, b = _problem(n, d, 1e1, 16)
    xs = O.solve_direct(A, b)
    H = np.zeros((trials, T + 1))
    for k in range(trials):
        _, it, st, hist = O.ihs(A, b, kind=kind, m=m, seed=50000 + k, mu=mu, beta=beta, tol=0.0,
                                maxit=T, rho_hat=d / m, xstar=xs)
        H[k] = hist
    return H


def test_refreshed_ihs_exact_expected_error():
    """E[delta_t] / delta_0 = prod (1 - 2 mu theta1 + mu^2 theta2) (theorem theoremexacterrorrefreshed)."""
    t1, t2 = O.theta_gaussian(16, 4)
    for mu in (t1 / t2, 0.5 * t1 / t2):
        H = _mc_refreshed(mu, 0.0, 3000, 4)
        f = O.refreshed_factor(t1, t2, mu)
        for t in range(1, 5):
            ratio = H[:, t] / H[:, 0]
            se = ratio.std() / np.sqrt(len(ratio))
            assert abs(ratio.mean() - f ** t) < 5 * se, (mu, t, ratio.mean(), f ** t)
    assert O.refreshed_rate(t1, t2) == pytest.approx(1 - t1 * t1 / t2)


def test_refreshed_polyak_expected_error_follows_linear_system():
    """E[delta_t] evolves by the 3x3 system EqnLDSMomentum (proof of theorem theoremmomentumrefreshed)."""
    t1, t2 = O.theta_gaussian(16, 4)
    mu, beta = t1 / t2, 0.3
    H = _mc_refreshed(mu, beta, 3000, 4)
    d0 = H[:, 0].mean()
    eta = (1 + beta) ** 2 - 2 * mu * t1 * (1 + beta) + mu * mu * t2
    gam = 1 + beta - mu * t1
    M = np.array([[eta, 2 * gam, 1.0], [-beta * gam, -beta, 0.0], [beta * beta, 0.0, 0.0]])
    d1 = O.refreshed_factor(t1, t2, mu) * d0     # first step is plain IHS (x_{-1} = x_0)
    X = np.array([d1, -beta * (1 - mu * t1) * d0, beta * beta * d0])
    pred = [d0, d1]
    for _ in range(3):
        X = M @ X
        pred.append(X[0])
    for t in range(5):
        se = H[:, t].std() / np.sqrt(H.shape[0])
        assert abs(H[:, t].mean() - pred[t]) < 5 * se + 1e-12 * d0, (t, H[:, t].mean(), pred[t])
    # the rate is not better than the refreshed IHS rate (theorem theoremminimalrootradius)
    assert max(abs(np.linalg.eigvals(M))) >= O.refreshed_rate(t1, t2) - 1e-12


def test_minimal_root_radius_on_a_grid():
    t1, t2 = O.theta_gaussian(256, 64)
    best = np.inf
    for mu in np.linspace(0.05, 1.5, 40) * t1 / t2:
        for beta in np.linspace(0.0, 0.95, 40):
            eta = (1 + beta) ** 2 - 2 * mu * t1 * (1 + beta) + mu * mu * t2
            gam = 1 + beta - mu * t1
            M = np.array([[eta, 2 * gam, 1.0], [-beta * gam, -beta, 0.0], [beta * beta, 0.0, 0.0]])
            best = min(best, max(abs(np.linalg.eigvals(M))))
    assert best >= O.refreshed_rate(t1, t2) - 1e-9
    assert best <= O.refreshed_rate(t1, t2) + 1e-2


# ---------------------------------------------------------------------------- pivoted QR
def test_pivoted_qr_matches_lapack():
    """Column-pivoted Householder QR against LAPACK's (scipy.linalg.qr with pivoting): the same
    column order where the column norms are well separated, the same R up to row signs."""
    from scipy.linalg import qr as sp_qr

    rng = np.random.default_rng(5)
    for m, d in [(60, 7), (300, 24), (257, 64)]:
        M = rng.standard_normal((m, d)) * np.logspace(0, 4, d)[rng.permutation(d)]
        R, perm, rank = O.qr_pivoted(M)
        Rs, Ps = sp_qr(M, pivoting=True, mode="r")
        Rs = Rs[:d]
        assert rank == d
        assert np.array_equal(perm, Ps)
        Rs = np.sign(np.diag(Rs))[:, None] * Rs
        np.testing.assert_allclose(R, Rs, rtol=1e-10, atol=1e-12 * np.abs(Rs).max())
        np.testing.assert_allclose(R.T @ R, M[:, perm].T @ M[:, perm], rtol=1e-12, atol=1e-13 * np.abs(R).max() ** 2)
        dg = np.diag(R)
        assert np.all(dg > 0) and np.all(dg[1:] <= dg[:-1] * (1 + 1e-12))
        assert np.all(np.tril(R, -1) == 0)


def test_pivoted_qr_reveals_rank():
    rng = np.random.default_rng(6)
    B = rng.standard_normal((200, 5))
    M = np.column_stack([B, B @ rng.standard_normal((5, 3))])  # rank 5 with 8 columns
    R, perm, rank = O.qr_pivoted(M, tol=1e-10)
    assert rank == 5
    assert np.all(R[5:] == 0)
    # the leading columns span M: the trailing ones are combinations of them
    lead = M[:, perm[:5]]
    coef = np.linalg.lstsq(lead, M[:, perm[5:]], rcond=None)[0]
    np.testing.assert_allclose(lead @ coef, M[:, perm[5:]], atol=1e-9 * np.abs(M).max())
    # and a full-rank input with tol = 0 keeps every column
    assert O.qr_pivoted(B)[2] == 5
