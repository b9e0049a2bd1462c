"""Pins for the oracle's flexible CG with refreshed embeddings (GCC / FCG / IPCG).

* GCC with a *fixed* embedding is PCG: with every S_t equal (m = N orthogonal SRHT gives
  H_S = H for every draw), GCC reaches x* in one step, as PCG does.
* Local optimality (eq. eqnoptimalityconditionrefreshed): GCC's x_{t+1} minimises the H-norm
  error over x_0 + span{v_0, ..., v_t}; checked against a direct least-squares over that span.
* Corollary corollaryupperboundfcg: E[delta_t]/delta_0 <= (1 - theta1^2/theta2)^t for FCG with
  refreshed Gaussian embeddings (Monte Carlo), and on average GCC <= IPCG <= IHS (Section 5).
"""
import numpy as np

import oracle as O
import workloads as W


def _prob(n, d, kappa, seed):
    P = W.make_problem(n, d, kappa, seed=seed)
    return P["A"], P["b"]


def test_gcc_orthogonal_sketch_one_step():
    A, b = _prob(64, 5, 1e2, 31)
    xs = O.solve_direct(A, b)
    x, it, st, _ = O.fcg(A, b, kind="srht", m=64, kmax=-1, tol=0.0, maxit=1, rho_hat=0.5)
    assert O.rel_h_err(A, x, xs) < 1e-12


def test_gcc_is_locally_optimal_over_its_span():
    n, d, m = 200, 8, 30
    A, b = _prob(n, d, 1e2, 32)
    xs = O.solve_direct(A, b)
    T = 4
    # the directions v_t are the same whatever the orthogonalisation (they depend on x_t),
    # so rebuild them from GCC's own iterates and compare with the span minimiser
    xg, it, st, _ = O.fcg(A, b, kind="gauss", m=m, seed=3, kmax=-1, tol=0.0, maxit=T, rho_hat=0.5)
    xs_t = [np.zeros(d)]
    for t in range(1, T + 1):
        xt, *_ = O.fcg(A, b, kind="gauss", m=m, seed=3, kmax=-1, tol=0.0, maxit=t, rho_hat=0.5)
        xs_t.append(xt)
    V = []
    for t in range(T):
        R = O.factor(O.sketch_gauss(A, m, 3, t))
        V.append(O.precond_solve(R, b - A.T @ (A @ xs_t[t])))
    V = np.stack(V, axis=1)
    # min_c ||A (V c - x*)||
    c = np.linalg.lstsq(A @ V, A @ xs, rcond=None)[0]
    best = V @ c
    assert O.rel_h_err(A, xg, xs) <= O.rel_h_err(A, best, xs) * (1 + 1e-6) + 1e-13


def test_fcg_bound_and_ordering_monte_carlo():
    n, d, m, T, trials = 64, 4, 16, 4, 600
    A, b = _prob(n, d, 1e1, 33)
    xs = O.solve_direct(A, b)
    t1, t2 = O.theta_gaussian(m, d)
    rate = O.refreshed_rate(t1, t2)
    out = {}
    for name, kmax in (("gcc", -1), ("ipcg", 1)):
        H = np.array([O.fcg(A, b, kind="gauss", m=m, seed=7000 + k, kmax=kmax, tol=0.0, maxit=T, rho_hat=d / m,
                            xstar=xs)[3] for k in range(trials)])
        out[name] = H.mean(axis=0) / H[:, 0].mean()
    Hi = np.array([O.ihs(A, b, kind="gauss", m=m, seed=7000 + k, mu=t1 / t2, tol=0.0, maxit=T, rho_hat=d / m,
                         xstar=xs)[3] for k in range(trials)])
    out["ihs"] = Hi.mean(axis=0) / Hi[:, 0].mean()
    for t in range(1, T + 1):
        assert out["ipcg"][t] <= rate ** t * 1.1
        assert out["gcc"][t] <= out["ipcg"][t] * 1.05
        assert out["ipcg"][t] <= out["ihs"][t] * 1.05
