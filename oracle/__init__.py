"""FP64 CPU oracle for the randomized-preconditioned least-squares method of
Lacotte & Pilanci, "Faster Least Squares Optimization" (arXiv 1911.02675).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  It shares no code with the CUDA library (``paper_1911_02675_gb300``)
and never imports it.  The arithmetic lives in ``lsq_oracle.c`` (plain C,
FP64 / double-double); this module only marshals numpy arrays and adds the
closed-form parameters of the paper.

Functions and the passages they follow:
  philox4x32_10          Philox4x32-10 (Salmon et al., SC'11), the generator every sketch draws from
  gauss_matrix, sketch_gauss, sketch_gauss_rows   Gaussian embedding N(0, 1/m)   Section 2
  srht_signs, srht_rows, sketch_srht   S = R H E with zero padding      Section 2 (+ footnote)
  sjlt_hash, sketch_sjlt  s nonzeros +-1/sqrt(s) per column of S         Section 2 (last paragraph)
  gram, cholesky_upper, qr_r, qr_pivoted, tri_inv_upper, precond_solve
                          factorisations of H_S                         Section 1 (PCG), Section 6
  hmatvec, residual_dd    H p = A^T A p, b - H x                         Section 1 (problem)
  pcg                     PCG with a fixed embedding                     Section 1, eq. (PCG)
  ihs                     IHS / Polyak-IHS, fixed or refreshed           Section 1, eqs. eqnihs / eqnpolyakihs
  fcg                     GCC / FCG / IPCG, refreshed                    Section 1, eqs. eqnconjugatedirectionsrefreshed / eqnflexiblecg
  solve_direct, solve_refined   x* (QR + double-double refinement)     Section 1 (definition of x*)
  grad_a, solve_grads     gradients of L(x*) w.r.t. A and b              implicit differentiation of H x* = b
  theta_gaussian, theta_srht   inverse moments                           Section 2, eqs. eqngaussianmoments, eqnsrhtmoments
  ihs_fixed_params, polyak_fixed_params                                  Section 3, theorem theoremihsfixed
  refreshed_rate                                                         Section 4, theorem theoremexacterrorrefreshed
  pcg_iterations_bound                                                   Section 6 (T = ceil(log(4/eps)/log(1/rho)))
  optimal_sketch_size                                                    Section 6, theorems theoremoptimalcomplexitysrht / -gaussian
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

from . import build as _build

STATUS = {0: "ok", 1: "bad argument", 2: "rank deficient", 3: "breakdown", 4: "max iterations"}

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        P = ctypes.c_void_p
        i64, i32, u32, u64, dbl = ctypes.c_int64, ctypes.c_int, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double
        sigs = {
            "orc_num_threads": (i32, []),
            "orc_philox4x32_10": (None, [P, P, P]),
            "orc_philox_batch": (None, [i64, P, P, P]),
            "orc_gauss_z": (dbl, [u64, u32, i64, i64]),
            "orc_gauss_matrix": (None, [i64, i64, u64, u32, P]),
            "orc_sketch_gauss": (None, [P, i64, i64, i64, i64, u64, u32, P]),
            "orc_sketch_gauss_rows": (None, [P, i64, i64, i64, i64, u64, u32, P, i64, P]),
            "orc_next_pow2": (i64, [i64]),
            "orc_srht_signs": (None, [i64, u64, u32, P]),
            "orc_srht_rows": (None, [i64, i64, u64, u32, P]),
            "orc_fwht_rows": (None, [P, i64, i64]),
            "orc_sketch_srht": (i32, [P, i64, i64, i64, i64, u64, u32, P]),
            "orc_sjlt_hash": (i32, [i64, i64, i32, u64, u32, P, P]),
            "orc_sketch_sjlt": (i32, [P, i64, i64, i64, i64, i32, u64, u32, P]),
            "orc_gram": (None, [P, i64, i64, P]),
            "orc_cholesky_upper": (i32, [P, i64, P]),
            "orc_qr_r": (i32, [P, i64, i64, P]),
            "orc_qr_pivoted": (i32, [P, i64, i64, dbl, P, P, P]),
            "orc_tri_inv_upper": (None, [P, i64, P]),
            "orc_precond_solve": (None, [P, i64, P, P]),
            "orc_hmatvec": (None, [P, i64, i64, i64, P, P, P]),
            "orc_residual_dd": (None, [P, i64, i64, i64, P, P, P]),
            "orc_pcg": (i32, [P, i64, i64, i64, P, P, P, dbl, i32, dbl, P, P, P]),
            "orc_ihs": (i32, [P, i64, i64, i64, P, P, i32, i64, i32, u64, dbl, dbl, P, dbl, i32, dbl, P, P, P]),
            "orc_solve_direct": (i32, [P, i64, i64, i64, P, P]),
            "orc_solve_refined": (i32, [P, i64, i64, i64, P, P, dbl, P, i32]),
            "orc_rel_h_err": (dbl, [P, i64, i64, i64, P, P]),
            "orc_grad_a": (None, [P, i64, i64, i64, P, P, P]),
            "orc_fcg": (i32, [P, i64, i64, i64, P, i32, i64, i32, u64, i32, P, dbl, i32, dbl, P, P, P]),
        }
        for name, (res, args) in sigs.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _mat(A):
    """(contiguous FP64 copy-or-view, n, d, ld); rows may be strided."""
    A = np.asarray(A)
    if A.dtype != np.float64:
        A = A.astype(np.float64)
    if A.ndim != 2:
        raise ValueError("A must be 2-D")
    n, d = A.shape
    if A.strides[1] != 8 or A.strides[0] % 8 or A.strides[0] < 8 * d:
        A = np.ascontiguousarray(A)
    return A, n, d, A.strides[0] // 8


def num_threads() -> int:
    return lib().orc_num_threads()


# ----------------------------------------------------------------------------- generator
def philox4x32_10(ctr, key) -> np.ndarray:
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    key = np.ascontiguousarray(key, dtype=np.uint32).reshape(2)
    out = np.empty_like(ctr)
    lib().orc_philox_batch(ctr.shape[0], _ptr(ctr), _ptr(key), _ptr(out))
    return out


# ----------------------------------------------------------------------------- sketches
def gauss_z(seed: int, t: int, j: int, i: int) -> float:
    return lib().orc_gauss_z(seed, t, j, i)


def gauss_matrix(m: int, n: int, seed: int, t: int = 0) -> np.ndarray:
    S = np.empty((m, n))
    lib().orc_gauss_matrix(m, n, seed, t, _ptr(S))
    return S


def sketch_gauss(A, m: int, seed: int, t: int = 0) -> np.ndarray:
    A, n, d, ld = _mat(A)
    SA = np.empty((m, d))
    lib().orc_sketch_gauss(_ptr(A), n, d, ld, m, seed, t, _ptr(SA))
    return SA


def sketch_gauss_rows(A, m: int, seed: int, rows, t: int = 0) -> np.ndarray:
    """Rows `rows` of the Gaussian SA (m rows in all) without the others."""
    A, n, d, ld = _mat(A)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    if rows.size and (rows.min() < 0 or rows.max() >= m):
        raise ValueError("row index outside the sketch")
    out = np.empty((rows.size, d))
    lib().orc_sketch_gauss_rows(_ptr(A), n, d, ld, m, seed, t, _ptr(rows), rows.size, _ptr(out))
    return out


def next_pow2(n: int) -> int:
    return lib().orc_next_pow2(n)


def srht_signs(N: int, seed: int, t: int = 0) -> np.ndarray:
    s = np.empty(N, dtype=np.int8)
    lib().orc_srht_signs(N, seed, t, _ptr(s))
    return s


def srht_rows(N: int, m: int, seed: int, t: int = 0) -> np.ndarray:
    rows = np.empty(m, dtype=np.int64)
    lib().orc_srht_rows(N, m, seed, t, _ptr(rows))
    return rows


def fwht_rows(X) -> np.ndarray:
    X = _f64(X).copy()
    N, d = X.shape
    lib().orc_fwht_rows(_ptr(X), N, d)
    return X


def sketch_srht(A, m: int, seed: int, t: int = 0) -> np.ndarray:
    A, n, d, ld = _mat(A)
    SA = np.empty((m, d))
    st = lib().orc_sketch_srht(_ptr(A), n, d, ld, m, seed, t, _ptr(SA))
    if st:
        raise ValueError(f"sketch_srht: {STATUS.get(st, st)}")
    return SA


def sjlt_hash(n: int, m: int, s: int, seed: int, t: int = 0):
    h = np.empty((n, s), dtype=np.int32)
    sg = np.empty((n, s), dtype=np.int8)
    st = lib().orc_sjlt_hash(n, m, s, seed, t, _ptr(h), _ptr(sg))
    if st:
        raise ValueError(f"sjlt_hash: {STATUS.get(st, st)}")
    return h, sg


def sketch_sjlt(A, m: int, s: int, seed: int, t: int = 0) -> np.ndarray:
    A, n, d, ld = _mat(A)
    SA = np.empty((m, d))
    st = lib().orc_sketch_sjlt(_ptr(A), n, d, ld, m, s, seed, t, _ptr(SA))
    if st:
        raise ValueError(f"sketch_sjlt: {STATUS.get(st, st)}")
    return SA


SKETCH_TYPES = {"gauss": 0, "srht": 1, "sjlt": 2}


def sketch(A, kind: str, m: int, seed: int, t: int = 0, s: int = 8) -> np.ndarray:
    if kind == "gauss":
        return sketch_gauss(A, m, seed, t)
    if kind == "srht":
        return sketch_srht(A, m, seed, t)
    if kind == "sjlt":
        return sketch_sjlt(A, m, s, seed, t)
    raise ValueError(kind)


# ----------------------------------------------------------------------------- factor
def gram(M) -> np.ndarray:
    M = _f64(M)
    m, d = M.shape
    G = np.empty((d, d))
    lib().orc_gram(_ptr(M), m, d, _ptr(G))
    return G


def cholesky_upper(G) -> np.ndarray:
    G = _f64(G)
    d = G.shape[0]
    R = np.empty((d, d))
    st = lib().orc_cholesky_upper(_ptr(G), d, _ptr(R))
    if st:
        raise np.linalg.LinAlgError(f"non-positive pivot at column {st - 1}")
    return R


def qr_r(M) -> np.ndarray:
    M = _f64(M)
    m, d = M.shape
    R = np.empty((d, d))
    st = lib().orc_qr_r(_ptr(M), m, d, _ptr(R))
    if st:
        raise np.linalg.LinAlgError(f"zero column {st - 1}")
    return R


def qr_pivoted(M, tol: float = 0.0):
    """Householder QR with column pivoting: (R, perm, rank) with M[:, perm] = Q R, R upper with a
    positive, non-increasing diagonal; rows of R from `rank` on are zero (Section 1, PCG paragraph)."""
    M = _f64(M)
    m, d = M.shape
    R = np.empty((d, d))
    perm = np.empty(d, dtype=np.int32)
    rank = ctypes.c_int64(0)
    lib().orc_qr_pivoted(_ptr(M), m, d, float(tol), _ptr(R), _ptr(perm), ctypes.byref(rank))
    return R, perm, rank.value


def factor(SA) -> np.ndarray:
    """R (upper, positive diagonal) with R^T R = (SA)^T (SA), by Gram + Cholesky."""
    return cholesky_upper(gram(SA))


def tri_inv_upper(R) -> np.ndarray:
    R = _f64(R)
    d = R.shape[0]
    W = np.empty((d, d))
    lib().orc_tri_inv_upper(_ptr(R), d, _ptr(W))
    return W


def precond_solve(R, r) -> np.ndarray:
    R = _f64(R)
    r = _f64(r)
    z = np.empty_like(r)
    lib().orc_precond_solve(_ptr(R), R.shape[0], _ptr(r), _ptr(z))
    return z


# ----------------------------------------------------------------------------- H products
def hmatvec(A, p):
    A, n, d, ld = _mat(A)
    p = _f64(p)
    v = np.empty(d)
    q = np.empty(1)
    lib().orc_hmatvec(_ptr(A), n, d, ld, _ptr(p), _ptr(v), _ptr(q))
    return v, float(q[0])


def residual_dd(A, b, x) -> np.ndarray:
    A, n, d, ld = _mat(A)
    b, x = _f64(b), _f64(x)
    r = np.empty(d)
    lib().orc_residual_dd(_ptr(A), n, d, ld, _ptr(b), _ptr(x), _ptr(r))
    return r


# ----------------------------------------------------------------------------- solvers
def pcg(A, b, R, x0=None, tol=1e-10, maxit=1000, rho_hat=None, xstar=None):
    """PCG (Section 1).  Returns (x, iters, status, hist)."""
    A, n, d, ld = _mat(A)
    b, R = _f64(b), _f64(R)
    x = np.zeros(d) if x0 is None else _f64(x0).copy()
    if rho_hat is None:
        raise ValueError("rho_hat is required (deviation parameter of the stopping rule)")
    hist = np.full(maxit + 1, np.nan)
    it = ctypes.c_int(0)
    xs = _f64(xstar) if xstar is not None else None
    st = lib().orc_pcg(_ptr(A), n, d, ld, _ptr(b), _ptr(R), _ptr(x), tol, maxit, rho_hat,
                       _ptr(xs) if xs is not None else None, ctypes.byref(it), _ptr(hist))
    return x, it.value, st, hist[: it.value + 1]


def ihs(A, b, *, R=None, kind="gauss", m=None, s=8, seed=0, mu, beta=0.0, x0=None, tol=1e-10,
        maxit=1000, rho_hat, xstar=None):
    """IHS / Polyak-IHS (Section 1); R=None draws refreshed sketches (Section 4).
    Returns (x, iters, status, hist)."""
    A, n, d, ld = _mat(A)
    b = _f64(b)
    x = np.zeros(d) if x0 is None else _f64(x0).copy()
    Rp = _f64(R) if R is not None else None
    if Rp is None and m is None:
        raise ValueError("refreshed IHS needs the sketch size m")
    hist = np.full(maxit + 1, np.nan)
    it = ctypes.c_int(0)
    xs = _f64(xstar) if xstar is not None else None
    st = lib().orc_ihs(_ptr(A), n, d, ld, _ptr(b), _ptr(Rp) if Rp is not None else None,
                       SKETCH_TYPES[kind], int(m or 0), s, seed, mu, beta, _ptr(x), tol, maxit, rho_hat,
                       _ptr(xs) if xs is not None else None, ctypes.byref(it), _ptr(hist))
    return x, it.value, st, hist[: it.value + 1]


def fcg(A, b, *, kind="gauss", m, s=8, seed=0, kmax=-1, x0=None, tol=1e-10, maxit=100, rho_hat, xstar=None):
    """Flexible CG with refreshed embeddings: kmax = -1 GCC, kmax = 1 IPCG (Sections 1, 4).
    Returns (x, iters, status, hist)."""
    A, n, d, ld = _mat(A)
    b = _f64(b)
    x = np.zeros(d) if x0 is None else _f64(x0).copy()
    hist = np.full(maxit + 1, np.nan)
    it = ctypes.c_int(0)
    xs = _f64(xstar) if xstar is not None else None
    st = lib().orc_fcg(_ptr(A), n, d, ld, _ptr(b), SKETCH_TYPES[kind], m, s, seed, kmax, _ptr(x), tol, maxit, rho_hat,
                       _ptr(xs) if xs is not None else None, ctypes.byref(it), _ptr(hist))
    return x, it.value, st, hist[: it.value + 1]


def solve_batched(problems, *, kind="sjlt", s=8, m_factor=4.0, seed=0, tol=1e-10, maxit=1000, X0=None):
    """Batched PCG (Section 1, eq. (PCG)) done problem by problem and right-hand side by
    right-hand side: problem p draws sketch instance t = p of `seed` with m = max(d, ceil(m_factor d))
    rows (an SJLT with min(s, m) nonzeros per column), factors it, and runs the oracle's PCG (rho_hat = d / m) from x0 (zero by default) on
    each right-hand side.  problems: list of (A (n x d), B (k x d)).
    Returns a list of (X (k x d), iters (k,), status (k,))."""
    out = []
    for p, (A, B) in enumerate(problems):
        A64 = np.ascontiguousarray(A, dtype=np.float64)
        n, d = A64.shape
        m = max(d, int(math.ceil(m_factor * d)))
        R = factor(sketch(A64, kind, m, seed, t=p, s=min(s, m)))
        X = np.zeros((B.shape[0], d))
        its = np.zeros(B.shape[0], dtype=np.int64)
        sts = np.zeros(B.shape[0], dtype=np.int64)
        for j in range(B.shape[0]):
            x0 = None if X0 is None else X0[p][j]
            X[j], its[j], sts[j], _ = pcg(A64, B[j], R, x0=x0, tol=tol, maxit=maxit, rho_hat=d / m)
        out.append((X, its, sts))
    return out


def solve_direct(A, b) -> np.ndarray:
    A, n, d, ld = _mat(A)
    b = _f64(b)
    x = np.empty(d)
    st = lib().orc_solve_direct(_ptr(A), n, d, ld, _ptr(b), _ptr(x))
    if st:
        raise np.linalg.LinAlgError("A is rank deficient")
    return x


def solve_refined(A, b, R, rho_hat, outer=6) -> np.ndarray:
    A, n, d, ld = _mat(A)
    b, R = _f64(b), _f64(R)
    x = np.empty(d)
    st = lib().orc_solve_refined(_ptr(A), n, d, ld, _ptr(b), _ptr(R), rho_hat, _ptr(x), outer)
    if st:
        raise RuntimeError(f"solve_refined: {STATUS.get(st, st)}")
    return x


def rel_h_err(A, x, xstar) -> float:
    A, n, d, ld = _mat(A)
    return lib().orc_rel_h_err(_ptr(A), n, d, ld, _ptr(_f64(x)), _ptr(_f64(xstar)))


def grad_a(A, x, lam) -> np.ndarray:
    """dL/dA = -(A x) lam^T - (A lam) x^T for x = H^{-1} b, lam = H^{-1} dL/dx."""
    A, n, d, ld = _mat(A)
    gA = np.empty((n, d))
    lib().orc_grad_a(_ptr(A), n, d, ld, _ptr(_f64(x)), _ptr(_f64(lam)), _ptr(gA))
    return gA


def solve_grads(A, b, g):
    """(x*, dL/dA, dL/db) of L with dL/dx* = g, by the definitions (direct solves)."""
    xs = solve_direct(A, b)
    lam = solve_direct(A, g)
    return xs, grad_a(A, xs, lam), lam


# ----------------------------------------------------------------------------- closed forms
def theta_gaussian(m: int, d: int):
    """E[C_S^-1] = theta1 I, E[C_S^-2] = theta2 I for Gaussian S, m >= d + 4
    (Section 2, eq. eqngaussianmoments)."""
    if m < d + 4:
        raise ValueError("the Gaussian inverse moments need m >= d + 4")
    t1 = m / (m - d - 1)
    t2 = m * m * (m - 1) / ((m - d) * (m - d - 1) * (m - d - 3))
    return t1, t2


def theta_srht(m: int, d: int, N: int):
    """Haar finite-sample approximations (Section 2, eq. eqnsrhtmoments), used for the SRHT
    via its trace formula (eq. eqnsrhttrace).  The paper's formulas are for an embedding
    with orthonormal rows; this build scales every sketch so that E[S^T S] = I, i.e.
    S = sqrt(N/m) S_orth, which multiplies C_S^-j by (m/N)^j."""
    t1 = (N - d) / (m - d)
    t2 = (N - d) / (m - d) ** 3 * (d * d + m * N - 2 * d * m)
    return (m / N) * t1, (m / N) ** 2 * t2


def refreshed_rate(theta1: float, theta2: float) -> float:
    """Per-step rate 1 - theta1^2/theta2 of refreshed IHS with mu = theta1/theta2
    (Section 4, theorem theoremexacterrorrefreshed)."""
    return 1.0 - theta1 * theta1 / theta2


def refreshed_factor(theta1: float, theta2: float, mu: float) -> float:
    """E[delta_{t+1}] / E[delta_t] = 1 - 2 mu theta1 + mu^2 theta2 (proof of the same theorem)."""
    return 1.0 - 2.0 * mu * theta1 + mu * mu * theta2


def ihs_fixed_params(rho: float):
    """IHS with a fixed embedding: mu = (1-rho)^2/(1+rho), rate 4 rho/(1+rho)^2
    (Section 3, theorem theoremihsfixed)."""
    return (1 - rho) ** 2 / (1 + rho), 4 * rho / (1 + rho) ** 2


def polyak_fixed_params(rho: float):
    """Polyak-IHS with a fixed embedding: mu = (1-rho)^2, beta = rho (same theorem)."""
    return (1 - rho) ** 2, rho


def optimal_sketch_size(n: int, d: int, eps: float, kind: str):
    """Section 6: (m*, cost ratio) of the flop model with constants dropped.
    Gaussian (theorem theoremoptimalcomplexitygaussian): alpha* log alpha* = (n/d^2) log(1/eps),
    m* = d alpha* = d exp(W0(.)), ratio = 1/log(n/d^2).  SRHT (theorem
    theoremoptimalcomplexitysrht): cases (i) / (ii) by sqrt(log 1/eps) vs log(n/d^2)."""
    from scipy.special import lambertw

    L, Lr = math.log(1 / eps), math.log(n / d**2)
    if n <= d * d:
        raise ValueError("the analysis assumes n > d^2")
    if kind == "gauss":
        return d * math.exp(lambertw((n / d**2) * L).real), 1.0 / Lr
    if kind == "srht":
        if math.sqrt(L) < Lr:
            return math.exp(math.sqrt(L)) * d * math.log(d), (math.log(d) + math.sqrt(L)) / (math.log(d) + L)
        return (n / d) * max(math.log(d), L / Lr), (math.log(d) + L / Lr) / (math.log(d) + L)
    raise ValueError(kind)


def pcg_iterations_bound(eps: float, rho: float) -> int:
    """T = ceil(log(4/eps) / log(1/rho)) iterations give delta_T/delta_0 <= eps (Section 6)."""
    return int(math.ceil(math.log(4.0 / eps) / math.log(1.0 / rho)))
