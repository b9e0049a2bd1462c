"""Pins for the oracle's random embeddings (Section 2 of the paper).

Each check compares the oracle with something that does not come from it: published
known-answer vectors, a library Hadamard matrix, an explicit matrix product, exact
identities of the embedding, or the inverse moments of Section 2 by Monte Carlo.
"""
import os

import numpy as np
import pytest
import scipy.linalg
import scipy.stats

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------- Philox
def test_philox_known_answer_vectors():
    rows = []
    with open(os.path.join(GOLDEN, "philox_kat.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([int(w, 16) for w in line.split()])
    for r in rows:
        out = O.philox4x32_10(r[:4], r[4:6])[0]
        assert [int(v) for v in out] == r[6:10]


def test_philox_words_uniform():
    ctr = np.zeros((50000, 4), dtype=np.uint32)
    ctr[:, 0] = np.arange(50000)
    ctr[:, 3] = 7
    w = O.philox4x32_10(ctr, [12345, 678]).ravel()
    counts = np.bincount((w >> 28).astype(np.int64), minlength=16)
    assert scipy.stats.chisquare(counts).pvalue > 1e-4
    # each bit is balanced
    bits = ((w[:, None] >> np.arange(32, dtype=np.uint32)) & 1).mean(axis=0)
    assert np.all(np.abs(bits - 0.5) < 0.01)


# ---------------------------------------------------------------------------- Gaussian
def test_gaussian_entries_standard_normal():
    z = np.array([O.gauss_z(3, 0, j, i) for j in range(40) for i in range(500)])
    assert abs(z.mean()) < 4 / np.sqrt(z.size)
    assert abs(z.var() - 1) < 0.05
    assert scipy.stats.kstest(z, "norm").pvalue > 1e-4
    # cosine and sine branches of one Box-Muller pair are uncorrelated
    pairs = np.array([[O.gauss_z(5, 0, 2 * q, i), O.gauss_z(5, 0, 2 * q + 1, i)] for q in range(20) for i in range(500)])
    assert abs(np.corrcoef(pairs.T)[0, 1]) < 4 / np.sqrt(len(pairs))


def test_gaussian_instances_differ_and_repeat():
    a = O.gauss_matrix(8, 16, seed=1, t=0)
    assert np.array_equal(a, O.gauss_matrix(8, 16, seed=1, t=0))
    assert not np.allclose(a, O.gauss_matrix(8, 16, seed=1, t=1))
    assert not np.allclose(a, O.gauss_matrix(8, 16, seed=2, t=0))


def test_gaussian_sketch_is_explicit_product():
    rng = np.random.default_rng(0)
    A = rng.standard_normal((37, 5))
    S = O.gauss_matrix(9, 37, seed=4, t=2)
    np.testing.assert_allclose(O.sketch_gauss(A, 9, seed=4, t=2), S @ A, rtol=1e-13, atol=1e-13)
    # entries have variance 1/m
    assert abs((O.gauss_matrix(64, 400, 11) ** 2).mean() * 64 - 1) < 0.03


def test_gaussian_sketch_rows_are_rows_of_the_explicit_product():
    rng = np.random.default_rng(3)
    A = rng.standard_normal((53, 6))
    S = O.gauss_matrix(12, 53, seed=5, t=1)
    rows = np.array([11, 0, 7, 7])
    np.testing.assert_allclose(O.sketch_gauss_rows(A, 12, seed=5, rows=rows, t=1), (S @ A)[rows], rtol=1e-13,
                               atol=1e-13)
    np.testing.assert_array_equal(O.sketch_gauss_rows(A, 12, 5, rows, t=1), O.sketch_gauss(A, 12, 5, t=1)[rows])


def test_gaussian_inverse_moments_monte_carlo():
    """E[C_S^-1] = theta1 I and E[C_S^-2] = theta2 I (Section 2, Gaussian moments)."""
    n, d, m, trials = 40, 4, 16, 3000
    U, _ = np.linalg.qr(np.random.default_rng(1).standard_normal((n, d)))
    t1, t2 = O.theta_gaussian(m, d)
    M1 = np.zeros((trials, d, d))
    M2 = np.zeros((trials, d, d))
    for k in range(trials):
        SU = O.sketch_gauss(U, m, seed=1000 + k)
        Ci = np.linalg.inv(SU.T @ SU)
        M1[k] = Ci
        M2[k] = Ci @ Ci
    for M, theta in ((M1, t1), (M2, t2)):
        mean = M.mean(axis=0)
        se = M.std(axis=0) / np.sqrt(trials)
        np.testing.assert_array_less(np.abs(mean - theta * np.eye(d)), 5 * se + 1e-12)
    # a sketch scaled 1/m instead of 1/sqrt(m) would be off by a factor of m
    assert abs(np.trace(M1.mean(axis=0)) / d / t1 - 1) < 0.05


# ---------------------------------------------------------------------------- SRHT
def test_fwht_matches_library_hadamard():
    rng = np.random.default_rng(2)
    for N in (1, 2, 8, 64):
        X = rng.standard_normal((N, 3))
        np.testing.assert_allclose(O.fwht_rows(X), scipy.linalg.hadamard(N) @ X, rtol=1e-13, atol=1e-12)


@pytest.mark.parametrize("n", [64, 50, 33])
def test_srht_is_explicit_RHE(n):
    rng = np.random.default_rng(n)
    d, m, seed, t = 3, 12, 9, 4
    A = rng.standard_normal((n, d))
    N = O.next_pow2(n)
    sg = O.srht_signs(N, seed, t)
    rows = O.srht_rows(N, m, seed, t)
    S = scipy.linalg.hadamard(N)[rows] * sg[None, :] / np.sqrt(m)
    A_pad = np.vstack([A, np.zeros((N - n, d))])
    np.testing.assert_allclose(O.sketch_srht(A, m, seed, t), S @ A_pad, rtol=1e-13, atol=1e-13)
    # S S^T = (N/m) I_m exactly: distinct rows of a Hadamard matrix are orthogonal
    np.testing.assert_allclose(S @ S.T, (N / m) * np.eye(m), atol=1e-12)


def test_srht_rows_distinct_sorted_uniform():
    N, m = 256, 16
    counts = np.zeros(N)
    for seed in range(2000):
        r = O.srht_rows(N, m, seed)
        assert np.all(np.diff(r) > 0) and r[0] >= 0 and r[-1] < N
        counts[r] += 1
    assert scipy.stats.chisquare(counts).pvalue > 1e-4
    s = O.srht_signs(1 << 14, 3)
    assert set(np.unique(s)) == {-1, 1} and abs(s.mean()) < 4 / np.sqrt(s.size)


def test_srht_unbiased_gram():
    """E[S^T S] = I_n for the scaling used here; the diagonal is exactly 1 for every draw."""
    n, m = 16, 4
    acc = np.zeros((n, n))
    for seed in range(3000):
        S = O.sketch_srht(np.eye(n), m, seed)  # = S itself (m x n)
        G = S.T @ S
        np.testing.assert_allclose(np.diag(G), 1.0, atol=1e-14)
        acc += G
    acc /= 3000
    assert np.max(np.abs(acc - np.eye(n))) < 0.06


# ---------------------------------------------------------------------------- SJLT
def test_sjlt_positions_and_signs():
    n, m, s = 3000, 50, 8
    h, sg = O.sjlt_hash(n, m, s, seed=5)
    assert h.shape == (n, s)
    assert np.all(np.diff(h, axis=1) > 0), "distinct and sorted in every column of S"
    assert h.min() >= 0 and h.max() < m
    assert set(np.unique(sg)) == {-1, 1}
    counts = np.bincount(h.ravel(), minlength=m)
    assert scipy.stats.chisquare(counts).pvalue > 1e-4
    assert abs(sg.mean()) < 4 / np.sqrt(sg.size)


@pytest.mark.parametrize("m", [3, 7])
def test_sjlt_bounded_integers_unbiased(m):
    h, _ = O.sjlt_hash(60000, m, 1, seed=1)
    counts = np.bincount(h.ravel(), minlength=m)
    assert scipy.stats.chisquare(counts).pvalue > 1e-4


def test_sjlt_is_explicit_product():
    rng = np.random.default_rng(3)
    n, d, m, s = 41, 4, 10, 3
    A = rng.standard_normal((n, d))
    h, sg = O.sjlt_hash(n, m, s, seed=2, t=1)
    S = np.zeros((m, n))
    for i in range(n):
        S[h[i], i] = sg[i] / np.sqrt(s)
    np.testing.assert_allclose(O.sketch_sjlt(A, m, s, seed=2, t=1), S @ A, rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(np.diag(S.T @ S), 1.0, atol=1e-14)


def test_sjlt_rejects_bad_sizes():
    with pytest.raises(ValueError):
        O.sjlt_hash(10, 4, 5, seed=0)
