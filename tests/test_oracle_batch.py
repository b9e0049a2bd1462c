"""Pins for the oracle's batched solve and the uneven-batch input recipe.

The batched oracle is the pinned single-problem PCG applied per problem and right-hand side;
what is pinned here is the composition: every right-hand side of every problem reaches x*
(the exact solution of H x = b_j, by QR and double-double refinement) to the requested
relative H-norm error, each problem uses its own sketch instance, and the shapes follow
their log-uniform / uniform laws."""
import math

import numpy as np

import oracle as O
import workloads as W


def test_batched_oracle_reaches_xstar():
    shapes = [(300, 4, 1), (1000, 17, 3), (2048, 33, 5), (777, 40, 2), (4096, 8, 4)]
    probs = W.make_batch(shapes, seed=5, scale_max=1e3, dtype=np.float32)
    res = O.solve_batched([(q["A"], q["B"]) for q in probs], kind="sjlt", s=4, m_factor=4.0, seed=3, tol=1e-11)
    for q, (X, its, sts) in zip(probs, res):
        A64 = q["A"].astype(np.float64)
        assert X.shape == q["B"].shape
        for j in range(q["B"].shape[0]):
            xs = O.solve_direct(A64, q["B"][j])
            assert sts[j] == 0
            assert O.rel_h_err(A64, X[j], xs) <= 1e-10


def test_batched_oracle_uses_instance_p():
    shapes = [(500, 6, 1), (500, 6, 1)]
    probs = W.make_batch(shapes, seed=6, scale_max=1e2, dtype=np.float64)
    # the same matrix in both slots: the iterates differ only through the sketch instance
    pb = [(probs[0]["A"], probs[0]["B"]), (probs[0]["A"], probs[0]["B"])]
    res = O.solve_batched(pb, kind="gauss", m_factor=3.0, seed=9, tol=0.0, maxit=2)
    assert not np.allclose(res[0][0], res[1][0])
    m = 18
    R1 = O.factor(O.sketch(probs[0]["A"], "gauss", m, 9, t=1))
    x1, *_ = O.pcg(probs[0]["A"], probs[0]["B"][0], R1, tol=0.0, maxit=2, rho_hat=6 / m)
    assert np.allclose(res[1][0][0], x1, rtol=0, atol=1e-12 * np.abs(x1).max())


def test_batch_shapes_laws():
    sh = W.batch_shapes(4000, seed=2)
    n = np.array([a for a, _, _ in sh]); d = np.array([b for _, b, _ in sh]); k = np.array([c for _, _, c in sh])
    assert n.min() >= 1 << 12 and n.max() <= 1 << 18
    assert d.min() >= 32 and d.max() <= 512
    assert k.min() == 1 and k.max() == 16
    # log-uniform: log n uniform on [12 ln 2, 18 ln 2] -> mean at the midpoint, within 3 sigma
    u = (np.log(n) - 12 * math.log(2)) / (6 * math.log(2))
    assert abs(u.mean() - 0.5) < 3 * math.sqrt(1 / 12 / len(u)) + 1e-3
    v = (np.log(d) - math.log(32)) / math.log(16)
    assert abs(v.mean() - 0.5) < 3 * math.sqrt(1 / 12 / len(v)) + 2e-3
    assert abs(k.mean() - 8.5) < 3 * math.sqrt((16 ** 2 - 1) / 12 / len(k))
