"""Parity of lsq_solve_batched (many problems, k right-hand sides each, one persistent launch)
with the FP64 oracle.

Bar: every right-hand side of every problem reaches relative H-norm error <= 1e-10 against
x* (QR + double-double refinement of the oracle); in the FP64 mode, with FP64 sketches, the
iterates follow the oracle's PCG (same sketch instance t = p per problem).  Shapes are uneven
(d not a multiple of 32, n not a multiple of the 32-row tile, problems smaller than one work
unit, k from 1 to 16, d up to the 512 limit)."""
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


SHAPES = [(700, 5, 1), (3001, 37, 3), (5000, 64, 16), (1200, 130, 7), (20000, 96, 2), (4100, 200, 9),
          (999, 33, 4), (6000, 250, 12), (2500, 31, 16), (1500, 300, 5)]


def _dev(probs, dtype):
    return [(to_dev(q["A"].astype(dtype)), to_dev(q["B"])) for q in probs]


@pytest.mark.parametrize("precision,sketch_precision", [("mixed", "f32"), ("f64", "f32"), ("mixed", "bf16")])
def test_batch_reaches_xstar(L, ctx, precision, sketch_precision):
    """Every right-hand side reaches 1e-10 against x*, also with the SJLT over BF16-rounded A
    (the sketch is only the preconditioner's embedding; PCG wins the accuracy back)."""
    probs = W.make_batch(SHAPES, seed=11, scale_max=1e4, dtype=np.float32)
    X, per, info = L.lsq_solve_batched(ctx, _dev(probs, np.float32), tol=1e-10, maxit=300, precision=precision,
                                       sketch_precision=sketch_precision, seed=4)
    assert info["status"] == 0, (info, per)
    for q, Xp, (it, st) in zip(probs, X, per):
        A64 = q["A"].astype(np.float64)
        assert st == 0 and it > 0
        Xh = Xp.cpu().numpy()
        for j in range(q["B"].shape[0]):
            xs = O.solve_direct(A64, q["B"][j])
            assert O.rel_h_err(A64, Xh[j], xs) <= 1e-10, (q["A"].shape, j)


def test_batch_f64_follows_oracle(L, ctx):
    shapes = SHAPES[:6]
    probs = W.make_batch(shapes, seed=12, scale_max=1e3, dtype=np.float64)
    for T in (1, 4):
        X, per, info = L.lsq_solve_batched(ctx, _dev(probs, np.float64), tol=0.0, maxit=T, precision="f64",
                                           sketch_precision="f64", seed=7, s=8)
        ref = O.solve_batched([(q["A"], q["B"]) for q in probs], kind="sjlt", s=8, m_factor=4.0, seed=7, tol=0.0,
                              maxit=T)
        for Xp, (Xr, its, sts), (it, st) in zip(X, ref, per):
            assert it == T and st == L.LSQ_ERR_MAXIT
            assert rel_fro(Xp.cpu().numpy(), Xr) < 1e-10
    # converged iteration counts agree with the oracle's (same sketches, same rule)
    X, per, info = L.lsq_solve_batched(ctx, _dev(probs, np.float64), tol=1e-10, maxit=300, precision="f64",
                                       sketch_precision="f64", seed=7)
    ref = O.solve_batched([(q["A"], q["B"]) for q in probs], kind="sjlt", s=8, m_factor=4.0, seed=7, tol=1e-10)
    for (it, st), (Xr, its, sts) in zip(per, ref):
        assert st == 0 and abs(it - int(its.max())) <= 1


def test_batch_nonzero_x0_and_statuses(L, ctx):
    shapes = [(2000, 40, 3), (3000, 64, 1), (1000, 20, 5)]
    probs = W.make_batch(shapes, seed=13, scale_max=1e2, dtype=np.float32)
    rng = np.random.default_rng(1)
    X0 = [to_dev(rng.standard_normal(q["B"].shape)) for q in probs]
    X, per, info = L.lsq_solve_batched(ctx, _dev(probs, np.float32), X0=X0, tol=1e-10, maxit=300, seed=2)
    assert info["status"] == 0
    for q, Xp in zip(probs, X):
        A64 = q["A"].astype(np.float64)
        for j in range(q["B"].shape[0]):
            assert O.rel_h_err(A64, Xp[j].cpu().numpy(), O.solve_direct(A64, q["B"][j])) <= 1e-10
    # zero right-hand sides converge at once; a tight tolerance with 2 iterations hits maxit
    dev = _dev(probs, np.float32)
    dev[1] = (dev[1][0], torch.zeros_like(dev[1][1]))
    X, per, info = L.lsq_solve_batched(ctx, dev, tol=1e-10, maxit=300, seed=2)
    assert per[1] == (0, 0) and not X[1].abs().sum().item()
    X, per, info = L.lsq_solve_batched(ctx, _dev(probs, np.float32), tol=1e-15, maxit=2, seed=2)
    assert all(st == L.LSQ_ERR_MAXIT and it == 2 for it, st in per)
    assert info["status"] == L.LSQ_ERR_MAXIT


def test_batch_largest_shape(L, ctx):
    shapes = [(6000, 512, 16), (4096, 1, 1), (3000, 512, 2)]
    probs = W.make_batch(shapes, seed=14, scale_max=1e4, dtype=np.float32)
    X, per, info = L.lsq_solve_batched(ctx, _dev(probs, np.float32), tol=1e-10, maxit=400, seed=1)
    assert info["status"] == 0, per
    for q, Xp in zip(probs, X):
        A64 = q["A"].astype(np.float64)
        for j in range(q["B"].shape[0]):
            assert O.rel_h_err(A64, Xp[j].cpu().numpy(), O.solve_direct(A64, q["B"][j])) <= 1e-10


def test_batch_one_column_problem_is_stable(L, ctx):
    """A d = 1 problem is solved by the first step up to rounding; its FP32 recursive residual
    then drops far below FP32's resolution, and the exact residual that replaces it is much
    larger.  Every repeat (the reduction order of the passes varies) must restart the direction
    there and stop within a few iterations instead of stepping along the stale direction."""
    shapes = [(6000, 512, 16), (4096, 1, 1), (3000, 512, 2)]
    probs = W.make_batch(shapes, seed=14, scale_max=1e4, dtype=np.float32)
    dev = _dev(probs, np.float32)
    for _ in range(12):
        X, per, info = L.lsq_solve_batched(ctx, dev, tol=1e-10, maxit=400, seed=1)
        assert info["status"] == 0, per
        assert per[1][0] <= 10, per


def test_batch_autotuner_and_device_loop(L, ctx):
    """The first call of a batch shape runs the autotuner (one timed pass per candidate work-unit
    size and grid); the next call of the same shape reuses its choice; either way, and with the
    autotuner off, every right-hand side reaches the tolerance and the device-driven loop reports
    the iterations it ran."""
    shapes = [(5000, 40, 3), (3000, 17, 1), (12000, 64, 6), (2500, 33, 16)]
    data = W.make_batch(shapes, seed=77)
    probs = [(to_dev(q["A"]), to_dev(q["B"])) for q in data]
    xs = [np.stack([O.solve_direct(q["A"].astype(np.float64), q["B"][j]) for j in range(q["B"].shape[0])])
          for q in data]
    infos = []
    for kw in ({}, {}, {"autotune": 0}):
        X, per, info = L.lsq_solve_batched(ctx, probs, tol=1e-10, maxit=300, **kw)
        assert info["status"] == 0 and all(st == 0 for _, st in per), (per, info)
        for (q, Xp, xsp) in zip(data, X, xs):
            A64 = q["A"].astype(np.float64)
            for j in range(Xp.shape[0]):
                assert O.rel_h_err(A64, Xp[j].cpu().numpy(), xsp[j]) <= 1e-10
        assert info["iters_max"] == max(it for it, _ in per) and info["passes"] >= info["iters_max"]
        infos.append(info)
    assert infos[0]["tuned"] == 1 and infos[1]["tuned"] == 0 and infos[2]["tuned"] == 0
    assert (infos[0]["pass_chunk_elems"], infos[0]["pass_grid"]) == (infos[1]["pass_chunk_elems"], infos[1]["pass_grid"])
    assert infos[0]["pass_chunk_elems"] in (1 << 19, 1 << 20, 1 << 21)
    assert infos[2]["pass_chunk_elems"] == 1 << 20


@pytest.mark.parametrize("x0", [False, True])
def test_batch_mixed_first_iterations_follow_oracle(L, ctx, x0):
    """Mixed precision over FP32 A (the pass whose rows are staged by bulk copies): the first
    iterates follow the FP64 oracle's PCG on the same FP64 sketches to FP32 accuracy, from x0 = 0
    (FP32 passes only) and from a nonzero x0 (the initial residual from the double-FP32 exact
    pass).  Shapes take every column width class (dp 32 .. 512, 8 .. 32 lanes per row), every
    padded count of right-hand sides, rows not a multiple of 4 elements, and problems larger than
    one 32 KB stage and one work unit."""
    shapes = [(3001, 37, 3), (5000, 64, 16), (1201, 130, 7), (4100, 200, 9), (999, 33, 4), (6000, 250, 12),
              (2503, 31, 16), (1500, 300, 5), (70001, 19, 11), (9000, 511, 14)]
    probs = W.make_batch(shapes, seed=21, scale_max=1e3, dtype=np.float32)
    rng = np.random.default_rng(5)
    X0 = [rng.standard_normal(q["B"].shape) for q in probs] if x0 else None
    for T in (1, 3):
        X, per, info = L.lsq_solve_batched(ctx, _dev(probs, np.float32), tol=0.0, maxit=T, precision="mixed",
                                           sketch_precision="f64", seed=3, s=8,
                                           X0=[to_dev(v) for v in X0] if x0 else None)
        ref = O.solve_batched([(q["A"].astype(np.float64), q["B"]) for q in probs], kind="sjlt", s=8, m_factor=4.0,
                              seed=3, tol=0.0, maxit=T, X0=X0)
        for sh, Xp, (Xr, its, sts), (it, st) in zip(shapes, X, ref, per):
            assert it == T and st == L.LSQ_ERR_MAXIT, (sh, it, st)
            err = rel_fro(Xp.cpu().numpy() - (X0[shapes.index(sh)] if x0 else 0.0),
                          Xr - (X0[shapes.index(sh)] if x0 else 0.0))
            assert err < 1e-5, (sh, T, err)


def test_batch_strided_or_unaligned_rows_take_the_tiled_pass(L, ctx):
    """The ring pass needs every problem's rows contiguous and 16-byte aligned; a batch with a
    strided problem (ld = d + 3) and one whose first element sits at an odd float offset runs the
    tiled pass instead.  Either way every right-hand side reaches 1e-10 against x*."""
    shapes = [(3001, 37, 3), (5000, 130, 9), (2500, 31, 16)]
    probs = W.make_batch(shapes, seed=31, scale_max=1e3, dtype=np.float32)
    aligned = _dev(probs, np.float32)
    A1 = torch.from_numpy(probs[1]["A"]).cuda()
    wide = torch.zeros((A1.shape[0], A1.shape[1] + 3), dtype=torch.float32, device=A1.device)
    wide[:, :A1.shape[1]] = A1
    A2 = torch.from_numpy(probs[2]["A"]).cuda()
    flat = torch.zeros(A2.numel() + 1, dtype=torch.float32, device=A2.device)
    flat[1:] = A2.reshape(-1)
    shifted = flat[1:].view(A2.shape)
    assert shifted.data_ptr() % 16 != 0 and wide[:, :A1.shape[1]].stride(0) == A1.shape[1] + 3
    odd = [aligned[0], (wide[:, :A1.shape[1]], aligned[1][1]), (shifted, aligned[2][1])]
    for name, batch in (("aligned", aligned), ("strided and shifted", odd)):
        X, per, info = L.lsq_solve_batched(ctx, batch, tol=1e-10, maxit=300, seed=2)
        assert info["status"] == 0, (name, per)
        for q, Xp in zip(probs, X):
            A64 = q["A"].astype(np.float64)
            for j in range(q["B"].shape[0]):
                assert O.rel_h_err(A64, Xp[j].cpu().numpy(), O.solve_direct(A64, q["B"][j])) <= 1e-10


def test_batch_a_non_finite_problem_stays_isolated(L, ctx):
    """One problem of the batch has a NaN in A: it ends with a non-zero status while every other
    problem converges as without it (no non-finite value crosses problems, in shared memory or
    in the state the passes share), and a later batch on the same context, whose state and
    shared memory the failed solve has dirtied, converges too."""
    shapes = [(3000, 40, 3), (2000, 24, 2), (4096, 100, 12)]
    probs = W.make_batch(shapes, seed=41, scale_max=1e3, dtype=np.float32)
    bad = probs[1]["A"].copy()
    bad[777, 5] = np.nan
    batch = _dev(probs, np.float32)
    batch[1] = (to_dev(bad), batch[1][1])
    X, per, info = L.lsq_solve_batched(ctx, batch, tol=1e-10, maxit=300, seed=5)
    assert per[1][1] != 0 and info["status"] != 0, per
    for i in (0, 2):
        q = probs[i]
        assert per[i][1] == 0, per
        A64 = q["A"].astype(np.float64)
        for j in range(q["B"].shape[0]):
            assert O.rel_h_err(A64, X[i][j].cpu().numpy(), O.solve_direct(A64, q["B"][j])) <= 1e-10
    shapes2 = [(3001, 37, 3), (5000, 130, 9), (2500, 31, 16)]
    probs2 = W.make_batch(shapes2, seed=42, scale_max=1e3, dtype=np.float32)
    X2, per2, info2 = L.lsq_solve_batched(ctx, _dev(probs2, np.float32), tol=1e-10, maxit=300, seed=5)
    assert info2["status"] == 0, per2
    for q, Xp in zip(probs2, X2):
        A64 = q["A"].astype(np.float64)
        for j in range(q["B"].shape[0]):
            assert O.rel_h_err(A64, Xp[j].cpu().numpy(), O.solve_direct(A64, q["B"][j])) <= 1e-10
