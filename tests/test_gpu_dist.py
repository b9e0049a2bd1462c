"""The row partition on one GPU: three slabs of A stand in for three ranks, run one after the
other in this process (nothing waits on another launch), with the library's kernels.

* lsq_sketch with row0 / n_total gives each slab's share of the whole matrix's sketch: the
  shares sum to lsq_sketch of the whole matrix and to the oracle's sketch, bit for bit on
  integer data (SRHT through the staged tensor-copy kernel, the SIMT kernels and the SJLT);
  the Gaussian shares agree to rounding (FP64) or to the BF16 sketch's own error;
* the partitioned PCG (lsq_hmatvec per slab, fixed-order sums, lsq_pcg_tail) reaches 1e-10
  against the oracle's x*, in the iterations of the one-GPU solve.
"""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as W
from gpu_util import int_matrix, rel_fro, to_dev

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


def _slabs(n, world):
    from paper_1911_02675_gb300.dist import slab_rows

    return [slab_rows(n, world, r) for r in range(world)]


@pytest.mark.parametrize("n,d,kind,m,s,prec", [
    (9 * 2048 + 555, 24, "srht", 256, 8, "f64"),    # shared-memory transform, ragged last slab
    (9 * 2048 + 555, 24, "srht", 256, 8, "f32"),    # staged (tensor copy) transform
    (40000, 64, "srht", 1024, 8, "f32"),            # the staged kernel with wider d
    (9 * 2048 + 555, 24, "sjlt", 64, 4, "f64"),
    (9 * 2048 + 555, 24, "sjlt", 64, 4, "f32"),
])
def test_slab_shares_sum_to_the_whole_sketch(L, ctx, n, d, kind, m, s, prec):
    A = int_matrix(n, d, seed=n + m)
    Ad = to_dev(A)
    whole = L.lsq_sketch(ctx, Ad, kind, m, 9, s=s, precision=prec)
    parts = [L.lsq_sketch(ctx, Ad[r0:r1], kind, m, 9, s=s, precision=prec, row0=r0, n_total=n)
             for r0, r1 in _slabs(n, 3)]
    from paper_1911_02675_gb300.dist import all_sum

    summed = all_sum(parts)
    assert torch.equal(summed, whole)
    assert np.array_equal(summed.cpu().numpy(), O.sketch(A, kind, m, 9, s=s))


@pytest.mark.parametrize("prec,tol", [("f64", 1e-13), ("bf16", 1e-2)])
def test_gaussian_slab_shares(L, ctx, prec, tol):
    n, d, m = 3 * 2048 + 100, 40, 256
    A = W.make_problem(n, d, 1e2, seed=2)["A"].astype(np.float32 if prec == "bf16" else np.float64)
    Ad = to_dev(A)
    whole = L.lsq_sketch(ctx, Ad, "gauss", m, 4, precision=prec)
    from paper_1911_02675_gb300.dist import all_sum

    parts = [L.lsq_sketch(ctx, Ad[r0:r1], "gauss", m, 4, precision=prec, row0=r0, n_total=n)
             for r0, r1 in _slabs(n, 3)]
    summed = all_sum(parts).cpu().numpy()
    ref = O.sketch_gauss(A.astype(np.float64), m, 4)
    assert rel_fro(summed, ref) < tol
    assert rel_fro(summed, whole.cpu().numpy()) < (1e-14 if prec == "f64" else 1e-5)


def test_slab_arguments_are_checked(L, ctx):
    A = to_dev(np.ones((4096, 8)))
    with pytest.raises(L.LsqError):  # SRHT slabs start on a 2048-row block
        L.lsq_sketch(ctx, A[:2000], "srht", 64, 0, row0=100, n_total=4096)
    with pytest.raises(L.LsqError):  # the slab must lie inside the whole matrix
        L.lsq_sketch(ctx, A, "gauss", 64, 0, row0=2048, n_total=4096)


@pytest.mark.parametrize("kind", ["srht", "gauss"])
def test_partitioned_pcg_reaches_xstar(L, ctx, kind):
    from paper_1911_02675_gb300.dist import CudaSlabOps, pcg_slabs, sketch_slabs

    n, d, m = 7 * 2048 + 901, 48, 384
    P = W.make_problem(n, d, 1e5, seed=11)
    A, b = P["A"], P["b"]
    Ad, bd = to_dev(A), to_dev(b)
    ops = CudaSlabOps(ctx)
    slabs = [(Ad[r0:r1], r0) for r0, r1 in _slabs(n, 3)]
    SA = sketch_slabs(ops, slabs, kind, m, 0, n)
    Wm = ops.factor(SA)
    x, info = pcg_slabs(ops, slabs, bd, Wm, tol=1e-10, maxit=300, m=m)
    assert info["status"] == "ok", info
    xs = O.solve_direct(A, b)
    assert O.rel_h_err(A, x.cpu().numpy(), xs) <= 1e-10
    # the one-GPU solve with the whole matrix's sketch takes the same number of iterations
    _, W1 = L.lsq_factor(ctx, L.lsq_sketch(ctx, Ad, kind, m, 0))
    x1, info1 = L.lsq_solve(ctx, Ad, bd, "pcg", W1, tol=1e-10, maxit=300, m=m)
    assert abs(info1["iters"] - info["iters"]) <= 1
    # and a nonzero start
    x0 = to_dev(np.random.default_rng(1).standard_normal(d))
    x2, info2 = pcg_slabs(ops, slabs, bd, Wm, tol=1e-10, maxit=300, m=m, x0=x0)
    assert info2["status"] == "ok" and O.rel_h_err(A, x2.cpu().numpy(), xs) <= 1e-10


def test_pcg_tail_reports_breakdown(L, ctx):
    d = 8
    Wm = torch.eye(d, dtype=torch.float64, device="cuda")
    b = torch.ones(d, dtype=torch.float64, device="cuda")
    state = torch.zeros(4 * d + 8, dtype=torch.float64, device="cuda")
    vq = torch.zeros(d + 1, dtype=torch.float64, device="cuda")
    assert L.lsq_pcg_tail(ctx, Wm, b, vq, 0, 1e-10, 0.25, state) == 0
    vq[d] = -1.0  # p^T H p <= 0
    with pytest.raises(L.LsqError) as e:
        L.lsq_pcg_tail(ctx, Wm, b, vq, 1, 1e-10, 0.25, state)
    assert e.value.status == L.LSQ_ERR_BREAKDOWN
