"""The row partition across ranks (paper_1911_02675_gb300.dist) on CPU: gloo, world size 2.

Each rank holds a row slab of A (whole 2048-row blocks); the local computations are done by
the oracle (its sketch of the slab placed in a zero matrix of the whole height is, by
definition, the slab's share S[:, slab] A), and the product's driver does the rest: the slab
assignment, the fixed-order sums across ranks, and the PCG loop that exchanges d + 1 numbers
per iteration.  Checked: the summed sketch equals the one-rank oracle sketch bit for bit on
integer data (exact sums, power-of-two scales), both ranks end with the same iterate bit for
bit, and it reaches 1e-10 in relative H-norm error against the oracle's x*.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle as O
import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


class OracleSlabOps:
    """Local computations of a slab on the CPU by the oracle (test infrastructure)."""

    def sketch(self, A_slab, kind, m, seed, row0, n_total, s=8):
        A = np.zeros((n_total, A_slab.shape[1]))
        A[row0:row0 + A_slab.shape[0]] = A_slab.numpy()
        return torch.from_numpy(O.sketch(A, kind, m, seed, s=s))

    def factor(self, SA):
        return torch.from_numpy(O.factor(SA.numpy()))  # R; the tail applies H_S^-1 with it

    def hmatvec(self, A_slab, p):
        v, q = O.hmatvec(A_slab.numpy(), p.numpy())
        return torch.from_numpy(np.concatenate([v, [q]]))

    def zeros(self, k, like):
        return torch.zeros(k, dtype=torch.float64)

    def tail(self, R, b, vq, phase, tol, rho, state):
        """One PCG tail (Section 1, eq. (PCG)) in numpy around the oracle's H_S^-1 solve."""
        d = b.numel()
        st = state.numpy()
        x, r, z, p, sc = st[:d], st[d:2 * d], st[2 * d:3 * d], st[3 * d:4 * d], st[4 * d:]
        bb, v = b.numpy(), vq.numpy()
        if phase == 0:
            sc[:] = 0
            r[:] = bb - v[:d]
        else:
            if sc[4] != 0:
                return int(sc[4])
            alpha = sc[0] / v[d]
            x += alpha * p
            r -= alpha * v[:d]
        z[:] = O.precond_solve(R.numpy(), r)
        rz = float(r @ z)
        beta = 0.0 if phase == 0 else rz / sc[0]
        p[:] = z + beta * p if phase else z
        sc[0], sc[1] = rz, float(bb @ x)
        if rz == 0 or (1 + np.sqrt(rho)) ** 2 * rz <= tol * tol * sc[1]:
            sc[4] = 1
        return int(sc[4])


def test_slab_rows_cover_whole_blocks():
    from paper_1911_02675_gb300.dist import slab_rows

    for n, world in [(5 * 2048 + 777, 2), (2048, 3), (100, 1), (9 * 2048, 4), (40000, 7)]:
        slabs = [slab_rows(n, world, r) for r in range(world)]
        assert slabs[0][0] == 0 and slabs[-1][1] == n
        for (a0, a1), (b0, b1) in zip(slabs, slabs[1:]):
            assert a1 == b0
        for r0, r1 in slabs:
            assert r0 % 2048 == 0 and r0 <= r1
        sizes = [r1 - r0 for r0, r1 in slabs if r1 < n]
        if sizes:
            assert max(sizes) - min(sizes) <= 2048
    with pytest.raises(ValueError):
        slab_rows(10, 0, 0)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import sys

    sys.path.insert(0, ROOT)
    from paper_1911_02675_gb300.dist import pcg_slabs, sketch_slabs, slab_rows

    ops = OracleSlabOps()
    res = {}
    # sketches of integer data: exact sums, and 1/sqrt(m) = 1/16, 1/sqrt(s) = 1/2 are exact scales
    n, d = 5 * 2048 + 777, 12
    A = np.random.default_rng(3).integers(-8, 9, size=(n, d)).astype(np.float64)
    r0, r1 = slab_rows(n, world, rank)
    slab = [(torch.from_numpy(A[r0:r1].copy()), r0)]
    for kind, m, s in [("srht", 256, 8), ("sjlt", 64, 4), ("gauss", 32, 8)]:
        SA = sketch_slabs(ops, slab, kind, m, 5, n, s=s)
        res[kind] = SA.numpy()
    # the partitioned PCG on a conditioned problem
    P = W.make_problem(n, d, 1e4, seed=7)
    A2, b2 = P["A"], P["b"]
    slab2 = [(torch.from_numpy(A2[r0:r1].copy()), r0)]
    SA2 = sketch_slabs(ops, slab2, "srht", 128, 0, n)
    R = ops.factor(SA2)
    x, info = pcg_slabs(ops, slab2, torch.from_numpy(b2), R, tol=1e-10, maxit=200, m=128)
    res["x"], res["info"], res["rows"] = x.numpy(), info, (r0, r1)
    out[rank] = res
    dist.destroy_process_group()


def test_partitioned_sketch_and_pcg_two_ranks_gloo():
    world = 2
    out = mp.Manager().dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    n, d = 5 * 2048 + 777, 12
    A = np.random.default_rng(3).integers(-8, 9, size=(n, d)).astype(np.float64)
    assert out[0]["rows"] == (0, 3 * 2048) and out[1]["rows"] == (3 * 2048, n)
    for kind, m, s in [("srht", 256, 8), ("sjlt", 64, 4)]:
        ref = O.sketch(A, kind, m, 5, s=s)
        for r in range(world):
            assert np.array_equal(out[r][kind], ref), kind
    ref = O.sketch(A, "gauss", 32, 5)
    for r in range(world):
        np.testing.assert_allclose(out[r]["gauss"], ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())
    assert np.array_equal(out[0]["gauss"], out[1]["gauss"])
    # same iterate on both ranks, converged against the oracle's x*
    assert np.array_equal(out[0]["x"], out[1]["x"])
    P = W.make_problem(n, d, 1e4, seed=7)
    xs = O.solve_direct(P["A"], P["b"])
    assert out[0]["info"]["status"] == "ok"
    assert O.rel_h_err(P["A"], out[0]["x"], xs) <= 1e-10
    # the iteration count of the one-rank oracle PCG with the same sketch
    _, it, _, _ = O.pcg(P["A"], P["b"], O.factor(O.sketch(P["A"], "srht", 128, 0)), tol=1e-10, maxit=200,
                        rho_hat=d / 128)
    assert abs(out[0]["info"]["iters"] - it) <= 1
