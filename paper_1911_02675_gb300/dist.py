"""Row-partitioned solves: A split by rows across ranks (one GPU each), the data plane of the
method when A does not fit one GPU or is produced in pieces.

Every step of the method is a sum over the rows of A (Section 2: S A = sum_i S[:, i] a_i^T;
Section 1: H p = sum_i a_i (a_i^T p)), so with A in row slabs A_k:

* sketch: each rank forms its slab's share S[:, slab] A_k with the whole matrix's S
  (lsq_sketch with row0 / n_total: the Philox counters take global row indices, and the SRHT's
  signs, sampled rows and zero padding are the whole matrix's); the m x d shares are summed
  across ranks (one exchange per sketch);
* factor: replicated (every rank factors the same summed sketch, d x d);
* each PCG iteration: each rank runs the fused pass over its slab (lsq_hmatvec), the d + 1 sums
  v = A^T A p, q = p^T H p are added across ranks (one exchange of d + 1 doubles), and every
  rank runs the same tail on them (lsq_pcg_tail), so all ranks keep the same iterate.

Sums across ranks are taken in a fixed order (this rank's slabs in order, then ranks in order,
after an all-gather), so every rank holds the same bits and a run repeats bit for bit.

The local computations are an `ops` object (CudaSlabOps: this library's kernels on the rank's
GPU); the collective is torch.distributed when it is initialised (NCCL on GPUs, gloo on CPU).
A process may hold several slabs (they are summed first), which also lets one GPU stand in for
several ranks run one after the other.
"""
from __future__ import annotations

import torch

SRHT_BLOCK = 2048  # SRHT slabs are whole blocks of the two-level Hadamard transform


def slab_rows(n_total: int, world: int, rank: int, align: int = SRHT_BLOCK) -> tuple[int, int]:
    """Rows [row0, row1) of rank `rank` among `world` ranks: contiguous, whole `align`-row blocks
    (the last slab ends at n_total), as even as whole blocks allow; empty when there are more
    ranks than blocks."""
    if world < 1 or not 0 <= rank < world or n_total < 1 or align < 1:
        raise ValueError("bad partition arguments")
    blocks = -(-n_total // align)
    b0 = blocks * rank // world
    b1 = blocks * (rank + 1) // world
    return min(n_total, b0 * align), min(n_total, b1 * align)


def _world(group=None):
    import torch.distributed as dist

    if dist.is_available() and dist.is_initialized():
        return dist.get_world_size(group), dist.get_rank(group)
    return 1, 0


def all_sum(parts, group=None) -> torch.Tensor:
    """The sum of every slab's partial result over every rank, in a fixed order: this rank's
    parts in order, then the ranks' sums in rank order (all-gather, then added in order on every
    rank), so that all ranks get the same bits."""
    if not parts:
        raise ValueError("no partial results")
    local = parts[0].clone()
    for t in parts[1:]:
        local += t
    world, _ = _world(group)
    if world == 1:
        return local
    import torch.distributed as dist

    gathered = [torch.empty_like(local) for _ in range(world)]
    dist.all_gather(gathered, local, group=group)
    out = gathered[0].clone()
    for t in gathered[1:]:
        out += t
    return out


class CudaSlabOps:
    """The local computations of a slab on this rank's GPU, through the library's C ABI."""

    def __init__(self, ctx):
        self.ctx = ctx

    def sketch(self, A_slab, kind, m, seed, row0, n_total, **kw):
        from . import lsq_sketch

        return lsq_sketch(self.ctx, A_slab, kind, m, seed, row0=row0, n_total=n_total, **kw)

    def factor(self, SA, precision="f64"):
        from . import lsq_factor

        return lsq_factor(self.ctx, SA, precision=precision)[1]

    def hmatvec(self, A_slab, p):
        from . import lsq_hmatvec

        v, q = lsq_hmatvec(self.ctx, A_slab, p)
        return torch.cat([v, q])

    def zeros(self, k, like):
        return torch.zeros(k, dtype=torch.float64, device=like.device)

    def tail(self, W, b, vq, phase, tol, rho, state):
        from . import lsq_pcg_tail

        return lsq_pcg_tail(self.ctx, W, b, vq, phase, tol, rho, state)


def sketch_slabs(ops, slabs, kind, m, seed, n_total, group=None, **kw):
    """The sketch of the whole matrix from this rank's slabs [(A_k, row0_k), ...]."""
    return all_sum([ops.sketch(A, kind, m, seed, row0, n_total, **kw) for A, row0 in slabs], group)


def pcg_slabs(ops, slabs, b, W, tol=1e-10, maxit=1000, rho=None, m=None, x0=None, group=None):
    """PCG (Section 1, eq. (PCG)) over the row slabs [(A_k, row0_k), ...] of every rank with the
    preconditioner W = R^{-1} of the summed sketch.  rho defaults to d / m.  Returns (x, info) on
    every rank; info: iters, status ("ok", "maxit"), flag."""
    d = b.numel()
    if rho is None:
        if m is None:
            raise ValueError("give rho or the sketch size m")
        rho = d / m
    state = ops.zeros(4 * d + 8, b)
    if x0 is not None and bool((x0 != 0).any()):
        state[:d] = x0
        vq = all_sum([ops.hmatvec(A, state[:d]) for A, _ in slabs], group)
    else:
        vq = ops.zeros(d + 1, b)
    flag = ops.tail(W, b, vq, 0, tol, rho, state)
    it = 0
    while flag == 0 and it < maxit:
        vq = all_sum([ops.hmatvec(A, state[3 * d:4 * d]) for A, _ in slabs], group)
        flag = ops.tail(W, b, vq, 1, tol, rho, state)
        it += 1
    status = "ok" if flag == 1 else "maxit"
    return state[:d].clone(), {"iters": it, "status": status, "flag": flag}
