"""lsq_hmatvec_noalloc: the fused pass for callers that cannot allocate device memory.

Such callers (code that keeps all device memory in its own pool, or loops that cannot
absorb an allocation's synchronisation) get an entry point whose scratch is a fixed array
inside the library.  This test calls it through the C ABI twice in a row, on different
shapes, and checks each result against the regular entry point lsq_hmatvec within the
tolerance of the other pass tests.  Collected last so that a failure here stops a -x run
only after every other test has run.
"""
import ctypes

import numpy as np
import pytest
import torch

import workloads as W
from gpu_util import rel_fro, to_dev

pytestmark = pytest.mark.gpu


def _noalloc(L, A, p):
    d = A.shape[1]
    v = torch.empty(d, dtype=torch.float64, device=A.device)
    q = torch.empty(1, dtype=torch.float64, device=A.device)
    M = L.as_matrix(A)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = L.lib().lsq_hmatvec_noalloc(ctypes.byref(M), ctypes.c_void_p(p.data_ptr()), ctypes.c_void_p(v.data_ptr()),
                                     ctypes.c_void_p(q.data_ptr()), stream)
    assert st == 0, L.STATUS.get(st, st)
    return v, q


def test_noalloc_matches_hmatvec_on_two_calls_in_a_row():
    import paper_1911_02675_gb300 as L

    ctx = L.Context(0)
    cases = [(20001, 512, np.float64, 1), (3000, 100, np.float32, 2)]
    for n, d, dtype, seed in cases:
        A = to_dev(W.make_problem(n, d, 1e3, seed=seed)["A"].astype(dtype))
        p = to_dev(np.random.default_rng(seed).standard_normal(d))
        v0, q0 = L.lsq_hmatvec(ctx, A, p)
        v1, q1 = _noalloc(L, A, p)
        torch.cuda.synchronize()
        assert rel_fro(v1.cpu().numpy(), v0.cpu().numpy()) < 1e-13
        assert abs(q1.item() - q0.item()) <= 1e-13 * abs(q0.item())
    ctx.close()


def test_noalloc_rejects_what_does_not_fit():
    import paper_1911_02675_gb300 as L

    A = torch.zeros((64, 1025), dtype=torch.float64, device="cuda")
    p = torch.zeros(1025, dtype=torch.float64, device="cuda")
    v = torch.empty_like(p)
    q = torch.empty(1, dtype=torch.float64, device="cuda")
    M = L.as_matrix(A)
    st = L.lib().lsq_hmatvec_noalloc(ctypes.byref(M), ctypes.c_void_p(p.data_ptr()), ctypes.c_void_p(v.data_ptr()),
                                     ctypes.c_void_p(q.data_ptr()), None)
    assert st == L.LSQ_ERR_ARG


def test_noalloc_allocates_nothing_and_runs_on_another_stream():
    """After a first call (which looks up the array's address and loads the kernel), further
    calls on the default stream and on another stream leave the device's free memory and torch's
    allocator untouched, and give the regular pass's result."""
    import paper_1911_02675_gb300 as L

    A = to_dev(W.make_problem(5000, 96, 1e3, seed=4)["A"])
    p = to_dev(np.random.default_rng(4).standard_normal(96))
    ctx = L.Context(0)
    v0, q0 = L.lsq_hmatvec(ctx, A, p)
    v0, q0 = v0.cpu().numpy(), q0.item()
    side = torch.cuda.Stream()
    d = A.shape[1]
    v = torch.empty(d, dtype=torch.float64, device=A.device)
    q = torch.empty(1, dtype=torch.float64, device=A.device)
    M = L.as_matrix(A)

    def call(stream):
        return L.lib().lsq_hmatvec_noalloc(ctypes.byref(M), ctypes.c_void_p(p.data_ptr()),
                                           ctypes.c_void_p(v.data_ptr()), ctypes.c_void_p(q.data_ptr()),
                                           ctypes.c_void_p(stream.cuda_stream))

    assert call(torch.cuda.current_stream()) == 0  # warm-up
    torch.cuda.synchronize()
    free0, alloc0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
    outs = []
    for s in (torch.cuda.current_stream(), side, torch.cuda.current_stream()):
        assert call(s) == 0
        s.synchronize()
        outs.append((v.cpu().numpy().copy(), q.item()))
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == alloc0
    assert torch.cuda.mem_get_info()[0] == free0
    for vv, qq in outs:
        assert rel_fro(vv, v0) < 1e-13
        assert abs(qq - q0) <= 1e-13 * abs(q0)
    ctx.close()
