"""GB300 (sm_103a) randomized-preconditioned least squares, after Lacotte & Pilanci,
"Faster Least Squares Optimization" (arXiv 1911.02675).

This module is a thin ctypes binding over the C ABI of ``include/lsq.h`` (library
``_build/liblsq.so``, built by ``build.py``).  It only marshals arguments: torch
tensors give device pointers and the current CUDA stream; every step of the method
runs in the library's kernels.  If the library is missing the import fails; there
is no CPU path.

Entry points (same names as the C ABI):
    lsq_sketch(ctx, A, kind, m, seed, t=0, s=8, precision="f64") -> SA      (Section 2)
    lsq_factor(ctx, SA, precision) -> (R, W)                                (Section 1, PCG; Section 6)
    lsq_solve(ctx, A, b, method, W, x0=None, tol=1e-10, maxit=..., **opts)  (Section 1; Sections 3-4)
    lsq_hmatvec(ctx, A, p) -> (v, q)                                        (one fused pass over A)
    lsq_solve_batched(ctx, [(A_p, B_p), ...], tol, maxit, **opts)            (many problems, k_p RHS each)
"""
from __future__ import annotations

import ctypes
import math
import os

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "liblsq.so")

STATUS = {0: "LSQ_OK", 1: "LSQ_ERR_ARG", 2: "LSQ_ERR_RANK", 3: "LSQ_ERR_BREAKDOWN", 4: "LSQ_ERR_MAXIT",
          5: "LSQ_ERR_TIMEOUT", 6: "LSQ_ERR_CUDA", 7: "LSQ_ERR_ALLOC"}
LSQ_OK, LSQ_ERR_ARG, LSQ_ERR_RANK, LSQ_ERR_BREAKDOWN, LSQ_ERR_MAXIT, LSQ_ERR_TIMEOUT, LSQ_ERR_CUDA, LSQ_ERR_ALLOC = range(8)
SKETCH = {"gauss": 0, "srht": 1, "sjlt": 2}
METHOD = {"pcg": 0, "ihs": 1, "polyak": 2, "fcg": 3}
PRECISION = {"f64": 0, "mixed": 1}
SKETCH_PRECISION = {"f64": 0, "f32": 1, "bf16": 2}
DTYPE = {torch.float64: 0, torch.float32: 1}

# every symbol the header declares
EXPORTS = ("lsq_create", "lsq_destroy", "lsq_set_stream", "lsq_set_deferred_checks", "lsq_sync", "lsq_sketch", "lsq_upload_sketch", "lsq_factor", "lsq_factor_ex", "lsq_solve",
           "lsq_solve_opts_default", "lsq_hmatvec", "lsq_status_str", "lsq_version", "lsq_launch_count",
           "lsq_hmatvec_noalloc", "lsq_grad_a", "lsq_advise_sketch_size", "lsq_batch_opts_default",
           "lsq_solve_batched", "lsq_selftest_wait", "lsq_pcg_tail", "lsq_factor_qr")


class LsqError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {STATUS.get(status, status)} ({_status_str(status)})")


class LsqMatrix(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("n", ctypes.c_int64), ("d", ctypes.c_int64), ("ld", ctypes.c_int64),
                ("dtype", ctypes.c_int32)]


class LsqSketchOpts(ctypes.Structure):
    _fields_ = [("t", ctypes.c_uint32), ("s", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("a32", ctypes.c_void_p), ("ld32", ctypes.c_int64), ("row0", ctypes.c_int64), ("n_total", ctypes.c_int64)]


class LsqSolveOpts(ctypes.Structure):
    _fields_ = [("rho", ctypes.c_double), ("mu", ctypes.c_double), ("beta", ctypes.c_double),
                ("refresh", ctypes.c_int32), ("sketch_type", ctypes.c_int32), ("m", ctypes.c_int64),
                ("seed", ctypes.c_uint64), ("s", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("refresh_every", ctypes.c_int32), ("grid_blocks", ctypes.c_int32), ("x0_zero", ctypes.c_int32),
                ("fcg_k", ctypes.c_int32), ("a32", ctypes.c_void_p), ("ld32", ctypes.c_int64),
                ("a32_copy", ctypes.c_int32), ("w_dense", ctypes.c_int32)]


class LsqProblem(ctypes.Structure):
    _fields_ = [("A", LsqMatrix), ("B", ctypes.c_void_p), ("X", ctypes.c_void_p), ("k", ctypes.c_int32),
                ("iters", ctypes.c_int32), ("status", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class LsqBatchOpts(ctypes.Structure):
    _fields_ = [("sketch_type", ctypes.c_int32), ("s", ctypes.c_int32), ("m_factor", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("sketch_precision", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("rho", ctypes.c_double), ("x0_zero", ctypes.c_int32), ("refresh_every", ctypes.c_int32),
                ("chunk_rows", ctypes.c_int32), ("grid_blocks", ctypes.c_int32), ("profile_phases", ctypes.c_int32),
                ("autotune", ctypes.c_int32)]


class LsqBatchInfo(ctypes.Structure):
    _fields_ = [("iters_max", ctypes.c_int32), ("status", ctypes.c_int32), ("passes", ctypes.c_int32),
                ("exact_passes", ctypes.c_int32), ("ms_total", ctypes.c_double), ("ms_sketch", ctypes.c_double),
                ("ms_factor", ctypes.c_double), ("ms_solve", ctypes.c_double), ("ms_phase", ctypes.c_double * 8),
                ("pass_chunk_elems", ctypes.c_int64), ("pass_grid", ctypes.c_int32), ("tuned", ctypes.c_int32)]

    def as_dict(self):
        out = {k: getattr(self, k) for k, _ in self._fields_}
        out["ms_phase"] = dict(zip(("pass", "update", "wt_r", "w_t", "direction"), list(self.ms_phase)[:5]))
        return out


class LsqAdvice(ctypes.Structure):
    _fields_ = [("m_star", ctypes.c_double), ("cost_ratio", ctypes.c_double), ("predicted_iters", ctypes.c_double),
                ("regime", ctypes.c_int32)]


class LsqSolveInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("status", ctypes.c_int32), ("passes", ctypes.c_int32),
                ("exact_passes", ctypes.c_int32), ("est_err", ctypes.c_double), ("ms_total", ctypes.c_double),
                ("ms_sketch", ctypes.c_double), ("a32_copy", ctypes.c_int32), ("reserved", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: run `python -m paper_1911_02675_gb300.build` (no CPU fallback)")
    L = ctypes.CDLL(LIB_PATH)
    P, i64, i32, u64, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64, ctypes.c_double
    L.lsq_create.argtypes = [ctypes.POINTER(P), P]
    L.lsq_destroy.argtypes = [P]
    L.lsq_set_stream.argtypes = [P, P]
    L.lsq_set_deferred_checks.argtypes = [P, i32]
    L.lsq_sync.argtypes = [P]
    L.lsq_sketch.argtypes = [P, ctypes.POINTER(LsqMatrix), i32, i64, u64, ctypes.POINTER(LsqSketchOpts), P]
    L.lsq_upload_sketch.argtypes = [P, P, i64, ctypes.POINTER(LsqMatrix), i32, i64, u64, ctypes.POINTER(LsqSketchOpts), P]
    L.lsq_factor.argtypes = [P, P, i64, i64, P, P]
    L.lsq_factor_ex.argtypes = [P, P, i64, i64, P, P, i32]
    L.lsq_solve.argtypes = [P, ctypes.POINTER(LsqMatrix), P, i32, P, P, dbl, i32, ctypes.POINTER(LsqSolveOpts),
                            ctypes.POINTER(LsqSolveInfo)]
    L.lsq_solve_opts_default.argtypes = [ctypes.POINTER(LsqSolveOpts)]
    L.lsq_solve_opts_default.restype = None
    L.lsq_hmatvec.argtypes = [P, ctypes.POINTER(LsqMatrix), P, P, P]
    L.lsq_hmatvec_noalloc.argtypes = [ctypes.POINTER(LsqMatrix), P, P, P, P]
    L.lsq_hmatvec_noalloc.restype = ctypes.c_int
    L.lsq_grad_a.argtypes = [P, ctypes.POINTER(LsqMatrix), P, P, P, i64]
    L.lsq_grad_a.restype = ctypes.c_int
    L.lsq_advise_sketch_size.argtypes = [i64, i64, dbl, i32, ctypes.POINTER(LsqAdvice)]
    L.lsq_advise_sketch_size.restype = ctypes.c_int
    L.lsq_batch_opts_default.argtypes = [ctypes.POINTER(LsqBatchOpts)]
    L.lsq_batch_opts_default.restype = None
    L.lsq_solve_batched.argtypes = [P, i32, ctypes.POINTER(LsqProblem), dbl, i32, ctypes.POINTER(LsqBatchOpts),
                                    ctypes.POINTER(LsqBatchInfo)]
    L.lsq_solve_batched.restype = ctypes.c_int
    L.lsq_factor_qr.argtypes = [P, P, i64, i64, dbl, P, P, P, ctypes.POINTER(i64)]
    L.lsq_factor_qr.restype = ctypes.c_int
    L.lsq_pcg_tail.argtypes = [P, i64, P, P, P, i32, dbl, dbl, P, ctypes.POINTER(i32)]
    L.lsq_pcg_tail.restype = ctypes.c_int
    L.lsq_selftest_wait.argtypes = [P, i32, i32, i64]
    L.lsq_selftest_wait.restype = ctypes.c_int
    L.lsq_status_str.argtypes = [i32]
    L.lsq_status_str.restype = ctypes.c_char_p
    L.lsq_version.restype = ctypes.c_char_p
    L.lsq_launch_count.restype = ctypes.c_uint64
    for name in ("lsq_create", "lsq_destroy", "lsq_set_stream", "lsq_sketch", "lsq_factor", "lsq_factor_ex", "lsq_solve",
                 "lsq_hmatvec"):
        getattr(L, name).restype = ctypes.c_int
    return L


_L = _load()


def lib():
    return _L


def _status_str(s: int) -> str:
    return _L.lsq_status_str(int(s)).decode()


def lsq_launch_count() -> int:
    return int(_L.lsq_launch_count())


def lsq_version() -> str:
    return _L.lsq_version().decode()


def _ptr(t: torch.Tensor | None):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream_handle(device) -> ctypes.c_void_p:
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _check_vec(v: torch.Tensor, d: int, name: str):
    if not v.is_cuda or v.dtype != torch.float64 or v.numel() != d or not v.is_contiguous():
        raise ValueError(f"{name} must be a contiguous CUDA float64 tensor of {d} entries")


def as_matrix(A: torch.Tensor) -> LsqMatrix:
    if A.dim() != 2 or not A.is_cuda or A.dtype not in DTYPE or A.stride(1) != 1 or A.stride(0) < A.shape[1]:
        raise ValueError("A must be a 2-D CUDA float64/float32 tensor with unit column stride")
    return LsqMatrix(A.data_ptr(), A.shape[0], A.shape[1], A.stride(0), DTYPE[A.dtype])


class Context:
    """Owns an lsq_ctx (stream = the current torch stream of `device` at creation)."""

    def __init__(self, device=None):
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else torch.device(device).index or 0)
        with torch.cuda.device(self.device):
            h = ctypes.c_void_p()
            st = _L.lsq_create(ctypes.byref(h), _stream_handle(self.device))
            if st:
                raise LsqError(st, "lsq_create")
        self.handle = h

    def sync_stream(self):
        _L.lsq_set_stream(self.handle, _stream_handle(self.device))

    def set_deferred_checks(self, on: bool = True):
        """Sketch and factor calls stop waiting for their own work; their errors (a timed-out
        wait, LSQ_ERR_RANK) are raised by the next lsq_solve or lsq_sync on this context."""
        st = _L.lsq_set_deferred_checks(self.handle, 1 if on else 0)
        if st:
            raise LsqError(st, "lsq_set_deferred_checks")

    def close(self):
        if getattr(self, "handle", None):
            _L.lsq_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def lsq_create(device=None) -> Context:
    return Context(device)


def lsq_destroy(ctx: Context) -> None:
    ctx.close()


def _check_a32(A: torch.Tensor, a32: torch.Tensor):
    if (a32.dtype != torch.float32 or not a32.is_cuda or a32.dim() != 2 or a32.shape[0] != A.shape[0]
            or a32.shape[1] < A.shape[1] or a32.stride(1) != 1 or a32.stride(0) % 4):
        raise ValueError("a32 must be a CUDA float32 n x (>= d) matrix with a row stride that is a multiple of 4")


def narrow_buffer(A: torch.Tensor) -> torch.Tensor:
    """An uninitialised buffer of the shape lsq_sketch(..., a32=) fills (n x ceil32(d) FP32)."""
    return torch.empty((A.shape[0], (A.shape[1] + 31) // 32 * 32), dtype=torch.float32, device=A.device)


def lsq_sketch(ctx: Context, A: torch.Tensor, kind: str, m: int, seed: int, t: int = 0, s: int = 8,
               precision: str = "f64", out: torch.Tensor | None = None, a32: torch.Tensor | None = None,
               row0: int = 0, n_total: int = 0) -> torch.Tensor:
    """SA (m x d FP64).  With `a32` (FP64 A), also writes the FP32 narrowing of A into it for a later
    mixed lsq_solve(..., a32=a32).  With row0 / n_total, A is the row slab [row0, row0 + n) of a
    matrix of n_total rows and SA its share of that matrix's sketch."""
    ctx.sync_stream()
    M = as_matrix(A)
    SA = out if out is not None else torch.empty((m, A.shape[1]), dtype=torch.float64, device=A.device)
    opts = LsqSketchOpts(t, s, SKETCH_PRECISION[precision], None, 0, int(row0), int(n_total))
    if a32 is not None:
        _check_a32(A, a32)
        opts.a32, opts.ld32 = a32.data_ptr(), a32.stride(0)
    st = _L.lsq_sketch(ctx.handle, ctypes.byref(M), SKETCH[kind], m, seed, ctypes.byref(opts), _ptr(SA))
    if st:
        raise LsqError(st, "lsq_sketch")
    return SA


def lsq_upload_sketch(ctx: Context, A_host: torch.Tensor, A: torch.Tensor, kind: str, m: int, seed: int, t: int = 0,
                      s: int = 8, precision: str = "f64", out: torch.Tensor | None = None,
                      a32: torch.Tensor | None = None) -> torch.Tensor:
    """Copies the host matrix A_host (CPU, row-major, pinned for overlap) into the device matrix A
    (same shape and dtype) and returns SA as lsq_sketch(ctx, A, ...) would, the SRHT transform
    running on each row range as it lands."""
    ctx.sync_stream()
    if A_host.device.type != "cpu" or A_host.dtype != A.dtype or A_host.shape != A.shape or A_host.stride(1) != 1:
        raise ValueError("A_host must be a CPU matrix of A's shape and dtype with unit column stride")
    M = as_matrix(A)
    SA = out if out is not None else torch.empty((m, A.shape[1]), dtype=torch.float64, device=A.device)
    opts = LsqSketchOpts(t, s, SKETCH_PRECISION[precision], None, 0, 0, 0)
    if a32 is not None:
        _check_a32(A, a32)
        opts.a32, opts.ld32 = a32.data_ptr(), a32.stride(0)
    st = _L.lsq_upload_sketch(ctx.handle, A_host.data_ptr(), A_host.stride(0), ctypes.byref(M), SKETCH[kind], m, seed,
                              ctypes.byref(opts), _ptr(SA))
    if st:
        raise LsqError(st, "lsq_upload_sketch")
    return SA


def lsq_factor(ctx: Context, SA: torch.Tensor, R: torch.Tensor | None = None, W: torch.Tensor | None = None,
               precision: str = "f64"):
    """(R, W) with R^T R = SA^T SA and W = R^{-1}; precision "mixed" forms the Gram in double-FP32."""
    ctx.sync_stream()
    if SA.dtype != torch.float64 or not SA.is_contiguous() or not SA.is_cuda:
        raise ValueError("SA must be a contiguous CUDA float64 matrix")
    m, d = SA.shape
    R = R if R is not None else torch.empty((d, d), dtype=torch.float64, device=SA.device)
    W = W if W is not None else torch.empty((d, d), dtype=torch.float64, device=SA.device)
    st = _L.lsq_factor_ex(ctx.handle, _ptr(SA), m, d, _ptr(R), _ptr(W), PRECISION[precision])
    if st:
        raise LsqError(st, "lsq_factor")
    return R, W


def lsq_factor_qr(ctx: Context, SA: torch.Tensor, tol: float = 0.0, raise_on_rank: bool = True):
    """(R, W, perm, rank) by Householder QR with column pivoting of SA: SA[:, perm] = Q R and
    W = P R^{-1} (dense: lsq_solve(..., w_dense=1)).  With raise_on_rank=False a rank-deficient SA
    returns W = None instead of raising."""
    ctx.sync_stream()
    if SA.dtype != torch.float64 or not SA.is_contiguous() or not SA.is_cuda:
        raise ValueError("SA must be a contiguous CUDA float64 matrix")
    m, d = SA.shape
    R = torch.empty((d, d), dtype=torch.float64, device=SA.device)
    W = torch.empty((d, d), dtype=torch.float64, device=SA.device)
    perm = torch.empty(d, dtype=torch.int32, device=SA.device)
    rank = ctypes.c_int64(0)
    st = _L.lsq_factor_qr(ctx.handle, _ptr(SA), m, d, float(tol), _ptr(R), _ptr(W), _ptr(perm), ctypes.byref(rank))
    if st == LSQ_ERR_RANK and not raise_on_rank:
        return R, None, perm, rank.value
    if st:
        raise LsqError(st, "lsq_factor_qr")
    return R, W, perm, rank.value


def solve_opts(**kw) -> LsqSolveOpts:
    o = LsqSolveOpts()
    _L.lsq_solve_opts_default(ctypes.byref(o))
    for k, v in kw.items():
        if k == "sketch_type" and isinstance(v, str):
            v = SKETCH[v]
        if k == "precision" and isinstance(v, str):
            v = PRECISION[v]
        setattr(o, k, v)
    return o


def lsq_solve(ctx: Context, A: torch.Tensor, b: torch.Tensor, method: str, W: torch.Tensor | None,
              x0: torch.Tensor | None = None, tol: float = 1e-10, maxit: int = 1000, raise_on_maxit: bool = False,
              **opts):
    """Returns (x, info dict).  Raises LsqError for errors other than LSQ_ERR_MAXIT."""
    ctx.sync_stream()
    M = as_matrix(A)
    d = A.shape[1]
    _check_vec(b, d, "b")
    x = torch.zeros(d, dtype=torch.float64, device=A.device) if x0 is None else x0.clone()
    _check_vec(x, d, "x0")
    if W is not None and (W.shape != (d, d) or W.dtype != torch.float64 or not W.is_contiguous()):
        raise ValueError("W must be a contiguous d x d float64 tensor")
    if x0 is None:
        opts.setdefault("x0_zero", 1)
    a32 = opts.pop("a32", None)
    o = solve_opts(**opts)
    if a32 is not None:
        _check_a32(A, a32)
        o.a32, o.ld32 = a32.data_ptr(), a32.stride(0)
    info = LsqSolveInfo()
    st = _L.lsq_solve(ctx.handle, ctypes.byref(M), _ptr(b), METHOD[method], _ptr(W), _ptr(x), float(tol), int(maxit),
                      ctypes.byref(o), ctypes.byref(info))
    if st and not (st == LSQ_ERR_MAXIT and not raise_on_maxit):
        raise LsqError(st, "lsq_solve")
    return x, info.as_dict()


def lsq_sync(ctx: Context) -> None:
    """Waits for the context's stream; raises LsqError for a deferred sketch or factor error."""
    ctx.sync_stream()
    st = _L.lsq_sync(ctx.handle)
    if st:
        raise LsqError(st, "lsq_sync")


def lsq_hmatvec(ctx: Context, A: torch.Tensor, p: torch.Tensor):
    ctx.sync_stream()
    M = as_matrix(A)
    d = A.shape[1]
    _check_vec(p, d, "p")
    v = torch.empty(d, dtype=torch.float64, device=A.device)
    q = torch.empty(1, dtype=torch.float64, device=A.device)
    st = _L.lsq_hmatvec(ctx.handle, ctypes.byref(M), _ptr(p), _ptr(v), _ptr(q))
    if st:
        raise LsqError(st, "lsq_hmatvec")
    return v, q


def lsq_grad_a(ctx: Context, A: torch.Tensor, x: torch.Tensor, lam: torch.Tensor,
               out: torch.Tensor | None = None) -> torch.Tensor:
    """dL/dA = -(A x) lam^T - (A lam) x^T (same dtype as A)."""
    ctx.sync_stream()
    M = as_matrix(A)
    d = A.shape[1]
    _check_vec(x, d, "x")
    _check_vec(lam, d, "lam")
    gA = out if out is not None else torch.empty(A.shape, dtype=A.dtype, device=A.device)
    st = _L.lsq_grad_a(ctx.handle, ctypes.byref(M), _ptr(x), _ptr(lam), _ptr(gA), gA.stride(0))
    if st:
        raise LsqError(st, "lsq_grad_a")
    return gA


class LeastSquaresSolve(torch.autograd.Function):
    """x* = argmin 1/2 <x, A^T A x> - <b, x> as a differentiable op.

    forward: sketch (SRHT by default), factor, PCG to `tol`.  backward: lambda = H^{-1} g by
    PCG with the forward's preconditioner W (no stored iterates), grad_b = lambda,
    grad_A = -(A x*) lambda^T - (A lambda) x*^T (lsq_grad_a)."""

    @staticmethod
    def forward(fctx, A, b, lsq: Context, sketch: str = "srht", m: int = 1024, seed: int = 0, tol: float = 1e-10,
                precision: str = "mixed", maxit: int = 1000):
        SA = lsq_sketch(lsq, A, sketch, m, seed, precision="f32" if precision == "mixed" else "f64")
        _, W = lsq_factor(lsq, SA)
        x, info = lsq_solve(lsq, A, b.contiguous(), "pcg", W, tol=tol, maxit=maxit, m=m, precision=precision,
                            raise_on_maxit=True)
        fctx.lsq, fctx.m, fctx.tol, fctx.precision, fctx.maxit = lsq, m, tol, precision, maxit
        fctx.save_for_backward(A, x, W)
        return x

    @staticmethod
    def backward(fctx, g):
        A, x, W = fctx.saved_tensors
        lam, _ = lsq_solve(fctx.lsq, A, g.contiguous().to(torch.float64), "pcg", W, tol=fctx.tol, maxit=fctx.maxit,
                           m=fctx.m, precision=fctx.precision, raise_on_maxit=True)
        gA = lsq_grad_a(fctx.lsq, A, x, lam) if fctx.needs_input_grad[0] else None
        gb = lam if fctx.needs_input_grad[1] else None
        return gA, gb, None, None, None, None, None, None, None


def lstsq_solve(A: torch.Tensor, b: torch.Tensor, lsq: Context, **kw) -> torch.Tensor:
    """Differentiable x* = H^{-1} b (see LeastSquaresSolve)."""
    return LeastSquaresSolve.apply(A, b, lsq, kw.get("sketch", "srht"), kw.get("m", 1024), kw.get("seed", 0),
                                   kw.get("tol", 1e-10), kw.get("precision", "mixed"), kw.get("maxit", 1000))


def batch_opts(**kw) -> LsqBatchOpts:
    o = LsqBatchOpts()
    _L.lsq_batch_opts_default(ctypes.byref(o))
    for k, v in kw.items():
        if k == "sketch_type" and isinstance(v, str):
            v = SKETCH[v]
        if k == "precision" and isinstance(v, str):
            v = PRECISION[v]
        if k == "sketch_precision" and isinstance(v, str):
            v = SKETCH_PRECISION[v]
        setattr(o, k, v)
    return o


def lsq_solve_batched(ctx: Context, problems, tol: float = 1e-10, maxit: int = 1000, X0=None, **opts):
    """Solves every problem (A_p, B_p) of the list: A_p an n_p x d_p CUDA tensor (FP64 or FP32, one
    type for the batch), B_p a k_p x d_p FP64 CUDA tensor of right-hand sides (row j = b_j).
    Returns (X list (k_p x d_p FP64), per-problem (iters, status) list, info dict).  Raises
    LsqError for errors other than LSQ_ERR_MAXIT / LSQ_ERR_BREAKDOWN / LSQ_ERR_RANK, which
    are reported per problem."""
    ctx.sync_stream()
    n = len(problems)
    arr = (LsqProblem * n)()
    Xs = []
    for p, (A, B) in enumerate(problems):
        M = as_matrix(A)
        d = A.shape[1]
        if B.dim() != 2 or B.shape[1] != d or B.dtype != torch.float64 or not B.is_cuda or not B.is_contiguous():
            raise ValueError("B must be a contiguous CUDA float64 tensor of shape (k, d)")
        if X0 is not None:
            X = X0[p].clone()
        else:
            X = torch.zeros_like(B)
        Xs.append(X)
        arr[p] = LsqProblem(M, B.data_ptr(), X.data_ptr(), B.shape[0], 0, 0, 0)
    if X0 is None:
        opts.setdefault("x0_zero", 1)
    else:
        opts.setdefault("x0_zero", 0)
    o = batch_opts(**opts)
    info = LsqBatchInfo()
    st = _L.lsq_solve_batched(ctx.handle, n, arr, float(tol), int(maxit), ctypes.byref(o), ctypes.byref(info))
    if st not in (LSQ_OK, LSQ_ERR_MAXIT, LSQ_ERR_BREAKDOWN, LSQ_ERR_RANK):
        raise LsqError(st, "lsq_solve_batched")
    per = [(arr[p].iters, arr[p].status) for p in range(n)]
    return Xs, per, info.as_dict()


def lsq_pcg_tail(ctx: Context, W: torch.Tensor, b: torch.Tensor, vq: torch.Tensor, phase: int, tol: float, rho: float,
                 state: torch.Tensor, wait: bool = True) -> int:
    """One PCG tail on the summed pass result vq (d + 1 FP64); returns the state's flag (0 running,
    1 converged) when `wait`, else -1.  Raises LsqError on breakdown."""
    ctx.sync_stream()
    d = b.numel()
    if vq.numel() != d + 1 or state.numel() != 4 * d + 8 or W.shape != (d, d):
        raise ValueError("vq must hold d + 1 and state 4 d + 8 FP64 entries, W d x d")
    flag = ctypes.c_int32(-1)
    st = _L.lsq_pcg_tail(ctx.handle, d, _ptr(W), _ptr(b), _ptr(vq), int(phase), float(tol), float(rho), _ptr(state),
                         ctypes.byref(flag) if wait else None)
    if st:
        raise LsqError(st, "lsq_pcg_tail")
    return int(flag.value)


def lsq_selftest_wait(ctx: Context, kind: int = 0, missing: int = 1, wait_ns: int = 0) -> int:
    """Runs one bounded grid barrier that waits for `missing` arrivals more than its grid has and
    returns the status code it ends with (LSQ_ERR_TIMEOUT when missing > 0)."""
    ctx.sync_stream()
    return int(_L.lsq_selftest_wait(ctx.handle, int(kind), int(missing), int(wait_ns)))


def lsq_advise_sketch_size(n: int, d: int, eps: float, kind: str = "srht") -> dict:
    """Section 6's optimized sketch size m*, the model cost ratio and the predicted iterations."""
    out = LsqAdvice()
    st = _L.lsq_advise_sketch_size(n, d, eps, SKETCH[kind], ctypes.byref(out))
    if st:
        raise LsqError(st, "lsq_advise_sketch_size")
    return {k: getattr(out, k) for k, _ in out._fields_}


def default_rho(d: int, m: int) -> float:
    return d / m


def lam1_bound(rho: float) -> float:
    return (1 + math.sqrt(rho)) ** 2
