"""Parity of lsq_sketch (Section 2) with the FP64 oracle.

Bar: SRHT signs / sample indices and SJLT positions bit for bit (integer-valued A makes
every sum exact, so SA must equal the oracle's SA exactly); SA in FP64 to 1e-12 relative
Frobenius error; the FP32 variant within its own rounding bound."""
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


@pytest.mark.parametrize("n,d,m,seed,t", [(1000, 37, 70, 3, 0), (4096, 64, 256, 0, 0), (777, 130, 129, 5, 2),
                                          (33, 1, 2, 9, 1)])
def test_gaussian_fp64(L, ctx, n, d, m, seed, t):
    A = W.make_problem(n, d, 1e3, seed=seed + 1)["A"]
    SA = L.lsq_sketch(ctx, to_dev(A), "gauss", m, seed, t=t).cpu().numpy()
    assert rel_fro(SA, O.sketch_gauss(A, m, seed, t)) < 1e-12


def test_gaussian_fp32_storage_and_arithmetic(L, ctx):
    A32 = W.make_problem(3000, 48, 1e2, seed=2)["A"].astype(np.float32)
    ref = O.sketch_gauss(A32.astype(np.float64), 96, 4)
    SA = L.lsq_sketch(ctx, to_dev(A32), "gauss", 96, 4).cpu().numpy()
    assert rel_fro(SA, ref) < 1e-12          # FP32 storage, FP64 arithmetic
    SA32 = L.lsq_sketch(ctx, to_dev(A32), "gauss", 96, 4, precision="f32").cpu().numpy()
    assert rel_fro(SA32, ref) < 5e-6         # FP32 arithmetic: u32 * sqrt-growth


@pytest.mark.parametrize("n,d,m,seed,t", [(64, 5, 16, 1, 0), (1000, 7, 64, 2, 3), (5000, 33, 300, 7, 1),
                                          (70000, 3, 1000, 4, 0), (2048, 16, 2048, 3, 0)])
def test_srht_indices_and_signs_bit_exact(L, ctx, n, d, m, seed, t):
    A = int_matrix(n, d, seed)
    SA = L.lsq_sketch(ctx, to_dev(A), "srht", m, seed, t=t).cpu().numpy()
    ref = O.sketch_srht(A, m, seed, t)
    assert np.array_equal(SA, ref)


@pytest.mark.parametrize("n,d,m,seed", [(3000, 40, 200, 1), (4096, 64, 256, 0), (20000, 130, 1024, 2)])
def test_srht_fp64(L, ctx, n, d, m, seed):
    A = W.make_problem(n, d, 1e4, seed=seed)["A"]
    SA = L.lsq_sketch(ctx, to_dev(A), "srht", m, seed).cpu().numpy()
    assert rel_fro(SA, O.sketch_srht(A, m, seed)) < 1e-12
    SA32 = L.lsq_sketch(ctx, to_dev(A), "srht", m, seed, precision="f32").cpu().numpy()
    assert rel_fro(SA32, O.sketch_srht(A, m, seed)) < 5e-6


@pytest.mark.parametrize("n,d,m,dtype,ld", [(5000, 13, 700, np.float64, 14), (5000, 13, 700, np.float32, 16),
                                             (9000, 24, 4096, np.float64, 24), (9000, 24, 4097, np.float64, 24),
                                             (3000, 20, 300, np.float64, 21), (2048, 8, 64, np.float64, 8),
                                             (2048, 3, 64, np.float64, 4), (3000, 5, 100, np.float32, 8),
                                             (20000, 40, 9000, np.float64, 40), (12000, 16, 8192, np.float32, 16)])
def test_srht_fp32_arithmetic_layouts(L, ctx, n, d, m, dtype, ld):
    """FP32-arithmetic SRHT over row strides and sizes that take the staged (tensor-copy) kernel
    -- ragged n and d, FP32 storage, 8 sampled rows per thread, more than 4096 sampled rows in
    slices of 4096 -- and ones that do not (a row stride that is not a multiple of 16 bytes)."""
    A = W.make_problem(n, d, 1e4, seed=n + d)["A"].astype(dtype)
    big = torch.zeros((n, ld), dtype=torch.float64 if dtype == np.float64 else torch.float32, device="cuda")
    big[:, :d] = to_dev(A)
    SA = L.lsq_sketch(ctx, big[:, :d], "srht", m, 5, t=2, precision="f32").cpu().numpy()
    ref = O.sketch_srht(A.astype(np.float64), m, 5, 2)
    assert rel_fro(SA, ref) < 5e-6
    # repeatable bit for bit
    SA2 = L.lsq_sketch(ctx, big[:, :d], "srht", m, 5, t=2, precision="f32").cpu().numpy()
    assert np.array_equal(SA, SA2)


@pytest.mark.parametrize("n,d,m,s,seed,t", [(100, 4, 10, 3, 1, 0), (5000, 33, 64, 8, 2, 2), (20000, 130, 512, 8, 3, 0),
                                            (3000, 9, 7, 7, 5, 1), (1000, 2, 40, 1, 6, 0)])
def test_sjlt_positions_bit_exact(L, ctx, n, d, m, s, seed, t):
    A = int_matrix(n, d, seed)
    SA = L.lsq_sketch(ctx, to_dev(A), "sjlt", m, seed, t=t, s=s).cpu().numpy()
    ref = O.sketch_sjlt(A, m, s, seed, t)
    # sqrt(s) SA holds exact integer sums of +-A rows; the two sides round the scale in a
    # different order (per term vs per sum), so compare the integers those sums must be
    k_gpu, k_ref = SA * np.sqrt(s), ref * np.sqrt(s)
    assert np.max(np.abs(k_gpu - np.rint(k_gpu))) < 1e-6 and np.max(np.abs(k_ref - np.rint(k_ref))) < 1e-6
    assert np.array_equal(np.rint(k_gpu), np.rint(k_ref))
    assert rel_fro(SA, ref) < 1e-14


def test_sjlt_fp64_and_fp32(L, ctx):
    A = W.make_problem(8000, 64, 1e4, seed=3)["A"]
    ref = O.sketch_sjlt(A, 512, 8, 11)
    assert rel_fro(L.lsq_sketch(ctx, to_dev(A), "sjlt", 512, 11, s=8).cpu().numpy(), ref) < 1e-12
    assert rel_fro(L.lsq_sketch(ctx, to_dev(A), "sjlt", 512, 11, s=8, precision="f32").cpu().numpy(), ref) < 5e-6


def test_strided_rows(L, ctx):
    A = W.make_problem(2000, 24, 1e2, seed=4)["A"]
    big = torch.zeros((2000, 40), dtype=torch.float64, device="cuda")
    big[:, :24] = to_dev(A)
    for kind in ("gauss", "srht", "sjlt"):
        SA = L.lsq_sketch(ctx, big[:, :24], kind, 128, 1).cpu().numpy()
        assert rel_fro(SA, O.sketch(A, kind, 128, 1)) < 1e-12


def test_rejects_bad_arguments(L, ctx):
    A = to_dev(np.ones((64, 4)))
    with pytest.raises(L.LsqError):
        L.lsq_sketch(ctx, A, "srht", 65, 0)       # m > N
    with pytest.raises(L.LsqError):
        L.lsq_sketch(ctx, A, "sjlt", 4, 0, s=5)   # s > m


@pytest.mark.parametrize("n,m", [(256, 256), (512, 128), (300, 200), (1024, 256), (800, 130)])
def test_gaussian_bf16_tensor_core_layout(L, ctx, n, m):
    """A = I_n makes SA = S: every entry of the tensor-core product must be the BF16 rounding of
    z(j, i) (up to one BF16 step where FP32 and FP64 evaluations straddle a rounding boundary),
    so any error in the operand layouts or descriptors shows up entry by entry.  The kernel is
    also deterministic: a second run agrees bit for bit."""
    A = np.eye(n)
    SA = L.lsq_sketch(ctx, to_dev(A), "gauss", m, 7, t=1, precision="bf16").cpu().numpy() * np.sqrt(m)
    SA2 = L.lsq_sketch(ctx, to_dev(A), "gauss", m, 7, t=1, precision="bf16").cpu().numpy() * np.sqrt(m)
    assert np.array_equal(SA, SA2)
    Z = O.gauss_matrix(m, n, 7, 1) * np.sqrt(m)
    Zb = torch.from_numpy(Z).to(torch.bfloat16).to(torch.float64).numpy()
    # FP32 generation (24-bit uniforms, fast sin/cos) moves tiny |z| by up to ~1e-4 absolute
    assert np.all(np.abs(SA - Zb) <= 2.0 ** -7 * np.abs(Zb) + 1e-4)
    # equal up to the rounding of the final 1/sqrt(m) scale, except at straddled boundaries
    assert np.mean(np.isclose(SA, Zb, rtol=1e-12, atol=0)) > 0.99


@pytest.mark.parametrize("n,d,m,dtype", [(20000, 256, 512, np.float32), (9000, 700, 384, np.float64),
                                         (4096, 64, 256, np.float32)])
def test_gaussian_bf16_accuracy(L, ctx, n, d, m, dtype):
    A = W.make_problem(n, d, 1e2, seed=5)["A"].astype(dtype)
    SA = L.lsq_sketch(ctx, to_dev(A), "gauss", m, 3, precision="bf16").cpu().numpy()
    ref = O.sketch_gauss(A.astype(np.float64), m, 3)
    assert rel_fro(SA, ref) < 1e-2  # BF16 operands: about 2^-9 per product, random signs


def narrow_truncate(A):
    """FP64 -> FP32 by mantissa truncation with the exponent clamped to FP32's range (the
    narrowing of the mixed solve's FP32 passes), written out on the bits."""
    u = np.ascontiguousarray(A, dtype=np.float64).view(np.uint64)
    hi, lo = (u >> np.uint64(32)).astype(np.uint64), (u & np.uint64(0xFFFFFFFF)).astype(np.uint64)
    e = (hi >> np.uint64(20)) & np.uint64(0x7FF)
    ec = np.clip(e, 896, 1151).astype(np.uint64) - np.uint64(896)
    mant = (((hi & np.uint64(0xFFFFF)) << np.uint64(3)) | (lo >> np.uint64(29))) & np.uint64(0x7FFFFF)
    sign = hi & np.uint64(0x80000000)
    return (sign | (ec << np.uint64(23)) | mant).astype(np.uint32).view(np.float32)


@pytest.mark.parametrize("kind,precision,n,d", [("srht", "f32", 5000, 13), ("srht", "f32", 9000, 64),
                                                ("srht", "f64", 3000, 20), ("gauss", "f32", 1000, 40),
                                                ("sjlt", "f32", 2000, 33)])
def test_sketch_writes_fp32_copy(L, ctx, kind, precision, n, d):
    """lsq_sketch(..., a32=) leaves the FP32 narrowing of A (the values of a mixed solve's FP32
    passes): written by the staged SRHT on the way, by a separate pass otherwise."""
    A = W.make_problem(n, d, 1e6, seed=d)["A"]
    Ad = to_dev(A)
    a32 = torch.full((n, (d + 31) // 32 * 32), np.nan, dtype=torch.float32, device="cuda")
    SA = L.lsq_sketch(ctx, Ad, kind, 256, 3, precision=precision, a32=a32).cpu().numpy()
    got = a32.cpu().numpy()[:, :d]
    want = narrow_truncate(A)
    assert np.array_equal(got, want)
    # truncation: |a32| <= |A| within one FP32 unit in the last place
    assert np.all(np.abs(want.astype(np.float64)) <= np.abs(A))
    assert np.all(np.abs(A - want) <= 2.0 ** -23 * np.abs(A))
    # the sketch itself is unchanged by the extra output (SJLT: up to the order of its atomic sums)
    SA0 = L.lsq_sketch(ctx, Ad, kind, 256, 3, precision=precision).cpu().numpy()
    if kind == "sjlt":
        assert rel_fro(SA, SA0) < 1e-6
    else:
        assert np.array_equal(SA, SA0)


@pytest.mark.parametrize("n,d,m,dtype,kind,pinned", [
    (2**17 + 777, 64, 512, np.float64, "srht", True),     # many row-block groups, ragged tail
    (300000, 512, 4096, np.float64, "srht", True),         # the headline's shape class
    (70000, 40, 256, np.float32, "srht", True),            # FP32 A, d not a multiple of 8
    (50000, 48, 6000, np.float64, "srht", True),           # two slices of sampled rows
    (1500, 24, 64, np.float64, "srht", False),             # one zero-padded block, pageable host memory
    (900, 24, 64, np.float64, "srht", True),               # padded length under 2048: whole copy
    (5000, 33, 128, np.float64, "gauss", True),            # other sketches: whole copy, then sketch
    (600001, 1024, 4096, np.float32, "gauss-bf16", True),  # tensor-core Gaussian: 2 chunks, ragged tail
    (2**21 + 333, 40, 256, np.float32, "gauss-bf16", True),  # narrow d: 2 chunks of 2^21 rows
    (3000, 24, 64, np.float64, "gauss-bf16", False),       # one chunk, pageable host memory
    (600001, 600, 1000, np.float32, "sjlt-bf16", True),    # tensor-core SJLT: CTA pairs, 2 chunks
])
def test_upload_sketch_matches_sketch_of_device_copy(L, ctx, n, d, m, dtype, kind, pinned):
    """lsq_upload_sketch copies A while the SRHT transforms the row groups that have landed (the
    tensor-core Gaussian sketch: the chunks that have landed): A on the device, SA and the FP32
    copy equal those of lsq_sketch on A already resident."""
    rng = np.random.default_rng(n + d)
    A = rng.standard_normal((n, d)).astype(dtype) * np.logspace(0, 3, d).astype(dtype)
    A_host = torch.from_numpy(A)
    if pinned:
        A_host = A_host.pin_memory()
    Ad = torch.empty(A_host.shape, dtype=A_host.dtype, device="cuda")
    prec = {"srht": "f32", "gauss-bf16": "bf16", "sjlt-bf16": "bf16"}.get(kind, "f64")
    kind = kind.split("-")[0]
    a32 = L.narrow_buffer(Ad) if dtype == np.float64 else None
    SA_up = L.lsq_upload_sketch(ctx, A_host, Ad, kind, m, 5, precision=prec, a32=a32)
    a32_up = a32.clone() if a32 is not None else None
    assert torch.equal(Ad.cpu(), torch.from_numpy(A))
    SA_ref = L.lsq_sketch(ctx, Ad, kind, m, 5, precision=prec, a32=a32)
    assert torch.equal(SA_up, SA_ref)
    if a32 is not None:  # the pad columns past d are never written nor read
        assert torch.equal(a32_up[:, :d], a32[:, :d])


def _narrow_f32(A):
    """FP64 -> FP32 by truncating the mantissa (the library's narrowing, for normal values), FP32 as is."""
    if A.dtype == np.float32:
        return A
    u = np.ascontiguousarray(A).view(np.uint64)
    sign = (u >> 63) << 31
    e = ((u >> 52) & 0x7FF).astype(np.int64) - 896
    assert e.min() > 0 and e.max() < 255, "test data in the normal FP32 range"
    f = sign | (e.astype(np.uint64) << 23) | ((u >> 29) & 0x7FFFFF)
    return f.astype(np.uint32).view(np.float32)


def _round_bf16(A):
    """The library's FP32 narrowing, then BF16 (nearest, ties to even) by the bit pattern, back to FP64."""
    u = np.ascontiguousarray(_narrow_f32(A)).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


@pytest.mark.parametrize("n,d,m,s,dtype", [(5000, 33, 256, 8, np.float32), (3000, 20, 128, 4, np.float64),
                                           (20000, 64, 512, 8, np.float32), (70001, 600, 1000, 8, np.float64),
                                           (9000, 300, 96, 32, np.float32), (2000, 16, 8, 8, np.float32)])
def test_sjlt_bf16_is_the_sketch_of_rounded_a(L, ctx, n, d, m, s, dtype):
    """LSQ_SKETCH_BF16 for the SJLT (on the tensor cores): the FP64 sketch of A narrowed to BF16 (exact
    +-1 signs and positions), up to the FP32 sums; and it repeats bit for bit."""
    A = W.make_problem(n, d, 1e3, seed=n + s)["A"].astype(dtype)
    Ab = _round_bf16(A)
    assert np.max(np.abs(Ab - A)) > 0  # the rounding does something
    Ad = to_dev(A)
    SA = L.lsq_sketch(ctx, Ad, "sjlt", m, 3, s=s, precision="bf16").cpu().numpy()
    ref = O.sketch_sjlt(Ab, m, s, 3, 0)
    assert rel_fro(SA, ref) < 1e-6
    assert np.array_equal(SA, L.lsq_sketch(ctx, Ad, "sjlt", m, 3, s=s, precision="bf16").cpu().numpy())
    assert rel_fro(SA, O.sketch_sjlt(A.astype(np.float64), m, s, 3, 0)) < 1e-2  # ~ BF16 resolution


@pytest.mark.parametrize("n,d,m,s", [(5000, 24, 200, 4), (20001, 600, 1000, 16), (3000, 300, 64, 4),
                                     (70000, 512, 4096, 4), (999, 7, 8, 4)])
def test_sjlt_bf16_tensor_core_bit_exact_on_integers(L, ctx, n, d, m, s):
    """Small integers are exact in BF16 and their FP32 sums are exact, and 1/sqrt(s) is a power
    of two for s = 4, 16: the tensor-core SJLT equals the oracle's sketch bit for bit, which
    pins every target row and sign it writes into the tiles of S (window edges at m not a
    multiple of 128, CTA pairs for d > 512, ragged n)."""
    A = int_matrix(n, d, seed=n + d)
    SA = L.lsq_sketch(ctx, to_dev(A), "sjlt", m, 6, s=s, precision="bf16").cpu().numpy()
    assert np.array_equal(SA, O.sketch_sjlt(A, m, s, 6, 0))


@pytest.mark.parametrize("n,d,m,dtype", [(20000, 130, 512, np.float32), (20001, 600, 1000, np.float32),
                                         (9000, 300, 256, np.float64)])
def test_sjlt_bf16_tensor_core_repeats_bit_for_bit(L, ctx, n, d, m, dtype):
    """The tensor-core SJLT sums its exact +-1 products in a fixed order, so on real-valued A two
    runs agree bit for bit (single CTAs and CTA pairs), unlike the FP32 scatter's atomic sums."""
    A = to_dev(W.make_problem(n, d, 1e4, seed=d)["A"].astype(dtype))
    SA1 = L.lsq_sketch(ctx, A, "sjlt", m, 9, s=8, precision="bf16")
    SA2 = L.lsq_sketch(ctx, A, "sjlt", m, 9, s=8, precision="bf16")
    assert torch.equal(SA1, SA2)
    assert torch.isfinite(SA1).all()
