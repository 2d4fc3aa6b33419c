"""The tensor-core GEMM (tcgen05, TF32 or BF16 operands, FP32 accumulation)
that the mixed factorizations use for their contractions, through the C ABI
(hs_gemm_tc).

* Exactness: with small integer operands every product and every partial
  sum is exact in TF32, BF16 and FP32, so the result must equal the FP64
  product bit for bit -- any error in the shared-memory layout, the
  transposes, the ragged edges or alpha/beta shows as a wrong integer.
* Rounding: with normal operands the result must match the FP64 product of
  the operands rounded as the kernel rounds them (TF32: nearest, ties away
  from zero; BF16: nearest even), within FP32 accumulation error.
"""
import numpy as np
import pytest

from paper_1611_03189_gb300 import _lib

from gpu_util import need_gpu

pytestmark = pytest.mark.gpu

SHAPES = [(1, 1, 1), (5, 7, 3), (128, 128, 32), (130, 129, 33), (64, 64, 64), (300, 200, 513), (17, 250, 1000)]


def _operand(torch, rows, cols, vals, pad, shift):
    """rows x cols float32 view with leading dimension cols + pad, starting
    `shift` elements into its storage (shift = 1 breaks 16-byte alignment)."""
    base = torch.zeros((rows, cols + pad + shift), dtype=torch.float32, device="cuda")
    v = base[:, shift:shift + cols]
    v.copy_(torch.as_tensor(vals, dtype=torch.float32))
    return v


def _round_tf32(x):
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = ((b + 0x1000) & 0xFFFFE000) & 0xFFFFFFFF
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def _round_bf16(torch, x):
    return torch.as_tensor(np.asarray(x, dtype=np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


@pytest.mark.parametrize("prec", [_lib.HS_PREC_TF32, _lib.HS_PREC_BF16, _lib.HS_PREC_TF32X3],
                         ids=["tf32", "bf16", "tf32x3"])
@pytest.mark.parametrize("bn", [64, 128])
@pytest.mark.parametrize("ta,tb", [(0, 0), (0, 1), (1, 0), (1, 1)])
def test_integer_operands_give_the_exact_product(prec, bn, ta, tb):
    torch = need_gpu()
    rng = np.random.default_rng(7 + 2 * ta + tb + bn + prec)
    for M, N, K in SHAPES:
        for pad, shift in ((0, 0), (3, 1)):
            a = rng.integers(-4, 5, size=(M, K)).astype(np.float64)
            b = rng.integers(-4, 5, size=(K, N)).astype(np.float64)
            c0 = rng.integers(-8, 9, size=(M, N)).astype(np.float64)
            A = _operand(torch, *(a.T.shape if ta else a.shape), a.T if ta else a, pad, shift)
            B = _operand(torch, *(b.T.shape if tb else b.shape), b.T if tb else b, pad, shift)
            C = _operand(torch, M, N, c0, pad, shift)
            _lib.gemm_tc(prec, A, B, C, alpha=2.0, beta=-1.0, ta=ta, tb=tb, bn=bn)
            torch.cuda.synchronize()
            want = 2.0 * (a @ b) - c0
            got = C.double().cpu().numpy()
            assert np.array_equal(got, want), (M, N, K, pad, shift, np.abs(got - want).max())


@pytest.mark.parametrize("prec", [_lib.HS_PREC_TF32, _lib.HS_PREC_BF16], ids=["tf32", "bf16"])
def test_rounded_operands_within_fp32_accumulation(prec):
    torch = need_gpu()
    rng = np.random.default_rng(3)
    for M, N, K in ((200, 300, 700), (129, 64, 2048)):
        a = rng.standard_normal((M, K)).astype(np.float32)
        b = rng.standard_normal((K, N)).astype(np.float32)
        A = torch.as_tensor(a, device="cuda")
        B = torch.as_tensor(b, device="cuda")
        C = torch.zeros((M, N), dtype=torch.float32, device="cuda")
        _lib.gemm_tc(prec, A, B, C)
        got = C.double().cpu().numpy()
        if prec == _lib.HS_PREC_TF32:
            ar, br = _round_tf32(a), _round_tf32(b)
        else:
            ar, br = _round_bf16(torch, a), _round_bf16(torch, b)
        want = ar @ br
        # FP32 accumulation: each partial sum rounds with u = 2^-24
        bound = 2.0 * K * 2.0 ** -24 * (np.abs(ar) @ np.abs(br))
        assert np.all(np.abs(got - want) <= bound + 1e-30)
        # and the rounding of the operands is visible against the FP64 product
        exact = a.astype(np.float64) @ b.astype(np.float64)
        u = 2.0 ** -11 if prec == _lib.HS_PREC_TF32 else 2.0 ** -8
        assert np.max(np.abs(got - exact)) <= 2.5 * u * np.max(np.abs(a).astype(np.float64) @ np.abs(b))


@pytest.mark.parametrize("prec", [_lib.HS_PREC_TF32, _lib.HS_PREC_BF16, _lib.HS_PREC_TF32X3],
                         ids=["tf32", "bf16", "tf32x3"])
def test_empty_inner_dimension_scales_c(prec):
    """K = 0: op(A) op(B) is the zero matrix, so C becomes beta C."""
    import ctypes as C

    torch = need_gpu()
    M, N = 257, 65
    c0 = torch.arange(M * N, dtype=torch.float32, device="cuda").reshape(M, N) % 17 - 8
    Cm = c0.clone()
    dummy = torch.zeros(4, dtype=torch.float32, device="cuda")
    code = _lib.lib().hs_gemm_tc(prec, M, N, 0, 2.0, dummy.data_ptr(), 1, 0, dummy.data_ptr(), N, 0, -1.0,
                                 Cm.data_ptr(), N, 0, C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert code == _lib.HS_OK
    assert torch.equal(Cm, -c0)


def test_tf32x3_keeps_near_fp32_accuracy():
    """3xTF32: a = a_hi + a_lo (TF32 parts, a_lo = tf32(a - a_hi)), products
    a_hi b_hi + a_hi b_lo + a_lo b_hi.  The split leaves |a - a_hi - a_lo| <=
    2^-22 |a| and the dropped a_lo b_lo is <= 2^-22 |a b|, so each product is
    within 3 2^-22 |a b|; the sums add the tensor core's FP32 accumulation,
    whose additions are coarser than IEEE round-to-nearest (measured: about
    1e-4 relative at K = 700 against 2e-3 for plain TF32 operands).  Checked
    against the FP64 product with the FP32 accumulation bound, and at least
    ten times closer than plain TF32."""
    torch = need_gpu()
    rng = np.random.default_rng(11)
    for M, N, K in ((200, 300, 700), (129, 64, 2048)):
        a = rng.standard_normal((M, K)).astype(np.float32)
        b = rng.standard_normal((K, N)).astype(np.float32)
        C = torch.zeros((M, N), dtype=torch.float32, device="cuda")
        _lib.gemm_tc(_lib.HS_PREC_TF32X3, torch.as_tensor(a, device="cuda"), torch.as_tensor(b, device="cuda"), C)
        got = C.double().cpu().numpy()
        exact = a.astype(np.float64) @ b.astype(np.float64)
        absab = np.abs(a).astype(np.float64) @ np.abs(b).astype(np.float64)
        bound = (3.0 * 2.0 ** -22 + 2.0 * K * 2.0 ** -24) * absab
        assert np.all(np.abs(got - exact) <= bound)
        # at least 10x closer than plain TF32 on the largest entry error
        C1 = torch.zeros((M, N), dtype=torch.float32, device="cuda")
        _lib.gemm_tc(_lib.HS_PREC_TF32, torch.as_tensor(a, device="cuda"), torch.as_tensor(b, device="cuda"), C1)
        e3 = np.max(np.abs(got - exact))
        e1 = np.max(np.abs(C1.double().cpu().numpy() - exact))
        assert e3 * 10 < e1, (e3, e1)


def test_invalid_arguments_are_rejected():
    torch = need_gpu()
    A = torch.zeros((4, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(_lib.HsError) as e:
        _lib.gemm_tc(_lib.HS_PREC_F32, A, A, A.clone())
    assert e.value.code == _lib.HS_ERR_INVALID
    with pytest.raises(_lib.HsError) as e:
        _lib.gemm_tc(_lib.HS_PREC_TF32, A, A, A.clone(), bn=96)
    assert e.value.code == _lib.HS_ERR_INVALID
