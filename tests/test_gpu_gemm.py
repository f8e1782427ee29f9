"""GPU parity of the GEMM that carries every network layer, SIMT fp32 and tcgen05 bf16.

Reference: the plain definition C = A B^T (+ bias) (ReLU) in float64 on the CPU, computed
from the very operand values the kernel reads (bf16 operands are exact in float64, so
the only difference is the kernel's fp32 accumulation): within 1e-5 of sqrt(K) times
the largest |a||b| product scale, i.e. fp32 rounding of a length-K dot product.
"""
import numpy as np
import pytest
import torch

from paper_1911_00357_gb300 import binding as B

pytestmark = pytest.mark.gpu

SHAPES = [
    (128, 128, 64), (256, 256, 128), (129, 65, 72), (1000, 300, 520), (37, 2048, 512),
    (5, 1152, 128), (64, 2048, 512), (4096, 32, 288), (32, 288, 24576), (128, 1152, 4096),
    (3, 7, 40), (200, 17, 16), (8192, 512, 2048),
    # M <= 64 with K % 16 == 0: the small-M kernel (LSTM recurrences of one rollout step)
    (32, 512, 2048), (1, 64, 16), (64, 33, 48), (17, 100, 32), (64, 2048, 576),
]


def _ref(A, Bm, C0, beta, bias, relu):
    r = A.double().cpu() @ Bm.double().cpu().T
    if beta:
        r = r + beta * C0.double().cpu()
    if bias is not None:
        r = r + bias.double().cpu()
    if relu:
        r = r.clamp_min(0)
    return r


@pytest.mark.parametrize("M,N,K", SHAPES)
@pytest.mark.parametrize("dtype", [torch.bfloat16, torch.float32])
def test_gemm_parity(M, N, K, dtype):
    g = torch.Generator(device="cuda").manual_seed(M * 7 + N * 13 + K)
    A = torch.randn(M, K, device="cuda", generator=g).to(dtype)
    Bm = torch.randn(N, K, device="cuda", generator=g).to(dtype)
    C = torch.zeros(M, N, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    B.ddppo_gemm(A, Bm, C, status=st)
    torch.cuda.synchronize()
    assert st.item() == 0
    ref = _ref(A, Bm, None, 0.0, None, False)
    tol = 1e-5 * np.sqrt(K) * 4.0
    err = (C.double().cpu() - ref).abs().max().item()
    assert err <= tol, (err, tol, B.ddppo_gemm_backend(A, Bm))
    if dtype == torch.bfloat16 and M >= 1 and K >= 16:
        assert B.ddppo_gemm_backend(A, Bm)


TRANS_SHAPES = [(32, 288, 24576), (64, 576, 4100), (2048, 576, 1000), (2048, 512, 4096),
                (512, 2048, 64), (37, 56, 3000), (300, 200, 136)]


@pytest.mark.parametrize("M,N,K", TRANS_SHAPES)
@pytest.mark.parametrize("a_t,b_t", [(1, 1), (1, 0), (0, 1)])
@pytest.mark.parametrize("dtype", [torch.bfloat16, torch.float32])
def test_gemm_mn_major_operands(M, N, K, a_t, b_t, dtype):
    """Operands stored [K, M] / [K, N] (the weight-gradient contractions)."""
    g = torch.Generator(device="cuda").manual_seed(M + 3 * N + 7 * K + a_t + 2 * b_t)
    A = torch.randn(M, K, device="cuda", generator=g).to(dtype)
    Bm = torch.randn(N, K, device="cuda", generator=g).to(dtype)
    At = A.t().contiguous() if a_t else A
    Bt = Bm.t().contiguous() if b_t else Bm
    C = torch.zeros(M, N, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    B.ddppo_gemm(At, Bt, C, status=st, a_t=bool(a_t), b_t=bool(b_t))
    torch.cuda.synchronize()
    assert st.item() == 0
    ref = _ref(A, Bm, None, 0.0, None, False)
    tol = 1e-5 * np.sqrt(K) * 4.0
    err = (C.double().cpu() - ref).abs().max().item()
    assert err <= tol, (err, tol)


@pytest.mark.parametrize("dtype", [torch.bfloat16, torch.float32])
@pytest.mark.parametrize("M", [300, 40])   # 40: the small-M kernel
def test_gemm_epilogue_and_strides(dtype, M):
    N, K = 200, 144
    g = torch.Generator(device="cuda").manual_seed(5)
    Abig = torch.randn(M, K + 24, device="cuda", generator=g).to(dtype)   # lda = K + 24
    A = Abig[:, :K]
    Bm = torch.randn(N, K, device="cuda", generator=g).to(dtype)
    bias = torch.randn(N, device="cuda", generator=g)
    C0 = torch.randn(M, N + 8, device="cuda", generator=g)
    C = C0.clone()
    B.ddppo_gemm(A, Bm, C, beta=0.5, bias=bias, relu=True, M=M, N=N, K=K, lda=K + 24, ldc=N + 8)
    torch.cuda.synchronize()
    ref = _ref(A, Bm, C0[:, :N], 0.5, bias, True)
    assert (C[:, :N].double().cpu() - ref).abs().max().item() <= 1e-4
    assert torch.equal(C[:, N:], C0[:, N:])            # columns beyond N untouched
    # bf16 output
    Cb = torch.zeros(M, N, device="cuda", dtype=torch.bfloat16)
    B.ddppo_gemm(A, Bm, Cb, bias=bias, M=M, N=N, K=K, lda=K + 24)
    torch.cuda.synchronize()
    ref2 = _ref(A, Bm, None, 0.0, bias, False)
    assert ((Cb.double().cpu() - ref2).abs() <= 2 ** -8 * ref2.abs() + 1e-3).all()
