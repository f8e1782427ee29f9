"""The tensor-store epilogue of the tcgen05 GEMM changes how a tile's result leaves the SM
(one tensor copy per 32 x 32 block from swizzled shared memory, instead of a transpose and
one store per row), never the values: each output is formed by the same operations in the
same order (scale, + beta C as one fused multiply-add with C read by a tensor load, + bias,
ReLU, output type; split-K partials raw). With the epilogue on and off, plain contractions
(fp32 and bf16 outputs, beta, bias and ReLU, ragged M and N, split-K partials),
convolutions on the 4-D gather and the row halo (ragged last tiles, Cout below 32, beta),
and whole rollout-then-update iterations (captured collect and update graphs) are
bit-identical."""
import numpy as np
import pytest
import torch

from paper_1911_00357_gb300 import binding as B
from paper_1911_00357_gb300.worker import Worker

pytestmark = pytest.mark.gpu


def _both(fn):
    before = B.ddppo_tma_epilogue()
    try:
        B.ddppo_set_tma_epilogue(True)
        a = fn()
        B.ddppo_set_tma_epilogue(False)
        b = fn()
    finally:
        B.ddppo_set_tma_epilogue(before)
    return a, b


# (M, N, K, c dtype, beta, bias, relu): tiles of 128 rows; N tiles of 64 / 128 with
# 32-column store blocks; ragged M and N (the stores stop at the tensor's edge); K >= 512
# with few tiles takes split-K (partials through the tensor store, then the reduction)
GEMMS = [
    (4096, 64, 288, torch.float32, 0.0, False, False),
    (4096, 64, 288, torch.float32, 1.0, False, False),
    (1000, 300, 520, torch.float32, 0.0, True, True),
    (1000, 300, 520, torch.float32, 0.5, True, True),
    (8192, 512, 2048, torch.bfloat16, 0.0, True, True),
    (777, 96, 64, torch.bfloat16, 0.0, False, True),
    (300, 40, 128, torch.float32, -0.75, True, False),
    (129, 33, 72, torch.float32, 0.0, False, False),
    (2000, 128, 1024, torch.float32, 1.0, False, True),
]


@pytest.mark.parametrize("M,N,K,cdt,beta,bias,relu", GEMMS)
def test_gemm_epilogues_bit_identical(M, N, K, cdt, beta, bias, relu):
    g = torch.Generator(device="cuda").manual_seed(M + 3 * N + 7 * K)
    A = torch.randn(M, K, device="cuda", generator=g).to(torch.bfloat16)
    Bm = torch.randn(N, K, device="cuda", generator=g).to(torch.bfloat16)
    bv = torch.randn(N, device="cuda", generator=g) if bias else None
    C0 = torch.randn(M, N, device="cuda", generator=g)

    def run():
        C = C0.clone() if beta else torch.full((M, N), float("nan"), device="cuda").to(cdt)
        B.ddppo_gemm(A, Bm, C, beta=beta, bias=bv, relu=relu)
        torch.cuda.synchronize()
        return C.cpu()

    a, b = _both(run)
    assert torch.equal(a.view(torch.int16) if cdt == torch.bfloat16 else a.view(torch.int32),
                       b.view(torch.int16) if cdt == torch.bfloat16 else b.view(torch.int32))
    ref = A.double().cpu() @ Bm.double().cpu().T
    if beta:
        ref = ref + beta * C0.double().cpu()
    if bias:
        ref = ref + bv.double().cpu()
    if relu:
        ref = ref.clamp_min(0)
    tol = (4e-3 if cdt == torch.bfloat16 else 1e-5) * np.sqrt(K) * max(ref.abs().max().item(), 1.0)
    assert (a.double() - ref).abs().max().item() <= tol


# (N, H, W, C, Cout, k, s, p)
CONVS = [
    (6, 32, 32, 32, 32, 3, 1, 1),     # row halo, 4 rows per tile
    (3, 20, 8, 32, 16, 3, 1, 1),      # row halo, 16 rows per tile, ragged last tile, Cout 16
    (2, 35, 32, 32, 32, 3, 1, 1),     # row halo, ragged last tile
    (5, 16, 16, 64, 64, 3, 1, 1),     # 4-D gather
    (7, 8, 8, 128, 256, 3, 2, 1),     # 4-D gather, 8 images per tile
    (4, 16, 16, 64, 128, 1, 2, 0),    # 1x1 stride-2 shortcut
    (3, 15, 15, 32, 32, 3, 1, 1),     # anchor halo (tile rows are not output rows): per-row stores
]


@pytest.mark.parametrize("beta", [0.0, 1.0])
@pytest.mark.parametrize("N,H,W,C,Co,k,s,p", CONVS)
def test_conv_epilogues_bit_identical(N, H, W, C, Co, k, s, p, beta):
    g = torch.Generator(device="cuda").manual_seed(N * 131 + C * 7 + Co + k + s)
    x = torch.randn(N, H, W, C, device="cuda", generator=g).to(torch.bfloat16)
    wg = (torch.randn(Co, k * k * C, device="cuda", generator=g) / np.sqrt(C * k * k)).to(torch.bfloat16)
    Ho, Wo = (H + 2 * p - k) // s + 1, (W + 2 * p - k) // s + 1

    y0 = torch.randn(N, Ho, Wo, Co, device="cuda", generator=g)

    def run():
        y = y0.clone() if beta else torch.full((N, Ho, Wo, Co), float("nan"), device="cuda")
        st = torch.zeros(1, dtype=torch.int32, device="cuda")
        B.ddppo_conv2d(x, wg, y, k, s, p, beta=beta, status=st)
        torch.cuda.synchronize()
        assert st.item() == 0
        return y.cpu()

    a, b = _both(run)
    assert not torch.isnan(a).any()
    assert torch.equal(a.view(torch.int32), b.view(torch.int32))


SMALL = dict(num_envs=8, rollout_T=8, minibatches=2)


def _iterations(preset, precision=None):
    kw = dict(SMALL)
    if precision is not None:
        kw["precision"] = precision
    w = Worker(preset, seed=11, **kw)
    try:
        B.ddppo_autotune(w.h, False)  # the same contraction configurations in both runs
        rec = []
        for _ in range(3):
            w.iterate()
            torch.cuda.synchronize()
            rec.append((w.stats.cpu().clone(), w.t["actions"].cpu().clone(), w.t["values"].cpu().clone()))
        P = B.ddppo_num_params(w.h)
        p = torch.zeros(P, device="cuda")
        B.ddppo_get_params(w.h, p)
        torch.cuda.synchronize()
        assert B.ddppo_device_status(w.h) == 0
        return rec, p.cpu()
    finally:
        w.close()


@pytest.mark.parametrize("preset,precision", [("resnet", None), ("wide_256_fp8", None)])
def test_iterations_bit_identical(preset, precision):
    (ra, pa), (rb, pb) = _both(lambda: _iterations(preset, precision))
    for it, (a, b) in enumerate(zip(ra, rb)):
        for x, y in zip(a, b):
            assert torch.equal(x, y), it
    assert torch.equal(pa, pb)
