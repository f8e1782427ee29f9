"""GPU parity of the implicit-im2col convolution (4-D TMA gathers inside the tcgen05 GEMM).

Reference: float64 convolution (torch.nn.functional.conv2d on the CPU, itself pinned to
the loop definition in test_oracle_rl.py) of exactly the bf16 values the kernel reads;
the only difference is the kernel's fp32 accumulation: within 4e-5 sqrt(K).
"""
import numpy as np
import pytest
import torch
import torch.nn.functional as F

from paper_1911_00357_gb300 import binding as B

pytestmark = pytest.mark.gpu

# (N, H, W, C, Cout, k, s, p): the encoder's layer shapes plus ragged and odd cases
SHAPES = [
    (3, 32, 32, 32, 32, 3, 1, 1),     # C = 32: 64-byte swizzle, 4 output rows per tile
    (2, 32, 32, 32, 64, 3, 2, 1),     # stride 2
    (5, 16, 16, 64, 64, 3, 1, 1),     # C = 64: 128-byte swizzle
    (3, 16, 16, 64, 128, 3, 2, 1),    # tiles span 2 images, ragged last tile
    (9, 8, 8, 128, 128, 3, 1, 1),
    (7, 8, 8, 128, 256, 3, 2, 1),     # 4x4 outputs: 8 images per tile
    (6, 4, 4, 256, 128, 3, 1, 1),     # compression conv shape
    (4, 16, 16, 64, 128, 1, 2, 0),    # 1x1 stride-2 shortcut
    (2, 64, 64, 32, 32, 3, 1, 1),     # 64-wide rows
    (3, 32, 32, 96, 64, 3, 1, 1),     # C = 96: 32-channel K-blocks
    (33, 8, 8, 256, 256, 3, 1, 1),    # many tiles
]


@pytest.mark.parametrize("N,H,W,C,Co,k,s,p", SHAPES)
def test_implicit_conv_parity(N, H, W, C, Co, k, s, p):
    g = torch.Generator(device="cuda").manual_seed(N * 131 + C * 7 + Co + k + s)
    x = torch.randn(N, H, W, C, device="cuda", generator=g).to(torch.bfloat16)
    wt = (torch.randn(Co, C, k, k, device="cuda", generator=g) / np.sqrt(C * k * k)).to(torch.bfloat16)
    wg = wt.permute(0, 2, 3, 1).contiguous().reshape(Co, k * k * C)   # K ordered (ky, kx, c)
    Ho, Wo = (H + 2 * p - k) // s + 1, (W + 2 * p - k) // s + 1
    y = torch.full((N, Ho, Wo, Co), float("nan"), device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    B.ddppo_conv2d(x, wg, y, k, s, p, status=st)
    torch.cuda.synchronize()
    assert st.item() == 0
    ref = F.conv2d(x.double().cpu().permute(0, 3, 1, 2), wt.double().cpu(), stride=s, padding=p)
    ref = ref.permute(0, 2, 3, 1)
    err = (y.double().cpu() - ref).abs().max().item()
    assert err <= 4e-5 * np.sqrt(k * k * C), err


def test_unsupported_shape_is_rejected():
    x = torch.zeros(2, 15, 15, 32, device="cuda", dtype=torch.bfloat16)   # 15-wide output
    w = torch.zeros(32, 9 * 32, device="cuda", dtype=torch.bfloat16)
    y = torch.zeros(2, 15, 15, 32, device="cuda")
    with pytest.raises(B.DDPPOError) as ei:
        B.ddppo_conv2d(x, w, y, 3, 1, 1)
    assert ei.value.code == -2
