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
    # stride-1 'same' convolutions of 32-channel inputs take the halo path: one input
    # box per tile, every tap a row-shifted view of it; odd widths and sizes that no
    # tile divides
    (3, 15, 15, 32, 32, 3, 1, 1),     # 17-wide anchor rows, tiles straddle rows
    (4, 7, 7, 32, 64, 3, 1, 1),       # 9x9 anchors: one image per tile
    (5, 5, 5, 32, 32, 3, 1, 1),       # 7x7 anchors: two images per tile, ragged last tile
    (3, 12, 20, 32, 32, 3, 1, 1),     # non-square
    (2, 16, 16, 32, 32, 5, 1, 2),     # 5x5 filter, halo of two
    (3, 9, 9, 32, 64, 1, 1, 0),       # 1x1 filter
    # 3x3 filters on rows of 8, 16 or 32 pixels take the row halo: whole rows per tile,
    # the three column taps in one N = 96 MMA, combined by lane shuffles
    (2, 16, 16, 32, 32, 3, 1, 1),     # 8 rows per tile
    (3, 20, 8, 32, 16, 3, 1, 1),      # 16 rows per tile, the last one ragged; Cout 16
    (2, 35, 32, 32, 32, 3, 1, 1),     # 4 rows per tile, 35 rows: ragged last tile
    (5, 8, 16, 32, 24, 3, 1, 1),      # one tile per image, Cout 24
    (3, 8, 16, 64, 32, 3, 1, 1),      # 64 channels: 4-D gather path
    (2, 16, 16, 64, 64, 5, 1, 2),     # 5x5, 64 channels: 4-D gather path
    # one input channel (the stem): patches gathered in shared memory, no im2col matrix
    (3, 128, 128, 1, 32, 7, 2, 3),    # the bench's stem (64x64 outputs, 32 tiles per image)
    (2, 64, 64, 1, 16, 7, 2, 3),      # 16 output channels
    (3, 30, 22, 1, 64, 7, 2, 3),      # 64 output channels, ragged last tile
    (2, 9, 9, 1, 32, 3, 1, 1),        # 3x3 / stride 1: a tile spans images
    (1, 17, 13, 1, 32, 8, 3, 2),      # k^2 = 64: every tap column used
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


# y = beta y + conv(x, w): the accumulating form the encoder backward uses for the
# identity-skip input gradient (halo path: per-row output addresses; gather path)
BETA_SHAPES = [
    (3, 15, 15, 32, 32, 3, 1, 1),     # halo, tiles straddle rows
    (5, 5, 5, 32, 32, 3, 1, 1),       # halo, two images per tile
    (2, 30, 30, 32, 32, 3, 1, 1),     # halo only (no whole rows per 128-pixel tile)
    (3, 32, 32, 32, 32, 3, 1, 1),     # row halo
    (2, 20, 8, 32, 16, 3, 1, 1),      # row halo, ragged last tile, Cout 16
    (3, 16, 16, 64, 64, 3, 1, 1),     # 4-D gather path
    (2, 40, 40, 1, 32, 7, 2, 3),      # one input channel
]


@pytest.mark.parametrize("N,H,W,C,Co,k,s,p", BETA_SHAPES)
def test_implicit_conv_beta_parity(N, H, W, C, Co, k, s, p):
    g = torch.Generator(device="cuda").manual_seed(N * 17 + H + C + Co)
    x = torch.randn(N, H, W, C, device="cuda", generator=g).to(torch.bfloat16)
    wt = (torch.randn(Co, C, k, k, device="cuda", generator=g) / np.sqrt(C * k * k)).to(torch.bfloat16)
    wg = wt.permute(0, 2, 3, 1).contiguous().reshape(Co, k * k * C)
    Ho, Wo = (H + 2 * p - k) // s + 1, (W + 2 * p - k) // s + 1
    y0 = torch.randn(N, Ho, Wo, Co, device="cuda", generator=g)
    y = y0.clone()
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    B.ddppo_conv2d(x, wg, y, k, s, p, beta=0.5, status=st)
    torch.cuda.synchronize()
    assert st.item() == 0
    ref = F.conv2d(x.double().cpu().permute(0, 3, 1, 2), wt.double().cpu(), stride=s, padding=p)
    ref = ref.permute(0, 2, 3, 1) + 0.5 * y0.double().cpu()
    err = (y.double().cpu() - ref).abs().max().item()
    assert err <= 4e-5 * np.sqrt(k * k * C) + 1e-6, err


def test_unsupported_shape_is_rejected():
    # stride 2 (no halo path) with a 15-wide output (no whole rows per 128-pixel tile)
    x = torch.zeros(2, 30, 30, 32, device="cuda", dtype=torch.bfloat16)
    w = torch.zeros(32, 9 * 32, device="cuda", dtype=torch.bfloat16)
    y = torch.zeros(2, 15, 15, 32, device="cuda")
    with pytest.raises(B.DDPPOError) as ei:
        B.ddppo_conv2d(x, w, y, 3, 2, 1)
    assert ei.value.code == -2


# (N, H, W, C, Cout, k, s, p) for the weight gradient: 64-pixel K blocks of whole rows or
# whole images; C = 32 (64-byte swizzled MN-major boxes) and C % 64 == 0 (128-byte);
# 3x3 / stride-1 / 32 -> 32 shapes take the halo weight gradient
WGRAD_SHAPES = [
    (3, 32, 32, 32, 32, 3, 1, 1),     # layer-1 shape: 2 output rows per K block, 4 boxes per tile
    (2, 32, 32, 32, 64, 3, 2, 1),     # stride 2 (16x16 outputs)
    (5, 16, 16, 64, 64, 3, 1, 1),     # 2 boxes (taps) per 128-row tile
    (3, 16, 16, 64, 128, 3, 2, 1),    # 8x8 outputs: one image per K block
    (9, 8, 8, 128, 128, 3, 1, 1),
    (7, 8, 8, 128, 256, 3, 2, 1),     # 4x4 outputs: 4 images per K block, ragged image tail
    (6, 4, 4, 256, 128, 3, 1, 1),     # ragged (tap, channel) tile: 2304 = 18 x 128
    (4, 16, 16, 64, 128, 1, 2, 0),    # 1x1 stride-2 shortcut
    (2, 64, 64, 32, 32, 3, 1, 1),     # 64-wide rows: one row per K block
    (70, 32, 32, 32, 32, 3, 1, 1),    # long reduction (split K)
    # 3x3 / stride 1, 32 -> 32 channels: the halo weight gradient (whole-row units of Wp
    # anchors, three taps per MMA); widths that no 64-pixel block divides
    (3, 15, 15, 32, 32, 3, 1, 1),
    (2, 7, 9, 32, 32, 3, 1, 1),
    (5, 33, 20, 32, 32, 3, 1, 1),
]


@pytest.mark.parametrize("N,H,W,C,Co,k,s,p", WGRAD_SHAPES)
def test_implicit_wgrad_parity(N, H, W, C, Co, k, s, p):
    g = torch.Generator(device="cuda").manual_seed(N * 17 + C * 5 + Co + 3 * k + s)
    x = torch.randn(N, H, W, C, device="cuda", generator=g).to(torch.bfloat16)
    Ho, Wo = (H + 2 * p - k) // s + 1, (W + 2 * p - k) // s + 1
    dy = torch.randn(N, Ho, Wo, Co, device="cuda", generator=g).to(torch.bfloat16)
    dw0 = torch.randn(Co, k * k * C, device="cuda", generator=g)
    dw = dw0.clone()
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    B.ddppo_conv2d_wgrad(x, dy, dw, k, s, p, beta=1.0, status=st)
    torch.cuda.synchronize()
    assert st.item() == 0
    # float64 weight gradient of the same bf16 values through autograd of conv2d
    xd = x.double().cpu().permute(0, 3, 1, 2)
    wd = torch.zeros(Co, C, k, k, dtype=torch.float64, requires_grad=True)
    out = F.conv2d(xd, wd, stride=s, padding=p)
    out.backward(dy.double().cpu().permute(0, 3, 1, 2))
    ref = wd.grad.permute(0, 2, 3, 1).reshape(Co, k * k * C) + dw0.double().cpu()
    red = N * Ho * Wo
    err = (dw.double().cpu() - ref).abs().max().item()
    assert err <= 4e-5 * np.sqrt(red) * 4, err


def test_wgrad_unsupported_shape_is_rejected():
    # stride 2 (no halo path) with a 15-wide output (no whole rows per 64-pixel block)
    x = torch.zeros(2, 30, 30, 32, device="cuda", dtype=torch.bfloat16)
    dy = torch.zeros(2, 15, 15, 32, device="cuda", dtype=torch.bfloat16)
    dw = torch.zeros(32, 9 * 32, device="cuda")
    with pytest.raises(B.DDPPOError) as ei:
        B.ddppo_conv2d_wgrad(x, dy, dw, 3, 2, 1)
    assert ei.value.code == -2
