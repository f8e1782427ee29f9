"""Shared-memory staging geometry of the halo convolution and the halo weight gradient,
checked on the CPU against the reads their MMAs make.

The kernels read shifted views of one staged box. A view that reaches past the rows TMA
wrote reads stale shared memory, and one that reaches past the allocation reads another
stage. This test recomputes, for every tile of a sweep of shapes, the farthest anchor row
each MMA reads (the read pattern is restated here from the kernels' definition). It then
checks the two rules: rows that produce a stored output read only rows the box delivers,
and every read stays inside the rows allocated per ring stage.
"""
import itertools

import pytest

from paper_1911_00357_gb300 import binding as B

TC_BM = 128          # output rows (anchors) per tensor-core tile
SMEM_MAX = 205 * 1024


def _fwd_shapes():
    for (H, W), k, cout, n in itertools.product(
            [(5, 5), (7, 9), (15, 15), (12, 20), (30, 30), (32, 32), (33, 20), (64, 64), (3, 40)],
            [3, 5], [32, 64], [1, 3]):
        if 2 * (k // 2) < min(H, W) + 4:
            yield n, H, W, k, cout


@pytest.mark.parametrize("N,H,W,k,Cout", list(_fwd_shapes()))
def test_halo_forward_reads_stay_in_the_staged_box(N, H, W, k, Cout):
    p = k // 2
    plan = B.ddppo_conv_plan(N, H, W, 32, Cout, k, 1, p)
    if not plan[1]:
        # declined: the resident weights (Cout x k^2 x 32 bf16) or the ring exceed their caps
        assert Cout * k * k * 32 * 2 > 96 * 1024 or W + 2 * p > 256 or H > 200
        return
    Wp, Hh, ni, tpi, rows_box, alloc, delivered, tiles = plan[2:10]
    if plan[1] == 2:
        _check_row_halo(N, H, W, k, Cout, plan)
        return
    assert Wp == W + 2 * p and Hh == H + 2 * p
    assert delivered == rows_box * Wp * (ni if ni else 1)
    assert tiles == ((N + ni - 1) // ni if ni else N * tpi)
    far = (k - 1) * Wp + (k - 1)          # largest tap offset, in anchors
    for tm in range(tiles if ni else tpi):  # the geometry repeats per image when ni == 0
        for m in range(TC_BM):
            if ni:
                # ni whole padded images per tile; anchors run over (image, row, column)
                i, rem = divmod(m, Hh * Wp)
                y, x = divmod(rem, Wp)
                valid = i < ni and tm * ni + i < N and y < H and x < W
                base = m
                if valid:   # every tap stays inside this image's padded block
                    assert rem + far < Hh * Wp
            else:
                a0 = (tm % tpi) * TC_BM
                y, x = divmod(a0 + m, Wp)
                valid = y < H and x < W
                base = a0 % Wp + m         # the tile's first anchor sits at column a0 % Wp
            last = base + far
            assert last < alloc, (tm, m, last, alloc)
            if valid:
                assert last < delivered, (tm, m, last, delivered)


def _check_row_halo(N, H, W, k, Cout, plan):
    # whole image rows per tile: R = 128 / W rows, the box R + 2 rows of W pixels starting
    # one row above the tile; filter row ky reads box pixels m + ky W for tile pixel m, and
    # the column taps are neighbours in the same image row (the epilogue's lane shuffles)
    Wp, Hh, ni, tpi, rows_box, alloc, delivered, tiles = plan[2:10]
    assert k == 3 and W in (8, 16, 32) and Cout <= 32
    R = TC_BM // W
    assert H >= R and Wp == W and Hh == H and ni == 0
    assert rows_box == R + 2 and tpi == (H + R - 1) // R and tiles == N * tpi
    assert delivered == (R + 2) * W and alloc >= delivered and (alloc * 64) % 1024 == 0
    for m in range(TC_BM):
        rr, x = divmod(m, W)
        for ky in range(3):
            rd = m + ky * W                  # box pixel this lane's row of the MMA reads
            assert rd < delivered
            assert rd // W == rr + ky and rd % W == x  # image row y + ky - 1, same column
        # a lane's image row lies within its warp: the shuffles never cross warps
        assert (m // 32) == ((m - x) // 32) == ((m - x + W - 1) // 32)
    # each filter row's view starts on a 512-byte (8-row) swizzle atom
    assert all((ky * W * 64) % 512 == 0 for ky in range(3))


@pytest.mark.parametrize("N,H,W", [(1, 4, 32), (3, 32, 32), (2, 35, 32), (2, 16, 16), (3, 20, 8),
                                   (1, 16, 8)])
def test_row_halo_geometry(N, H, W):
    plan = B.ddppo_conv_plan(N, H, W, 32, 32, 3, 1, 1)
    assert plan[1] == 2
    _check_row_halo(N, H, W, 3, 32, plan)


def test_row_halo_is_declined_where_it_does_not_apply():
    for N, H, W, Cout, k in [(2, 2, 32, 32, 3),     # fewer rows than one tile
                             (2, 30, 30, 32, 3),    # width 30
                             (2, 32, 32, 64, 3),    # 64 output channels
                             (2, 32, 32, 32, 5),    # 5x5 filter
                             (2, 64, 64, 32, 3)]:   # a row wider than a warp
        plan = B.ddppo_conv_plan(N, H, W, 32, Cout, k, 1, k // 2)
        assert plan[1] != 2, (N, H, W, Cout, k)


def _wgrad_shapes():
    for H, W in [(3, 3), (5, 5), (7, 9), (15, 15), (16, 16), (30, 30), (32, 32), (33, 20),
                 (64, 64), (40, 3), (100, 100), (250, 250)]:
        yield H, W


@pytest.mark.parametrize("H,W", list(_wgrad_shapes()))
def test_halo_weight_gradient_reads_stay_in_the_staged_box(H, W):
    plan = B.ddppo_conv_plan(2, H, W, 32, 32, 3, 1, 1)
    if not plan[11]:
        # declined: two ring stages of (RB + 3) + RB rows of 64-byte anchors do not fit
        assert W >= 96
        return
    RB, Wp, x_rows, dz_rows, stages, smem = plan[12:18]
    assert Wp == W + 2 and dz_rows == RB
    assert (RB * Wp) % 16 == 0 and RB * Wp >= 128   # whole 16-anchor K steps, a full M tile
    assert 2 <= stages and smem <= SMEM_MAX
    # per 16-anchor K step a0 and filter row ky the A operand's four atoms read anchors
    # a0 + t + ky Wp + j, t < 16, j < 4 (atom 3 is discarded but still read)
    last = (RB * Wp - 1) + 2 * Wp + 3
    assert last < x_rows * Wp, (last, x_rows, Wp)
    # a dz anchor that carries gradient (x < W) reads the input at column x + kx <= W + 1:
    # the same box row, inside the pitch
    assert (W - 1) + 2 < Wp
    assert RB - 1 + 2 < x_rows


def test_workload_shapes_take_the_halo_paths():
    # the first ResNet stage of the 32-base encoder at 128x128 input (32x32 maps) and of
    # the 64x64 input variants: forward, input gradient and weight gradient on the halo path
    for H in (32, 64):
        plan = B.ddppo_conv_plan(4096, H, H, 32, 32, 3, 1, 1)
        assert plan[1] == (2 if H == 32 else 1) and plan[11] == 1
    assert B.ddppo_conv_plan(64, 32, 32, 32, 64, 3, 1, 1)[1] == 1


def test_unsupported_shapes_are_reported():
    # stride 2 with a 15-wide output: neither halo path nor whole rows per tile
    plan = B.ddppo_conv_plan(2, 30, 30, 32, 32, 3, 2, 1)
    assert plan[0] == 0 and plan[1] == 0 and plan[11] == 0
    # 64 channels: no halo weight gradient (it is specific to 32 -> 32)
    assert B.ddppo_conv_plan(2, 16, 16, 64, 64, 3, 1, 1)[11] == 0
    with pytest.raises(B.DDPPOError):
        B.ddppo_conv_plan(0, 16, 16, 32, 32, 3, 1, 1)
