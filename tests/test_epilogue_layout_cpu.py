"""Shared-memory layouts and store coordinates of the tcgen05 contraction's epilogue,
checked on the CPU (the index arithmetic is restated here from the kernel's definition).

Tensor-store path: each epilogue warp stages its 32 x 32 block with lane l owning row l;
fp32 rows are 128 bytes, 16-byte chunk c at c ^ (l & 7); bf16 rows are 64 bytes, chunk c at
c ^ ((l >> 1) & 3). A tensor copy with SWIZZLE_128B / SWIZZLE_64B reads a 1024-byte-aligned
buffer with address bits [4:6] / [4:5] XORed with bits [7:9] / [7:8]; the staged layout must
be exactly that swizzle of the row-major block, cover the block once, and let the warp's
16-byte stores run without bank conflicts (each group of 8 lanes, one shared-memory
wavefront, touches 8 distinct 16-byte bank groups).

Transpose path: element (row i, column j) at word i * 32 + (j ^ i); the row writes (lane =
row) and the column reads (lane = column) each hit 32 distinct banks.

Row halo: the warp's 3-D store [images, H W, C] at pixel (tm mod tpi) R W + 32 q of image
tm / tpi must write exactly the tile's output pixels, and every output pixel of the
convolution exactly once.
"""
import pytest

from paper_1911_00357_gb300 import binding as B


def swizzle(addr, span):
    # the tensor copy's swizzle on shared-memory address bits: span 128 -> bits [4:6] ^= [7:9],
    # span 64 -> bits [4:5] ^= [7:8]
    mask = 7 if span == 128 else 3
    return addr ^ (((addr >> 7) & mask) << 4)


def staged_fp32(lane, c):
    return lane * 128 + ((c ^ (lane & 7)) << 4)


def staged_bf16(lane, c):
    return lane * 64 + ((c ^ ((lane >> 1) & 3)) << 4)


@pytest.mark.parametrize("row_bytes,chunks,staged,span", [(128, 8, staged_fp32, 128),
                                                          (64, 4, staged_bf16, 64)])
def test_staging_is_the_tensor_copy_swizzle(row_bytes, chunks, staged, span):
    seen = set()
    for lane in range(32):
        for c in range(chunks):
            off = staged(lane, c)
            assert off == swizzle(lane * row_bytes + c * 16, span)
            assert 0 <= off < 32 * row_bytes and off % 16 == 0
            seen.add(off)
    assert len(seen) == 32 * chunks  # the block is covered once


@pytest.mark.parametrize("chunks,staged", [(8, staged_fp32), (4, staged_bf16)])
def test_staging_stores_are_conflict_free(chunks, staged):
    # a 16-byte store of 32 lanes runs as 4 wavefronts of 8 lanes; 32 banks x 4 bytes =
    # 8 groups of 16 bytes
    for c in range(chunks):
        for w in range(4):
            groups = {(staged(lane, c) >> 4) & 7 for lane in range(8 * w, 8 * w + 8)}
            assert len(groups) == 8


def test_transpose_layout_is_conflict_free_both_ways():
    idx = lambda i, j: i * 32 + (j ^ i)
    assert sorted(idx(i, j) for i in range(32) for j in range(32)) == list(range(1024))
    for j in range(32):  # row writes: lane = row i, element j
        assert len({idx(lane, j) % 32 for lane in range(32)}) == 32
    for i in range(32):  # column reads: lane = column j, row i
        assert len({idx(i, lane) % 32 for lane in range(32)}) == 32


ROW_HALO = [(2, 16, 16, 32), (3, 20, 8, 16), (2, 35, 32, 32), (5, 8, 16, 24), (3, 32, 32, 32),
            (1, 9, 16, 32), (2, 33, 8, 32)]


@pytest.mark.parametrize("N,H,W,Cout", ROW_HALO)
def test_row_halo_stores_write_each_output_pixel_once(N, H, W, Cout):
    plan = B.ddppo_conv_plan(N, H, W, 32, Cout, 3, 1, 1)
    if plan[1] != 2:
        pytest.skip("not a row-halo shape")
    R = 128 // W
    tpi = (H + R - 1) // R
    assert plan[9] == N * tpi  # tiles
    written = {}
    for tm in range(N * tpi):
        img = tm // tpi
        for q in range(4):
            y0 = (tm - img * tpi) * R * W + q * 32
            for lane in range(32):
                r = q * 32 + lane
                # the tile row's output pixel (as the transpose path computes it)
                yy, x = (tm - img * tpi) * R + r // W, r % W
                pix = y0 + lane
                if yy < H:
                    assert pix == yy * W + x
                # the 3-D store writes pixel indices below H W only
                if pix < H * W:
                    key = (img, pix)
                    assert key not in written
                    written[key] = tm
    assert len(written) == N * H * W
