"""Pins of the oracle's ordered concealment (blocks concealed in order, the
samples concealed so far reused as support at weight beta times Eq. (3))."""
import numpy as np
import pytest

from oracle import image as oimage
from paper_2204_14193_gb300 import synth

C = dict(block=8, border=8, fft=32, rho=0.8, gamma=0.5, iters=30)


def test_non_adjacent_blocks_are_independent():
    """No block lies in another's area: ordered = independent concealment."""
    img = synth.make_image(91, 96, 96, u8=False)[None]
    blocks = np.array([[0, 8, 8, 0], [0, 48, 8, 0], [0, 8, 56, 0], [0, 64, 64, 0]], np.int32)
    mask = synth.loss_mask(blocks, [8], 1, 96, 96)
    res, _ = oimage.conceal_ordered(img, mask, blocks, C, 0.5)
    for (patch, _r), (_, x, y, _c) in zip(res, blocks):
        ref, _ = oimage.conceal_block(img[0], mask[0], int(x), int(y), C)
        np.testing.assert_array_equal(patch, ref)


def test_first_block_is_independent_and_beta_weights():
    """The first block sees no concealed samples; the second sees the first
    block's concealed samples at beta times Eq. (3)."""
    img = synth.make_image(92, 64, 64, u8=False)[None]
    blocks = np.array([[0, 24, 24, 0], [0, 32, 24, 0]], np.int32)   # side by side
    mask = synth.loss_mask(blocks, [8], 1, 64, 64)
    res, work = oimage.conceal_ordered(img, mask, blocks, C, 0.25)
    ref0, _ = oimage.conceal_block(img[0], mask[0], 24, 24, C)
    np.testing.assert_array_equal(res[0][0], ref0)
    np.testing.assert_array_equal(work[0, 24:32, 24:32], ref0)
    reused = np.zeros((64, 64), bool)
    reused[24:32, 24:32] = True
    s, w, off = oimage.area_inputs_ordered(work[0], mask[0], reused, 32, 24, 8, 8, 32, 0.8, 0.25)
    full = oimage.area_inputs(img[0], np.zeros_like(mask[0]), 32, 24, 8, 8, 32, 0.8)[1]
    # area of block 1 starts at (y, x) = (16, 24); block 0 occupies area rows 8..15, columns 0..7
    a = w[off:off + 24, off:off + 24]
    fa = full[off:off + 24, off:off + 24]
    np.testing.assert_allclose(a[8:16, 0:8], 0.25 * fa[8:16, 0:8], rtol=1e-15, atol=0)
    assert np.all(a[8:16, 8:16] == 0)                           # its own B
    np.testing.assert_array_equal(a[0:8, :], fa[0:8, :])          # ordinary support
    np.testing.assert_array_equal(s[off + 8:off + 16, off:off + 8], ref0)
