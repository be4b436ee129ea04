"""Pins of the oracle's warm start (the model starts from an estimate of the
area, Algorithm 1 runs on the residual) and of the learned network's input.

Warm start: conceal_block_init(img, est) runs Algorithm 1 on s - est over the
support and returns est + Re{g} on the lost block.  Pins: est = 0 is plain
concealment; a constant est = c is plain concealment of the shifted image
img - c, shifted back (the weighting and the argmax see the same residual);
an exact est leaves a zero residual, so the model stays zero and the output
is est on the block."""
import numpy as np
import pytest

from oracle import image as oimage
from paper_2204_14193_gb300 import synth

CLS = dict(block=8, border=12, fft=32, rho=0.8, gamma=0.5, iters=40)


def _scene():
    img = synth.make_image(4, 64, 64, u8=False).astype(np.float64)
    blocks = np.array([[0, 24, 20, 0]], np.int32)
    mask = synth.loss_mask(blocks, [8], 1, 64, 64)[0]
    return img, mask


def test_zero_estimate_is_plain_concealment():
    img, mask = _scene()
    M = 8 + 24
    plain, _ = oimage.conceal_block(img, mask, 24, 20, CLS)
    warm, _ = oimage.conceal_block_init(img, mask, 24, 20, CLS, np.zeros((M, M)))
    np.testing.assert_allclose(warm, plain, rtol=0, atol=1e-9)


@pytest.mark.parametrize("c", [37.5, 128.0, 240.0])
def test_constant_estimate_is_shifted_plain_concealment(c):
    img, mask = _scene()
    M = 8 + 24
    warm, _ = oimage.conceal_block_init(img, mask, 24, 20, CLS, np.full((M, M), c))
    plain, _ = oimage.conceal_block(img - c, mask, 24, 20, CLS)
    np.testing.assert_allclose(warm, plain + c, rtol=0, atol=1e-9)


def test_exact_estimate_returns_estimate():
    img, mask = _scene()
    est = img[20 - 12:20 - 12 + 32, 24 - 12:24 - 12 + 32]
    warm, res = oimage.conceal_block_init(img, mask, 24, 20, CLS, est)
    np.testing.assert_array_equal(warm, est[12:20, 12:20])
    assert np.all(res.g == 0)


def test_cnn_input_hand_case():
    """4x4 image, 2x2 block at the top-left corner with a 1-sample border
    (area rows and columns -1..2), one further lost sample at (2, 2)."""
    img = np.arange(16, dtype=np.float64).reshape(4, 4) * 10.0
    mask = np.zeros((4, 4), np.uint8)
    mask[0:2, 0:2] = 1
    mask[2, 2] = 1
    x = oimage.cnn_input(img, mask, 0, 0, 2, 1)
    sup = np.array([[0, 0, 0, 0],
                    [0, 0, 0, 1],
                    [0, 0, 0, 1],
                    [0, 1, 1, 0]], dtype=np.float64)
    np.testing.assert_array_equal(x[1], sup)
    vals = np.array([[0, 0, 0, 0],
                     [0, 0, 0, 20],
                     [0, 0, 0, 60],
                     [0, 80, 90, 0]], dtype=np.float64) / 255.0
    np.testing.assert_array_equal(x[0], vals)
