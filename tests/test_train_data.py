"""The training-set construction of the learned initialisation (torch, runs
on the CPU here) builds the same network input as the oracle's definition of
it, and the loss weights follow Eq. (3) on the support."""
import numpy as np
import pytest

from oracle import image as oimage
from oracle import weight as oweight
from paper_2204_14193_gb300 import synth, train_init

torch = pytest.importorskip("torch")


def test_area_tensors_match_oracle_cnn_input():
    H, W = 80, 72
    frames = np.stack([synth.make_image(s, H, W) for s in (1, 2)])
    blocks = np.concatenate([synth.grid_losses(10 + k, H, W, 16, 0.3, image=k) for k in range(2)])
    mask = synth.loss_mask(blocks, [16], 2, H, W)
    x, s, sup, own = train_init.area_tensors(torch.from_numpy(frames), torch.from_numpy(mask), blocks)
    for i, (im, bx, by, _c) in enumerate(blocks):
        ref = oimage.cnn_input(frames[im], mask[im], int(bx), int(by), 16, 16)
        np.testing.assert_array_equal(x[i, 1].numpy(), ref[1])
        np.testing.assert_allclose(x[i, 0].numpy(), ref[0], rtol=1e-6, atol=0)


def test_weight_table_is_eq3():
    w = train_init.weight_table("cpu").double().numpy()
    ref = oweight(48, 48, 0.8, np.ones((48, 48), np.uint8))
    np.testing.assert_allclose(w, ref, rtol=1e-6, atol=0)
