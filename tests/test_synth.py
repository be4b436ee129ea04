"""The seeded input recipe that stands in for the paper's test images: the
generators are deterministic per seed, draw their parameters from the stated
ranges, and the loss patterns have the stated geometry (b-aligned, inside the
image, the requested amount, no shared edges where asked for, no overlap for
mixed sizes)."""
import numpy as np
import pytest

from paper_2204_14193_gb300 import synth


def test_images_are_seeded_and_in_range():
    a = synth.make_image(11, 64, 80)
    b = synth.make_image(11, 64, 80)
    c = synth.make_image(12, 64, 80)
    assert a.dtype == np.uint8 and a.shape == (64, 80)
    np.testing.assert_array_equal(a, b)
    assert np.any(a != c)
    f = synth.make_image(11, 64, 80, u8=False)
    assert f.dtype == np.float32 and f.min() >= 0.0 and f.max() <= 255.0
    # u8 content is the float content rounded (same parameters and noise)
    np.testing.assert_array_equal(a, np.rint(f).astype(np.uint8))


def test_parameters_follow_the_recipe():
    rng = np.random.default_rng(3)
    for _ in range(50):
        p = synth._params(rng, 1080, 1920)
        assert np.all((p["a"] >= 5) & (p["a"] <= 25))
        fmag = np.hypot(p["fx"], p["fy"])
        assert np.all((fmag >= 0.005) & (fmag <= 0.2))
        assert 0 <= p["theta"] <= np.pi and -60 <= p["h"] <= 60
        assert np.all(np.abs(p["omega"]) <= 0.3) and abs(p["drift"]) <= 2


def test_video_frames_drift_smoothly():
    v = synth.make_video(5, 3, 96, 128, u8=False)
    d01 = np.abs(v[1] - v[0]).mean()
    assert d01 > 0.5                      # the content moves
    assert d01 < np.abs(v[0] - synth.make_video(6, 1, 96, 128, u8=False)[0]).mean()


@pytest.mark.parametrize("non_adjacent", [False, True])
def test_grid_losses_geometry(non_adjacent):
    H, W, b = 512, 512, 16
    blocks = synth.grid_losses(3, H, W, b, 0.25, non_adjacent=non_adjacent, image=2, cls=1)
    assert len(blocks) == 256
    assert np.all(blocks[:, 0] == 2) and np.all(blocks[:, 3] == 1)
    assert np.all(blocks[:, 1] % b == 0) and np.all(blocks[:, 2] % b == 0)
    assert np.all(blocks[:, 1] + b <= W) and np.all(blocks[:, 2] + b <= H)
    cells = {(int(y) // b, int(x) // b) for _i, x, y, _c in blocks}
    assert len(cells) == len(blocks)
    if non_adjacent:
        for r, c in cells:
            assert not ({(r - 1, c), (r + 1, c), (r, c - 1), (r, c + 1)} & cells)


def test_uneven_losses_geometry():
    H, W = 1080, 1920
    blocks = synth.uneven_losses(5000, H, W)
    sizes = np.array([4, 8, 16])[blocks[:, 3]]
    assert np.all(blocks[:, 1] % sizes == 0) and np.all(blocks[:, 2] % sizes == 0)
    assert np.all(blocks[:, 1] + sizes <= W) and np.all(blocks[:, 2] + sizes <= H)
    mask = synth.loss_mask(blocks, [4, 8, 16], 1, H, W)
    assert int(mask.sum()) == int(np.sum(sizes * sizes))          # no overlap
    assert 0.03 <= mask.mean() < 0.03 + 256 / (H * W)              # the target, at most one block over
    counts = np.bincount(blocks[:, 3], minlength=3)
    assert counts.min() >= 0.25 * len(blocks)      # each size drawn about a third of the time
