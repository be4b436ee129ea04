"""The host-buffer entry point over several images runs as a pipeline of
chunks (upload, conceal, read back on three streams).  Its patches must equal
those of the device entry point bit for bit, whatever the order of the block
list (image order, shuffled, blocks of the last image first), for video
volumes (which read the neighbouring frames), for mixed block sizes, for FP32
images, and from pageable or pinned host memory."""
import numpy as np
import pytest

from paper_2204_14193_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

C64 = dict(block=16, border=16, fft=64, rho=0.8, gamma=0.5, iters=60)
C32 = dict(block=8, border=12, fft=32, rho=0.8, gamma=0.5, iters=60)
C16 = dict(block=4, border=6, fft=16, rho=0.8, gamma=0.5, iters=40)
V32 = dict(block=8, border=12, fft=32, rho=0.8, gamma=0.5, iters=60, frames=3)


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2204_14193_gb300 as P
    return P


def _device(P, classes, video, mask, blocks):
    eng = P.Engine(classes)
    n = eng.patch_total(blocks)
    patches = torch.zeros(max(n, 1), dtype=torch.float32, device="cuda")
    eng.run(torch.from_numpy(video).cuda(), torch.from_numpy(mask).cuda(), blocks, patches=patches)
    torch.cuda.synchronize()
    eng.close()
    return patches.cpu().numpy()[:n]


def _host(P, classes, video, mask, blocks, pinned=False, repeat=1):
    eng = P.Engine(classes)
    n = eng.patch_total(blocks)
    if pinned:
        video = torch.from_numpy(video).pin_memory().numpy()
        mask = torch.from_numpy(mask).pin_memory().numpy()
        out = torch.full((max(n, 1),), -1.0).pin_memory().numpy()
    else:
        out = np.full(max(n, 1), -1.0, np.float32)
    for _ in range(repeat):
        eng.run_host(video, mask, blocks, out)
    eng.close()
    return out[:n]


def _frames(seed, T, H, W, b, frac):
    video = synth.make_video(seed, T, H, W)
    blocks = np.concatenate([synth.grid_losses(seed + 1 + t, H, W, b, frac, image=t) for t in range(T)])
    return video, blocks


@pytest.mark.parametrize("pinned", [False, True])
def test_pipeline_image_order(P, pinned):
    video, blocks = _frames(300, 11, 96, 128, 16, 0.25)
    mask = synth.loss_mask(blocks, [16], *video.shape)
    d = _device(P, [C64], video, mask, blocks)
    h = _host(P, [C64], video, mask, blocks, pinned=pinned, repeat=2)
    np.testing.assert_array_equal(h, d)


def test_pipeline_any_block_order(P):
    video, blocks = _frames(310, 9, 96, 128, 16, 0.25)
    mask = synth.loss_mask(blocks, [16], *video.shape)
    rng = np.random.default_rng(311)
    for order in (rng.permutation(len(blocks)), np.argsort(-blocks[:, 0], kind="stable")):
        blk = blocks[order]
        np.testing.assert_array_equal(_host(P, [C64], video, mask, blk), _device(P, [C64], video, mask, blk))


def test_pipeline_video_volumes_read_neighbour_frames(P):
    video, blocks = _frames(320, 10, 80, 96, 8, 0.08)
    mask = synth.loss_mask(blocks, [8], *video.shape)
    np.testing.assert_array_equal(_host(P, [V32], video, mask, blocks), _device(P, [V32], video, mask, blocks))


def test_pipeline_mixed_sizes_and_few_blocks(P):
    T, H, W = 5, 80, 96
    video = synth.make_video(330, T, H, W)
    rng = np.random.default_rng(331)
    rows, occ = [], np.zeros((T, H, W), bool)
    for c, (b, n) in enumerate(((4, 60), (8, 20), (16, 6))):
        placed = 0
        while placed < n:
            t, y, x = int(rng.integers(0, T)), int(rng.integers(0, H // b)) * b, int(rng.integers(0, W // b)) * b
            if occ[t, y:y + b, x:x + b].any():
                continue
            occ[t, y:y + b, x:x + b] = True
            rows.append((t, x, y, c))
            placed += 1
    blocks = np.array(sorted(rows), np.int32)
    classes = [C16, C32, C64]
    mask = synth.loss_mask(blocks, [4, 8, 16], T, H, W)
    np.testing.assert_array_equal(_host(P, classes, video, mask, blocks), _device(P, classes, video, mask, blocks))
    # two blocks: two chunks of one block each
    two = blocks[blocks[:, 3] == 2][:2]
    m2 = synth.loss_mask(two, [4, 8, 16], T, H, W)
    np.testing.assert_array_equal(_host(P, classes, video, m2, two), _device(P, classes, video, m2, two))


def test_pipeline_fp32_images(P):
    video, blocks = _frames(340, 6, 96, 128, 16, 0.25)
    video = (video.astype(np.float32) * 0.75 + 0.125).astype(np.float32)
    mask = synth.loss_mask(blocks, [16], *video.shape)
    np.testing.assert_array_equal(_host(P, [C64], video, mask, blocks, pinned=True),
                                  _device(P, [C64], video, mask, blocks))
