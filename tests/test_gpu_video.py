"""GPU parity of video-volume classes (frames = 3: the block's frame and its
two neighbours, a 4 x F x F transform grid) against the 3-D FP64 oracle,
alone and mixed with image classes in one launch; blocks in the first and
last frames (one neighbour missing) and co-located losses in consecutive
frames are included."""
import numpy as np
import pytest

from paper_2204_14193_gb300 import synth
import parity

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

V32 = dict(block=8, border=12, fft=32, rho=0.8, gamma=0.5, iters=100, frames=3)
V16 = dict(block=4, border=6, fft=16, rho=0.8, gamma=0.5, iters=60, frames=3)
C64 = dict(block=16, border=16, fft=64, rho=0.8, gamma=0.5, iters=100)


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2204_14193_gb300 as P
    return P


def _run(P, classes, video, mask, blocks):
    eng = P.Engine(classes, trace=True)
    n = eng.patch_total(blocks)
    patches = torch.zeros(max(n, 1), dtype=torch.float32, device="cuda")
    eng.run(torch.from_numpy(np.ascontiguousarray(video)).cuda(), torch.from_numpy(mask).cuda(), blocks,
            patches=patches)
    eng.sync()
    sel, energy, _ = eng.trace()
    eng.close()
    return patches.cpu().numpy()[:n], sel, energy


def _check(video, mask, blocks, classes, patches, sel, energy):
    res, off = [], 0
    for i, blk in enumerate(blocks):
        k = classes[int(blk[3])]
        b = k["block"]
        p = patches[off:off + b * b].astype(np.float64).reshape(b, b)
        off += b * b
        if k.get("frames", 0) > 1:
            res.append(parity.check_block3(video, mask, blk, classes, p, sel[i], energy[i]))
        else:
            res.append(parity.check_block(video[int(blk[0])], mask[int(blk[0])], blk, classes, p, sel[i], energy[i]))
    s = parity.summarize(res)
    print("video parity:", s)
    assert s["ok"], s
    parity.assert_strict_bounds(s)


def test_video_volume_parity(P):
    T, H, W = 5, 96, 128
    video = synth.make_video(71, T, H, W)
    blocks = np.concatenate([synth.grid_losses(72 + t, H, W, 8, 0.05, image=t) for t in range(T)])
    # the same block lost in three consecutive frames
    extra = np.array([[1, 40, 40, 0], [2, 40, 40, 0], [3, 40, 40, 0]], np.int32)
    keep = ~np.any(np.all(blocks[:, None, 1:3] == extra[None, :, 1:3], axis=2), axis=1)
    blocks = np.concatenate([blocks[keep], extra])
    blocks = np.unique(blocks, axis=0)
    mask = synth.loss_mask(blocks, [8], T, H, W)
    patches, sel, energy = _run(P, [V32], video, mask, blocks)
    _check(video, mask, blocks, [V32], patches, sel, energy)


def test_video_mixed_with_image_classes(P):
    T, H, W = 3, 80, 96
    video = synth.make_video(81, T, H, W)
    rows = []
    rng = np.random.default_rng(82)
    occ = np.zeros((T, H, W), bool)
    for c, (b, n) in enumerate(((4, 40), (8, 12), (16, 3))):
        placed = 0
        while placed < n:
            t = int(rng.integers(0, T))
            y = int(rng.integers(0, H // b)) * b
            x = int(rng.integers(0, W // b)) * b
            if occ[t, y:y + b, x:x + b].any():
                continue
            occ[t, y:y + b, x:x + b] = True
            rows.append((t, x, y, c))
            placed += 1
    blocks = np.array(rows, np.int32)
    classes = [V16, V32, C64]
    mask = synth.loss_mask(blocks, [4, 8, 16], T, H, W)
    patches, sel, energy = _run(P, classes, video, mask, blocks)
    _check(video, mask, blocks, classes, patches, sel, energy)


def test_video_class_rejected_where_unsupported(P):
    with pytest.raises(P.FseError) as ei:
        P.Engine([V32], init="learned", init_iters=10)
    assert ei.value.status == 2
    eng = P.Engine([V32], trace=True)
    with pytest.raises(P.FseError) as ei:
        eng.area_model()
    assert ei.value.status == 2
    video = torch.zeros((3, 64, 64), dtype=torch.uint8, device="cuda")
    mask = torch.zeros((3, 64, 64), dtype=torch.uint8, device="cuda")
    mask[1, 16:24, 16:24] = 1
    est = torch.zeros((1, 32 * 32), dtype=torch.float32, device="cuda")
    with pytest.raises(P.FseError) as ei:
        eng.run_init(video, mask, np.array([[1, 16, 16, 0]], np.int32), est,
                     patches=torch.zeros(64, dtype=torch.float32, device="cuda"))
    assert ei.value.status == 2
    eng.close()
