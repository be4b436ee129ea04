"""Video volumes and ordered concealment in the launches the benchmark times,
checked on sampled blocks against the oracles:
  - video volumes: 30 frames of 1920x1080 u8, 3% of the 8x8 blocks lost
    (29,160 blocks), 3-frame volumes on a 4 x 32 x 32 grid, I = 200;
  - ordered concealment: 64 frames of 3840x2160 u8, 10% of the 16x16 blocks
    lost (207,360 blocks) in image order, reuse weight 0.5, I = 200.  A
    sampled block is checked on its own: its support holds the original
    samples and, where the blocks before it in the list lie in its area,
    the values the GPU concealed there (read back from the output image),
    exactly the inputs the kernel used.
Both launches are also bit-identical with and without the trace."""
import numpy as np
import pytest

import oracle
from oracle import image as oimage
from paper_2204_14193_gb300 import synth
import parity

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

N_SAMPLE = 32


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2204_14193_gb300 as P
    return P


def test_video_volumes_full_size_sampled(P):
    T, H, W, b = 30, 1080, 1920, 8
    cls = dict(block=b, border=12, fft=32, rho=0.8, gamma=0.5, iters=200, frames=3)
    vid = synth.make_video_torch(4040, T, H, W, device="cuda")
    blocks = np.concatenate([synth.grid_losses(6000 + t, H, W, b, 0.03, image=t) for t in range(T)])
    mask_np = synth.loss_mask(blocks, [b], T, H, W)
    dmask = torch.from_numpy(mask_np).cuda()
    n = len(blocks)
    res = {}
    for trace in (False, True):
        eng = P.Engine([cls], trace=trace)
        pt = torch.zeros(n * b * b, dtype=torch.float32, device="cuda")
        eng.run(vid, dmask, blocks, patches=pt)
        eng.sync()
        torch.cuda.synchronize()
        res[trace] = (pt.cpu().numpy(), eng.trace()[:2] if trace else None)
        eng.close()
    np.testing.assert_array_equal(res[False][0], res[True][0])
    sel, energy = res[True][1]
    video = vid.cpu().numpy()
    rng = np.random.default_rng(9)
    out = []
    for i in np.sort(rng.choice(n, N_SAMPLE, replace=False)):
        p = res[True][0][b * b * i:b * b * (i + 1)].reshape(b, b).astype(np.float64)
        out.append(parity.check_block3(video, mask_np, blocks[i], [cls], p, sel[i], energy[i]))
    s = parity.summarize(out)
    print("full-size video volume sample:", s)
    assert s["ok"], s
    parity.assert_strict_bounds(s)


def test_ordered_full_size_sampled(P):
    T, H, W, b, beta = 64, 2160, 3840, 16, 0.5
    cls = dict(block=b, border=16, fft=64, rho=0.8, gamma=0.5, iters=200)
    vid = synth.make_video_torch(21, T, H, W, device="cuda")
    blocks = np.concatenate([synth.grid_losses(1000 + t, H, W, b, 0.10, image=t) for t in range(T)])
    mask_np = synth.loss_mask(blocks, [b], T, H, W)
    dmask = torch.from_numpy(mask_np).cuda()
    n = len(blocks)
    res = {}
    for trace in (False, True):
        eng = P.Engine([cls], trace=trace, ordered=True, reuse_weight=beta)
        out = torch.zeros(vid.shape, dtype=torch.float32, device="cuda")
        pt = torch.zeros(n * b * b, dtype=torch.float32, device="cuda")
        eng.run(vid, dmask, blocks, out=out, patches=pt)
        eng.sync()
        torch.cuda.synchronize()
        res[trace] = (pt.cpu().numpy(), eng.trace()[:2] if trace else None, out)
        eng.close()
    np.testing.assert_array_equal(res[False][0], res[True][0])
    patches, (sel, energy), out = res[True]
    rng = np.random.default_rng(10)
    pick = np.sort(rng.choice(n, N_SAMPLE, replace=False))
    worst_pix, worst_gap, max_delta, reusing = 0.0, 0.0, 0.0, 0
    d, M, I = cls["border"], b + 2 * cls["border"], cls["iters"]
    for j in pick:
        im, x, y, _c = (int(v) for v in blocks[j])
        frame = vid[im].cpu().numpy().astype(np.float64)
        concealed = out[im].cpu().numpy().astype(np.float64)
        reused = np.zeros((H, W), dtype=bool)
        work = frame.copy()
        # earlier blocks of the list whose B meets this block's area
        same = np.nonzero(blocks[:j, 0] == im)[0]
        near = same[(np.abs(blocks[same, 1] - x) < M) & (np.abs(blocks[same, 2] - y) < M)]
        for i in near:
            xi, yi = int(blocks[i, 1]), int(blocks[i, 2])
            reused[yi:yi + b, xi:xi + b] = True
            work[yi:yi + b, xi:xi + b] = concealed[yi:yi + b, xi:xi + b]
        reusing += int(len(near) > 0)
        s, w, off = oimage.area_inputs_ordered(work, mask_np[im], reused, x, y, b, d, 64, cls["rho"], beta)
        r = oracle.cfse(s, w, cls["gamma"], I, forced=sel[j, :I].astype(np.int32))
        ratio = r.e_sel / np.maximum(r.e_max, 1e-300)
        delta = np.abs(energy[j, :I] - r.e_sel) / np.maximum(r.e_sel, 1e-300)
        assert np.all(1.0 - ratio <= parity.EPS_TIE), j
        assert delta.max() <= parity.DELTA_MAX, (j, delta.max())
        r0 = off + d
        got = patches[j * b * b:(j + 1) * b * b].reshape(b, b)
        worst_pix = max(worst_pix, float(np.abs(got - r.g.real[r0:r0 + b, r0:r0 + b]).max()))
        worst_gap = max(worst_gap, float((1.0 - ratio).max()))
        max_delta = max(max_delta, float(delta.max()))
    print(f"full-size ordered sample: {len(pick)} blocks, {reusing} reuse neighbours, worst pix "
          f"{worst_pix:.2e}, worst gap {worst_gap:.2e}, max delta {max_delta:.2e}")
    assert reusing > 0
    assert worst_pix <= parity.PIX_TOL
