"""GPU ordered concealment (FSE_FLAG_ORDERED) against the oracle's ordered
concealment: blocks concealed in the caller's order, each reusing the
concealed samples of the earlier blocks in its area (weight beta x Eq. (3)).
The oracle replays every block along the GPU's selections with its own
working image; picks must be epsilon-argmaxes and pixels within the parity
tolerance.  With no block in another's area the result equals independent
concealment bit for bit."""
import numpy as np
import pytest

from oracle import image as oimage
from paper_2204_14193_gb300 import synth
import parity

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

C64 = dict(block=16, border=16, fft=64, rho=0.8, gamma=0.5, iters=60)
C32 = dict(block=8, border=12, fft=32, rho=0.8, gamma=0.5, iters=60)


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2204_14193_gb300 as P
    return P


def _run(P, cls, img, mask, blocks, ordered, beta=0.5, trace=True):
    eng = P.Engine([cls], trace=trace, ordered=ordered, reuse_weight=beta)
    dimg = torch.from_numpy(img).cuda()
    out = dimg.float().contiguous()
    patches = torch.zeros(len(blocks) * cls["block"] ** 2, dtype=torch.float32, device="cuda")
    eng.run(dimg, torch.from_numpy(mask).cuda(), blocks, out=out, patches=patches)
    eng.sync()
    tr = eng.trace() if trace else None
    eng.close()
    return patches.cpu().numpy(), tr


@pytest.mark.parametrize("cls,b", [(C64, 16), (C32, 8)])
def test_ordered_matches_oracle(P, cls, b):
    H, W = 160, 192
    img = synth.make_image(93, H, W)[None]
    blocks = synth.grid_losses(94, H, W, b, 0.3)            # adjacent losses allowed
    rng = np.random.default_rng(95)
    blocks = blocks[rng.permutation(len(blocks))]           # an arbitrary caller order
    mask = synth.loss_mask(blocks, [b], 1, H, W)
    patches, (sel, energy, _) = _run(P, cls, img, mask, blocks, True, beta=0.5)
    I = cls["iters"]
    res, _ = oimage.conceal_ordered(img, mask, blocks, cls, 0.5, forced=[sel[j, :I] for j in range(len(blocks))])
    worst_pix, worst_gap, max_delta, reusing = 0.0, 0.0, 0.0, 0
    for j, (patch, r) in enumerate(res):
        ratio = r.e_sel / np.maximum(r.e_max, 1e-300)
        delta = np.abs(energy[j, :I] - r.e_sel) / np.maximum(r.e_sel, 1e-300)
        assert np.all(1.0 - ratio <= parity.EPS_TIE), j
        assert delta.max() <= parity.DELTA_MAX, (j, delta.max())
        got = patches[j * b * b:(j + 1) * b * b].reshape(b, b)
        worst_pix = max(worst_pix, float(np.abs(got - patch).max()))
        worst_gap = max(worst_gap, float((1.0 - ratio).max()))
        max_delta = max(max_delta, float(delta.max()))
    # how many blocks actually reused a neighbour (the test must exercise it)
    ind = [oimage.conceal_block(img[0], mask[0], int(x), int(y), cls, forced=sel[j, :I])[0]
           for j, (_, x, y, _c) in enumerate(blocks)]
    reusing = sum(not np.array_equal(p, q) for (p, _r), q in zip(res, ind))
    print(f"ordered F={cls['fft']}: {len(blocks)} blocks, {reusing} reuse neighbours, worst pix {worst_pix:.2e}, "
          f"worst gap {worst_gap:.2e}, max delta {max_delta:.2e}")
    assert reusing > len(blocks) // 4
    assert worst_pix <= parity.PIX_TOL


def test_ordered_without_neighbours_is_independent(P):
    H, W = 128, 128
    img = synth.make_image(96, H, W)[None]
    blocks = np.array([[0, 0, 0, 0], [0, 64, 16, 0], [0, 16, 80, 0], [0, 96, 96, 0]], np.int32)
    mask = synth.loss_mask(blocks, [16], 1, H, W)
    a, _ = _run(P, C64, img, mask, blocks, True, trace=False)
    b, _ = _run(P, C64, img, mask, blocks, False, trace=False)
    np.testing.assert_array_equal(a, b)


def test_ordered_needs_the_output_image(P):
    img = synth.make_image(97, 64, 64)[None]
    blocks = np.array([[0, 16, 16, 0]], np.int32)
    mask = synth.loss_mask(blocks, [16], 1, 64, 64)
    eng = P.Engine([C64], ordered=True)
    patches = torch.zeros(256, dtype=torch.float32, device="cuda")
    with pytest.raises(P.FseError) as ei:
        eng.run(torch.from_numpy(img).cuda(), torch.from_numpy(mask).cuda(), blocks, patches=patches)
    assert ei.value.status == 1
    eng.close()
