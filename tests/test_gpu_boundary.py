"""GPU tests of the C-ABI's boundary options: outputs clamped and rounded to
8-bit values (FSE_FLAG_CLAMP_U8), a block list in device memory, the top-two
gap of the selection trace (fse_get_trace_gap) against the oracle's, and the
report of a block whose loss area is not marked lost in the mask."""
import numpy as np
import pytest

import oracle
from oracle import image as oimage
from paper_2204_14193_gb300 import synth
import parity

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

C64 = dict(block=16, border=16, fft=64, rho=0.8, gamma=0.5, iters=120)
C32 = dict(block=8, border=12, fft=32, rho=0.8, gamma=0.5, iters=120)
C16 = dict(block=4, border=6, fft=16, rho=0.8, gamma=0.5, iters=120)


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2204_14193_gb300 as P
    return P


def _saturated_image(seed, H, W):
    """Synthetic content pushed against both ends of the 8-bit range, so that
    the extrapolation overshoots below 0 and above 255."""
    img = synth.make_image(seed, H, W, u8=False).astype(np.float64)
    img = np.clip((img - 128.0) * 3.0 + 128.0, 0, 255)
    return np.rint(img).astype(np.uint8)[None]


def _run(P, classes, img, mask, blocks, **kw):
    eng = P.Engine(classes, **kw)
    n = eng.patch_total(blocks)
    patches = torch.zeros(n, dtype=torch.float32, device="cuda")
    eng.run(torch.from_numpy(img).cuda(), torch.from_numpy(mask).cuda(), blocks, patches=patches)
    torch.cuda.synchronize()
    return eng, patches.cpu().numpy()


def test_clamp_u8_is_round_half_even_of_the_clipped_output(P):
    H, W = 256, 256
    img = _saturated_image(61, H, W)
    blocks = synth.uneven_losses(62, H, W)
    mask = synth.loss_mask(blocks, [4, 8, 16], 1, H, W)
    cls = [C16, C32, C64]
    eng, raw = _run(P, cls, img, mask, blocks)
    eng.close()
    eng, clamped = _run(P, cls, img, mask, blocks, clamp_u8=True)
    eng.close()
    print("outputs below 0:", int(np.sum(raw < 0)), "above 255:", int(np.sum(raw > 255)),
          "halves:", int(np.sum(np.abs(raw - np.floor(raw) - 0.5) < 1e-3)))
    assert np.sum(raw < 0) + np.sum(raw > 255) > 0, "content does not exercise the clamp"
    np.testing.assert_array_equal(clamped, np.rint(np.clip(raw, 0.0, 255.0)).astype(np.float32))


def test_device_block_list_equals_host_list(P):
    H, W = 192, 224
    img = synth.make_image(63, H, W)[None]
    blocks = synth.uneven_losses(64, H, W)
    mask = synth.loss_mask(blocks, [4, 8, 16], 1, H, W)
    cls = [C16, C32, C64]
    eng, host = _run(P, cls, img, mask, blocks)
    dblocks = torch.from_numpy(np.ascontiguousarray(blocks, dtype=np.int32)).cuda()
    dimg, dmask = torch.from_numpy(img).cuda(), torch.from_numpy(mask).cuda()   # held until the launch ran
    patches = torch.zeros(eng.patch_total(blocks), dtype=torch.float32, device="cuda")
    P.fse_extrapolate_batch(eng.h, dimg.data_ptr(), P.FSE_DTYPE_U8, 1, H, W, W, dmask.data_ptr(),
                            dblocks.data_ptr(), len(blocks), None, patches.data_ptr(),
                            torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    eng.close()
    np.testing.assert_array_equal(patches.cpu().numpy(), host)


@pytest.mark.parametrize("classes", [[C64], [C16, C32, C64]])
def test_trace_gap_matches_the_oracle(P, classes):
    """The kernel's top-two gap (e1 - e2) / e1 at every selection equals the
    oracle's along the same selections (guided replay), within the FP32
    energy deviation bound of the parity harness."""
    H, W = 192, 192
    img = synth.make_image(65, H, W)[None]
    if len(classes) == 1:
        blocks = synth.grid_losses(66, H, W, 16, 0.2, non_adjacent=True)
        mask = synth.loss_mask(blocks, [16], 1, H, W)
    else:
        blocks = synth.uneven_losses(66, H, W)
        mask = synth.loss_mask(blocks, [4, 8, 16], 1, H, W)
    eng, _ = _run(P, classes, img, mask, blocks, trace=True)
    sel, energy, _ = eng.trace()
    gap = eng.trace_gap()
    eng.close()
    assert np.all(gap >= 0.0)
    worst = 0.0
    for i, (im, x, y, c) in enumerate(blocks):
        k = classes[int(c)]
        I = k["iters"]
        s, w, _ = oimage.area_inputs(img[0], mask[0], int(x), int(y), k["block"], k["border"], k["fft"], k["rho"])
        r = oracle.cfse(s, w, k["gamma"], I, forced=sel[i, :I])
        e2 = np.where(r.e_sel >= r.e_max, r.e_second, r.e_max)   # largest energy besides the pick
        ref = (r.e_sel - e2) / r.e_sel
        worst = max(worst, float(np.max(np.abs(gap[i, :I] - ref))))
    print("largest |gap - oracle gap|:", worst)
    assert worst <= 2 * parity.DELTA_MAX


def test_unmarked_loss_area_is_reported(P):
    H, W = 128, 128
    img = synth.make_image(67, H, W)[None]
    blocks = np.array([[0, 32, 32, 0], [0, 80, 64, 0]], np.int32)
    mask = synth.loss_mask(blocks[:1], [16], 1, H, W)     # the second block is not marked
    eng, _ = _run(P, [C64], img, mask, blocks)
    with pytest.raises(P.FseError) as e:
        eng.sync()
    assert e.value.status == 1   # FSE_ERR_INVALID_ARG
    # reported once; a correctly marked batch on the same handle is clean
    mask2 = synth.loss_mask(blocks, [16], 1, H, W)
    patches = torch.zeros(512, dtype=torch.float32, device="cuda")
    eng.run(torch.from_numpy(img).cuda(), torch.from_numpy(mask2).cuda(), blocks, patches=patches)
    eng.sync()
    eng.close()
