"""GPU parity of reduced-precision residual storage (FSE_FLAG_FIXED_W): after
FSE_FIXED_W_FROM FP32 updates the kernel holds W as 16-bit fixed-point codes
of W / W[0,0].  Two bars:
  - the C7 criteria against the oracle of the same form (oracle.cfse with
    wfix_from): 1e-2 pixels under guided replay, the divergence bound, and
    picks and energies within the mode's own band (parity.EPS_FIX,
    parity.DELTA_FIX: the kernel decides its codes from FP32 W, the oracle
    from FP64 W, so a few codes differ by one step);
  - the 1e-2 pixel bar against the exact oracle (Algorithm 1 in FP64)
    replayed along the GPU's selections.
Batches of at most FSE_FIXED_W_FROM + 1 iterations never read the codes and
match the FP32 kernel bit for bit.
"""
import numpy as np
import pytest

from paper_2204_14193_gb300 import synth
import parity

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

C64 = dict(block=16, border=16, fft=64, rho=0.8, gamma=0.5, iters=200)
MAX_WIDE_FIX = 1e-3   # of all picks of a batch


@pytest.fixture(scope="module")
def fse():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2204_14193_gb300 as P
    return P


def run(P, classes, images, mask, blocks, fixed_w=True, trace=True, out_image=False):
    eng = P.Engine(classes, trace=trace, fixed_w=fixed_w)
    dimg = torch.from_numpy(np.ascontiguousarray(images)).cuda()
    dmask = torch.from_numpy(np.ascontiguousarray(mask)).cuda()
    n = eng.patch_total(blocks)
    patches = torch.zeros(max(n, 1), dtype=torch.float32, device="cuda")
    out = torch.zeros(images.shape, dtype=torch.float32, device="cuda") if out_image else None
    eng.run(dimg, dmask, blocks, out=out, patches=patches)
    torch.cuda.synchronize()
    tr = eng.trace()[:2] if trace else None
    res = (patches.cpu().numpy()[:n], tr, out.cpu().numpy() if out_image else None)
    eng.close()
    return res


def check(P, images, mask, blocks, classes, patches, tr):
    res = parity.check_batch(images, mask, blocks, classes, patches, tr[0], tr[1],
                             wfix_from=P.FSE_FIXED_W_FROM)
    s = parity.summarize(res)
    print("fixed-point parity:", s)
    assert s["ok"], s
    # picks outside the FP32 path's 1e-5 band: 2 of 51,200 measured
    parity.assert_strict_bounds(s, max_wide=MAX_WIDE_FIX)
    assert s["exact_pix"] <= parity.PIX_TOL, s
    return s


def test_fixw_512_u8_256_blocks_i200(fse):
    """512x512 8-bit image, 25% of 16x16 blocks lost (non-adjacent), I=200."""
    img = synth.make_image(2, 512, 512)[None]
    blocks = synth.grid_losses(3, 512, 512, 16, 0.25, non_adjacent=True)
    mask = synth.loss_mask(blocks, [16], 1, 512, 512)
    patches, tr, out = run(fse, [C64], img, mask, blocks, out_image=True)
    check(fse, img, mask, blocks, [C64], patches, tr)
    for i, (_, x, y, _c) in enumerate(blocks[:16]):
        np.testing.assert_array_equal(out[0, y:y + 16, x:x + 16].ravel(), patches[256 * i:256 * (i + 1)])


def test_fixw_fp32_area_and_edges(fse):
    """FP32 input (plain loads, no TMA) with supports past the image edges
    and lost diagonal neighbours; I = 100."""
    H, W = 96, 80
    img = synth.make_image(7, H, W, u8=False)[None]
    blocks = np.array([[0, 0, 0, 0], [0, 16, 16, 0], [0, 64, 0, 0], [0, 0, 80, 0],
                       [0, 64, 80, 0], [0, 32, 48, 0], [0, 48, 32, 0]], np.int32)
    mask = synth.loss_mask(blocks, [16], 1, H, W)
    cls = [dict(C64, iters=100)]
    patches, tr, _ = run(fse, cls, img, mask, blocks)
    check(fse, img, mask, blocks, cls, patches, tr)


def test_fixw_switch_boundary_is_the_fp32_kernel(fse):
    """Up to FSE_FIXED_W_FROM + 1 iterations no update reads the codes (the
    last iteration has no update): bit-identical to the FP32 kernel.  One
    and two iterations more read them and still meet both bars."""
    K = fse.FSE_FIXED_W_FROM
    img = synth.make_image(5, 256, 256)[None]
    blocks = synth.grid_losses(6, 256, 256, 16, 0.2, non_adjacent=True)
    mask = synth.loss_mask(blocks, [16], 1, 256, 256)
    for I in (0, 1, K, K + 1):
        cls = [dict(C64, iters=I)]
        a, _, _ = run(fse, cls, img, mask, blocks, fixed_w=True, trace=False)
        b, _, _ = run(fse, cls, img, mask, blocks, fixed_w=False, trace=False)
        np.testing.assert_array_equal(a, b)
    for I in (K + 2, K + 3):
        cls = [dict(C64, iters=I)]
        patches, tr, _ = run(fse, cls, img, mask, blocks)
        check(fse, img, mask, blocks, cls, patches, tr)


def test_fixw_graph_replay_and_uneven_counts(fse):
    """Two calls of one handle (the second replays the captured graph) on
    batches of 1, 151 and 457 blocks (items that are not a multiple of the
    grid) give the same patches as fresh handles."""
    img = synth.make_image(9, 1024, 1024)[None]
    allb = synth.grid_losses(10, 1024, 1024, 16, 0.15, non_adjacent=True)
    mask = synth.loss_mask(allb, [16], 1, 1024, 1024)
    dimg = torch.from_numpy(img).cuda()
    dmask = torch.from_numpy(mask).cuda()
    eng = fse.Engine([C64], fixed_w=True)
    try:
        for n in (1, 151, 457):
            blocks = allb[:n]
            p1 = torch.zeros(256 * n, device="cuda")
            p2 = torch.zeros(256 * n, device="cuda")
            eng.run(dimg, dmask, blocks, patches=p1)
            eng.run(dimg, dmask, blocks, patches=p2)
            torch.cuda.synchronize()
            fresh, _, _ = run(fse, [C64], img, mask, blocks, trace=False)
            np.testing.assert_array_equal(p1.cpu().numpy(), fresh)
            np.testing.assert_array_equal(p2.cpu().numpy(), fresh)
    finally:
        eng.close()


def test_fixw_trace_gap_is_unsupported(fse):
    img = synth.make_image(5, 128, 128)[None]
    blocks = synth.grid_losses(6, 128, 128, 16, 0.2, non_adjacent=True)
    mask = synth.loss_mask(blocks, [16], 1, 128, 128)
    eng = fse.Engine([dict(C64, iters=30)], trace=True, fixed_w=True)
    try:
        p = torch.zeros(256 * len(blocks), device="cuda")
        eng.run(torch.from_numpy(img).cuda(), torch.from_numpy(mask).cuda(), blocks, patches=p)
        with pytest.raises(fse.FseError) as ei:
            eng.trace_gap()
        assert ei.value.status == 2
    finally:
        eng.close()


def test_fixw_warm_start_parity(fse):
    """Warm start (fse_extrapolate_batch_init: the model starts from the
    residual of caller estimates) with the fixed-point spectrum."""
    img = synth.make_image(31, 256, 256)[None]
    blocks = synth.grid_losses(32, 256, 256, 16, 0.25, non_adjacent=True)
    mask = synth.loss_mask(blocks, [16], 1, 256, 256)
    est = synth.noisy_estimates(33, img, blocks, [C64])
    eng = fse.Engine([C64], trace=True, fixed_w=True)
    try:
        n = eng.patch_total(blocks)
        patches = torch.zeros(n, dtype=torch.float32, device="cuda")
        eng.run_init(torch.from_numpy(img).cuda(), torch.from_numpy(mask).cuda(), blocks,
                     torch.from_numpy(est).cuda(), patches=patches)
        torch.cuda.synchronize()
        sel, energy = eng.trace()[:2]
    finally:
        eng.close()
    res = parity.check_batch(img, mask, blocks, [C64], patches.cpu().numpy(), sel, energy, ests=est,
                             wfix_from=fse.FSE_FIXED_W_FROM)
    s = parity.summarize(res)
    print("fixed-point warm start parity:", s)
    assert s["ok"], s
    parity.assert_strict_bounds(s, max_wide=MAX_WIDE_FIX)
    assert s["exact_pix"] <= parity.PIX_TOL, s


def test_fixw_host_pipeline_equals_device_path(fse):
    """The host-buffer pipeline (several chunks) runs the same kernel set:
    bit-identical patches to the device entry point."""
    T, H, W = 6, 256, 320
    video = synth.make_video(41, T, H, W)
    blocks = np.concatenate([synth.grid_losses(42 + t, H, W, 16, 0.2, image=t) for t in range(T)])
    mask = synth.loss_mask(blocks, [16], T, H, W)
    cls = [dict(C64, iters=60)]
    dev, _, _ = run(fse, cls, video, mask, blocks, trace=False)
    eng = fse.Engine(cls, fixed_w=True)
    try:
        out = np.full(eng.patch_total(blocks), -1.0, np.float32)
        eng.run_host(video, mask, blocks, out)
    finally:
        eng.close()
    np.testing.assert_array_equal(out, dev)


def test_fixw_full_size_sampled(fse):
    """The benchmark's headline launch (64 x 3840x2160 u8 frames, 10% 16x16
    losses, F=64, I=200) with FSE_FLAG_FIXED_W: bit-identical with and
    without the trace, and 48 sampled blocks meet both bars."""
    T, H, W = 64, 2160, 3840
    vid = synth.make_video_torch(21, T, H, W, device="cuda")
    blocks = np.concatenate([synth.grid_losses(1000 + t, H, W, 16, 0.10, image=t) for t in range(T)])
    mask_np = synth.loss_mask(blocks, [16], T, H, W)
    dmask = torch.from_numpy(mask_np).cuda()
    n = len(blocks)
    res = {}
    for trace in (False, True):
        eng = fse.Engine([C64], trace=trace, fixed_w=True)
        patches = torch.zeros(n * 256, dtype=torch.float32, device="cuda")
        eng.run(vid, dmask, blocks, patches=patches)
        torch.cuda.synchronize()
        res[trace] = (patches.cpu().numpy(), eng.trace()[:2] if trace else None)
        eng.close()
    np.testing.assert_array_equal(res[False][0], res[True][0])
    rng = np.random.default_rng(6)
    pick = np.sort(rng.choice(n, 48, replace=False))
    host = {f: vid[f].cpu().numpy() for f in sorted(set(int(blocks[i, 0]) for i in pick))}
    sel, energy = res[True][1]
    out = []
    for i in pick:
        bk = blocks[i].copy()
        f = int(bk[0])
        bk[0] = 0
        p = res[True][0][256 * i:256 * (i + 1)].reshape(16, 16).astype(np.float64)
        out.append(parity.check_block(host[f], mask_np[f], bk, [C64], p, sel[i], energy[i],
                                      wfix_from=fse.FSE_FIXED_W_FROM))
    s = parity.summarize(out)
    print("fixed-point full-size sample:", s)
    assert s["ok"], s
    parity.assert_strict_bounds(s, max_wide=MAX_WIDE_FIX)
    assert s["exact_pix"] <= parity.PIX_TOL, s


def test_fixw_after_learned_initialisation(fse):
    """The learned pipeline with reduced-precision storage: the network's
    estimate on B (taken from the same handle configuration with zero
    iterations) starts the fixed-point iterations, which meet both bars."""
    from paper_2204_14193_gb300 import train_init as T
    w = T.load_weights()
    img = synth.make_image(51, 384, 384)[None]
    blocks = synth.grid_losses(52, 384, 384, 16, 0.2, non_adjacent=True)
    mask = synth.loss_mask(blocks, [16], 1, 384, 384)
    dimg, dmask = torch.from_numpy(img).cuda(), torch.from_numpy(mask).cuda()
    n = len(blocks)
    est_b = torch.zeros(n * 256, device="cuda")
    e0 = fse.Engine([dict(C64, iters=0)], init="learned", init_iters=0, weights=w, fixed_w=True)
    e0.run(dimg, dmask, blocks, patches=est_b)
    e0.close()
    eng = fse.Engine([C64], trace=True, init="learned", init_iters=60, weights=w, fixed_w=True)
    out = torch.zeros(n * 256, device="cuda")
    eng.run(dimg, dmask, blocks, patches=out)
    eng.sync()
    torch.cuda.synchronize()
    sel, energy = eng.trace()[:2]
    eng.close()
    est = np.zeros((n, 48 * 48))
    eb = est_b.cpu().numpy().reshape(n, 16, 16)
    for i in range(n):
        a = np.zeros((48, 48))
        a[16:32, 16:32] = eb[i]
        est[i] = a.ravel()
    res = parity.check_batch(img, mask, blocks, [C64], out.cpu().numpy(), sel, energy, ests=est, iters=60,
                             wfix_from=fse.FSE_FIXED_W_FROM)
    s = parity.summarize(res)
    print("fixed-point after learned initialisation:", s)
    assert s["ok"], s
    parity.assert_strict_bounds(s, max_wide=MAX_WIDE_FIX)
    assert s["exact_pix"] <= parity.PIX_TOL, s
