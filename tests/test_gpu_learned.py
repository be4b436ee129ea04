"""GPU tests of the warm start and the learned initialisation.

Warm start (fse_extrapolate_batch_init): the caller's per-block estimates
are the oracle's input too (seeded noisy stand-ins), so the guided replay of
the parity harness applies unchanged on the residual.

Learned initialisation: the network output on the lost block is compared
with the FP64 network oracle (bf16-rounded weights, input and activations)
at the CNN tolerances; the whole pipeline is checked for consistency with
the warm start fed by the standalone network forward on the same input.
"""
import numpy as np
import pytest

from oracle import cnn as ocnn
from oracle import image as oimage
from paper_2204_14193_gb300 import synth
import parity

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

C64 = dict(block=16, border=16, fft=64, rho=0.8, gamma=0.5, iters=100)
C32 = dict(block=8, border=12, fft=32, rho=0.8, gamma=0.5, iters=100)
C16 = dict(block=4, border=6, fft=16, rho=0.8, gamma=0.5, iters=100)


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2204_14193_gb300 as P
    return P


def _warm(P, classes, images, mask, blocks, est, out_image=False):
    eng = P.Engine(classes, trace=True)
    dimg = torch.from_numpy(np.ascontiguousarray(images)).cuda()
    dmask = torch.from_numpy(np.ascontiguousarray(mask)).cuda()
    n = eng.patch_total(blocks)
    patches = torch.zeros(max(n, 1), dtype=torch.float32, device="cuda")
    out = torch.zeros(images.shape, dtype=torch.float32, device="cuda") if out_image else None
    eng.run_init(dimg, dmask, blocks, torch.from_numpy(est).cuda(), out=out, patches=patches)
    torch.cuda.synchronize()
    sel, energy = eng.trace()[:2]
    eng.close()
    return patches.cpu().numpy()[:n], sel, energy, (out.cpu().numpy() if out_image else None)


def test_warm_start_parity_f64(P):
    img = synth.make_image(31, 256, 256)[None]
    blocks = synth.grid_losses(32, 256, 256, 16, 0.25, non_adjacent=True)
    mask = synth.loss_mask(blocks, [16], 1, 256, 256)
    est = synth.noisy_estimates(33, img, blocks, [C64])
    patches, sel, energy, out = _warm(P, [C64], img, mask, blocks, est, out_image=True)
    s = parity.summarize(parity.check_batch(img, mask, blocks, [C64], patches, sel, energy, ests=est))
    print("warm start parity:", s)
    assert s["ok"], s
    parity.assert_strict_bounds(s)
    for i, (_, x, y, _c) in enumerate(blocks[:8]):
        np.testing.assert_array_equal(out[0, y:y + 16, x:x + 16].ravel(), patches[256 * i:256 * (i + 1)])


def test_warm_start_parity_uneven(P):
    """Three classes in one launch; estimates at the largest area's stride."""
    img = synth.make_image(34, 384, 384)[None]
    blocks = synth.uneven_losses(35, 384, 384)
    cls = [C16, C32, C64]
    mask = synth.loss_mask(blocks, [4, 8, 16], 1, 384, 384)
    est = synth.noisy_estimates(36, img, blocks, cls, sigma=5.0)
    patches, sel, energy, _ = _warm(P, cls, img, mask, blocks, est)
    s = parity.summarize(parity.check_batch(img, mask, blocks, cls, patches, sel, energy, ests=est))
    print("warm start parity (uneven):", s)
    assert s["ok"], s
    parity.assert_strict_bounds(s)


def _learned_scene():
    img = synth.make_image(41, 256, 256)[None]
    blocks = synth.grid_losses(42, 256, 256, 16, 0.25, non_adjacent=True)
    mask = synth.loss_mask(blocks, [16], 1, 256, 256)
    return img, mask, blocks


def _learned(P, img, mask, blocks, cls, weights, init_iters, trace=False):
    eng = P.Engine([cls], trace=trace, init="learned", init_iters=init_iters, weights=weights)
    dimg = torch.from_numpy(img).cuda()
    dmask = torch.from_numpy(mask).cuda()
    patches = torch.zeros(eng.patch_total(blocks), dtype=torch.float32, device="cuda")
    eng.run(dimg, dmask, blocks, patches=patches)
    eng.sync()                       # raises on an expired device-side wait
    torch.cuda.synchronize()
    tr = eng.trace() if trace else None
    eng.close()
    return patches.cpu().numpy(), tr


@pytest.mark.parametrize("geom", ["b16d16", "b8d12", "b16d16_f32"])
def test_learned_estimate_matches_network_oracle(P, geom):
    """Zero FSE iterations: the output on each block is the network's estimate
    (16x16 blocks with a 16-sample border: the tensor-core kernel on B;
    other geometries: the whole-area network in chunks)."""
    img, mask, blocks = _learned_scene()
    w = P.he_init(43)
    if geom == "b16d16_f32":   # FP32 samples (not integers) through the same kernel
        img = (img.astype(np.float32) + synth.make_image(47, 256, 256, u8=False)[None] * 0.25) * 0.8
    if geom.startswith("b16d16"):
        cls, b, d = dict(C64, iters=0), 16, 16
    else:
        cls, b, d = dict(C32, iters=0), 8, 12
        blocks = synth.grid_losses(46, 256, 256, 8, 0.2, non_adjacent=True)
        mask = synth.loss_mask(blocks, [8], 1, 256, 256)
    patches, _ = _learned(P, img, mask, blocks, cls, w, 0)
    x = np.stack([oimage.cnn_input(img[0], mask[0], int(bx), int(by), b, d) for _, bx, by, _c in blocks])
    # the input's bf16 rounding is decided on the kernel's FP32 value s * (1/255)
    # (the same decision on both sides; it matters for non-integer samples)
    M = b + 2 * d
    for i, (_, bx, by, _c) in enumerate(blocks):
        ys = np.clip(np.arange(by - d, by - d + M), 0, img.shape[1] - 1)
        xs = np.clip(np.arange(bx - d, bx - d + M), 0, img.shape[2] - 1)
        s32 = img[0][np.ix_(ys, xs)].astype(np.float32) * np.float32(1.0 / 255.0)
        x[i, 0] = np.where(x[i, 1] > 0, s32, 0.0)
    ref = 255.0 * ocnn.forward(w.astype(np.float64), x.astype(np.float32).astype(np.float64))
    ref_b = ref[:, d:d + b, d:d + b].reshape(len(blocks), -1)
    got = patches.reshape(len(blocks), -1).astype(np.float64)
    rms = np.sqrt(np.mean(ref ** 2))
    err = np.abs(got - ref_b)
    print("learned estimate: rms", rms, "max", err.max(), "p99.9", np.quantile(err, 0.999))
    assert err.max() <= 2.0 ** -6 * rms
    assert np.quantile(err, 0.999) <= 2.0 ** -9 * rms


def test_learned_pipeline_equals_warm_start_from_network(P):
    """The captured learned pipeline (network, its output kept on B as the
    estimate, then init_iters FSE iterations) gives what the warm start gives
    on the standalone network forward of the same input, cropped to B."""
    img, mask, blocks = _learned_scene()
    w = P.he_init(44)
    b, d, M = 16, 16, 48
    learned, _ = _learned(P, img, mask, blocks, dict(C64, iters=200), w, 60)
    sup = np.stack([oimage.cnn_input(img[0], mask[0], int(bx), int(by), b, d)[1] for _, bx, by, _c in blocks])
    vals = np.zeros_like(sup, dtype=np.float32)
    for i, (_, bx, by, _c) in enumerate(blocks):
        ys = np.clip(np.arange(by - d, by - d + M), 0, 255)
        xs = np.clip(np.arange(bx - d, bx - d + M), 0, 255)
        vals[i] = img[0][np.ix_(ys, xs)].astype(np.float32) * np.float32(1.0 / 255.0)
    x = np.stack([np.where(sup > 0, vals, np.float32(0)), sup.astype(np.float32)], axis=1).astype(np.float32)
    net = P.Cnn(M, M, max_batch=len(blocks))
    net.set_params(w)
    y = net.forward(torch.from_numpy(np.ascontiguousarray(x)).cuda())
    est = torch.zeros_like(y)
    est[:, d:d + b, d:d + b] = y[:, d:d + b, d:d + b] * 255.0
    est = est.reshape(len(blocks), M * M).contiguous()
    net.close()
    eng = P.Engine([dict(C64, iters=60)])
    patches = torch.zeros(len(blocks) * b * b, dtype=torch.float32, device="cuda")
    eng.run_init(torch.from_numpy(img).cuda(), torch.from_numpy(mask).cuda(), blocks, est, patches=patches)
    torch.cuda.synchronize()
    eng.close()
    # the two network implementations (tensor-core kernel on B, chunked
    # whole-area kernels) accumulate in different orders: CNN tolerances
    diff = np.abs(patches.cpu().numpy() - learned)
    rms = float(torch.sqrt((est ** 2).sum() / (len(blocks) * b * b)))
    print("learned vs warm start: max", diff.max(), "p99.9", np.quantile(diff, 0.999), "rms", rms)
    assert diff.max() <= 2.0 ** -6 * rms
    assert np.quantile(diff, 0.999) <= 2.0 ** -9 * rms


def test_learned_trace_stride_follows_init_iters(P):
    img, mask, blocks = _learned_scene()
    patches, tr = _learned(P, img, mask, blocks, dict(C64, iters=20), P.he_init(45), 90, trace=True)
    sel, energy = tr[0], tr[1]
    assert sel.shape == (len(blocks), 90)
    assert np.all((sel >= 0) & (sel < 64 * 64))
    assert np.all(np.isfinite(patches))


def test_learned_without_weights_is_rejected(P):
    img, mask, blocks = _learned_scene()
    eng = P.Engine([C64], init="learned", init_iters=10)
    patches = torch.zeros(eng.patch_total(blocks), dtype=torch.float32, device="cuda")
    with pytest.raises(P.FseError) as ei:
        eng.run(torch.from_numpy(img).cuda(), torch.from_numpy(mask).cuda(), blocks, patches=patches)
    assert ei.value.status == 6
    eng.close()
    plain = P.Engine([C64])
    with pytest.raises(P.FseError) as ei:
        plain.load_init_weights(P.he_init(1))
    assert ei.value.status == 1
    plain.close()


def test_argument_errors(P):
    img, mask, blocks = _learned_scene()
    dimg, dmask = torch.from_numpy(img).cuda(), torch.from_numpy(mask).cuda()
    eng = P.Engine([C64])
    short = torch.zeros((len(blocks), 47 * 47), dtype=torch.float32, device="cuda")
    patches = torch.zeros(len(blocks) * 256, dtype=torch.float32, device="cuda")
    with pytest.raises(P.FseError) as ei:       # estimate stride below M*M
        eng.run_init(dimg, dmask, blocks, short, patches=patches)
    assert ei.value.status == 1
    eng.run(dimg, dmask, blocks, patches=patches)
    with pytest.raises(P.FseError) as ei:       # area model needs a trace handle
        eng.area_model()
    assert ei.value.status == 1
    eng.sync()
    eng.close()
