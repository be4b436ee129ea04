"""The learned initialisation in the launch the benchmark times: 64 frames of
3840x2160 u8 video, 10% of the 16x16 blocks lost (207,360 blocks), the
shipped network on the tensor cores, then I = 50 iterations.  Sampled blocks
are checked against the oracles at full size:
  - with zero iterations the output on B is the network's estimate, which
    must match the FP64 network oracle (bf16-rounded weights, input and
    activations) at the CNN tolerances of tests/test_gpu_learned.py;
  - with 50 iterations (traced) the output must match the FSE oracle started
    from that same estimate (guided replay, every C7 criterion).
"""
import numpy as np
import pytest

from oracle import cnn as ocnn
from oracle import image as oimage
from paper_2204_14193_gb300 import synth
import parity

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

C64 = dict(block=16, border=16, fft=64, rho=0.8, gamma=0.5, iters=200)
N_SAMPLE = 32


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2204_14193_gb300 as P
    return P


def _run(eng, vid, dmask, blocks):
    patches = torch.zeros(len(blocks) * 256, dtype=torch.float32, device="cuda")
    eng.run(vid, dmask, blocks, patches=patches)
    eng.sync()
    torch.cuda.synchronize()
    return patches.cpu().numpy()


def test_learned_full_size_sampled(P):
    from paper_2204_14193_gb300 import train_init as T
    w = T.load_weights()
    Tn, H, W = 64, 2160, 3840
    vid = synth.make_video_torch(21, Tn, H, W, device="cuda")
    blocks = np.concatenate([synth.grid_losses(1000 + t, H, W, 16, 0.10, image=t) for t in range(Tn)])
    mask_np = synth.loss_mask(blocks, [16], Tn, H, W)
    dmask = torch.from_numpy(mask_np).cuda()
    n = len(blocks)
    # the network alone (zero iterations): the estimate on B
    eng0 = P.Engine([dict(C64, iters=0)], init="learned", init_iters=0, weights=w)
    est_b = _run(eng0, vid, dmask, blocks).reshape(n, 16, 16)
    eng0.close()
    # the benchmark's learned pipeline: network, then 50 iterations, traced
    eng = P.Engine([C64], trace=True, init="learned", init_iters=50, weights=w)
    out = _run(eng, vid, dmask, blocks)
    sel, energy = eng.trace()[:2]
    eng.close()

    rng = np.random.default_rng(8)
    pick = np.sort(rng.choice(n, N_SAMPLE, replace=False))
    host = {f: vid[f].cpu().numpy() for f in sorted(set(int(blocks[i, 0]) for i in pick))}
    # network estimate against the FP64 network oracle
    x = np.stack([oimage.cnn_input(host[int(blocks[i, 0])], mask_np[int(blocks[i, 0])],
                                   int(blocks[i, 1]), int(blocks[i, 2]), 16, 16) for i in pick])
    ref = 255.0 * ocnn.forward(w.astype(np.float64), x.astype(np.float32).astype(np.float64))
    ref_b = ref[:, 16:32, 16:32]
    got = est_b[pick].astype(np.float64)
    rms = np.sqrt(np.mean(ref ** 2))
    err = np.abs(got - ref_b)
    print("full-size learned estimate: rms", rms, "max", err.max(), "p99.9", np.quantile(err, 0.999))
    assert err.max() <= 2.0 ** -6 * rms
    assert np.quantile(err, 0.999) <= 2.0 ** -9 * rms
    # the iterations from that estimate (kept on B, zero elsewhere)
    res = []
    for i in pick:
        bk = blocks[i].copy()
        f = int(bk[0])
        bk[0] = 0
        est = np.zeros((48, 48))
        est[16:32, 16:32] = est_b[i]
        p = out[256 * i:256 * (i + 1)].reshape(16, 16).astype(np.float64)
        res.append(parity.check_block(host[f], mask_np[f], bk, [C64], p, sel[i], energy[i],
                                      est=est, iters=50))
    s = parity.summarize(res)
    print("full-size learned pipeline sample:", s)
    assert s["ok"], s
    parity.assert_strict_bounds(s)
