"""Training and evaluation of the learned initialisation, on the GPU.

The network (4 dilated 3x3 convolutions, 32 channels, bf16 weights and
activations, FP32 accumulation; every forward, backward and Adam step runs in
libfse.so) maps the support of an extrapolation area -- channel 0 the support
samples / 255, channel 1 the support indicator -- to an estimate e of the
whole M x M area.  In use, the frequency selective extrapolation then models
the residual s - e on the support for a few iterations and the output on the
lost block is e + Re{g}.

Training pairs are built from seeded synthetic frames with 10% of the 16x16
grid blocks lost.  The target is the model g that plain extrapolation
(Algorithm 1 from a zero model, I = 200) builds for the same area, over the
whole area (target "model"; the residual s - e the iterations then see is
what the plain model left unexplained plus the network's own error, which
they go on to model); with target "support", the support samples
themselves on the support and the plain extrapolation on the lost block;
with target "correction" (the default, and the reading the library's
learned launch uses), only the lost block counts: there the target is what
the plain extrapolation at I = 200 adds to the one at I = short_iters.  In
use the estimate is kept on the lost block only, the iterations run on the
unchanged support, and the network supplies the detail the short run
misses.  Measured on held-out frames (20k areas): the "model" reading left
the network's error on the lost block uncorrected (20.4 dB at I = 50 against
30.1 dB plain), the "correction" reading gains over plain at I = 50.
Loss weights: lam_b on the lost block; for "model" and "support" also the
weighting function of Eq. (3) on the support (the weight the model fitting
gives the residual there); 0 elsewhere (outside the frame, other lost
samples).
Test frames come from disjoint seeds.  PSNR is taken over all lost samples
against the original frame, with outputs clipped to [0, 255].

Usage (writes <out>/init_cnn_b16_d16.f32 and <out>/init_cnn_b16_d16.json):
    python -m paper_2204_14193_gb300.train_init --out DIR
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time

import numpy as np

B, D, FFT, RHO, GAMMA = 16, 16, 64, 0.8, 0.5
M = B + 2 * D
WEIGHTS_NAME = "init_cnn_b16_d16"
TRAIN_SEED0 = 1_000_000
TEST_SEED0 = 2_000_000


def weights_path() -> str:
    """The trained parameters shipped with the package (FP32, flat layout)."""
    return os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights", WEIGHTS_NAME + ".f32")


def shipped_networks():
    """(k, path) of every shipped network: the one of weights_path() trained
    for k = 50 iterations after it, and <name>_k<k>.f32 for other k."""
    import glob
    import re
    out = [(50, weights_path())] if os.path.exists(weights_path()) else []
    for p in sorted(glob.glob(os.path.join(os.path.dirname(weights_path()), WEIGHTS_NAME + "_k*.f32"))):
        m = re.search(r"_k(\d+)\.f32$", p)
        if m:
            out.append((int(m.group(1)), p))
    return sorted(out)


def load_weights(path: str | None = None) -> np.ndarray:
    from . import FSE_CNN_PARAMS
    p = np.fromfile(path or weights_path(), dtype="<f4")
    if p.size != FSE_CNN_PARAMS:
        raise ValueError(f"{path}: {p.size} parameters, expected {FSE_CNN_PARAMS}")
    return p


def frames_and_losses(seed0: int, n_frames: int, H: int, W: int, loss: float, device="cuda"):
    """n_frames seeded frames (one seed each), their lost blocks and mask."""
    import torch
    from . import synth
    frames = torch.empty((n_frames, H, W), dtype=torch.uint8, device=device)
    blocks = []
    for k in range(n_frames):
        frames[k] = synth.make_video_torch(seed0 + k, 1, H, W, device=device)[0]
        blocks.append(synth.grid_losses(seed0 + k, H, W, B, loss, image=k))
    blocks = np.concatenate(blocks).astype(np.int32)
    mask = synth.grid_mask_torch(blocks, B, n_frames, H, W, device=device)
    return frames, mask, blocks


def area_tensors(frames, mask, blocks):
    """Per-block area tensors on the frames' device: the network input
    x [n, 2, M, M] (float32), the area samples s [n, M, M] (float32, clamped
    at the frame edge), the support indicator and the lost-block indicator."""
    import torch
    dev = frames.device
    T, H, W = frames.shape
    bt = torch.from_numpy(np.asarray(blocks, dtype=np.int64)).to(dev)
    ar = torch.arange(M, device=dev)
    ys = bt[:, 2, None] - D + ar[None, :]            # [n, M]
    xs = bt[:, 1, None] - D + ar[None, :]
    inside = ((ys >= 0) & (ys < H))[:, :, None] & ((xs >= 0) & (xs < W))[:, None, :]
    yc = ys.clamp(0, H - 1)[:, :, None]
    xc = xs.clamp(0, W - 1)[:, None, :]
    im = bt[:, 0, None, None]
    s = frames[im, yc, xc].float()
    lost = mask[im, yc, xc] != 0
    own = torch.zeros((M, M), dtype=torch.bool, device=dev)
    own[D:D + B, D:D + B] = True
    sup = inside & ~lost & ~own[None]
    x0 = torch.where(sup, s * np.float32(1.0 / 255.0), torch.zeros((), device=dev))
    x = torch.stack([x0, sup.float()], dim=1).contiguous()
    return x, s, sup, own.expand_as(sup)


def plain_area_model(frames, mask, blocks, iters: int):
    """Re{g} of plain extrapolation over every block's whole area, [n, M, M]."""
    import torch
    from . import Engine
    eng = Engine([dict(block=B, border=D, fft=FFT, rho=RHO, gamma=GAMMA, iters=iters)], trace=True)
    p = torch.empty(len(blocks) * B * B, dtype=torch.float32, device=frames.device)
    eng.run(frames, mask, blocks, patches=p)
    g = eng.area_model()
    torch.cuda.synchronize()
    eng.close()
    return g.view(len(blocks), M, M)


def plain_patches(frames, mask, blocks, iters: int):
    """Plain extrapolation (zero initial model) of every block, [n, B, B]."""
    import torch
    from . import Engine
    eng = Engine([dict(block=B, border=D, fft=FFT, rho=RHO, gamma=GAMMA, iters=iters)])
    p = torch.empty(len(blocks) * B * B, dtype=torch.float32, device=frames.device)
    eng.run(frames, mask, blocks, patches=p)
    torch.cuda.synchronize()
    eng.close()
    return p.view(len(blocks), B, B)


def learned_patches(frames, mask, blocks, params, init_iters: int):
    import torch
    from . import Engine
    eng = Engine([dict(block=B, border=D, fft=FFT, rho=RHO, gamma=GAMMA, iters=max(init_iters, 0))],
                 init="learned", init_iters=init_iters, weights=params)
    p = torch.empty(len(blocks) * B * B, dtype=torch.float32, device=frames.device)
    eng.run(frames, mask, blocks, patches=p)
    torch.cuda.synchronize()
    eng.close()
    return p.view(len(blocks), B, B)


def truth_patches(frames, blocks):
    import torch
    dev = frames.device
    bt = torch.from_numpy(np.asarray(blocks, dtype=np.int64)).to(dev)
    ar = torch.arange(B, device=dev)
    ys = (bt[:, 2, None] + ar[None, :])[:, :, None]
    xs = (bt[:, 1, None] + ar[None, :])[:, None, :]
    return frames[bt[:, 0, None, None], ys, xs].float()


def psnr(est, truth) -> float:
    mse = float(((est.clamp(0.0, 255.0) - truth) ** 2).mean())
    return 10.0 * math.log10(255.0 ** 2 / max(mse, 1e-12))


def weight_table(device):
    """Eq. (3) on the M x M area (centre (M - 1) / 2), as float32."""
    import torch
    c = 0.5 * (M - 1)
    r = torch.arange(M, dtype=torch.float64, device=device) - c
    dist = torch.sqrt(r[:, None] ** 2 + r[None, :] ** 2)
    return (RHO ** dist).float()


def training_set(frames, mask, blocks, lam_b: float, target: str = "model", short_iters: int = 50):
    """x, target and per-sample loss weight of every training area."""
    import torch
    x, s, sup, own = area_tensors(frames, mask, blocks)
    if target == "model":
        t = plain_area_model(frames, mask, blocks, 200) / 255.0
    elif target == "correction":
        p200 = plain_patches(frames, mask, blocks, 200)
        p50 = plain_patches(frames, mask, blocks, short_iters)
        t = torch.zeros_like(s)
        t[:, D:D + B, D:D + B] = (p200 - p50) / 255.0
    else:
        fse = plain_patches(frames, mask, blocks, 200)
        t = s / 255.0
        t[:, D:D + B, D:D + B] = fse / 255.0
    w = weight_table(frames.device)
    if target == "correction":      # only the lost block's output is used
        lam = torch.zeros_like(s)
    else:
        lam = torch.where(sup, w[None].expand_as(s), torch.zeros((), device=s.device))
    lam[:, D:D + B, D:D + B] = lam_b
    return x, t.contiguous(), lam.contiguous()


def train(x, t, lam, steps: int, batch: int, lr: float, seed: int, init=None, log_every: int = 500,
          checkpoint: str | None = None, checkpoint_every: int = 0, resume: str | None = None, stop_at=None):
    """Adam on random minibatches with a cosine learning-rate decay; returns
    the parameters and the loss history.

    checkpoint / checkpoint_every: every checkpoint_every steps (and at the
    end) the whole state -- parameters, Adam moments and step count, the
    minibatch generator's state, the loop position and the loss history -- is
    written to checkpoint (.npz).  resume: continue from such a file; the run
    then goes on bit for bit as if it had not stopped.  stop_at: end the loop
    after that many steps (a run cut short, to be resumed)."""
    import torch
    from . import Cnn, he_init
    net = Cnn(M, M, max_batch=batch)
    g = torch.Generator(device=x.device)
    g.manual_seed(seed)
    hist, k0 = [], 0
    if resume is not None:
        z = np.load(resume)
        if int(z["steps"]) != steps or int(z["batch"]) != batch or float(z["lr"]) != lr or int(z["seed"]) != seed:
            raise ValueError(f"{resume}: checkpoint of another run (steps, batch, lr or seed differ)")
        net.set_state(z["params"], z["m"], z["v"], int(z["adam_step"]))
        g.set_state(torch.from_numpy(z["rng"]).to(torch.uint8))
        k0 = int(z["k"])
        hist = [tuple(h) for h in z["hist"].tolist()]
    else:
        net.set_params(he_init(seed) if init is None else init)

    def save(k):
        p, m, v, st = net.get_state()
        np.savez(checkpoint, params=p, m=m, v=v, adam_step=st, rng=g.get_state().numpy(), k=k,
                 hist=np.array(hist, dtype=np.float64).reshape(-1, 3), steps=steps, batch=batch, lr=lr, seed=seed)

    t0 = time.time()
    end = steps if stop_at is None else min(steps, stop_at)
    for k in range(k0, end):
        idx = torch.randint(0, x.shape[0], (batch,), device=x.device, generator=g)
        lr_k = 1e-5 + 0.5 * (lr - 1e-5) * (1.0 + math.cos(math.pi * k / steps))
        want = (k + 1) % log_every == 0 or k == steps - 1
        loss = net.train_step(x[idx].contiguous(), t[idx].contiguous(), lam[idx].contiguous(), lr_k,
                              want_loss=want)
        if want:
            hist.append((k + 1, float(loss), time.time() - t0))
            print(f"step {k + 1}: loss {float(loss):.6g} lr {lr_k:.3g} {time.time() - t0:.1f}s", flush=True)
        if checkpoint and checkpoint_every and (k + 1) % checkpoint_every == 0:
            save(k + 1)
    if checkpoint:
        save(end)
    p = net.get_params()
    net.close()
    return p, hist


def evaluate(frames, mask, blocks, params, plain_iters=(50, 60, 70, 80, 100, 150, 200), learned_iters=(0, 50)):
    """PSNR on the lost samples: plain extrapolation at each I of
    plain_iters, learned initialisation followed by each I of learned_iters."""
    import torch
    from . import Engine
    truth = truth_patches(frames, blocks)
    out = {"blocks": int(len(blocks))}
    # a perfect network: the plain I=200 model itself as the warm start
    g200 = plain_area_model(frames, mask, blocks, 200).reshape(len(blocks), M * M).contiguous()
    eng = Engine([dict(block=B, border=D, fft=FFT, rho=RHO, gamma=GAMMA, iters=50)])
    p = torch.empty(len(blocks) * B * B, dtype=torch.float32, device=frames.device)
    eng.run_init(frames, mask, blocks, g200, patches=p)
    torch.cuda.synchronize()
    eng.close()
    out["warm_from_plain_i200_model_i50_psnr"] = psnr(p.view(len(blocks), B, B), truth)
    del g200
    for I in plain_iters:
        out[f"plain_i{I}_psnr"] = psnr(plain_patches(frames, mask, blocks, I), truth)
    for I in learned_iters:
        out[f"learned_i{I}_psnr"] = psnr(learned_patches(frames, mask, blocks, params, I), truth)
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--out", required=True)
    ap.add_argument("--train-frames", type=int, default=62)     # ~200k areas at 4K, 10% losses
    ap.add_argument("--test-frames", type=int, default=6)       # ~20k areas
    ap.add_argument("--height", type=int, default=2160)
    ap.add_argument("--width", type=int, default=3840)
    ap.add_argument("--loss", type=float, default=0.10)
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--batch", type=int, default=128)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--lam-b", type=float, default=1.0)
    ap.add_argument("--seed", type=int, default=7)
    ap.add_argument("--target", choices=["model", "support", "correction"], default="correction")
    ap.add_argument("--short-iters", type=int, default=50)
    ap.add_argument("--init", default=None, help="start from these parameters (.f32)")
    ap.add_argument("--eval-only", default=None, help="evaluate these parameters (.f32) and exit")
    ap.add_argument("--checkpoint-every", type=int, default=0,
                    help="write <out>/train_state.npz every this many steps (0: only at the end)")
    ap.add_argument("--resume", default=None, help="continue the training run of this train_state.npz")
    a = ap.parse_args(argv)
    import torch
    if a.eval_only:
        fr, mk, bl = frames_and_losses(TEST_SEED0, a.test_frames, a.height, a.width, a.loss)
        print(json.dumps(evaluate(fr, mk, bl, load_weights(a.eval_only))), flush=True)
        return
    os.makedirs(a.out, exist_ok=True)
    t0 = time.time()
    fr, mk, bl = frames_and_losses(TRAIN_SEED0, a.train_frames, a.height, a.width, a.loss)
    x, t, lam = training_set(fr, mk, bl, a.lam_b, a.target, a.short_iters)
    del fr, mk
    print(f"training set: {x.shape[0]} areas, {time.time() - t0:.1f}s", flush=True)
    params, hist = train(x, t, lam, a.steps, a.batch, a.lr, a.seed,
                         init=None if a.init is None else load_weights(a.init),
                         checkpoint=os.path.join(a.out, "train_state.npz"), checkpoint_every=a.checkpoint_every,
                         resume=a.resume)
    train_s = hist[-1][2] if hist else 0.0
    del x, t, lam
    torch.cuda.empty_cache()
    fr, mk, bl = frames_and_losses(TEST_SEED0, a.test_frames, a.height, a.width, a.loss)
    ev = evaluate(fr, mk, bl, params, learned_iters=(0, a.short_iters))
    print(json.dumps(ev), flush=True)
    name = WEIGHTS_NAME if (a.target != "correction" or a.short_iters == 50) else f"{WEIGHTS_NAME}_k{a.short_iters}"
    params.astype("<f4").tofile(os.path.join(a.out, name + ".f32"))
    meta = dict(vars(a), train_seed0=TRAIN_SEED0, test_seed0=TEST_SEED0, block=B, border=D, fft=FFT, rho=RHO,
                gamma=GAMMA, train_seconds=train_s, loss_history=hist, eval=ev)
    with open(os.path.join(a.out, name + ".json"), "w") as f:
        json.dump(meta, f, indent=1)


if __name__ == "__main__":
    main()
