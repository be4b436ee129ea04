"""Workloads run once with the normal library and once with the bounds-checked
one (FSE_BOUNDS_CHECK=1 in the environment), by tests/test_gpu_bounds_checked.py.
Every kernel path runs: FFT-64 with the TMA gather and with plain FP32 loads,
mixed 16/32/64 sizes, video volumes of FFT 32 and 16, ordered concealment of
FFT 64 and 32, reduced-precision storage, a traced launch, the learned
initialisation, the host-buffer pipeline and the allocation-free entry point.
Each workload prints one line: its name and the SHA-256 of its output.  Any
failure (a bounds violation reported by fse_sync included) ends the script
with a non-zero status."""
import hashlib
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import numpy as np  # noqa: E402
import torch  # noqa: E402

import paper_2204_14193_gb300 as P  # noqa: E402
from paper_2204_14193_gb300 import synth  # noqa: E402

C64 = dict(block=16, border=16, fft=64, rho=0.8, gamma=0.5, iters=60)
C32 = dict(block=8, border=12, fft=32, rho=0.8, gamma=0.5, iters=60)
C16 = dict(block=4, border=6, fft=16, rho=0.8, gamma=0.5, iters=40)
V32 = dict(C32, iters=40, frames=3)
V16 = dict(C16, iters=30, frames=3)


def digest(name, *arrays):
    h = hashlib.sha256()
    for a in arrays:
        h.update(np.ascontiguousarray(a).tobytes())
    print(name, h.hexdigest()[:24], flush=True)


def run(classes, images, mask, blocks, out_image=False, **kw):
    eng = P.Engine(classes, **kw)
    n = eng.patch_total(blocks)
    dimg = torch.from_numpy(np.ascontiguousarray(images)).cuda()
    patches = torch.zeros(max(n, 1), device="cuda")
    out = dimg.float().contiguous() if out_image else None
    eng.run(dimg, torch.from_numpy(np.ascontiguousarray(mask)).cuda(), blocks, out=out, patches=patches)
    eng.sync()
    res = [patches.cpu().numpy()]
    if out is not None:
        res.append(out.cpu().numpy())
    if kw.get("trace"):
        res.extend(eng.trace()[:2])
    eng.close()
    return res


def main():
    print("library", os.path.basename(P.library_path()), flush=True)
    torch.manual_seed(0)
    # FFT 64, 8-bit (TMA gather), and FP32 samples with supports past every edge
    img = synth.make_image(2, 256, 256)[None]
    blocks = synth.grid_losses(3, 256, 256, 16, 0.25, non_adjacent=True)
    mask = synth.loss_mask(blocks, [16], 1, 256, 256)
    digest("f64_u8", *run([C64], img, mask, blocks, out_image=True))
    H, W = 96, 80
    imf = synth.make_image(7, H, W, u8=False)[None]
    be = np.array([[0, 0, 0, 0], [0, 16, 16, 0], [0, 64, 0, 0], [0, 0, 80, 0],
                   [0, 64, 80, 0], [0, 32, 48, 0], [0, 48, 32, 0]], np.int32)
    digest("f64_f32_edges", *run([C64], imf, synth.loss_mask(be, [16], 1, H, W), be, out_image=True))
    # mixed sizes in one launch
    vid = synth.make_video(4, 2, 540, 960)
    bu = np.concatenate([synth.uneven_losses(10 + t, 540, 960, image=t) for t in range(2)])
    digest("uneven", *run([C16, C32, C64], vid, synth.loss_mask(bu, [4, 8, 16], 2, 540, 960), bu))
    # video volumes, FFT 32 and 16
    v5 = synth.make_video(71, 5, 96, 128)
    b8 = np.concatenate([synth.grid_losses(72 + t, 96, 128, 8, 0.05, image=t) for t in range(5)])
    digest("vol32", *run([V32], v5, synth.loss_mask(b8, [8], 5, 96, 128), b8))
    b4 = np.concatenate([synth.grid_losses(82 + t, 96, 128, 4, 0.03, image=t) for t in range(5)])
    digest("vol16", *run([V16], v5, synth.loss_mask(b4, [4], 5, 96, 128), b4))
    # ordered concealment, FFT 64 and 32
    im2 = synth.make_image(93, 160, 192)[None]
    for cls, b in ((C64, 16), (C32, 8)):
        bo = synth.grid_losses(94, 160, 192, b, 0.3)
        digest(f"ordered{cls['fft']}", *run([cls], im2, synth.loss_mask(bo, [b], 1, 160, 192), bo,
                                           out_image=True, ordered=True, reuse_weight=0.5))
    # reduced-precision storage (traced) and a traced FP32 launch
    digest("fixed_w", *run([dict(C64, iters=80)], img, mask, blocks, fixed_w=True, trace=True))
    digest("traced", *run([dict(C64, iters=30)], img, mask, blocks, trace=True))
    # learned initialisation with the shipped network
    from paper_2204_14193_gb300 import train_init
    w = train_init.load_weights()
    digest("learned", *run([C64], img, mask, blocks, init="learned", init_iters=30, weights=w))
    # host-buffer pipeline over several frames
    v6 = synth.make_video(41, 6, 256, 320)
    b6 = np.concatenate([synth.grid_losses(42 + t, 256, 320, 16, 0.2, image=t) for t in range(6)])
    m6 = synth.loss_mask(b6, [16], 6, 256, 320)
    eng = P.Engine([C64])
    hp = np.zeros(eng.patch_total(b6), np.float32)
    eng.run_host(v6, m6, b6, hp)
    eng.sync()
    eng.close()
    digest("host_pipeline", hp)
    # allocation-free entry point (image output only)
    dv, dm = torch.from_numpy(v6).cuda(), torch.from_numpy(m6).cuda()
    out = dv.float().contiguous()
    P.fse_extrapolate_batch_noalloc([C64], dv.data_ptr(), P.FSE_DTYPE_U8, 6, 256, 320, 320, dm.data_ptr(),
                                    b6, len(b6), out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    digest("noalloc", out.cpu().numpy())


if __name__ == "__main__":
    main()
