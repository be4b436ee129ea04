#!/usr/bin/env python3
"""Throughput benchmark of the cFSE hot path on GB300.

Workload (the paper's Section IV setup at video scale): 64 frames of
3840x2160 8-bit synthetic content, 10% of the 16x16 blocks of every frame
lost, 16-sample support border (48x48 areas), 64x64 FFT, rho 0.8, gamma 0.5,
I = 200 selected basis functions per block.  One step conceals the whole
batch (207,360 blocks) in one graph-captured persistent launch.

Metric: lost 16x16 blocks concealed per second (higher is better).
  value  device-resident inputs, CUDA events on the launch stream
  e2e    the host-buffer C-ABI entry point: H2D of frames + mask, kernel,
         D2H of the concealed patches, per step (average of up to 10 calls;
         pipelined inside the call:
         uploads, launches and read-backs of up to eight chunks overlap)
Under torchrun every rank conceals its own 64-frame batch (weak scaling, no
collective on the data path); rank 0 prints one JSON line.

--impl reference times the FP64 CPU oracle (the only baseline: the paper
ships no code) on the host cores over a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

CLS = dict(block=16, border=16, fft=64, rho=0.8, gamma=0.5, iters=200)
T, H, W = 64, 2160, 3840
LOSS = 0.10
METRIC = "16x16 blocks/s at I=200, 64x64 FFT"
PROFILE_NOTE = os.path.join(ROOT, "profiles", "fse_batch_kernel_4k64_i200.md")
KERNEL_SRC = os.path.join(ROOT, "paper_2204_14193_gb300", "csrc", "fse_device.cuh")
# multiply-adds of the network outputs that reach a 16x16 block (layers 0..3:
# 44^2 x 32 x 18, 40^2 x 32 x 288, 32^2 x 32 x 288, 16^2 x 1 x 288), x2 flops
NET_FLOPS_PER_BLOCK = 2.0 * (44 * 44 * 32 * 18 + 40 * 40 * 32 * 288 + 32 * 32 * 32 * 288 + 16 * 16 * 288)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--frames", type=int, default=T)
    ap.add_argument("--iters", type=int, default=CLS["iters"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the I sweep and the uneven-size batch")
    ap.add_argument("--init-iters", type=int, default=50)
    ap.add_argument("--init-weights", default=None, help="network parameters (.f32) for the learned leg")
    ap.add_argument("--fixed-w", action="store_true",
                    help="time the headline with reduced-precision residual storage (FSE_FLAG_FIXED_W)")
    return ap.parse_args()


def workload(rank: int, frames: int, device):
    import torch
    from paper_2204_14193_gb300 import synth
    vid = synth.make_video_torch(2022 + rank, frames, H, W, device=device)
    blocks = workload_blocks(rank, frames)
    mask = synth.grid_mask_torch(blocks, 16, frames, H, W, device=device)
    return vid, mask, blocks


def workload_blocks(rank: int, frames: int) -> np.ndarray:
    """The lost blocks of a rank's batch (seeds differ per rank and frame)."""
    from paper_2204_14193_gb300 import synth
    return np.concatenate([synth.grid_losses(100_000 * (rank + 1) + t, H, W, 16, LOSS, image=t)
                           for t in range(frames)])


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def max_sm_clock_mhz(gpu: int) -> float:
    """Maximum SM clock reported by nvidia-smi (fallback when the timed
    region was too short to sample the clock)."""
    try:
        out = subprocess.run(["nvidia-smi", "-i", str(gpu), "--query-gpu=clocks.max.sm",
                              "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=20)
        return float(out.stdout.strip().splitlines()[0])
    except (OSError, ValueError, IndexError, subprocess.TimeoutExpired):
        return 2070.0


def profile_traffic():
    """DRAM bytes per launch recorded by the committed ncu summary, if it was
    taken on the current kernel source; else None."""
    try:
        txt = open(PROFILE_NOTE).read()
        src_hash = hashlib.sha256(open(KERNEL_SRC, "rb").read()).hexdigest()[:16]
    except OSError:
        return None
    kv = {}
    for ln in txt.splitlines():
        if ":" in ln and ln.strip().startswith("- "):
            k, v = ln.strip()[2:].split(":", 1)
            kv[k.strip()] = v.strip().strip("`")
    if kv.get("kernel_source_sha256_16") != src_hash:
        return None
    try:
        return float(kv["dram_bytes_per_full_launch"])
    except (KeyError, ValueError):
        return None


def cpu_oracle_rate(frames_host, mask_host, blocks, seconds: float, seed: int = 7):
    """FP64 oracle over a seeded sample of the workload's blocks, on all host
    cores, until ~seconds of wall time; returns (blocks/s, cores, n_done)."""
    from concurrent.futures import ThreadPoolExecutor
    from oracle import image as oimage
    cores = len(os.sched_getaffinity(0))
    rng = np.random.default_rng(seed)
    order = rng.permutation(len(blocks))
    done = 0
    t0 = time.perf_counter()

    def one(i):
        im, x, y, _c = (int(v) for v in blocks[i])
        oimage.conceal_block(frames_host[im], mask_host[im], x, y, CLS)

    with ThreadPoolExecutor(max_workers=cores) as ex:
        chunk = 4 * cores
        while time.perf_counter() - t0 < seconds and done < len(order):
            idx = order[done:done + chunk]
            list(ex.map(one, idx))
            done += len(idx)
    dt = time.perf_counter() - t0
    return done / dt, cores, done


def job_throughput(ms_local: float, units_local: int, device):
    """Whole-job figures under weak scaling: every rank processes its own
    units (no collective on the data path); the step time is the maximum over
    ranks and the units are summed.  Returns (ms_max, units_total, units/s)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms_local], dtype=torch.float64, device=device)
    u = torch.tensor([float(units_local)], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
    ms_max, units = float(t.item()), float(u.item())
    return ms_max, units, units / (ms_max / 1e3)


def smem_bytes_per_block(F: int, I: int) -> float:
    """Algorithmic shared-memory bytes of one F x F block at I iterations:
    one 8-byte W operand per bin and iteration, and twelve 8-byte sweeps of
    the grid for the weighting, the two FFT passes (two steps each, loads and
    stores) and the split into R_w and W."""
    return 8.0 * I * F * F + 96.0 * F * F


def fixed_w_bytes_per_block(F: int, I: int, K: int) -> float:
    """smem_bytes_per_block with reduced-precision residual storage, counted
    the same way (one W operand per bin and iteration): 8-byte FP32 operands
    for the first K iterations, 4-byte codes for the other I - K."""
    k32 = min(K, I)
    return 8.0 * k32 * F * F + 4.0 * (I - k32) * F * F + 96.0 * F * F


def pinned_h2d_gbs(host, dev_buf, stream, dev, reps: int = 3) -> float:
    """Pinned host-to-device copy rate of one tensor (best of reps), GB/s."""
    import torch
    best = None
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        dev_buf.copy_(host, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1)
        best = ms if best is None else min(best, ms)
    return host.numel() * host.element_size() / (best / 1e3) / 1e9


def timed_runs(eng, vid, mask, blocks, patches, steps, warmup, stream, dev):
    import torch
    for _ in range(warmup):
        eng.run(vid, mask, blocks, patches=patches)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        eng.run(vid, mask, blocks, patches=patches)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    return e0.elapsed_time(e1) / steps


def learned_leg(P, vid, mask, blocks, plain_patches, args, stream, dev):
    """Learned initialisation (network, then init_iters iterations on the
    residual) against plain extrapolation at I=200 and at init_iters, on the
    same batch: blocks/s and PSNR of the lost samples against the frames."""
    import torch
    from paper_2204_14193_gb300 import train_init
    try:
        w = train_init.load_weights(args.init_weights)
    except (OSError, ValueError) as e:
        return {"available": False, "why": str(e)}
    n = len(blocks)
    truth = train_init.truth_patches(vid, blocks)
    ps = lambda p: train_init.psnr(p.view(n, 16, 16), truth)  # noqa: E731
    out = {"init_iters": args.init_iters, "plain_i200_psnr_db": ps(plain_patches)}
    k = max(3, min(args.steps, 10))
    eng = P.Engine([CLS], init="learned", init_iters=args.init_iters, weights=w)
    pl = torch.empty_like(plain_patches)
    ms = timed_runs(eng, vid, mask, blocks, pl, k, max(args.warmup, 2), stream, dev)
    eng.close()
    out.update(value=n / (ms / 1e3), unit="blocks/s", ms_per_step=ms, psnr_db=ps(pl))
    eng = P.Engine([dict(CLS, iters=args.init_iters)])
    ms_p = timed_runs(eng, vid, mask, blocks, pl, k, max(args.warmup, 2), stream, dev)
    eng.close()
    net_ms = ms - ms_p
    peaks = measured_peaks()
    peak = peaks.get("bf16_tflops_sustained")
    achieved = n * NET_FLOPS_PER_BLOCK / (net_ms / 1e3) / 1e12 if net_ms > 0 else None
    out.update({f"plain_i{args.init_iters}_blocks_per_s": n / (ms_p / 1e3),
                f"plain_i{args.init_iters}_psnr_db": ps(pl),
                "network_ms_per_step_est": net_ms,
                "network_roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                                     "frac": achieved / peak if (achieved and peak) else None,
                                     "basis": "network time = learned step - plain step at the same I; "
                                              f"{NET_FLOPS_PER_BLOCK / 1e6:.2f} MFLOP per block (the valid "
                                              "convolutions that reach B); peak = measured sustained bf16"},
                "weights": os.path.relpath(args.init_weights or train_init.weights_path(), ROOT)})
    return out


def _crossing(points, target):
    """points: (iters, ms per step, psnr) in increasing iters.  The time per
    step at which the curve first reaches PSNR `target`, interpolated linearly
    in PSNR between the bracketing points; None if it never does."""
    prev = None
    for it, ms, ps in points:
        if ps >= target:
            if prev is None or prev[2] >= target:
                return ms, it
            f = (target - prev[2]) / (ps - prev[2])
            return prev[1] + f * (ms - prev[1]), prev[0] + f * (it - prev[0])
        prev = (it, ms, ps)
    return None


def learned_curve(P, vid, mask, blocks, stream, dev, plain_iters=(50, 60, 75, 100, 125, 150, 175, 200),
                  learned_iters=(25, 50, 75, 100, 150)):
    """Learned initialisation against plain extrapolation at equal PSNR, on the
    headline batch: PSNR (lost samples against the frames) and blocks/s of
    plain extrapolation at each I of plain_iters and of the network followed
    by k iterations for each k of learned_iters (the network trained for that
    k -- it supplies what iterations beyond k add -- where one is shipped,
    else the one trained for k = 50; each point names its network).  The comparison point is
    plain I=200's PSNR - 0.1 dB: the blocks/s of each curve there
    (interpolated) and their ratio (learned over plain); and, for every learned
    point, plain extrapolation at that point's own PSNR and the ratio there."""
    import torch
    from paper_2204_14193_gb300 import train_init
    n = len(blocks)
    truth = train_init.truth_patches(vid, blocks)
    ps = lambda p: train_init.psnr(p.view(n, 16, 16), truth)  # noqa: E731
    pt = torch.empty(n * 256, dtype=torch.float32, device=dev)
    plain = []
    for I in plain_iters:
        eng = P.Engine([dict(CLS, iters=I)])
        ms = timed_runs(eng, vid, mask, blocks, pt, 3, 2, stream, dev)
        eng.close()
        plain.append((I, ms, ps(pt)))
    learned, nets = [], dict(train_init.shipped_networks())
    for k in learned_iters:
        # the network trained for k iterations after it, else the one trained for 50
        path = nets.get(k, nets.get(50))
        if path is None:
            continue
        eng = P.Engine([CLS], init="learned", init_iters=k, weights=train_init.load_weights(path))
        ms = timed_runs(eng, vid, mask, blocks, pt, 3, 2, stream, dev)
        eng.close()
        learned.append((k, ms, ps(pt), os.path.basename(path)))
    learned.sort()
    p200 = dict((it, q) for it, _m, q in plain).get(200)
    target = p200 - 0.1 if p200 is not None else None
    lpts = []
    for k, m, q, net in learned:
        cp = _crossing(plain, q)      # plain extrapolation at the learned point's own PSNR
        lpts.append({"init_iters": k, "network": net, "blocks_per_s": n / (m / 1e3), "psnr_db": q,
                     "plain_at_equal_psnr": None if cp is None else {"iters": cp[1], "blocks_per_s": n / (cp[0] / 1e3)},
                     "ratio_at_equal_psnr": None if cp is None else cp[0] / m})
    out = {"plain": [{"iters": it, "blocks_per_s": n / (m / 1e3), "psnr_db": q} for it, m, q in plain],
           "learned": lpts,
           "target_psnr_db": target, "target": "plain I=200 PSNR - 0.1 dB"}
    if target is not None:
        cp, cl = _crossing(plain, target), _crossing([t[:3] for t in learned], target)
        out["plain_at_target"] = None if cp is None else {"blocks_per_s": n / (cp[0] / 1e3), "iters": cp[1]}
        out["learned_at_target"] = None if cl is None else {"blocks_per_s": n / (cl[0] / 1e3), "init_iters": cl[1]}
        out["ratio_at_equal_psnr"] = (cp[0] / cl[0]) if (cp and cl) else None
        if learned and cl is None:
            best = max(learned, key=lambda t: t[2])
            out["learned_best"] = {"init_iters": best[0], "network": best[3], "psnr_db": best[2],
                                   "below_target_db": target - best[2], "blocks_per_s": n / (best[1] / 1e3)}
    return out


def oracle_rate(jobs, seconds: float, threads: int):
    """The FP64 oracle on (image, mask, x, y, class) jobs, `threads` host
    threads, until about `seconds` of wall time or the jobs are done.
    Returns (blocks/s, blocks done)."""
    from concurrent.futures import ThreadPoolExecutor
    from oracle import image as oimage
    done, t0 = 0, time.perf_counter()
    with ThreadPoolExecutor(max_workers=threads) as ex:
        while done < len(jobs) and (done == 0 or time.perf_counter() - t0 < seconds):
            part = jobs[done:done + 4 * threads]
            list(ex.map(lambda j: oimage.conceal_block(j[0], j[1], j[2], j[3], j[4]), part))
            done += len(part)
    return done / (time.perf_counter() - t0), done


def small_configs(P, stream, dev, with_oracle: bool, seconds: float):
    """The two small workloads, device-resident, one graph replay each:
    one 48x48 FP32 area with a centred 16x16 hole, I=100 (the latency of one
    block), and a 512x512 8-bit image with 256 non-adjacent 16x16 losses,
    I=200 (fewer items than the GPU's CTA slots: one wave).  Beside each, the
    FP64 oracle on the same blocks (one host thread for the single area, all
    host threads for the 256 blocks)."""
    import torch
    from paper_2204_14193_gb300 import synth
    cores = len(os.sched_getaffinity(0))
    out = {}
    img1 = synth.make_image(1, 48, 48, u8=False)[None]
    b1 = np.array([[0, 16, 16, 0]], np.int32)
    m1 = synth.loss_mask(b1, [16], 1, 48, 48)
    img2 = synth.make_image(2, 512, 512)[None]
    b2 = synth.grid_losses(3, 512, 512, 16, 0.25, non_adjacent=True)
    m2 = synth.loss_mask(b2, [16], 1, 512, 512)
    for name, img, bl, mk, I, threads in (("single_area_fp32_i100", img1, b1, m1, 100, 1),
                                          ("image_512_u8_256_blocks_i200", img2, b2, m2, 200, cores)):
        cls = dict(CLS, iters=I)
        eng = P.Engine([cls])
        dimg, dmask = torch.from_numpy(img).to(dev), torch.from_numpy(mk).to(dev)
        pt = torch.empty(len(bl) * 256, dtype=torch.float32, device=dev)
        ms = timed_runs(eng, dimg, dmask, bl, pt, 20, 5, stream, dev)
        eng.close()
        r = {"blocks": int(len(bl)), "ms_per_launch": ms, "value": len(bl) / (ms / 1e3), "unit": "blocks/s"}
        if with_oracle:
            jobs = [(img[0], mk[0], int(x), int(y), cls) for _, x, y, _c in bl]
            rate, nd = oracle_rate(jobs * max(1, int(8 * threads // len(jobs))), seconds, threads)
            r["oracle"] = {"value": rate, "unit": "blocks/s", "threads": threads, "blocks_done": nd, "kind": "oracle"}
        out[name] = r
    return out


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def iteration_sweep(P, vid, mask, blocks, patches, args, stream, dev, peak_gbs):
    """Plain extrapolation of the same batch at I = 50 and I = 500."""
    out = {}
    n = len(blocks)
    for I in (50, 500):
        eng = P.Engine([dict(CLS, iters=I)])
        ms = timed_runs(eng, vid, mask, blocks, patches, 3, 2, stream, dev)
        eng.close()
        achieved = n * smem_bytes_per_block(CLS["fft"], I) / (ms / 1e3) / 1e9
        out[f"i{I}"] = {"value": n / (ms / 1e3), "unit": "blocks/s", "ms_per_step": ms,
                        "smem_frac": achieved / peak_gbs}
    return out


def uneven_batch(P, args, stream, dev, peak_gbs, with_oracle=False, seconds=6.0):
    """30 frames of 1920x1080 u8 video, 3% of the samples lost in mixed
    4x4 / 8x8 / 16x16 blocks (borders 6/12/16, FFT 16/32/64), I = 200, one
    launch over all sizes."""
    import torch
    from paper_2204_14193_gb300 import synth
    T3, H3, W3 = 30, 1080, 1920
    vid = synth.make_video_torch(3030, T3, H3, W3, device=dev)
    blocks = np.concatenate([synth.uneven_losses(5000 + t, H3, W3, image=t) for t in range(T3)])
    mask = torch.from_numpy(synth.loss_mask(blocks, [4, 8, 16], T3, H3, W3)).to(dev)
    classes = [dict(block=4, border=6, fft=16, rho=0.8, gamma=0.5, iters=200),
               dict(block=8, border=12, fft=32, rho=0.8, gamma=0.5, iters=200),
               dict(block=16, border=16, fft=64, rho=0.8, gamma=0.5, iters=200)]
    eng = P.Engine(classes)
    pt = torch.empty(eng.patch_total(blocks), dtype=torch.float32, device=dev)
    ms = timed_runs(eng, vid, mask, blocks, pt, 5, 3, stream, dev)
    eng.close()
    counts = np.bincount(blocks[:, 3], minlength=3)
    oracle_line = None
    if with_oracle:
        # the FP64 oracle on a seeded sample of the same blocks, all host threads
        rng = np.random.default_rng(11)
        pick = rng.permutation(len(blocks))[:2048]
        frames = sorted(set(int(blocks[i, 0]) for i in pick))
        vh = {f: vid[f].cpu().numpy() for f in frames}
        mh = {f: mask[f].cpu().numpy() for f in frames}
        jobs = [(vh[int(blocks[i, 0])], mh[int(blocks[i, 0])], int(blocks[i, 1]), int(blocks[i, 2]),
                 classes[int(blocks[i, 3])]) for i in pick]
        cores = len(os.sched_getaffinity(0))
        rate, nd = oracle_rate(jobs, seconds, cores)
        oracle_line = {"value": rate, "unit": "blocks/s", "threads": cores, "blocks_done": nd, "kind": "oracle",
                       "sample": "seeded sample of the batch's blocks (all three sizes)"}
    # shared-memory roofline: each class's algorithmic bytes per block
    nbytes = sum(int(counts[c]) * smem_bytes_per_block(k["fft"], k["iters"]) for c, k in enumerate(classes))
    return {"value": len(blocks) / (ms / 1e3), "unit": "blocks/s", "ms_per_step": ms, "oracle": oracle_line,
            "workload": f"{T3} x {W3}x{H3} u8 frames, 3% of samples lost in 4/8/16 blocks "
                        f"({counts[0]}/{counts[1]}/{counts[2]}), F 16/32/64, I=200, one launch",
            "blocks": int(len(blocks)), "smem_bytes_per_launch": nbytes,
            "smem_frac": nbytes / (ms / 1e3) / 1e9 / peak_gbs}


def video_volumes(P, args, stream, dev, peak_gbs):
    """30 frames of 1920x1080 u8 video, 3% of the 8x8 blocks lost, concealed
    as 3-frame volumes (the block's frame and its neighbours, 4 x 32 x 32
    transform) and, for comparison, as image areas (32 x 32), I = 200:
    blocks/s and PSNR of the lost samples."""
    import torch
    from paper_2204_14193_gb300 import synth
    T3, H3, W3, b = 30, 1080, 1920, 8
    vid = synth.make_video_torch(4040, T3, H3, W3, device=dev)
    blocks = np.concatenate([synth.grid_losses(6000 + t, H3, W3, b, 0.03, image=t) for t in range(T3)])
    mask = synth.grid_mask_torch(blocks, b, T3, H3, W3, device=dev)
    bt = torch.from_numpy(blocks.astype(np.int64)).to(dev)
    ar = torch.arange(b, device=dev)
    truth = vid[bt[:, 0, None, None], (bt[:, 2, None] + ar)[:, :, None], (bt[:, 1, None] + ar)[:, None, :]].float()
    out = {"workload": f"{T3} x {W3}x{H3} u8 frames, 3% of the 8x8 blocks lost ({len(blocks)} blocks), "
                       "border 12, I=200", "blocks": int(len(blocks))}
    for name, frames in (("volume", 3), ("image", 0)):
        cls = dict(block=b, border=12, fft=32, rho=0.8, gamma=0.5, iters=200, frames=frames)
        eng = P.Engine([cls])
        pt = torch.empty(len(blocks) * b * b, dtype=torch.float32, device=dev)
        ms = timed_runs(eng, vid, mask, blocks, pt, 5, 3, stream, dev)
        eng.close()
        mse = float(((pt.view(-1, b, b).clamp(0, 255) - truth) ** 2).mean())
        bins = 32 * 32 * (4 if frames else 1)
        achieved = len(blocks) * (8.0 * 200 * bins + 96.0 * bins) / (ms / 1e3) / 1e9
        out[name] = {"value": len(blocks) / (ms / 1e3), "unit": "blocks/s", "ms_per_step": ms,
                     "psnr_db": 10 * np.log10(255.0 ** 2 / max(mse, 1e-12)), "smem_frac": achieved / peak_gbs}
    return out


def ordered_leg(P, vid, mask, blocks, plain_patches, stream, dev):
    """The headline batch concealed in order, each block reusing the concealed
    samples of earlier neighbours (weight 0.5 x Eq. (3)): blocks/s and PSNR
    against independent concealment."""
    import torch
    from paper_2204_14193_gb300 import train_init
    n = len(blocks)
    truth = train_init.truth_patches(vid, blocks)
    ps = lambda p: train_init.psnr(p.view(n, 16, 16), truth)  # noqa: E731
    eng = P.Engine([CLS], ordered=True, reuse_weight=0.5)
    out = torch.empty(vid.shape, dtype=torch.float32, device=dev)
    pt = torch.empty_like(plain_patches)
    for _ in range(2):
        eng.run(vid, mask, blocks, out=out, patches=pt)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(3):
        eng.run(vid, mask, blocks, out=out, patches=pt)
    e1.record(stream)
    eng.sync()
    ms = e0.elapsed_time(e1) / 3
    eng.close()
    return {"value": n / (ms / 1e3), "unit": "blocks/s", "ms_per_step": ms, "reuse_weight": 0.5,
            "psnr_db": ps(pt), "independent_psnr_db": ps(plain_patches)}


def fixed_w_leg(P, vid, mask, blocks, plain_patches, plain_ms, args, stream, dev, peak_gbs):
    """The headline batch with reduced-precision residual storage
    (FSE_FLAG_FIXED_W: 16-bit fixed-point W after FSE_FIXED_W_FROM FP32
    updates): blocks/s, speed-up over the FP32 kernel, PSNR of both, largest
    pixel difference, and the shared-memory roofline with the mode's own
    algorithmic bytes (8 B per bin for the FP32 iterations, 4 B after)."""
    import torch
    from paper_2204_14193_gb300 import train_init
    n = len(blocks)
    truth = train_init.truth_patches(vid, blocks)
    ps = lambda p: train_init.psnr(p.view(n, 16, 16), truth)  # noqa: E731
    eng = P.Engine([CLS], fixed_w=True)
    pf = torch.empty_like(plain_patches)
    ms = timed_runs(eng, vid, mask, blocks, pf, max(3, min(args.steps, 10)), max(args.warmup, 2), stream, dev)
    eng.close()
    F, I, K = CLS["fft"], CLS["iters"], P.FSE_FIXED_W_FROM
    bytes_block = fixed_w_bytes_per_block(F, I, K)
    achieved = n * bytes_block / (ms / 1e3) / 1e9
    return {"value": n / (ms / 1e3), "unit": "blocks/s", "ms_per_step": ms, "fixed_from": K,
            "speedup_vs_fp32_w": plain_ms / ms, "psnr_db": ps(pf), "fp32_w_psnr_db": ps(plain_patches),
            "max_abs_diff_vs_fp32_w": float((pf - plain_patches).abs().max().item()),
            "smem_bytes_per_block": bytes_block, "smem_frac": achieved / peak_gbs}


def run_reference(args):
    """The oracle as the reference arm (rank 0 only)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2204_14193_gb300 import synth
    frames = 2   # a bounded sample: two frames of the workload's content and losses
    vid = synth.make_video(2022, frames, H, W)
    blocks = np.concatenate([synth.grid_losses(100_000 + t, H, W, 16, LOSS, image=t) for t in range(frames)])
    mask = synth.loss_mask(blocks, [16], frames, H, W)
    import oracle
    oracle.build()
    cores = len(os.sched_getaffinity(0))
    per = max(8, min(len(blocks), int(args.cpu_seconds)))  # blocks per step, tuned below
    # calibrate: one block's time on one core -> blocks per ~3 s step on all cores
    t0 = time.perf_counter()
    from oracle import image as oimage
    im, x, y, _ = (int(v) for v in blocks[0])
    oimage.conceal_block(vid[im], mask[im], x, y, CLS)
    one = time.perf_counter() - t0
    per = int(max(cores, min(len(blocks), 3.0 * cores / max(one, 1e-4))))
    sample = blocks[:per]
    times = []
    from concurrent.futures import ThreadPoolExecutor

    def work(i):
        im, x, y, _c = (int(v) for v in sample[i])
        oimage.conceal_block(vid[im], mask[im], x, y, CLS)

    with ThreadPoolExecutor(max_workers=cores) as ex:
        for s in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            list(ex.map(work, range(len(sample))))
            if s >= args.warmup:
                times.append(time.perf_counter() - t0)
    ms = 1e3 * sum(times) / len(times)
    value = per / (ms / 1e3)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "blocks/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"FP64 CPU oracle, sample of {per} blocks of the 3840x2160 u8 "
                                   "10% 16x16-loss workload (48x48 areas, F=64, rho 0.8, gamma 0.5, I=200)",
                       "blocks_per_step": per},
            "cpu_baseline": {"value": value, "unit": "blocks/s", "cores": cores, "kind": "oracle",
                             "sample": f"{per} blocks x {args.steps} steps"},
            "e2e": {"value": value, "unit": "blocks/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    import paper_2204_14193_gb300 as P
    cls = dict(CLS, iters=args.iters)
    frames = args.frames
    vid, mask, blocks = workload(rank, frames, dev)
    n_blocks = len(blocks)
    eng = P.Engine([cls], device=local, fixed_w=args.fixed_w)
    patches = torch.empty(n_blocks * 256, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    for _ in range(args.warmup):
        eng.run(vid, mask, blocks, patches=patches)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clk:
        torch.cuda.nvtx.range_push("timed")
        e0.record(stream)
        for _ in range(args.steps):
            eng.run(vid, mask, blocks, patches=patches)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        torch.cuda.nvtx.range_pop()
    if world > 1:
        dist.barrier()
    ms = e0.elapsed_time(e1) / args.steps
    ms_max, _units, value = job_throughput(ms, n_blocks, dev)
    clocks = clk.summary()

    # ---- end to end through the host-buffer entry point ----
    e2e = None
    if not args.no_e2e:
        t_vid = vid.cpu().pin_memory()
        h_vid = t_vid.numpy()
        h_mask = mask.cpu().pin_memory().numpy()
        h_patch = torch.empty(n_blocks * 256, dtype=torch.float32).pin_memory().numpy()
        eng.run_host(h_vid, h_mask, blocks, h_patch)     # warm-up (staging buffers, graph)
        k = max(3, min(args.steps, 10))   # calls averaged: the host's own memory traffic varies
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(k):
            eng.run_host(h_vid, h_mask, blocks, h_patch)
        dt = (time.perf_counter() - t0) / k
        dt_ms, _units, e2e_value = job_throughput(dt * 1e3, n_blocks, dev)
        dt = dt_ms / 1e3
        e2e = {"value": e2e_value, "unit": "blocks/s",
               "h2d_bytes_per_step": int(h_vid.nbytes + h_mask.nbytes + blocks.nbytes),
               "d2h_bytes_per_step": int(h_patch.nbytes), "ms_per_step": dt * 1e3}
        # the e2e patches equal the device-path patches bit for bit
        assert np.array_equal(h_patch, patches.cpu().numpy()), "host entry point disagrees with device path"
        # context for e2e: this box's pinned host-to-device copy rate (the
        # pipeline hides the upload while it is faster than twice the rate
        # at which the kernel consumes frames)
        e2e["h2d_gbs"] = pinned_h2d_gbs(t_vid, vid, stream, dev)

    # the shared-memory peak: measured on this GPU (a stream of conflict-free
    # 16-byte shared loads on every SM), right after the timed region
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    sm_mhz = clocks["sm_mhz"] or clocks["sm_max_mhz"] or max_sm_clock_mhz(local)
    derived_peak = sms * 128.0 * sm_mhz * 1e6 / 1e9
    try:
        smem_peak = P.fse_measure_smem_bandwidth(local)
        peak_basis = (f"measured: conflict-free 16-byte shared-memory load stream on all {sms} SMs "
                      f"(fse_measure_smem_bandwidth, best of 5), {smem_peak / (sms * sm_mhz * 1e6 / 1e9):.1f} B/clk "
                      f"per SM at the {sm_mhz:.0f} MHz median SM clock of the timed region (derived 128 B/clk: "
                      f"{derived_peak:.0f} GB/s)")
    except P.FseError:
        smem_peak = derived_peak
        peak_basis = f"derived: {sms} SMs x 128 B/clk x {sm_mhz:.0f} MHz (the measurement failed)"

    learned = curve = None
    if not args.no_learned and args.iters == 200 and not args.fixed_w:
        learned = learned_leg(P, vid, mask, blocks, patches, args, stream, dev)
        curve = learned_curve(P, vid, mask, blocks, stream, dev)
    sweep = uneven = video = ordered = small = fixed = None
    if not args.no_extra and args.iters == 200 and not args.fixed_w:
        fixed = fixed_w_leg(P, vid, mask, blocks, patches, ms, args, stream, dev, smem_peak)
        ordered = ordered_leg(P, vid, mask, blocks, patches, stream, dev)
        sweep = iteration_sweep(P, vid, mask, blocks, patches, args, stream, dev, smem_peak)
        uneven = uneven_batch(P, args, stream, dev, smem_peak, with_oracle=rank == 0 and not args.no_cpu_baseline,
                              seconds=args.cpu_seconds / 2)
        video = video_volumes(P, args, stream, dev, smem_peak)
        small = small_configs(P, stream, dev, with_oracle=rank == 0 and not args.no_cpu_baseline,
                              seconds=args.cpu_seconds / 4)

    # ---- roofline of the persistent kernel (shared-memory bound) ----
    F, I = cls["fft"], cls["iters"]
    smem_bytes_block = (fixed_w_bytes_per_block(F, I, P.FSE_FIXED_W_FROM) if args.fixed_w
                        else smem_bytes_per_block(F, I))
    flops_block = I * F * F * 11.0 + 3 * 5.0 * F * F * np.log2(F * F)
    achieved = n_blocks * smem_bytes_block / (ms / 1e3) / 1e9
    peak = smem_peak
    fp32_peak = sms * 256.0 * sm_mhz * 1e6 / 1e12
    traffic = None if args.fixed_w else profile_traffic()
    roofline = {"bound": "smem", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "bytes_per_block": smem_bytes_block,
                "bytes_basis": ("8 K F^2 + 4 (I - K) F^2 (8-byte FP32 W operands for the first K iterations, "
                                "4-byte codes after) + 96 F^2" if args.fixed_w else
                                "8 I F^2 (one 8-byte W operand per bin and iteration) + 96 F^2 (the FFT passes, "
                                "the weighting and the split: twelve 8-byte sweeps of the F x F grid)"),
                "peak_basis": peak_basis,
                "fp32": {"achieved_tflops": n_blocks * flops_block / (ms / 1e3) / 1e12,
                         "peak_tflops": fp32_peak,
                         "frac": n_blocks * flops_block / (ms / 1e3) / 1e12 / fp32_peak}}

    # ---- CPU baseline: the oracle on the host cores ----
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        frames_used = sorted(set(int(b) for b in blocks[:4096, 0]))
        fh = {f: vid[f].cpu().numpy() for f in frames_used}
        mh = {f: mask[f].cpu().numpy() for f in frames_used}
        sub = blocks[:4096]
        rate, cores, ndone = cpu_oracle_rate(fh, mh, sub, args.cpu_seconds)
        cpu = {"value": rate, "unit": "blocks/s", "cores": cores, "kind": "oracle",
               "sample": f"{ndone} seeded blocks of the first {len(frames_used)} frames, FP64, "
                         f"{args.cpu_seconds:.0f} s budget"}
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "blocks/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": f"{frames} x 3840x2160 u8 frames, 10% 16x16 losses per frame "
                                       f"({n_blocks} blocks per GPU), 48x48 areas, F=64, rho 0.8, "
                                       f"gamma 0.5, I={I}, plain (zero) initialisation"
                                       + (f", 16-bit fixed-point W after {P.FSE_FIXED_W_FROM} FP32 updates"
                                          if args.fixed_w else ""),
                           "parallelism": f"replicas x{world}", "blocks_per_gpu": n_blocks,
                           "l2": f"inputs larger than L2 (frames + mask = {2 * frames * H * W / 1e6:.0f} MB per GPU, "
                                 "L2 129 MB)"},
                "clocks": clocks, "gpu_launches": args.steps, "roofline": roofline,
                "e2e": e2e, "cpu_baseline": cpu, "learned_init": learned, "learned_vs_plain": curve,
                "iteration_sweep": sweep, "uneven_batch": uneven, "video_volumes": video, "ordered": ordered,
                "small_configs": small, "fixed_w": fixed}
        print(json.dumps(line))
    eng.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
