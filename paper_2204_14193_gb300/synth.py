"""Seeded synthetic inputs: images, videos and loss patterns.

This module draws inputs only; it holds none of the extrapolation arithmetic
and imports neither the CUDA binding nor the oracle, so both can be fed the
same arrays.

Content model (stand-in for natural images such as the Kodak set used in
Section IV): 128 + sum of 8 random 2-D sinusoids + one random step edge +
Gaussian noise (sigma 2), clipped to [0, 255]; 8-bit content is rounded.
  amplitude a_i ~ U(5, 25), spatial frequency |f_i| ~ U(0.005, 0.2) cycles/px
  with uniform orientation, phase phi_i ~ U(0, 2 pi); edge normal theta ~
  U(0, pi), offset t uniform over the image's projected extent, height
  h ~ U(-60, 60).  Video frames advance phi_i by omega_i ~ U(-0.3, 0.3)
  rad/frame and t by a per-video drift ~ U(-2, 2) px/frame.
"""
from __future__ import annotations

import numpy as np


def _params(rng: np.random.Generator, H: int, W: int):
    a = rng.uniform(5.0, 25.0, 8)
    fmag = rng.uniform(0.005, 0.2, 8)
    ori = rng.uniform(0.0, 2.0 * np.pi, 8)
    phi = rng.uniform(0.0, 2.0 * np.pi, 8)
    theta = rng.uniform(0.0, np.pi)
    c, s = np.cos(theta), np.sin(theta)
    corners = np.array([0.0, (W - 1) * c, (H - 1) * s, (W - 1) * c + (H - 1) * s])
    t = rng.uniform(corners.min(), corners.max())
    h = rng.uniform(-60.0, 60.0)
    omega = rng.uniform(-0.3, 0.3, 8)
    drift = rng.uniform(-2.0, 2.0)
    return dict(a=a, fx=fmag * np.cos(ori), fy=fmag * np.sin(ori), phi=phi, theta=theta,
                t=t, h=h, omega=omega, drift=drift)


def _render(p, H: int, W: int, frame: int, rng: np.random.Generator, u8: bool) -> np.ndarray:
    x = np.arange(W, dtype=np.float64)
    y = np.arange(H, dtype=np.float64)
    img = np.full((H, W), 128.0, dtype=np.float64)
    for i in range(8):
        ph = p["phi"][i] + p["omega"][i] * frame
        ax = 2.0 * np.pi * p["fx"][i] * x + ph
        ay = 2.0 * np.pi * p["fy"][i] * y
        # cos(ay + ax) = cos(ay) cos(ax) - sin(ay) sin(ax), separable
        img += p["a"][i] * (np.outer(np.cos(ay), np.cos(ax)) - np.outer(np.sin(ay), np.sin(ax)))
    proj = np.add.outer(y * np.sin(p["theta"]), x * np.cos(p["theta"]))
    img += p["h"] * (proj > p["t"] + p["drift"] * frame)
    img += rng.normal(0.0, 2.0, size=(H, W))
    np.clip(img, 0.0, 255.0, out=img)
    if u8:
        return np.rint(img).astype(np.uint8)
    return img.astype(np.float32)


def _render_torch(p, H: int, W: int, frames: int, seed: int, u8: bool, device):
    """The same content model evaluated with torch on ``device`` (used for
    large benchmark batches).  Only the noise realisation differs from the
    numpy path (torch's generator on that device, seeded with ``seed``)."""
    import torch
    dev = torch.device(device)
    gen = torch.Generator(device=dev)
    gen.manual_seed(int(seed))
    x = torch.arange(W, dtype=torch.float64, device=dev)
    y = torch.arange(H, dtype=torch.float64, device=dev)
    out = torch.empty((frames, H, W), dtype=torch.uint8 if u8 else torch.float32, device=dev)
    proj = (y[:, None] * np.sin(p["theta"]) + x[None, :] * np.cos(p["theta"])).float()
    for t in range(frames):
        img = torch.full((H, W), 128.0, dtype=torch.float32, device=dev)
        for i in range(8):
            ph = float(p["phi"][i] + p["omega"][i] * t)
            ax = 2.0 * np.pi * float(p["fx"][i]) * x + ph
            ay = 2.0 * np.pi * float(p["fy"][i]) * y
            img += float(p["a"][i]) * (torch.outer(torch.cos(ay), torch.cos(ax))
                                       - torch.outer(torch.sin(ay), torch.sin(ax))).float()
        img += float(p["h"]) * (proj > float(p["t"] + p["drift"] * t)).float()
        img += 2.0 * torch.randn((H, W), generator=gen, device=dev, dtype=torch.float32)
        img.clamp_(0.0, 255.0)
        out[t] = torch.round(img).to(torch.uint8) if u8 else img
    return out


def make_video_torch(seed: int, frames: int, H: int, W: int, u8: bool = True, device="cuda"):
    """make_video rendered with torch on ``device`` (a torch tensor)."""
    rng = np.random.default_rng(seed)
    p = _params(rng, H, W)
    return _render_torch(p, H, W, frames, seed, u8, device)


def make_image(seed: int, H: int, W: int, u8: bool = True) -> np.ndarray:
    """One synthetic image [H, W] (uint8 or float32)."""
    rng = np.random.default_rng(seed)
    p = _params(rng, H, W)
    return _render(p, H, W, 0, rng, u8)


def make_video(seed: int, frames: int, H: int, W: int, u8: bool = True) -> np.ndarray:
    """A synthetic video [T, H, W] whose sinusoids and edge drift per frame."""
    rng = np.random.default_rng(seed)
    p = _params(rng, H, W)
    out = np.empty((frames, H, W), dtype=np.uint8 if u8 else np.float32)
    for t in range(frames):
        out[t] = _render(p, H, W, t, rng, u8)
    return out


def grid_losses(seed: int, H: int, W: int, b: int, frac: float, non_adjacent: bool = False,
                image: int = 0, cls: int = 0) -> np.ndarray:
    """Lose round(frac * cells) blocks of a b-aligned grid of one image.

    With ``non_adjacent`` no two lost blocks share an edge (4-neighbourhood);
    diagonal neighbours may both be lost.  Returns int32 rows (image, x, y, cls).
    """
    rng = np.random.default_rng(seed)
    gh, gw = H // b, W // b
    want = int(round(frac * gh * gw))
    order = rng.permutation(gh * gw)
    taken = np.zeros((gh, gw), dtype=bool)
    picked = []
    for cell in order:
        if len(picked) >= want:
            break
        r, c = divmod(int(cell), gw)
        if non_adjacent:
            nb = [(r - 1, c), (r + 1, c), (r, c - 1), (r, c + 1)]
            if any(0 <= rr < gh and 0 <= cc < gw and taken[rr, cc] for rr, cc in nb):
                continue
        taken[r, c] = True
        picked.append((image, c * b, r * b, cls))
    if len(picked) < want:
        raise ValueError("could not place the requested number of non-adjacent losses")
    picked.sort(key=lambda t: (t[2], t[1]))
    return np.array(picked, dtype=np.int32).reshape(-1, 4)


def uneven_losses(seed: int, H: int, W: int, sizes=(4, 8, 16), pixel_frac: float = 0.03,
                  image: int = 0) -> np.ndarray:
    """Non-overlapping b-aligned losses of mixed sizes covering ~pixel_frac of
    the image; the size class of each block is drawn uniformly from ``sizes``.
    Rows (image, x, y, cls) with cls the index into ``sizes``."""
    rng = np.random.default_rng(seed)
    g = min(sizes)
    occ = np.zeros((H // g + 1, W // g + 1), dtype=bool)
    target = pixel_frac * H * W
    lost = 0
    out = []
    attempts = 0
    while lost < target and attempts < 1_000_000:
        attempts += 1
        ci = int(rng.integers(len(sizes)))
        b = sizes[ci]
        ny, nx = H // b, W // b
        y = int(rng.integers(ny)) * b
        x = int(rng.integers(nx)) * b
        if y + b > H or x + b > W:
            continue
        sl = occ[y // g:(y + b) // g, x // g:(x + b) // g]
        if sl.any():
            continue
        sl[...] = True
        out.append((image, x, y, ci))
        lost += b * b
    out.sort(key=lambda t: (t[2], t[1]))
    return np.array(out, dtype=np.int32).reshape(-1, 4)


def loss_mask(blocks: np.ndarray, sizes, n_images: int, H: int, W: int) -> np.ndarray:
    """uint8 mask [N, H, W] with 1 on every lost sample.  ``sizes[cls]`` is
    the block edge of each class."""
    m = np.zeros((n_images, H, W), dtype=np.uint8)
    for im, x, y, c in np.asarray(blocks).reshape(-1, 4):
        b = sizes[int(c)]
        m[int(im), int(y):int(y) + b, int(x):int(x) + b] = 1
    return m


def noisy_estimates(seed: int, images: np.ndarray, blocks: np.ndarray, classes, sigma: float = 8.0,
                    stride: int | None = None) -> np.ndarray:
    """Seeded stand-ins for an initial estimate of each block's area: the
    unlost image over the area (edge-clamped outside the image) plus Gaussian
    noise of standard deviation sigma.  Returns float32 [n_blocks, stride]
    (area row-major in the first M*M entries)."""
    rng = np.random.default_rng(seed)
    blocks = np.asarray(blocks).reshape(-1, 4)
    Ms = [c["block"] + 2 * c["border"] for c in classes]
    stride = stride or max(M * M for M in Ms)
    est = np.zeros((len(blocks), stride), np.float32)
    for i, (im, x, y, c) in enumerate(blocks):
        d, M = classes[c]["border"], Ms[c]
        H, W = images.shape[1:]
        ys = np.clip(np.arange(y - d, y - d + M), 0, H - 1)
        xs = np.clip(np.arange(x - d, x - d + M), 0, W - 1)
        a = images[im][np.ix_(ys, xs)].astype(np.float64) + rng.normal(0.0, sigma, (M, M))
        est[i, :M * M] = a.ravel()
    return est


def grid_mask_torch(blocks: np.ndarray, b: int, n_images: int, H: int, W: int, device="cuda"):
    """Loss mask [N, H, W] uint8 on ``device`` for b-aligned grid blocks."""
    import torch
    cells = torch.zeros((n_images, (H + b - 1) // b, (W + b - 1) // b), dtype=torch.uint8)
    bt = torch.from_numpy(np.asarray(blocks, dtype=np.int64).reshape(-1, 4))
    cells[bt[:, 0], bt[:, 2] // b, bt[:, 1] // b] = 1
    full = cells.to(device).repeat_interleave(b, 1).repeat_interleave(b, 2)
    return full[:, :H, :W].contiguous()
