"""Image-level driver of the FP64 oracle (test infrastructure only).

For each lost block it builds the extrapolation area L = A u B of Fig. 1:
an M x M window (M = b + 2d) centred on the b x b loss area B, placed at
offset (F - M) // 2 of an F x F grid (the DFT period, Section IV uses a 64x64
FFT for a 48x48 area).  Samples of the window that fall outside the image, are
marked lost in the mask (any block) or belong to the block's own B are not
support: their weight is 0.
Eq. (3) then gives w on A, Algorithm 1 (``oracle.cfse``) the model g, and
Re{g} replaces the samples of B (the last loop of Algorithm 1).  Blocks are
concealed independently of each other from the original mask, except in
``conceal_ordered`` (earlier blocks' concealed samples reused as support).
``area_inputs3`` / ``conceal_block3`` build and conceal video volumes.
"""
from __future__ import annotations

from concurrent.futures import ThreadPoolExecutor
import os

import numpy as np

from . import cfse, cfse3, weight, weight3


def area_inputs(img: np.ndarray, mask: np.ndarray, x: int, y: int, b: int, d: int,
                F: int, rho: float):
    """Return (s_grid, w_grid, off): the F x F signal and weight of one block.

    img, mask: 2-D arrays of one image; (x, y) is the top-left sample of the
    lost block (x = column, y = row).
    """
    H, W = img.shape
    M = b + 2 * d
    off = (F - M) // 2
    ys = np.arange(y - d, y - d + M)
    xs = np.arange(x - d, x - d + M)
    inside = ((ys >= 0) & (ys < H))[:, None] & ((xs >= 0) & (xs < W))[None, :]
    yc = np.clip(ys, 0, H - 1)
    xc = np.clip(xs, 0, W - 1)
    s_area = img[np.ix_(yc, xc)].astype(np.float64)
    lost = mask[np.ix_(yc, xc)] != 0
    own_b = np.zeros((M, M), dtype=bool)
    own_b[d:d + b, d:d + b] = True          # Eq. (3): w = 0 on B
    support = inside & ~lost & ~own_b
    w_area = weight(M, M, rho, support.astype(np.uint8))
    s_grid = np.zeros((F, F))
    w_grid = np.zeros((F, F))
    s_grid[off:off + M, off:off + M] = np.where(support, s_area, 0.0)
    w_grid[off:off + M, off:off + M] = w_area
    return s_grid, w_grid, off


def cnn_input(img: np.ndarray, mask: np.ndarray, x: int, y: int, b: int, d: int) -> np.ndarray:
    """Input of the learned-initialisation network for one block: [2, M, M],
    channel 0 = support sample / 255 (0 off the support), channel 1 = the
    support indicator (inside the image, not lost, not in the block's B)."""
    H, W = img.shape
    M = b + 2 * d
    ys = np.arange(y - d, y - d + M)
    xs = np.arange(x - d, x - d + M)
    inside = ((ys >= 0) & (ys < H))[:, None] & ((xs >= 0) & (xs < W))[None, :]
    yc = np.clip(ys, 0, H - 1)
    xc = np.clip(xs, 0, W - 1)
    s_area = img[np.ix_(yc, xc)].astype(np.float64)
    own_b = np.zeros((M, M), dtype=bool)
    own_b[d:d + b, d:d + b] = True
    sup = inside & (mask[np.ix_(yc, xc)] == 0) & ~own_b
    return np.stack([np.where(sup, s_area / 255.0, 0.0), sup.astype(np.float64)])


def conceal_block_init(img, mask, x, y, cls, est, forced=None):
    """Warm start: Algorithm 1 on the residual s - est of the support (est:
    M x M estimate of the area, sample units); returns est + Re{g} on B."""
    b, d, F, rho, gamma, iters = (cls["block"], cls["border"], cls["fft"], cls["rho"],
                                  cls["gamma"], cls["iters"])
    s_grid, w_grid, off = area_inputs(img, mask, x, y, b, d, F, rho)
    M = b + 2 * d
    est = np.asarray(est, dtype=np.float64).reshape(M, M)
    e_grid = np.zeros((F, F))
    e_grid[off:off + M, off:off + M] = est
    s_res = np.where(w_grid > 0, s_grid - e_grid, 0.0)
    res = cfse(s_res, w_grid, gamma, iters, forced=forced)
    r0 = off + d
    patch = res.g.real[r0:r0 + b, r0:r0 + b] + est[d:d + b, d:d + b]
    return patch, res


def conceal_block(img, mask, x, y, cls, forced=None, wfix_from=None):
    """Run the oracle on one block; returns (patch b x b, CfseResult).
    wfix_from: reduced-precision residual storage from that iteration on
    (``oracle.cfse``)."""
    b, d, F, rho, gamma, iters = (cls["block"], cls["border"], cls["fft"], cls["rho"],
                                  cls["gamma"], cls["iters"])
    s_grid, w_grid, off = area_inputs(img, mask, x, y, b, d, F, rho)
    res = cfse(s_grid, w_grid, gamma, iters, forced=forced, wfix_from=wfix_from)
    r0 = off + d
    patch = res.g.real[r0:r0 + b, r0:r0 + b].copy()
    return patch, res


def conceal(images: np.ndarray, mask: np.ndarray, blocks: np.ndarray, classes,
            forced=None, threads: int | None = None, keep_results: bool = False,
            wfix_from: int | None = None):
    """Conceal every block of ``blocks`` (rows: image, x, y, class index).

    images: [N, H, W] (u8 or float); mask: [N, H, W] u8 (1 = lost).
    classes: list of dicts with keys block, border, fft, rho, gamma, iters.
    forced: optional list (per block) of forced selection sequences.
    wfix_from: reduced-precision residual storage (``oracle.cfse``).
    Returns (patches: list of b x b arrays, results or None).
    """
    images = np.asarray(images)
    mask = np.asarray(mask)
    blocks = np.asarray(blocks, dtype=np.int64).reshape(-1, 4)
    nthreads = threads or len(os.sched_getaffinity(0))

    def one(i):
        im, x, y, c = (int(v) for v in blocks[i])
        f = None if forced is None else forced[i]
        return conceal_block(images[im], mask[im], x, y, classes[c], forced=f, wfix_from=wfix_from)

    if len(blocks) == 0:
        return [], ([] if keep_results else None)
    with ThreadPoolExecutor(max_workers=nthreads) as ex:
        out = list(ex.map(one, range(len(blocks))))
    patches = [p for p, _ in out]
    return patches, ([r for _, r in out] if keep_results else None)


# ----------------------------------------------------------------- video volumes
def area_inputs3(video, mask, t0, x, y, b, d, F, Ft, T, rho):
    """Grid inputs of the 3-D extrapolation of the b x b block at (x, y) of
    frame t0: the T x M x M volume of frames t0 - (T-1)/2 .. t0 + (T-1)/2
    placed at offset ((Ft - T) // 2, (F - M) // 2, (F - M) // 2) of an
    Ft x F x F grid.  Support: inside the video, not lost, not the block
    itself (which is in the centre frame).  Returns (s_grid, w_grid, toff, off)."""
    NF, H, W = video.shape
    M = b + 2 * d
    tc = (T - 1) // 2
    sup = np.zeros((T, M, M), dtype=np.uint8)
    svol = np.zeros((T, M, M))
    for tau in range(T):
        f = t0 - tc + tau
        for m in range(M):
            for n in range(M):
                yy, xx = y - d + m, x - d + n
                own = tau == tc and d <= m < d + b and d <= n < d + b
                if 0 <= f < NF and 0 <= yy < H and 0 <= xx < W and not own and mask[f, yy, xx] == 0:
                    sup[tau, m, n] = 1
                    svol[tau, m, n] = float(video[f, yy, xx])
    w = weight3(T, M, rho, sup)
    toff, off = (Ft - T) // 2, (F - M) // 2
    s_grid = np.zeros((Ft, F, F))
    w_grid = np.zeros((Ft, F, F))
    s_grid[toff:toff + T, off:off + M, off:off + M] = svol
    w_grid[toff:toff + T, off:off + M, off:off + M] = w
    return s_grid, w_grid, toff, off


def conceal_block3(video, mask, t0, x, y, cls, forced=None):
    """The 3-D oracle on one block; cls has block, border, fft, fft_t, frames,
    rho, gamma, iters.  Returns (patch b x b, CfseResult)."""
    b, d, F, Ft, T = cls["block"], cls["border"], cls["fft"], cls["fft_t"], cls["frames"]
    s, w, toff, off = area_inputs3(video, mask, t0, x, y, b, d, F, Ft, T, cls["rho"])
    res = cfse3(s, w, cls["gamma"], cls["iters"], forced=forced)
    tc = toff + (T - 1) // 2
    return res.g.real[tc, off + d:off + d + b, off + d:off + d + b], res


# ----------------------------------------------------------- ordered concealment
def area_inputs_ordered(work, mask, reused, x, y, b, d, F, rho, beta):
    """Grid inputs when already-concealed samples count as support: `work`
    holds the original samples and the values concealed so far, `reused`
    marks the samples concealed so far (lost samples of earlier blocks).
    Support: inside the image and either not lost (weight w of Eq. (3)) or
    reused (weight beta w); the block's own B is excluded."""
    H, W = work.shape
    M = b + 2 * d
    off = (F - M) // 2
    ys = np.arange(y - d, y - d + M)
    xs = np.arange(x - d, x - d + M)
    inside = ((ys >= 0) & (ys < H))[:, None] & ((xs >= 0) & (xs < W))[None, :]
    yc = np.clip(ys, 0, H - 1)
    xc = np.clip(xs, 0, W - 1)
    s_area = work[np.ix_(yc, xc)].astype(np.float64)
    lost = mask[np.ix_(yc, xc)] != 0
    re = reused[np.ix_(yc, xc)]
    own_b = np.zeros((M, M), dtype=bool)
    own_b[d:d + b, d:d + b] = True
    support = inside & ~own_b & (~lost | re)
    w_area = weight(M, M, rho, support.astype(np.uint8)) * np.where(lost & re, beta, 1.0)
    s_grid = np.zeros((F, F))
    w_grid = np.zeros((F, F))
    s_grid[off:off + M, off:off + M] = np.where(support, s_area, 0.0)
    w_grid[off:off + M, off:off + M] = w_area
    return s_grid, w_grid, off


def conceal_ordered(images, mask, blocks, cls, beta, forced=None):
    """Blocks concealed one after another in the given order; each block's
    support also holds the samples of the blocks concealed before it (their
    concealed values, weight beta times Eq. (3)).  One class.  forced: None or
    per-block selection sequences for a guided replay.  Returns the list of
    (patch, CfseResult) and the working images."""
    work = np.asarray(images, dtype=np.float64).copy()
    reused = np.zeros(work.shape, dtype=bool)
    b, d, F = cls["block"], cls["border"], cls["fft"]
    out = []
    for j, (im, x, y, _c) in enumerate(np.asarray(blocks).reshape(-1, 4)):
        im, x, y = int(im), int(x), int(y)
        s, w, off = area_inputs_ordered(work[im], mask[im], reused[im], x, y, b, d, F, cls["rho"], beta)
        res = cfse(s, w, cls["gamma"], cls["iters"], forced=None if forced is None else forced[j])
        r0 = off + d
        patch = res.g.real[r0:r0 + b, r0:r0 + b].copy()
        work[im, y:y + b, x:x + b] = patch
        reused[im, y:y + b, x:x + b] = True
        out.append((patch, res))
    return out, work
