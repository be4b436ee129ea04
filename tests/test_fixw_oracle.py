"""Pins of the oracle's reduced-precision residual storage (oracle.cfse with
wfix_from = K): the residual updates of iterations K, K+1, ... read W as
16-bit fixed-point codes of W / W[0,0] (scale 32767), the form the
Conclusion's remark on fixed-point arithmetic suggests for the spectrum the
update re-reads I times.

Each test ties the mode to something other than its own code: the exact
oracle where the codes are exact or never used, the incremental-residual
identity of Eq. (18) with the quantised spectrum, the Hermitian symmetry a
real weight gives W, and the 1e-2 pixel bar against the exact oracle.
"""
import numpy as np
import pytest

import oracle
from oracle import image as oimage
from paper_2204_14193_gb300 import synth

FIX_FROM = 20     # FP32 updates before the switch (the kernel's switch point)


def _rand_support_w(rng, F, M, rho=0.8, hole=16):
    sup = np.ones((M, M), np.uint8)
    a = (M - hole) // 2
    sup[a:a + hole, a:a + hole] = 0
    sup[rng.random((M, M)) < 0.1] = 0
    w = oracle.weight(M, M, rho, sup)
    o = (F - M) // 2
    wg = np.zeros((F, F))
    wg[o:o + M, o:o + M] = w
    return wg


def _same(a, b):
    for f in ("sel", "coef", "e_sel", "e_max", "e_second", "g", "R", "W"):
        assert np.array_equal(getattr(a, f), getattr(b, f)), f


def test_fix_code_closed_forms():
    """Codes the definition fixes: 0, +-W00 -> +-32767, W00/2 -> 16384
    (16383.5 rounds to the even neighbour), out-of-range magnitudes held to
    +-32767, and odd symmetry (round to nearest is symmetric)."""
    for W00 in (1.0, 64.0, 1024.0, 1587.25):
        assert oracle.fix_code(0.0, W00) == 0
        assert oracle.fix_code(W00, W00) == 32767
        assert oracle.fix_code(-W00, W00) == -32767
        assert oracle.fix_code(1.5 * W00, W00) == 32767
        assert oracle.fix_code(-3.0 * W00, W00) == -32767
    assert oracle.fix_code(512.0, 1024.0) == 16384
    assert oracle.fix_code(-512.0, 1024.0) == -16384
    rng = np.random.default_rng(3)
    for x in rng.uniform(-900.0, 900.0, 200):
        c = oracle.fix_code(x, 900.0)
        assert oracle.fix_code(-x, 900.0) == -c
        # the nearest code: within half a step of x / W00 * 32767 (up to the
        # FP32 decision)
        assert abs(c - x / 900.0 * 32767.0) <= 0.5 + 1e-3


def test_fix_code_matches_float32_rounding():
    """The decision is round-to-nearest-even of an FP32 product: compare
    with numpy's float32 arithmetic and np.rint on random values."""
    rng = np.random.default_rng(4)
    for W00 in rng.uniform(50.0, 3000.0, 8):
        qs = np.float32(32767.0) * (np.float32(1.0) / np.float32(W00))
        for x in rng.uniform(-W00, W00, 100):
            want = int(np.clip(np.rint(np.float32(x) * qs), -32767, 32767))
            assert oracle.fix_code(x, W00) == want


@pytest.mark.parametrize("K", [60, 61, 1000])
def test_switch_at_or_after_the_last_update_is_the_exact_oracle(K):
    """wfix_from >= I never reads the codes: bit-identical to Algorithm 1."""
    F, I = 32, 60
    rng = np.random.default_rng(11)
    s = rng.normal(120, 40, (F, F))
    w = _rand_support_w(rng, F, 24, hole=8)
    _same(oracle.cfse(s, w, 0.5, I), oracle.cfse(s, w, 0.5, I, wfix_from=K))


def test_exact_codes_reproduce_the_exact_oracle():
    """w = 1 on the sub-lattice (a F/4, b F/4): W is 16 on the bins with
    k, l = 0 mod 4 and 0 elsewhere, so every code is exact (0 or 32767)
    and the fixed-point run equals the exact one from the first update."""
    F, I = 32, 40
    w = np.zeros((F, F))
    w[::F // 4, ::F // 4] = 1.0
    rng = np.random.default_rng(12)
    s = rng.normal(120, 40, (F, F))
    a = oracle.cfse(s, w, 0.5, I)
    b = oracle.cfse(s, w, 0.5, I, wfix_from=0)
    assert set(np.unique(np.round(a.W.real, 9))) == {0.0, 16.0}
    _same(a, b)


@pytest.mark.parametrize("K", [0, 7, FIX_FROM])
def test_incremental_residual_with_quantised_spectrum(K):
    """Eq. (18) with the switch: after I updates the residual equals
    FFT{w s} - FFT{w g_K} - FFT{w_q (g_I - g_K)}, where g_K is the model of
    the first K coefficients and w_q = IFFT{W_q} the weight whose spectrum
    is the quantised W.  W_q keeps the Hermitian symmetry of W (round to
    nearest is odd), so w_q is real.  A switch one iteration early or late
    leaves a residual error of |c_K| |W - W_q|, far above FP64 rounding."""
    F, I = 64, 50
    rng = np.random.default_rng(13)
    s = rng.normal(120, 40, (F, F))
    w = _rand_support_w(rng, F, 48)
    r = oracle.cfse(s, w, 0.5, I, wfix_from=K)
    W = np.fft.fft2(w)
    W00 = W[0, 0].real
    code = np.vectorize(lambda x: oracle.fix_code(x, W00))
    Wq = (code(W.real) + 1j * code(W.imag)) * W00 / 32767.0
    wq = np.fft.ifft2(Wq)
    assert np.max(np.abs(wq.imag)) <= 1e-12 * W00
    m = np.arange(F)

    def model(sel, coef):
        g = np.zeros((F, F), complex)
        for p, c in zip(sel, coef):
            u, v = divmod(int(p), F)
            g += c * np.exp(2j * np.pi * (u * m[:, None] + v * m[None, :]) / F)
        return g

    gK = model(r.sel[:K], r.coef[:K])
    gI = model(r.sel, r.coef)
    want = np.fft.fft2(w * s) - np.fft.fft2(w * gK) - np.fft.fft2(wq.real * (gI - gK))
    scale = np.max(np.abs(np.fft.fft2(w * s)))
    assert np.max(np.abs(r.R - want)) <= 1e-10 * scale
    # and the same identity with the switch moved by one fails
    for K2 in (K - 1, K + 1):
        if 0 <= K2 < I:
            g2 = model(r.sel[:K2], r.coef[:K2])
            alt = np.fft.fft2(w * s) - np.fft.fft2(w * g2) - np.fft.fft2(wq.real * (gI - g2))
            assert np.max(np.abs(r.R - alt)) > 1e3 * 1e-10 * scale


DELTA_FIX = 5e-3   # bound on the quantised residual's relative energy deviation (measured 2.2e-3)


@pytest.fixture(scope="module")
def against_exact():
    """Each of 12 lost blocks of a synthetic 512 x 512 image (F = 64,
    I = 200): the fixed-point run (switch at K) and the exact oracle replayed
    along its selections (guided replay).  Returns, per K, rows of
    (1 - e_sel / e_max of the exact residual at the worst pick, largest
    relative deviation of the fixed run's energies from the exact ones,
    largest pixel difference on B)."""
    H = W = 512
    img = synth.make_image(5, H, W)
    blocks = synth.grid_losses(6, H, W, 16, 0.10, non_adjacent=True)[:12]
    mask = synth.loss_mask(blocks, [16], 1, H, W)[0]
    out = {}
    for K in (0, FIX_FROM):
        rows = []
        for _i, x, y, _c in blocks:
            s, w, off = oimage.area_inputs(img, mask, int(x), int(y), 16, 16, 64, 0.8)
            fx = oracle.cfse(s, w, 0.5, 200, wfix_from=K)
            gd = oracle.cfse(s, w, 0.5, 200, forced=fx.sel)
            gap = 1.0 - gd.e_sel / gd.e_max
            delta = np.abs(fx.e_sel - gd.e_sel) / gd.e_sel
            r0 = off + 16
            pix = np.abs(fx.g.real - gd.g.real)[r0:r0 + 16, r0:r0 + 16].max()
            rows.append((gap.max(), delta.max(), pix))
        out[K] = np.array(rows)
    return out


def test_fixed_point_picks_are_near_argmaxes_of_the_exact_residual(against_exact):
    """The fixed-point run picks the argmax of its own residual, whose
    energies deviate from the exact ones by some delta (relative), so each
    pick is a (1 - 2 delta)-argmax of the exact residual along the same
    selections (delta as measured at the picks); delta stays below
    DELTA_FIX from the switch at K on."""
    a = against_exact[FIX_FROM]
    assert np.all(a[:, 1] <= DELTA_FIX)
    assert np.all(a[:, 0] <= 2.0 * a[:, 1] / (1.0 - a[:, 1]) + 1e-12)


def test_fixed_point_from_the_switch_meets_the_pixel_bar(against_exact):
    """Replayed along the fixed-point run's selections, the exact oracle's
    B samples lie within the 1e-2 pixel bar of the fixed-point run."""
    assert against_exact[FIX_FROM][:, 2].max() <= 1e-2


def test_fixed_point_from_the_start_misses_the_pixel_bar(against_exact):
    """Why the switch exists: codes from the first update move most blocks by
    more than 1e-2 along the same selections (the early coefficients are the
    large ones, and the update error is |c| |W - W_q|)."""
    assert np.mean(against_exact[0][:, 2] > 1e-2) >= 0.5
