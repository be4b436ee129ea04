"""Pins of the FP64 oracle against things other than itself.

Each test ties one part of the oracle to a library routine, a brute-force
evaluation of the paper's spatial-domain definitions, a closed form derived by
hand (tests/golden), or an invariant that follows from the paper's equations.
"""
import os

import numpy as np
import pytest

import oracle
from oracle import image as oimage

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    rows = []
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            rows.append(line.split())
    return rows


def _rand_support_w(rng, F, M=None, rho=0.8, hole=None):
    """A weighting function of Eq. (3) on an M x M area centred in F x F,
    with a centred square hole of edge ``hole`` and a few random exclusions."""
    M = M or F
    sup = np.ones((M, M), np.uint8)
    if hole:
        a = (M - hole) // 2
        sup[a:a + hole, a:a + hole] = 0
    sup[rng.random((M, M)) < 0.1] = 0
    w = oracle.weight(M, M, rho, sup)
    o = (F - M) // 2
    wg = np.zeros((F, F))
    wg[o:o + M, o:o + M] = w
    return wg


# --------------------------------------------------------------------- FFT
@pytest.mark.parametrize("F", [2, 4, 8, 16])
def test_fft_matches_direct_dft(F):
    rng = np.random.default_rng(F)
    x = rng.normal(size=(F, F)) + 1j * rng.normal(size=(F, F))
    for inv in (False, True):
        a = oracle.fft2(x, inverse=inv)
        b = oracle.dft2_direct(x, inverse=inv)
        assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(b))


@pytest.mark.parametrize("F", [16, 32, 64])
def test_fft_matches_numpy(F):
    rng = np.random.default_rng(100 + F)
    x = rng.normal(size=(F, F)) + 1j * rng.normal(size=(F, F))
    a = oracle.fft2(x)
    b = np.fft.fft2(x)
    assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(b))
    ai = oracle.fft2(x, inverse=True)
    bi = np.fft.ifft2(x) * F * F
    assert np.max(np.abs(ai - bi)) <= 1e-12 * np.max(np.abs(bi))


def test_fft_rejects_non_power_of_two():
    with pytest.raises(ValueError):
        oracle.fft2(np.zeros((12, 12)))


# --------------------------------------------------------------- weighting
def test_weight_pythagorean_distances():
    # M = 11: the centre sample is (5, 5).  Offsets (3, 4) and (4, 3) lie at
    # Euclidean distance 5, (0, 5) too, (5, 0) too: all get rho^5; offset
    # (0, 0) is the centre itself: rho^0 = 1.
    rho = 0.8
    sup = np.ones((11, 11), np.uint8)
    w = oracle.weight(11, 11, rho, sup)
    for (dm, dn) in [(3, 4), (4, 3), (-3, 4), (3, -4), (0, 5), (5, 0), (-5, 0)]:
        assert w[5 + dm, 5 + dn] == pytest.approx(rho ** 5, rel=1e-14)
    assert w[5, 5] == 1.0
    # distance sqrt(2) from the centre: (rho^sqrt(2))^sqrt(2) = rho^2
    assert w[6, 6] ** np.sqrt(2.0) == pytest.approx(rho ** 2, rel=1e-14)


def test_weight_zero_on_loss_area_and_symmetric():
    rng = np.random.default_rng(3)
    M = 48
    sup = np.ones((M, M), np.uint8)
    sup[16:32, 16:32] = 0
    w = oracle.weight(M, M, 0.8, sup)
    assert np.all(w[16:32, 16:32] == 0)
    assert np.all(w[sup == 1] > 0)
    # the 8 symmetries of the square leave a centred area's weights unchanged
    for t in (w.T, w[::-1], w[:, ::-1], np.rot90(w)):
        assert np.allclose(t, w, rtol=1e-14, atol=0)
    # exponent property: w(rho1) * w(rho2) = w(rho1 * rho2)
    w1 = oracle.weight(M, M, 0.9, sup)
    w2 = oracle.weight(M, M, 0.7, sup)
    w12 = oracle.weight(M, M, 0.63, sup)
    assert np.allclose(w1 * w2, w12, rtol=1e-12, atol=0)
    # rho = 1: every support sample has weight one
    assert np.all(oracle.weight(M, M, 1.0, sup) == sup)
    del rng


# -------------------------------------------------- Algorithm 1 vs spatial
@pytest.mark.parametrize("F,I", [(4, 12), (8, 20), (16, 8)])
def test_frequency_domain_matches_spatial_brute_force(F, I):
    """Section III: the frequency-domain selection and updates (Algorithm 1)
    equal the spatial-domain definitions evaluated literally."""
    rng = np.random.default_rng(7 * F + I)
    s = rng.normal(50, 20, (F, F)) + 1j * rng.normal(0, 20, (F, F))
    w = _rand_support_w(rng, F, hole=F // 4)
    fr = oracle.cfse(s, w, 0.5, I)
    sel, coef, crit, g = oracle.cfse_spatial(s, w, 0.5, I)
    assert np.array_equal(fr.sel, sel)
    assert np.max(np.abs(fr.coef - coef)) <= 1e-10 * np.max(np.abs(coef))
    # criterion |p|^2 sum(phi* w phi) = |R_w|^2 / W[0,0]
    assert np.allclose(crit, fr.e_sel / fr.W[0, 0].real, rtol=1e-9)
    assert np.max(np.abs(fr.g - g)) <= 1e-10 * np.max(np.abs(g))


def test_real_input_brute_force_modulo_mirror():
    """Real input: |R_w[k]| = |R_w[-k]| exactly, so the first pick may be
    either of a conjugate pair; Re{g} agrees either way."""
    F, I = 8, 16
    rng = np.random.default_rng(11)
    s = rng.normal(100, 30, (F, F))
    w = _rand_support_w(rng, F, hole=2)
    fr = oracle.cfse(s, w, 0.5, I)
    sel, coef, crit, g = oracle.cfse_spatial(s, w, 0.5, I)
    mirror = lambda p: ((-(p // F)) % F) * F + ((-(p % F)) % F)  # noqa: E731
    same = np.array_equal(fr.sel, sel)
    mirrored = np.array_equal(np.array([mirror(p) for p in fr.sel]), sel)
    assert same or mirrored
    assert np.max(np.abs(fr.g.real - g.real)) <= 1e-9 * np.max(np.abs(g))


# --------------------------------------------------------------- invariants
def test_energy_identity_and_monotone_decrease():
    """E_nu = sum w |s - g_nu|^2 drops by exactly gamma (2 - gamma)
    |R_w[u,v]|^2 / W[0,0] per iteration (from the projection of Section III
    and the coefficient of Eq. (13)), so it never increases for 0 < gamma < 2."""
    F, I = 16, 40
    rng = np.random.default_rng(5)
    s = rng.normal(120, 40, (F, F))
    w = _rand_support_w(rng, F, M=12, hole=4)
    for gamma in (0.2, 0.5, 1.0, 1.7):
        r = oracle.cfse(s, w, gamma, I)
        m = np.arange(F)
        g = np.zeros((F, F), complex)
        E = [np.sum(w * np.abs(s - g) ** 2)]
        for p, c in zip(r.sel, r.coef):
            u, v = divmod(int(p), F)
            g = g + c * np.exp(2j * np.pi * (u * m[:, None] + v * m[None, :]) / F)
            E.append(np.sum(w * np.abs(s - g) ** 2))
        E = np.array(E)
        drop = gamma * (2 - gamma) * r.e_sel / r.W[0, 0].real
        assert np.allclose(E[:-1] - E[1:], drop, rtol=1e-7, atol=1e-9 * E[0])
        assert np.all(np.diff(E) <= 1e-9 * E[0])
        # the model built from the coefficient list equals IFFT{G}
        assert np.max(np.abs(g - r.g)) <= 1e-9 * np.max(np.abs(g))


def test_incremental_residual_equals_recomputed():
    """R_w after the updates of Eq. (18) equals FFT{w (s - g)} from scratch."""
    F, I = 64, 60
    rng = np.random.default_rng(9)
    s = rng.normal(120, 40, (F, F))
    w = _rand_support_w(rng, F, M=48, hole=16)
    r = oracle.cfse(s, w, 0.5, I)
    R2 = np.fft.fft2(w * (s - r.g))
    assert np.max(np.abs(r.R - R2)) <= 1e-9 * np.max(np.abs(np.fft.fft2(w * s)))
    assert np.max(np.abs(r.W - np.fft.fft2(w))) <= 1e-12 * np.sum(w)


def test_shift_placement_invariance():
    """Circularly shifting s and w on the F grid shifts g and keeps picks."""
    F, I = 32, 30
    rng = np.random.default_rng(21)
    s = rng.normal(120, 40, (F, F))
    w = _rand_support_w(rng, F, M=24, hole=8)
    r0 = oracle.cfse(s, w, 0.5, I)
    a, b = 5, -3
    r1 = oracle.cfse(np.roll(s, (a, b), (0, 1)), np.roll(w, (a, b), (0, 1)), 0.5, I)
    mirror = lambda p: ((-(p // F)) % F) * F + ((-(p % F)) % F)  # noqa: E731
    assert (np.array_equal(r0.sel, r1.sel)
            or np.array_equal(np.array([mirror(p) for p in r0.sel]), r1.sel))
    assert np.max(np.abs(np.roll(r0.g.real, (a, b), (0, 1)) - r1.g.real)) <= 1e-9 * 255


def test_positive_scale_equivariance():
    F, I = 32, 30
    rng = np.random.default_rng(22)
    s = rng.normal(120, 40, (F, F)) + 1j * rng.normal(0, 10, (F, F))
    w = _rand_support_w(rng, F, M=24, hole=8)
    r0 = oracle.cfse(s, w, 0.5, I)
    r1 = oracle.cfse(4.0 * s, w, 0.5, I)   # power of two: exact scaling
    assert np.array_equal(r0.sel, r1.sel)
    assert np.allclose(4.0 * r0.g, r1.g, rtol=1e-12, atol=1e-12)


def test_conjugate_mirror_trajectory():
    """Real input: forcing the mirror bin at every step gives g' = conj(g)."""
    F, I = 16, 25
    rng = np.random.default_rng(23)
    s = rng.normal(120, 40, (F, F))
    w = _rand_support_w(rng, F, M=12, hole=4)
    r0 = oracle.cfse(s, w, 0.5, I)
    mir = np.array([((-(p // F)) % F) * F + ((-(p % F)) % F) for p in r0.sel], np.int32)
    r1 = oracle.cfse(s, w, 0.5, I, forced=mir)
    assert np.max(np.abs(r1.g - np.conj(r0.g))) <= 1e-9 * 255
    assert np.allclose(r1.coef, np.conj(r0.coef), rtol=1e-9, atol=1e-9)


# -------------------------------------------------------------- closed forms
def test_golden_constant_support():
    F = 64
    rng = np.random.default_rng(1)
    w = _rand_support_w(rng, F, M=48, hole=16)
    for c, gamma, I, expect in _rows("constant_support.txt"):
        c, gamma, I, expect = float(c), float(gamma), int(I), float(expect)
        r = oracle.cfse(np.full((F, F), c), w, gamma, I)
        assert np.all(r.sel == 0)
        assert np.max(np.abs(r.g - expect)) <= 1e-10 * c


def test_golden_f2_ties():
    rows = _rows("f2_delta_ties.txt")
    s = np.zeros((2, 2))
    s[0, 0] = 1.0
    r = oracle.cfse(s, np.ones((2, 2)), 1.0, 4)
    sel = [int(rw[1]) for rw in rows if rw[0] != "g"]
    coef = [float(rw[2]) + 1j * float(rw[3]) for rw in rows if rw[0] != "g"]
    g = [float(v) for rw in rows if rw[0] == "g" for v in rw[1:]]
    assert list(r.sel) == sel
    assert np.allclose(r.coef, coef, atol=1e-15)
    assert np.allclose(r.g.real.ravel(), g, atol=1e-15) and np.allclose(r.g.imag, 0, atol=1e-15)


def test_golden_single_basis_recovery():
    for F, k0, l0, ar, ai, idx in _rows("single_basis.txt"):
        F, k0, l0, idx = int(F), int(k0), int(l0), int(idx)
        a = float(ar) + 1j * float(ai)
        rng = np.random.default_rng(F + k0)
        M = 3 * F // 4
        w = _rand_support_w(rng, F, M=M, hole=F // 4)
        m = np.arange(F)
        phi = np.exp(2j * np.pi * (k0 * m[:, None] + l0 * m[None, :]) / F)
        s = a * phi
        if ai == "0.0" and (k0 in (0, F // 2)) and (l0 in (0, F // 2)):
            s = s.real                      # real-valued special case
        r = oracle.cfse(s, w, 1.0, 1)
        assert r.sel[0] == idx
        assert abs(r.coef[0] - a) <= 1e-12 * abs(a)
        assert np.max(np.abs(r.R)) <= 1e-10 * abs(a) * r.W[0, 0].real
        assert np.max(np.abs(r.g - s)) <= 1e-12 * abs(a)


# ------------------------------------------------------------- degenerate
def test_zero_iterations_and_no_support():
    F = 16
    rng = np.random.default_rng(2)
    s = rng.normal(100, 10, (F, F))
    w = _rand_support_w(rng, F, hole=4)
    r = oracle.cfse(s, w, 0.5, 0)
    assert r.sel.size == 0 and np.all(r.g == 0)
    r = oracle.cfse(s, np.zeros((F, F)), 0.5, 5)
    assert np.all(r.g == 0)


# ------------------------------------------------------- image-level driver
def test_image_driver_block_semantics():
    """Blocks at the image border and diagonal neighbours: samples outside
    the image or lost in any block get weight 0; a constant image is then
    extended by the closed form of constant_support.txt."""
    H = W = 64
    img = np.full((1, H, W), 90, np.uint8)
    blocks = np.array([[0, 0, 0, 0], [0, 16, 16, 0], [0, 48, 48, 0]], np.int32)
    mask = np.zeros((1, H, W), np.uint8)
    for _, x, y, _c in blocks:
        mask[0, y:y + 16, x:x + 16] = 1
    cls = [dict(block=16, border=16, fft=64, rho=0.8, gamma=0.5, iters=10)]
    patches, res = oimage.conceal(img, mask, blocks, cls, keep_results=True)
    for p in patches:
        assert np.allclose(p, 90 * (1 - 0.5 ** 10), atol=1e-9)
    # the corner block's area reaches 16 samples past the image edge
    s_grid, w_grid, off = oimage.area_inputs(img[0], mask[0], 0, 0, 16, 16, 64, 0.8)
    assert off == 8 and np.all(w_grid[:off + 16, :] == 0) and np.all(w_grid[:, :off + 16] == 0)
    # block (16,16)'s area contains the lost corner block (0..15) -> weight 0
    s_grid, w_grid, off = oimage.area_inputs(img[0], mask[0], 16, 16, 16, 16, 64, 0.8)
    assert np.all(w_grid[off:off + 16, off:off + 16] == 0)
    assert np.all(w_grid[off + 16:off + 32, off + 16:off + 32] == 0)
