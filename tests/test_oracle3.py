"""Pins of the 3-D (video volume) oracle against what the paper and the
mathematics fix: numpy's n-D FFT, the 2-D oracle when the volume has one
frame, brute force over the spatial-domain definitions on tiny grids, the
weighted-energy identity, and closed forms (constant support, a single 3-D
basis function recovered in one iteration at gamma = 1)."""
import numpy as np
import pytest

import oracle
from oracle import image as oimage


@pytest.mark.parametrize("Ft,F", [(1, 8), (2, 4), (4, 8), (4, 16), (4, 32), (8, 4)])
def test_fft3_matches_numpy(Ft, F):
    rng = np.random.default_rng(Ft * 100 + F)
    x = rng.normal(size=(Ft, F, F)) + 1j * rng.normal(size=(Ft, F, F))
    ref = np.fft.fftn(x)
    assert np.max(np.abs(oracle.fft3(x) - ref)) <= 1e-12 * np.max(np.abs(ref))
    back = oracle.fft3(ref, inverse=True) / x.size
    assert np.max(np.abs(back - x)) <= 1e-12 * np.max(np.abs(x))


def test_weight3_distances_and_reduction():
    rho = 0.8
    T, M = 3, 5                      # centre (1, 2, 2)
    w = oracle.weight3(T, M, rho, np.ones((T, M, M), np.uint8))
    assert w[1, 2, 2] == pytest.approx(1.0, abs=0)
    assert w[0, 2, 2] == pytest.approx(rho, rel=1e-15)                 # one frame away
    assert w[0, 0, 2] == pytest.approx(rho ** np.sqrt(5.0), rel=1e-15)  # (1, 2, 0)
    assert w[0, 0, 0] == pytest.approx(rho ** 3.0, rel=1e-15)           # (1, 2, 2): sqrt(9)
    np.testing.assert_array_equal(w, w[::-1])                          # symmetric in time
    # one frame: the 2-D weighting function of Eq. (3)
    rng = np.random.default_rng(3)
    sup = (rng.random((1, 7, 7)) > 0.3).astype(np.uint8)
    np.testing.assert_allclose(oracle.weight3(1, 7, 0.7, sup)[0], oracle.weight(7, 7, 0.7, sup[0]),
                               rtol=1e-15, atol=0)


@pytest.mark.parametrize("Ft,F,I", [(2, 4, 6), (4, 4, 5)])
def test_frequency_domain_matches_spatial_brute_force(Ft, F, I):
    rng = np.random.default_rng(Ft + F)
    s = rng.normal(size=(Ft, F, F)) + 1j * rng.normal(size=(Ft, F, F))
    w = rng.uniform(0.1, 1.0, size=(Ft, F, F)) * (rng.random((Ft, F, F)) > 0.25)
    res = oracle.cfse3(s, w, 0.6, I)
    sel, coef, g = oracle.cfse3_spatial(s, w, 0.6, I)
    np.testing.assert_array_equal(res.sel, sel)
    assert np.max(np.abs(res.coef - coef)) <= 1e-10
    assert np.max(np.abs(res.g - g)) <= 1e-10


def test_one_frame_is_the_2d_oracle():
    rng = np.random.default_rng(11)
    F = 16
    s = rng.normal(size=(F, F)) * 30 + 100
    w = oracle.weight(F, F, 0.8, (rng.random((F, F)) > 0.2).astype(np.uint8))
    r2 = oracle.cfse(s, w, 0.5, 25)
    r3 = oracle.cfse3(s[None], w[None], 0.5, 25)
    np.testing.assert_array_equal(r2.sel, r3.sel)
    assert np.max(np.abs(r2.coef - r3.coef)) <= 1e-9 * np.max(np.abs(r2.coef))
    assert np.max(np.abs(r2.g - r3.g[0])) <= 1e-9 * np.max(np.abs(r2.g))


def test_weighted_energy_identity():
    """E_nu = sum w |s - g_nu|^2 falls by gamma (2 - gamma) |R_w[pick]|^2 / W[0]
    at every iteration (W[0] = sum w)."""
    rng = np.random.default_rng(5)
    Ft, F, gamma = 4, 8, 0.7
    s = rng.normal(size=(Ft, F, F)) * 20 + 50
    w = rng.uniform(0.2, 1.0, size=(Ft, F, F)) * (rng.random((Ft, F, F)) > 0.3)
    W0 = w.sum()
    full = oracle.cfse3(s, w, gamma, 8)
    prev = np.sum(w * np.abs(s) ** 2)
    for nu in range(1, 9):
        g = oracle.cfse3(s, w, gamma, nu).g
        e = np.sum(w * np.abs(s - g) ** 2)
        assert prev - e == pytest.approx(gamma * (2 - gamma) * full.e_sel[nu - 1] / W0, rel=1e-9)
        prev = e


def test_constant_support_closed_form():
    """s = c on the support: every pick is the DC bin, g = c (1 - (1 - gamma)^I)."""
    rng = np.random.default_rng(8)
    Ft, F, c, gamma, I = 4, 16, 83.0, 0.5, 7
    w = rng.uniform(0.1, 1.0, size=(Ft, F, F)) * (rng.random((Ft, F, F)) > 0.4)
    res = oracle.cfse3(np.full((Ft, F, F), c), w, gamma, I)
    assert np.all(res.sel == 0)
    np.testing.assert_allclose(res.g, c * (1 - (1 - gamma) ** I), rtol=1e-12, atol=0)


def test_single_basis_recovered_in_one_iteration():
    Ft, F = 4, 16
    t, m, n = np.meshgrid(np.arange(Ft), np.arange(F), np.arange(F), indexing="ij")
    w0, u0, v0, c = 3, 5, 11, 2.5 - 1.25j
    phi = np.exp(2j * np.pi * (w0 * t / Ft + u0 * m / F + v0 * n / F))
    rng = np.random.default_rng(2)
    w = rng.uniform(0.1, 1.0, size=(Ft, F, F)) * (rng.random((Ft, F, F)) > 0.5)
    res = oracle.cfse3(c * phi, w, 1.0, 1)
    assert res.sel[0] == (w0 * F + u0) * F + v0
    assert res.coef[0] == pytest.approx(c, abs=1e-12)
    np.testing.assert_allclose(res.g, c * phi, rtol=0, atol=1e-12)


def test_area_inputs3_hand_case():
    """3 frames of 6 x 6, 2 x 2 block at (0, 0) of frame 1, 1-sample border:
    the volume's frames 0..2 at rows/columns -1..2; one further lost sample."""
    video = np.arange(3 * 36, dtype=np.float64).reshape(3, 6, 6)
    mask = np.zeros((3, 6, 6), np.uint8)
    mask[1, 0:2, 0:2] = 1           # the block
    mask[0, 1, 1] = 1               # lost in the previous frame
    s, w, toff, off = oimage.area_inputs3(video, mask, 1, 0, 0, 2, 1, 4, 4, 3, 0.5)
    assert (toff, off) == (0, 0)
    sup = w > 0
    # outside the video: row -1 and column -1 in every frame; the own block in
    # frame 1; the lost sample of frame 0 (volume position (0, 2, 2))
    assert not sup[:, 0, :].any() and not sup[:, :, 0].any()
    assert not sup[1, 1:3, 1:3].any()
    assert not sup[0, 2, 2]
    assert sup[0, 1, 1] and sup[2, 1, 1] and sup[1, 3, 3]
    assert not sup[3].any()         # temporal padding plane
    assert s[2, 1, 1] == video[2, 0, 0] and s[0, 3, 3] == video[0, 2, 2]
    # weights: centre (1, 1.5, 1.5); position (2, 1, 1) is at distance sqrt(1.5)
    assert w[2, 1, 1] == pytest.approx(0.5 ** np.sqrt(1.5), rel=1e-15)
