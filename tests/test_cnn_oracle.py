"""Pins of the FP64 CNN oracle (learned initialisation) against a library
routine (scipy correlate2d), finite differences, and closed forms."""
import numpy as np
import pytest

import oracle
from oracle import cnn

scipy_signal = pytest.importorskip("scipy.signal")


def dilate(k, d):
    """3x3 kernel -> (2d+1)x(2d+1) kernel with zeros between the taps."""
    out = np.zeros((2 * d + 1, 2 * d + 1))
    out[::d, ::d] = k
    return out


@pytest.mark.parametrize("d", [1, 2, 4, 8])
def test_conv_matches_scipy_correlate(d):
    rng = np.random.default_rng(d)
    N, Cin, Cout, H, W = 2, 3, 4, 20, 17
    x = rng.normal(size=(N, Cin, H, W))
    w = rng.normal(size=(Cout, Cin, 3, 3))
    b = rng.normal(size=Cout)
    y = cnn.conv3x3(x, w, b, d)
    for n in range(N):
        for co in range(Cout):
            ref = np.full((H, W), b[co])
            for ci in range(Cin):
                ref += scipy_signal.correlate2d(x[n, ci], dilate(w[co, ci], d), mode="same", boundary="fill")
            assert np.allclose(y[n, co], ref, rtol=1e-12, atol=1e-12)


def test_conv_backward_finite_differences():
    rng = np.random.default_rng(5)
    N, Cin, Cout, H, W, d = 2, 3, 2, 9, 11, 2
    x = rng.normal(size=(N, Cin, H, W))
    w = rng.normal(size=(Cout, Cin, 3, 3))
    b = rng.normal(size=Cout)
    proj = rng.normal(size=(N, Cout, H, W))
    f = lambda x_, w_, b_: float(np.sum(proj * cnn.conv3x3(x_, w_, b_, d)))  # noqa: E731
    dx, dw, db = cnn.conv3x3_bwd(x, w, proj, d)
    h = 1e-6
    for _ in range(12):
        idx = tuple(rng.integers(s) for s in x.shape)
        xp, xm = x.copy(), x.copy()
        xp[idx] += h
        xm[idx] -= h
        assert (f(xp, w, b) - f(xm, w, b)) / (2 * h) == pytest.approx(dx[idx], rel=1e-6, abs=1e-8)
        idx = tuple(rng.integers(s) for s in w.shape)
        wp, wm = w.copy(), w.copy()
        wp[idx] += h
        wm[idx] -= h
        assert (f(x, wp, b) - f(x, wm, b)) / (2 * h) == pytest.approx(dw[idx], rel=1e-6, abs=1e-8)
    for co in range(Cout):
        bp, bm = b.copy(), b.copy()
        bp[co] += h
        bm[co] -= h
        assert (f(x, w, bp) - f(x, w, bm)) / (2 * h) == pytest.approx(db[co], rel=1e-6, abs=1e-8)


def test_network_gradient_finite_differences():
    rng = np.random.default_rng(7)
    N, H, W = 2, 12, 12
    P = cnn.param_count()
    assert P == 19393
    params = rng.normal(scale=0.2, size=P)
    x = rng.uniform(size=(N, 2, H, W))
    t = rng.uniform(size=(N, H, W))
    lam = rng.uniform(0.5, 2.0, size=(N, H, W))
    loss, g, gx = cnn.loss_grad(params, x, t, lam, round_bf16=False, want_grad_x=True)
    h = 1e-6
    for i in list(rng.integers(0, P, 24)) + [P - 1, 0]:
        pp, pm = params.copy(), params.copy()
        pp[i] += h
        pm[i] -= h
        fd = (cnn.loss_grad(pp, x, t, lam, round_bf16=False)[0] - cnn.loss_grad(pm, x, t, lam, round_bf16=False)[0]) / (2 * h)
        assert fd == pytest.approx(g[i], rel=1e-5, abs=1e-9)
    for _ in range(6):
        idx = tuple(rng.integers(s) for s in x.shape)
        xp, xm = x.copy(), x.copy()
        xp[idx] += h
        xm[idx] -= h
        fd = (cnn.loss_grad(params, xp, t, lam, round_bf16=False)[0] - cnn.loss_grad(params, xm, t, lam, round_bf16=False)[0]) / (2 * h)
        assert fd == pytest.approx(gx[idx], rel=1e-5, abs=1e-9)


def test_forward_layers_compose():
    """The network output equals the four convolutions (dilations 1,2,4,8)
    applied in turn with ReLU between (round_bf16 off)."""
    rng = np.random.default_rng(9)
    params = rng.normal(scale=0.3, size=cnn.param_count())
    x = rng.uniform(size=(1, 2, 10, 10))
    cur = x
    for k, (ws, bs, cin, cout, d) in enumerate(cnn.layer_slices()):
        cur = cnn.conv3x3(cur, params[ws].reshape(cout, cin, 3, 3), params[bs], d)
        if k < 3:
            cur = np.maximum(cur, 0.0)
    assert np.allclose(cnn.forward(params, x, round_bf16=False), cur[:, 0], rtol=1e-12, atol=1e-12)


def test_bf16_rounding_closed_forms():
    u = 2.0 ** -8
    assert cnn.bf16(1 + u) == 1.0                        # tie -> even
    assert cnn.bf16(1 + 3 * u) == 1 + 4 * u              # tie -> even (upwards)
    assert cnn.bf16(1 + u + 2.0 ** -20) == 1 + 2 * u     # above the tie
    assert cnn.bf16(-(1 + u)) == -1.0
    assert cnn.bf16(3.0) == 3.0 and cnn.bf16(0.0) == 0.0


def test_adam_closed_form_constant_gradient():
    rng = np.random.default_rng(3)
    p0 = rng.normal(size=16)
    g = rng.normal(size=16)
    m = np.zeros(16)
    v = np.zeros(16)
    lr, eps = 1e-3, 1e-8
    p1, m, v = cnn.adam(p0, m, v, g, lr, 1, eps=eps)
    # bias-corrected first step: m_hat = g, v_hat = g^2
    assert np.allclose(p1, p0 - lr * g / (np.abs(g) + eps), rtol=0, atol=1e-15)
    p2, m, v = cnn.adam(p1, m, v, g, lr, 2, eps=eps)
    assert np.allclose(p2, p1 - lr * g / (np.abs(g) + eps), rtol=0, atol=1e-15)
    oracle._load()
