"""GPU parity of the learned-initialisation network (forward on the tensor
cores, FP32 backward, Adam) against the FP64 CNN oracle.

The oracle evaluates the same bf16-rounded weights, inputs and stored
activations in FP64; the GPU accumulates in FP32 in a different order, so a
stored activation can land on the other side of a bf16 rounding boundary.
Tolerances: forward, every output within 2^-6 of the output RMS and 99.9%
within 2^-9.  Gradients, element by element: |g - g_ref| <= GRAD_ATOL x the
RMS of the layer's reference weight (or bias) gradient + GRAD_RTOL x |g_ref|.
A gradient element sums, over every output position, products of a stored
bf16 activation (relative rounding 2^-9) and a back-propagated FP32 error
that itself carries the forward's bf16 differences; an element near zero is
a difference of such sums, hence the absolute part scaled by the layer's
RMS.  A stored activation that rounds the other way moves one term of such
a sum by at most 2^-8 of that term; the bounds are 2^-10 of the RMS plus
2^-10 relative (measured on the GB300: at most 1.5e-5 of the RMS).
"""
import numpy as np
import pytest

from oracle import cnn as ocnn

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2204_14193_gb300 as P
    return P


GRAD_ATOL = 2.0 ** -10   # x the layer's reference gradient RMS
GRAD_RTOL = 2.0 ** -10   # x |g_ref|


def _inputs(seed, n, H, W):
    rng = np.random.default_rng(seed)
    sup = (rng.random((n, H, W)) > 0.3).astype(np.float64)
    x = np.stack([rng.uniform(0, 1, (n, H, W)) * sup, sup], axis=1)
    t = rng.uniform(0, 1, (n, H, W))
    lam = rng.uniform(0.5, 2.0, (n, H, W))
    return x, t, lam


@pytest.mark.parametrize("n,H,W", [(3, 48, 48), (2, 20, 17)])
def test_forward_matches_oracle(P, n, H, W):
    params = P.he_init(11).astype(np.float64)
    params[np.arange(params.size) % 7 == 0] *= -1.0
    x, _, _ = _inputs(1, n, H, W)
    net = P.Cnn(H, W, max_batch=4)
    net.set_params(params.astype(np.float32))
    y = net.forward(torch.from_numpy(x.astype(np.float32)).cuda()).cpu().numpy().astype(np.float64)
    net.close()
    ref = ocnn.forward(params.astype(np.float32).astype(np.float64), x.astype(np.float32).astype(np.float64))
    rms = np.sqrt(np.mean(ref ** 2))
    d = np.abs(y - ref)
    print("forward: rms", rms, "max", d.max(), "p99.9", np.quantile(d, 0.999))
    assert d.max() <= 2.0 ** -6 * rms
    assert np.quantile(d, 0.999) <= 2.0 ** -9 * rms


def test_gradient_matches_oracle(P):
    n, H, W = 2, 48, 48
    params = P.he_init(12)
    x, t, lam = _inputs(2, n, H, W)
    xf, tf, lf = (a.astype(np.float32) for a in (x, t, lam))
    net = P.Cnn(H, W, max_batch=4)
    net.set_params(params)
    loss, g = net.loss_grad(torch.from_numpy(xf).cuda(), torch.from_numpy(tf).cuda(), torch.from_numpy(lf).cuda())
    net.close()
    rl, rg = ocnn.loss_grad(params.astype(np.float64), xf.astype(np.float64), tf.astype(np.float64),
                            lf.astype(np.float64))
    assert loss == pytest.approx(rl, rel=1e-3)
    for ws, bs, cin, cout, d in ocnn.layer_slices():
        for name, sl in (("weights", ws), ("biases", bs)):
            ref, got = rg[sl], g[sl].astype(np.float64)
            rms = max(np.sqrt(np.mean(ref ** 2)), 1e-30)
            excess = np.abs(got - ref) / (GRAD_ATOL * rms + GRAD_RTOL * np.abs(ref))
            print(f"layer dilation {d} {name}: max |d|/rms {np.max(np.abs(got - ref)) / rms:.2e}, "
                  f"worst element at {excess.max():.3f} of the bound")
            assert np.all(excess <= 1.0), (d, name, int(np.argmax(excess)), excess.max())


def test_adam_step_matches_oracle(P):
    n, H, W = 2, 24, 24
    params = P.he_init(13)
    x, t, lam = _inputs(3, n, H, W)
    xf, tf = (a.astype(np.float32) for a in (x, t))
    net = P.Cnn(H, W, max_batch=4)
    net.set_params(params)
    dx, dt = torch.from_numpy(xf).cuda(), torch.from_numpy(tf).cuda()
    _, g = net.loss_grad(dx, dt)
    lr = 1e-3
    net.train_step(dx, dt, lr=lr)
    p1 = net.get_params()
    net.close()
    want, _, _ = ocnn.adam(params.astype(np.float64), np.zeros(params.size), np.zeros(params.size),
                           g.astype(np.float64), lr, 1)
    assert np.max(np.abs(p1 - want)) <= 1e-6


def test_training_reduces_loss(P):
    n, H, W = 16, 48, 48
    rng = np.random.default_rng(4)
    x, _, _ = _inputs(4, n, H, W)
    t = 0.5 * x[:, 0] + 0.25      # a learnable target
    net = P.Cnn(H, W, max_batch=n)
    net.set_params(P.he_init(14))
    dx = torch.from_numpy(x.astype(np.float32)).cuda()
    dt = torch.from_numpy(t.astype(np.float32)).cuda()
    losses = [net.train_step(dx, dt, lr=3e-3) for _ in range(60)]
    net.close()
    print("loss", losses[0], "->", losses[-1])
    assert losses[-1] < 0.2 * losses[0]
    del rng
