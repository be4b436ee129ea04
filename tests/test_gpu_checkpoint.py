"""Checkpoint and resume of the network training: the full state (master
parameters, Adam moments and step count, the minibatch generator, the loop
position) saved half-way and restored in a new network continues bit for bit
as the uninterrupted run."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2204_14193_gb300 as P
    return P


def _set(seed, n, M):
    rng = np.random.default_rng(seed)
    sup = (rng.random((n, M, M)) > 0.3).astype(np.float32)
    x = np.stack([rng.uniform(0, 1, (n, M, M)).astype(np.float32) * sup, sup], axis=1)
    t = rng.uniform(0, 1, (n, M, M)).astype(np.float32)
    lam = rng.uniform(0.5, 2.0, (n, M, M)).astype(np.float32)
    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (x, t, lam)]


def test_state_round_trip(P):
    net = P.Cnn(48, 48, max_batch=8)
    net.set_params(P.he_init(21))
    x, t, lam = _set(22, 8, 48)
    for _ in range(3):
        net.train_step(x, t, lam, lr=1e-3)
    p, m, v, step = net.get_state()
    assert step == 3 and np.any(m != 0) and np.all(v >= 0)
    other = P.Cnn(48, 48, max_batch=8)
    other.set_state(p, m, v, step)
    p2, m2, v2, step2 = other.get_state()
    for a, b in ((p, p2), (m, m2), (v, v2)):
        np.testing.assert_array_equal(a, b)
    assert step2 == step
    # both continue identically
    net.train_step(x, t, lam, lr=1e-3)
    other.train_step(x, t, lam, lr=1e-3)
    np.testing.assert_array_equal(net.get_params(), other.get_params())
    net.close()
    other.close()


def test_training_resumes_bit_for_bit(P, tmp_path):
    from paper_2204_14193_gb300 import train_init as T
    x, t, lam = _set(23, 64, T.M)
    steps, batch, lr, seed = 40, 16, 2e-3, 9
    full, hist_full = T.train(x, t, lam, steps, batch, lr, seed, log_every=10)
    ck = str(tmp_path / "state.npz")
    T.train(x, t, lam, steps, batch, lr, seed, log_every=10, checkpoint=ck, stop_at=17)
    resumed, hist_res = T.train(x, t, lam, steps, batch, lr, seed, log_every=10, checkpoint=ck, resume=ck)
    np.testing.assert_array_equal(full, resumed)
    assert [h[:2] for h in hist_full] == [h[:2] for h in hist_res]
    z = np.load(ck)
    assert int(z["k"]) == steps and int(z["adam_step"]) == steps
    # a checkpoint of another run is refused
    with pytest.raises(ValueError):
        T.train(x, t, lam, steps + 1, batch, lr, seed, checkpoint=None, resume=ck)
