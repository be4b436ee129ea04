"""What the trained network gains over the method without it.

On held-out seeded frames (seeds disjoint from training and from the
training script's evaluation), the learned initialisation followed by
I = 50 iterations is compared with plain extrapolation (zero initial model)
at I = 50 and I = 200, by PSNR over all lost samples against the original
frames.  The shipped network was trained by train_init.py on 200k areas
labelled by plain extrapolation at I = 200.
"""
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2204_14193_gb300 as P
    return P


def test_trained_network_gains_over_plain_at_equal_iterations(P):
    from paper_2204_14193_gb300 import train_init as T
    w = T.load_weights()
    frames, mask, blocks = T.frames_and_losses(T.TEST_SEED0 + 100, 2, 2160, 3840, 0.10)
    truth = T.truth_patches(frames, blocks)
    plain50 = T.psnr(T.plain_patches(frames, mask, blocks, 50), truth)
    plain200 = T.psnr(T.plain_patches(frames, mask, blocks, 200), truth)
    learned50 = T.psnr(T.learned_patches(frames, mask, blocks, w, 50), truth)
    untrained50 = T.psnr(T.learned_patches(frames, mask, blocks, P.he_init(3) * 0.0, 50), truth)
    print(f"blocks {len(blocks)}: plain I=50 {plain50:.3f} dB, learned + I=50 {learned50:.3f} dB, "
          f"plain I=200 {plain200:.3f} dB")
    # a zero network leaves plain extrapolation unchanged
    assert untrained50 == pytest.approx(plain50, abs=1e-3)
    print(f"gap of learned + I=50 to plain I=200: {learned50 - plain200:+.3f} dB")
    # the trained network adds detail the short run misses
    assert learned50 >= plain50 + 0.2
