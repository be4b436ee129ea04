"""Failure detection without a GPU fault.

Bounded device waits: with the handle's wait limit set to 0 a wait expires at
its first failed poll; the kernel records it, waits (bounded) for its own
copies or MMAs in flight, and fse_sync reports FSE_ERR_TIMEOUT.  The handle
stays usable: with the default limit the same batch gives the normal result.
Three waits are exercised: the TMA gather of a 64 x 64-FFT window, an ordered
block's wait for the blocks it reuses, and the learned-initialisation
network's wait for its tensor-core MMAs.

Allocation failures are injected on the host (fse_test_fail_allocation):
every call that allocates returns FSE_ERR_OOM when one of its allocations
fails, leaks nothing (fse_test_live_allocations) and leaves no partial state
(the next call succeeds and gives the normal result)."""
import numpy as np
import pytest

from paper_2204_14193_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

C64 = dict(block=16, border=16, fft=64, rho=0.8, gamma=0.5, iters=80)
FSE_ERR_OOM, FSE_ERR_TIMEOUT = 4, 5


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2204_14193_gb300 as P
    return P


@pytest.fixture(scope="module")
def scene():
    H, W = 256, 256            # width a multiple of 16: the TMA gather path
    img = synth.make_image(81, H, W)[None]
    blocks = synth.grid_losses(82, H, W, 16, 0.25)
    mask = synth.loss_mask(blocks, [16], 1, H, W)
    return torch.from_numpy(img).cuda(), torch.from_numpy(mask).cuda(), blocks


def _patches(P, eng, scene, out=None):
    img, mask, blocks = scene
    p = torch.zeros(len(blocks) * 256, dtype=torch.float32, device="cuda")
    eng.run(img, mask, blocks, out=out, patches=p)
    return p


def _reference(P, scene, **kw):
    eng = P.Engine([C64], **kw)
    p = _patches(P, eng, scene)
    eng.sync()
    eng.close()
    return p.cpu().numpy()


def _expect_timeout_then_recover(P, eng, scene, ref, out=None):
    eng.set_wait_limit(0)
    _patches(P, eng, scene, out)
    with pytest.raises(P.FseError) as e:
        eng.sync()
    assert e.value.status == FSE_ERR_TIMEOUT
    eng.set_wait_limit(1_000_000_000)
    if out is not None:
        out.copy_(scene[0].float())
    p = _patches(P, eng, scene, out)
    eng.sync()                                 # no timeout now; the record was cleared
    np.testing.assert_array_equal(p.cpu().numpy(), ref)


def test_tma_gather_wait_expires(P, scene):
    ref = _reference(P, scene)
    eng = P.Engine([C64])
    _expect_timeout_then_recover(P, eng, scene, ref)
    eng.close()


def test_ordered_wait_expires(P, scene):
    img = scene[0]
    out = img.float().contiguous()
    eng = P.Engine([C64], ordered=True, reuse_weight=0.5)
    p = _patches(P, eng, scene, out)
    eng.sync()
    ref = p.cpu().numpy()
    out.copy_(img.float())
    _expect_timeout_then_recover(P, eng, scene, ref, out=out)
    eng.close()


def test_network_wait_expires(P):
    # a width that is not a multiple of 16: the concealment kernel gathers
    # with plain loads, so the only bounded wait is the network's
    from paper_2204_14193_gb300 import train_init
    H, W = 160, 200
    img = synth.make_image(85, H, W)[None]
    blocks = synth.grid_losses(86, H, W, 16, 0.25)
    mask = synth.loss_mask(blocks, [16], 1, H, W)
    sc = (torch.from_numpy(img).cuda(), torch.from_numpy(mask).cuda(), blocks)
    w = train_init.load_weights()
    ref = _reference(P, sc, init="learned", init_iters=20, weights=w)
    eng = P.Engine([C64], init="learned", init_iters=20, weights=w)
    _expect_timeout_then_recover(P, eng, sc, ref)
    eng.close()


def _lib(P):
    return P._load()


def test_failed_allocations_leak_nothing(P, scene):
    lib = _lib(P)
    live0 = lib.fse_test_live_allocations()
    ref = _reference(P, scene, trace=True)
    # fse_create: fail its 1st, 2nd, ... allocation until it needs no more
    n, created = 1, False
    while not created:
        lib.fse_test_fail_allocation(n)
        try:
            eng = P.Engine([C64], trace=True)
            created = True
        except P.FseError as e:
            assert e.status == FSE_ERR_OOM, e
            assert lib.fse_test_live_allocations() == live0
        lib.fse_test_fail_allocation(0)
        n += 1
    assert n > 3
    # a batch call: its allocations (block list, trace) fail one by one
    k = 1
    while True:
        lib.fse_test_fail_allocation(k)
        try:
            p = _patches(P, eng, scene)
            eng.sync()
            lib.fse_test_fail_allocation(0)
            break
        except P.FseError as e:
            assert e.status == FSE_ERR_OOM, e
        lib.fse_test_fail_allocation(0)
        k += 1
    assert k > 1
    np.testing.assert_array_equal(p.cpu().numpy(), ref)   # no partial state
    eng.close()
    assert lib.fse_test_live_allocations() == live0


def test_failed_allocations_of_the_network(P):
    from paper_2204_14193_gb300 import train_init
    lib = _lib(P)
    live0 = lib.fse_test_live_allocations()
    lib.fse_test_fail_allocation(5)
    with pytest.raises(P.FseError) as e:
        P.Cnn(48, 48, max_batch=4)
    lib.fse_test_fail_allocation(0)
    assert e.value.status == FSE_ERR_OOM
    assert lib.fse_test_live_allocations() == live0
    eng = P.Engine([C64], init="learned", init_iters=20)
    lib.fse_test_fail_allocation(2)
    with pytest.raises(P.FseError) as e:
        eng.load_init_weights(train_init.load_weights())
    lib.fse_test_fail_allocation(0)
    assert e.value.status == FSE_ERR_OOM
    eng.load_init_weights(train_init.load_weights())     # resumes the allocation
    eng.close()
    assert lib.fse_test_live_allocations() == live0


def test_failed_allocations_of_the_host_pipeline(P):
    lib = _lib(P)
    live0 = lib.fse_test_live_allocations()
    T, H, W = 3, 128, 160
    vid = synth.make_video(83, T, H, W)
    blocks = np.concatenate([synth.grid_losses(84 + t, H, W, 16, 0.2, image=t) for t in range(T)])
    mask = synth.loss_mask(blocks, [16], T, H, W)
    eng = P.Engine([C64])
    ref = eng.run_host(vid, mask, blocks).copy()
    eng.close()
    eng = P.Engine([C64])
    k = 1
    while True:
        lib.fse_test_fail_allocation(k)
        try:
            got = eng.run_host(vid, mask, blocks)
            lib.fse_test_fail_allocation(0)
            break
        except P.FseError as e:
            assert e.status == FSE_ERR_OOM, e
        lib.fse_test_fail_allocation(0)
        k += 1
    assert k > 3
    np.testing.assert_array_equal(got, ref)
    eng.close()
    assert lib.fse_test_live_allocations() == live0
