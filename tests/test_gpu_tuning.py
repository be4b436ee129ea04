"""Tuning modes of the launch shape (fse_set_tuning).  Every shape (128 or
256 threads per CTA, the two largest CTA counts per SM) must give the same
patches bit for bit; FSE_TUNE_ASYNC must not make any call wait for timing
runs, and must settle on a choice after the four candidates have run."""
import time

import numpy as np
import pytest

from paper_2204_14193_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CLS = dict(block=16, border=16, fft=64, rho=0.8, gamma=0.5, iters=500)


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2204_14193_gb300 as P
    return P


@pytest.fixture(scope="module")
def batch():
    """8 frames of 1920x1080, 10% of the 16x16 blocks lost (I = 500)."""
    T, H, W = 8, 1080, 1920
    video = synth.make_video(71, T, H, W)
    blocks = np.concatenate([synth.grid_losses(72 + t, H, W, 16, 0.10, image=t) for t in range(T)])
    mask = synth.loss_mask(blocks, [16], T, H, W)
    return video, mask, blocks


def _first_and_rest(P, mode, video, mask, blocks, calls):
    P.fse_test_clear_tuning_cache()
    eng = P.Engine([CLS])
    eng.set_tuning(mode)
    dv, dm = torch.from_numpy(video).cuda(), torch.from_numpy(mask).cuda()
    n = eng.patch_total(blocks)
    outs, pending = [], []
    try:
        for k in range(calls):
            p = torch.zeros(n, device="cuda")
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            eng.run(dv, dm, blocks, patches=p)
            dt = time.perf_counter() - t0
            if k == 0:
                first = dt
            torch.cuda.synchronize()
            outs.append(p.cpu().numpy())
            pending.append(eng.tuning()[1])
    finally:
        eng.close()
    return first, outs, pending


def test_async_tuning_never_waits_and_converges(P, batch):
    video, mask, blocks = batch
    t_async, outs_a, pend_a = _first_and_rest(P, "async", video, mask, blocks, 7)
    t_sync, outs_s, pend_s = _first_and_rest(P, "sync", video, mask, blocks, 2)
    print(f"first call: async {1e3 * t_async:.1f} ms, sync {1e3 * t_sync:.1f} ms; pending {pend_a}")
    # the synchronous first call waits for eight timed launches, the
    # asynchronous one for none
    assert t_async < t_sync / 4
    # four candidates, one per call, each polled by a later call
    assert pend_a[0] == 1 and pend_a[-1] == 0
    assert pend_s == [0, 0]
    # every launch shape gives the same patches
    for o in outs_a + outs_s[1:]:
        np.testing.assert_array_equal(o, outs_s[0])


def test_tuning_off_and_host_pipeline(P, batch):
    video, mask, blocks = batch
    P.fse_test_clear_tuning_cache()
    ref = P.Engine([CLS])
    off = P.Engine([CLS])
    off.set_tuning("off")
    asy = P.Engine([CLS])
    asy.set_tuning("async")
    try:
        n = ref.patch_total(blocks)
        dv, dm = torch.from_numpy(video).cuda(), torch.from_numpy(mask).cuda()
        a = torch.zeros(n, device="cuda")
        b = torch.zeros(n, device="cuda")
        ref.run(dv, dm, blocks, patches=a)
        off.run(dv, dm, blocks, patches=b)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(a.cpu().numpy(), b.cpu().numpy())
        assert off.tuning() == ("off", 0)
        # the host-buffer pipeline times its chunks asynchronously too
        for _ in range(6):
            h = np.full(n, -1.0, np.float32)
            asy.run_host(video, mask, blocks, h)
            np.testing.assert_array_equal(h, a.cpu().numpy())
    finally:
        ref.close()
        off.close()
        asy.close()


def test_switching_mode_closes_an_open_session(P, batch):
    """An ASYNC session left open when the handle switches to SYNC is closed
    by the synchronous choice (the mix then replays its captured launch)."""
    video, mask, blocks = batch
    P.fse_test_clear_tuning_cache()
    eng = P.Engine([CLS])
    try:
        eng.set_tuning("async")
        dv, dm = torch.from_numpy(video).cuda(), torch.from_numpy(mask).cuda()
        n = eng.patch_total(blocks)
        a = torch.zeros(n, device="cuda")
        eng.run(dv, dm, blocks, patches=a)
        assert eng.tuning() == ("async", 1)
        eng.set_tuning("sync")
        b = torch.zeros(n, device="cuda")
        eng.run(dv, dm, blocks, patches=b)
        assert eng.tuning() == ("sync", 0)
        c = torch.zeros(n, device="cuda")
        eng.run(dv, dm, blocks, patches=c)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(a.cpu().numpy(), b.cpu().numpy())
        np.testing.assert_array_equal(a.cpu().numpy(), c.cpu().numpy())
    finally:
        eng.close()
