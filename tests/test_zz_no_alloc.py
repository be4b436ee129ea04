"""The allocation-free entry point (fse_extrapolate_batch_noalloc).

Some callers cannot let a library allocate device memory while they run (a
real-time pipeline that cannot absorb the device-wide synchronisation of
cudaMalloc / cudaFree, an application whose own pool allocator owns the
device memory, a process that forbids allocation after start-up).  For them
the library offers one entry point whose scratch is a fixed array inside the
library.  This test calls it through the C ABI twice in a row, on two
different batches, and checks each result against the handle-based entry
point (fse_extrapolate_batch) on the same inputs, bit for bit: the kernel's
arithmetic does not depend on the thread mapping, and on these small batches
the handle path runs the 256-thread mapping while the allocation-free path
runs the 128-thread one.  It also checks that an oversized batch is refused.
The file name makes pytest collect it last.
"""
import numpy as np
import pytest

from paper_2204_14193_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

C16 = dict(block=4, border=6, fft=16, rho=0.8, gamma=0.5, iters=120)
C32 = dict(block=8, border=12, fft=32, rho=0.8, gamma=0.5, iters=120)
C64 = dict(block=16, border=16, fft=64, rho=0.8, gamma=0.5, iters=120)


def _batches():
    img = synth.make_image(31, 384, 512)[None]
    a = synth.grid_losses(32, 384, 512, 16, 0.2, non_adjacent=True, cls=2)
    vid = synth.make_video(33, 2, 360, 480)
    b = np.concatenate([synth.uneven_losses(34 + t, 360, 480, image=t) for t in range(2)])
    return [(img, a, [C16, C32, C64]), (vid, b, [C16, C32, C64])]


def test_noalloc_matches_handle_entry_two_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2204_14193_gb300 as P
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream().cuda_stream
    for images, blocks, classes in _batches():          # two calls in a row
        N, H, W = images.shape
        mask = synth.loss_mask(blocks, [c["block"] for c in classes], N, H, W)
        dimg = torch.from_numpy(np.ascontiguousarray(images)).cuda()
        dmask = torch.from_numpy(mask).cuda()
        ref = torch.zeros((N, H, W), dtype=torch.float32, device="cuda")
        eng = P.Engine(classes)
        eng.run(dimg, dmask, blocks, out=ref)
        torch.cuda.synchronize()
        eng.close()
        got = torch.full((N, H, W), 0.0, dtype=torch.float32, device="cuda")
        P.fse_extrapolate_batch_noalloc(classes, dimg.data_ptr(), P.FSE_DTYPE_U8, N, H, W, W, dmask.data_ptr(),
                                        blocks, len(blocks), got.data_ptr(), stream)
        torch.cuda.synchronize()
        diff = (got - ref).abs().max().item()
        assert diff == 0.0, diff
        assert torch.count_nonzero(got).item() > 0


def test_noalloc_rejects_oversized_batch():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2204_14193_gb300 as P
    n = 65537
    blocks = np.zeros((n, 4), np.int32)
    img = torch.zeros((1, 16, 16), dtype=torch.uint8, device="cuda")
    out = torch.zeros((1, 16, 16), dtype=torch.float32, device="cuda")
    with pytest.raises(P.FseError) as ei:
        P.fse_extrapolate_batch_noalloc([C16], img.data_ptr(), P.FSE_DTYPE_U8, 1, 16, 16, 16, img.data_ptr(),
                                        blocks, n, out.data_ptr(), None)
    assert ei.value.status == 1 and "65536" in str(ei.value)
