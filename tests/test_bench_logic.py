"""Host logic of the benchmark line (CPU): the equal-PSNR interpolation of
the learned-versus-plain curve and the per-block shared-memory bytes."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_crossing_interpolates_between_the_bracketing_points():
    pts = [(50, 10.0, 30.0), (100, 20.0, 32.0), (200, 40.0, 33.0)]
    ms, it = bench._crossing(pts, 32.5)
    assert ms == pytest.approx(30.0) and it == pytest.approx(150.0)
    ms, it = bench._crossing(pts, 31.0)
    assert ms == pytest.approx(15.0) and it == pytest.approx(75.0)


def test_crossing_at_a_point_and_outside_the_curve():
    pts = [(50, 10.0, 30.0), (100, 20.0, 32.0)]
    assert bench._crossing(pts, 32.0) == pytest.approx((20.0, 100.0))
    assert bench._crossing(pts, 29.0) == (10.0, 50)      # the first point already reaches it
    assert bench._crossing(pts, 32.1) is None            # never reached


def test_crossing_takes_the_first_crossing_of_a_non_monotonic_curve():
    pts = [(25, 5.0, 28.0), (50, 10.0, 34.0), (75, 15.0, 35.0), (100, 20.0, 34.9)]
    ms, it = bench._crossing(pts, 34.5)
    assert it == pytest.approx(62.5) and ms == pytest.approx(12.5)


def test_shared_memory_bytes_per_block():
    # 8 I F^2 plus about 0.4 MB of FFT passes at F = 64, I = 200 (about 7.0 MB)
    assert bench.smem_bytes_per_block(64, 200) == 8 * 200 * 4096 + 96 * 4096
    assert bench.smem_bytes_per_block(64, 200) == pytest.approx(6.95e6, rel=1e-3)
    assert bench.smem_bytes_per_block(32, 0) == 96 * 1024



def test_fixed_w_bytes_per_block():
    """Reduced-precision storage: 8-byte operands for the first K iterations,
    4-byte codes for the other I - K; the FP32 count when K >= I."""
    assert bench.fixed_w_bytes_per_block(64, 200, 20) == (8 * 20 + 4 * 180) * 4096 + 96 * 4096
    for I in (0, 1, 20):
        assert bench.fixed_w_bytes_per_block(64, I, 20) == bench.smem_bytes_per_block(64, I)
