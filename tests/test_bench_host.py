"""Host-side pieces of bench.py and of the paper-run input recipes (CPU only)."""
import numpy as np
import pytest

import bench
import synth


def test_fifo_latencies_single_server():
    lat, end = bench.fifo_latencies([0.0, 1.0, 1.5], [2.0, 1.0, 1.0])
    # starts at 0, 2, 3; ends at 2, 3, 4
    assert np.allclose(lat, [2.0, 2.0, 2.5]) and end == pytest.approx(4.0)
    lat, end = bench.fifo_latencies([0.0, 10.0], [1.0, 1.0])      # idle gap
    assert np.allclose(lat, [1.0, 1.0]) and end == pytest.approx(11.0)
    lat, _ = bench.fifo_latencies(np.zeros(3), [1.0, 2.0, 3.0])   # burst
    assert np.allclose(lat, [1.0, 3.0, 6.0])


def test_algorithmic_bytes_of_the_step_kernels():
    M, V, b, r, L = 36, 128 ** 3, 8, 4, 8
    n = M * V * b
    assert bench.kernel_bytes("k_plane", M, V, b, r, L) == 3 * n + V * L * r == 1879048192
    assert bench.kernel_bytes("k_zderiv(fixed)", M, V, b, r, L) == 2 * n
    assert bench.kernel_bytes("k_ypass_fixed(forward+coupling)", M, V, b, r, L) == 4 * n
    assert bench.kernel_bytes("k_xpass_fixed(pointwise)", M, V, b, r, L) == 2 * n + 16 * V
    assert bench.kernel_bytes("k_taps", M, V, b, r, L) is None


def test_job_value_and_traffic_record():
    assert bench.job_value(1e9, 4, 500.0) == pytest.approx(8e9)
    assert bench.measured_traffic("k_plane", "N=3 layout=full precision=fp64") is None
    v = bench.measured_traffic("k_plane", "N=7 layout=real precision=fp32")
    assert v is None or v > bench.kernel_bytes("k_plane", 36, 128 ** 3, 8, 4, 8)


def test_paper_run_recipes():
    e1 = synth.e1()
    assert e1.shape == (64, 64, 64) and e1.N == 21 and e1.nsteps == 400 and e1.pml_width == 0
    assert e1.dx == pytest.approx(50.0 / 64)
    x = (np.arange(64) + 0.5) * e1.dx
    assert np.all(e1.mus[..., x <= 15.0] == 5.0) and np.all(e1.mus[..., x > 15.0] == 1.0)
    assert np.all(e1.mua == 0.01) and np.all(e1.g == 0.9)
    e2 = synth.e2()
    assert e2.N == 7 and e2.nsteps == 25000 and e2.pml_mu0 == 0.01 and e2.pml_mu1 == 1.0
    assert e2.pml_width == round(7.25 / e2.dx) == 9
    z, y, xx = np.unravel_index(int(e2.src_voxel[0]), e2.shape)
    assert (z, y) == (32, 32) and (xx - 32) * e2.dx == pytest.approx(8.0, abs=e2.dx)
    assert np.all(e2.mus == 10.0) and np.all(e2.g == 0.95) and e2.src_fwhm[0] == 0.0
