"""Density-grid monopole (Sec. 3.4.4) on the GPU against the FP64 oracle:
TSC interpolation, overdensity, lag-averaged delta_i delta_j per bin.  The
GPU sums FP32 products with float-float accumulation, so the bound is a
relative 1e-5 of mean(delta^2), which bounds the mean |delta_i delta_j|."""
import numpy as np
import pytest

import oracle
from paper_1210_1833_gb300 import cute, synthetic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = cute.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("ngrid,weighted", [(32, False), (64, True)])
def test_density_grid_matches_oracle(ctx, ngrid, weighted):
    rng = np.random.default_rng(110 + ngrid)
    L = 400.0
    x = np.concatenate([synthetic.uniform_box(20000, L, rng),
                        synthetic.blobs_box(200, 100, L, 8.0, rng)])
    w = rng.uniform(0.5, 2.0, len(x)).astype(np.float32) if weighted else None
    edges = np.linspace(0.0, 100.0, 11)
    xi, lags = ctx.density_grid_xi(x, L, ngrid, edges, weights=w)
    rho = oracle.tsc_density(x, L, ngrid, w)
    delta = rho / rho.mean() - 1.0
    ref, ref_lags = oracle.lag_xi(delta, L, edges)
    np.testing.assert_array_equal(lags, ref_lags)
    scale = float(np.mean(delta * delta))
    m = ~np.isnan(ref)
    assert np.array_equal(np.isnan(xi), np.isnan(ref))
    assert np.all(np.abs(xi[m] - ref[m]) <= 1e-5 * scale)


def test_density_grid_device_inputs_and_errors(ctx):
    rng = np.random.default_rng(120)
    L = 100.0
    x = synthetic.uniform_box(5000, L, rng)
    edges = np.linspace(0, 30, 7)
    a, la = ctx.density_grid_xi(x, L, 32, edges)
    b, lb = ctx.density_grid_xi(torch.from_numpy(x).cuda(), L, 32, edges)
    np.testing.assert_allclose(a, b, rtol=1e-6, atol=1e-9)  # atomics add in any order
    with pytest.raises(cute.CuteError):
        ctx.density_grid_xi(x, L, 32, np.linspace(0, 60, 7))  # r_max >= L/2
    with pytest.raises(cute.CuteError):
        ctx.density_grid_xi(x, L, 48, edges)                 # ngrid not a multiple of 32
    bad = x.copy()
    bad[3, 1] = L                                            # outside [0, L)
    with pytest.raises(cute.CuteError):
        ctx.density_grid_xi(bad, L, 32, edges)


@pytest.mark.parametrize("ngrid", [128, 256, 384])
def test_density_grid_warp_kernel_matches_oracle(ctx, ngrid):
    """Rows of 128, 256 and 384 points take the warp-per-lag-window kernel
    (the bench's 256^3 grid among them); lags reach 45 grid steps, so the
    longest lag columns span three windows of the kernel.  The oracle's lag
    sums come from the FFT form (lag_xi_fft, pinned to the direct sums)."""
    rng = np.random.default_rng(120 + ngrid)
    L = 400.0
    x = np.concatenate([synthetic.uniform_box(40000, L, rng),
                        synthetic.blobs_box(300, 100, L, 6.0, rng)])
    w = rng.uniform(0.5, 2.0, len(x)).astype(np.float32)
    a = L / ngrid
    edges = np.linspace(0.0, 45.5 * a, 12)
    xi, lags = ctx.density_grid_xi(x, L, ngrid, edges, weights=w)
    rho = oracle.tsc_density(x, L, ngrid, w)
    delta = rho / rho.mean() - 1.0
    ref, ref_lags = oracle.lag_xi_fft(delta, L, edges)
    np.testing.assert_array_equal(lags, ref_lags)
    scale = float(np.mean(delta * delta))
    m = ~np.isnan(ref)
    assert np.array_equal(np.isnan(xi), np.isnan(ref))
    assert np.all(np.abs(xi[m] - ref[m]) <= 1e-5 * scale)
