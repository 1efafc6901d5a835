"""Pins for oracle.spectral: the naive DFT against numpy's FFT and known transforms."""
import numpy as np

from oracle import spectral


def test_dft2_matches_library_fft():
    rng = np.random.default_rng(0)
    for shape in [(8, 8), (12, 6), (16, 32), (6, 9)]:
        f = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
        np.testing.assert_allclose(spectral.dft2(f), np.fft.fft2(f), atol=1e-11)
        np.testing.assert_allclose(spectral.idft2(f), np.fft.ifft2(f), atol=1e-13)


def test_dft_accuracy_on_offset_signal():
    # A large mean on top of small fluctuations (as a neutral plasma's charge): the
    # fluctuation modes must keep full FP64 accuracy relative to the input norm.
    rng = np.random.default_rng(5)
    for n in (128, 512):
        f = 64.0 + rng.standard_normal((n, 4))
        ref = np.fft.fft2(f)
        err = np.abs(spectral.dft2(f) - ref)[1:].max()
        assert err < 2e-15 * np.linalg.norm(f) * np.sqrt(n), (n, err)


def test_delta_and_cosine():
    f = np.zeros((8, 4))
    f[0, 0] = 1.0
    np.testing.assert_allclose(spectral.dft2(f), np.ones((8, 4)), atol=1e-14)
    x = np.arange(8)[:, None] * np.ones((1, 4))
    g = np.cos(2 * np.pi * 3 * x / 8)
    gh = spectral.dft2(g)
    expect = np.zeros((8, 4), complex)
    expect[3, 0] = expect[5, 0] = 16.0
    np.testing.assert_allclose(gh, expect, atol=1e-12)


def test_parseval():
    rng = np.random.default_rng(1)
    f = rng.standard_normal((16, 8))
    fh = spectral.dft2(f)
    assert abs(np.sum(f * f) - np.sum(np.abs(fh) ** 2) / f.size) < 1e-10


def test_wavenumbers_nyquist_zero_and_signs():
    k = spectral.wavenumbers(8, 2.0)
    np.testing.assert_allclose(k, np.pi * np.array([0, 1, 2, 3, 0, -3, -2, -1]), atol=1e-15)
    k = spectral.wavenumbers(6, 1.0)
    np.testing.assert_allclose(k, 2 * np.pi * np.array([0, 1, 2, 0, -2, -1]), atol=1e-15)


def test_spectral_derivative_of_resolved_sine_is_exact():
    nx, ny, lx, ly = 16, 8, 1.7, 0.9
    kx, ky, K = spectral.wavenumber_grid(nx, ny, lx, ly)
    x = (np.arange(nx) * lx / nx)[:, None] * np.ones((1, ny))
    y = np.ones((nx, 1)) * (np.arange(ny) * ly / ny)[None, :]
    u = np.sin(2 * np.pi * 3 * x / lx) * np.cos(2 * np.pi * 2 * y / ly)
    uh = spectral.dft2(u)
    dux, duy = spectral.grad_hat(uh, kx, ky)
    np.testing.assert_allclose(spectral.idft2(dux).real,
                               (2 * np.pi * 3 / lx) * np.cos(2 * np.pi * 3 * x / lx)
                               * np.cos(2 * np.pi * 2 * y / ly), atol=1e-12)
    np.testing.assert_allclose(spectral.idft2(duy).real,
                               -(2 * np.pi * 2 / ly) * np.sin(2 * np.pi * 3 * x / lx)
                               * np.sin(2 * np.pi * 2 * y / ly), atol=1e-12)
    # Laplacian = div grad, mode by mode, including the Nyquist column.
    lap = spectral.div_hat(*spectral.grad_hat(uh, kx, ky), kx, ky)
    np.testing.assert_allclose(lap, -K * uh, atol=1e-12)


def test_derivative_of_real_field_stays_real():
    rng = np.random.default_rng(2)
    u = rng.standard_normal((8, 6))
    kx, ky, _ = spectral.wavenumber_grid(8, 6, 1.0, 1.0)
    d = spectral.idft2(1j * kx * spectral.dft2(u))
    assert np.max(np.abs(d.imag)) < 1e-13
