"""Naive DFT and spectral derivatives on the periodic collocated grid (oracle).

The paper restricts itself to doubly periodic domains and inverts the modified
Helmholtz operator L = I - alpha^-2 Laplacian with an FFT (section 3.1), and insists
that every spatial derivative (the divergence in the continuity equation, the
gradients fed to the particles) be taken "the same way as the solve", i.e.
spectrally (section 4, opening of the algorithm overview).  This module writes that
out with the DFT's definition as a dense matrix product -- no FFT anywhere:

    f_hat[m] = sum_j f[j] exp(-2 pi i m j / N),    f[j] = (1/N) sum_m f_hat[m] exp(+2 pi i m j / N)

Grid arrays are indexed [i, j] with i along x (nx nodes) and j along y (ny nodes),
node (i, j) sitting at (i dx, j dy).

Wavenumber reading (the paper does not spell it out): mode m carries
k(m) = 2 pi m'/L with m' = m for m < N/2 and m' = m - N for m > N/2, and k = 0 at
the Nyquist index m = N/2 of an even N.  The same k is used for the gradient (i k),
the divergence (i k .) and the Laplacian (-|k|^2), so that Laplacian = div grad holds
exactly mode by mode -- which the Gauss-law theorems of section 3 need -- and
derivatives of real fields stay real.
"""
import numpy as np


def dft_matrix(n, sign=-1):
    """Dense DFT matrix F[m, j] = exp(sign * 2 pi i m j / n).

    The kernel depends on m j only modulo n, so the exponent is taken at the reduced
    argument 2 pi ((m j) mod n) / n: evaluating it at m j up to (n-1)^2 would lose
    about log10(n^2) digits of the phase.
    """
    idx = np.arange(n)
    return np.exp(sign * 2j * np.pi * (np.outer(idx, idx) % n) / n)


def dft2(f):
    """Forward 2-D DFT of an (nx, ny) array, unnormalised."""
    f = np.asarray(f, dtype=np.complex128)
    nx, ny = f.shape
    return dft_matrix(nx) @ f @ dft_matrix(ny).T


def idft2(f_hat):
    """Inverse 2-D DFT of an (nx, ny) spectrum, with the 1/(nx ny) factor."""
    f_hat = np.asarray(f_hat, dtype=np.complex128)
    nx, ny = f_hat.shape
    return (dft_matrix(nx, +1) @ f_hat @ dft_matrix(ny, +1).T) / (nx * ny)


def wavenumbers(n, length):
    """Spectral wavenumbers k(m), m = 0..n-1, with k = 0 at the Nyquist index."""
    m = np.arange(n)
    signed = np.where(m < n / 2, m, m - n).astype(np.float64)
    if n % 2 == 0:
        signed[n // 2] = 0.0
    return 2.0 * np.pi * signed / length


def wavenumber_grid(nx, ny, lx, ly):
    """(kx, ky, K) on the (nx, ny) spectral grid, K = kx^2 + ky^2."""
    kx = wavenumbers(nx, lx)[:, None] * np.ones((1, ny))
    ky = np.ones((nx, 1)) * wavenumbers(ny, ly)[None, :]
    return kx, ky, kx * kx + ky * ky


def grad_hat(u_hat, kx, ky):
    """Spectral gradient (i kx u, i ky u)."""
    return 1j * kx * u_hat, 1j * ky * u_hat


def div_hat(fx_hat, fy_hat, kx, ky):
    """Spectral divergence i kx fx + i ky fy."""
    return 1j * kx * fx_hat + 1j * ky * fy_hat
