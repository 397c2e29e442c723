"""Prior covariance square roots on periodic grids (oracle).

The method works in the control variable v with x0 = xb + Gamma^{1/2} v, which is
the prior-preconditioned (first-level) form of Eq. gniterf1 / Eq. pcgsystem.
Gamma is stationary on a periodic grid, so Gamma^{1/2} is the circulant matrix
whose Fourier symbol is the square root of Gamma's symbol.

Squared-exponential prior (1D Burgers workloads):
  Gamma_ij = sigma_b^2 exp(-d_ij^2 / (2 L^2)),  d_ij = min(|i-j|, n-|i-j|) / n.
Its symbol is the DFT of the first column; eigenvalues below CLAMP_REL times the
largest one (round-off level, the kernel's spectrum decays like a Gaussian) are
set to zero before the square root.
"""
from __future__ import annotations

import numpy as np

CLAMP_REL = 1e-10


def se_first_column(n: int, sigma_b: float, length: float) -> np.ndarray:
    j = np.arange(n)
    d = np.minimum(j, n - j) / n
    return sigma_b ** 2 * np.exp(-(d ** 2) / (2.0 * length ** 2))


def se_sqrt_symbol(n: int, sigma_b: float, length: float) -> np.ndarray:
    c = se_first_column(n, sigma_b, length)
    lam = np.real(np.fft.fft(c))
    lam = np.where(lam < CLAMP_REL * lam.max(), 0.0, lam)
    return np.sqrt(lam)


def se_covariance_dense(n: int, sigma_b: float, length: float) -> np.ndarray:
    i = np.arange(n)
    d = np.abs(i[:, None] - i[None, :])
    d = np.minimum(d, n - d) / n
    return sigma_b ** 2 * np.exp(-(d ** 2) / (2.0 * length ** 2))


def apply_symbol(symbol, X):
    """Circulant product real(ifft(symbol * fft(X))) along axis 0 (1D grids)."""
    s = symbol if X.ndim == 1 else symbol[:, None]
    return np.real(np.fft.ifft(s * np.fft.fft(X, axis=0), axis=0))
