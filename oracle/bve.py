"""Barotropic vorticity model on a doubly periodic grid (oracle).

Sec. 5.2 uses the barotropic vorticity equation with an Arakawa-type Jacobian;
the workload here is its doubly periodic form on [0, 2 pi)^2 with N x N points,
d = 2 pi / N:

    q_t = -J_A(psi, q) + nu Lap_h q + F,     Lap psi = q  (spectral),  F = a sin(k_f y)

* psi = Lap^{-1} q with the spectral symbol -1/|kappa|^2 (psi_hat(0,0) = 0).
* Lap_h: five-point Laplacian.
* J_A: Arakawa's (1966) nine-point Jacobian, the mean of the three second-order
  forms J^{++}, J^{+x}, J^{x+} of J(a, b) = a_x b_y - a_y b_x.

Fields are stored row-major with y the slow index: array[j, i] = f(x_i, y_j),
flattened to length N*N; blocks of k fields are (N*N, k).

Linearization (each linear piece transposed separately):
    F(q) dq   = -J_A(Lap^{-1} dq, q) - J_A(psi, dq) + nu Lap_h dq
    F(q)^T w  = -Lap^{-1} J_A(q, w) + J_A(psi, w) + nu Lap_h w
using that Lap^{-1} and Lap_h are symmetric, J_A(a, b) = -J_A(b, a), and
b -> J_A(a, b) is skew-symmetric (Arakawa's enstrophy conservation).
"""
from __future__ import annotations

import numpy as np


class BVE2D:
    def __init__(self, N: int, nu: float, forcing_amp: float = 1.0, forcing_k: int = 4):
        self.N = int(N)
        self.n = self.N * self.N
        self.nu = float(nu)
        self.d = 2.0 * np.pi / self.N
        k = np.fft.fftfreq(self.N, 1.0 / self.N)          # integer wavenumbers
        KY, KX = np.meshgrid(k, k, indexing="ij")
        K2 = KX ** 2 + KY ** 2
        self.inv_lap = np.where(K2 > 0, -1.0 / np.where(K2 > 0, K2, 1.0), 0.0)
        self.K2 = K2
        y = np.arange(self.N) * self.d
        self.F = (forcing_amp * np.sin(forcing_k * y))[:, None] * np.ones((1, self.N))

    # -- shapes ----------------------------------------------------------------
    def _grid(self, f):
        return f.reshape((self.N, self.N) + f.shape[1:])

    def _flat(self, g, like):
        return g.reshape(like.shape)

    # -- operators ---------------------------------------------------------------
    def poisson(self, q):
        """psi = Lap^{-1} q (spectral)."""
        g = self._grid(q)
        s = self.inv_lap if g.ndim == 2 else self.inv_lap[:, :, None]
        psi = np.real(np.fft.ifft2(s * np.fft.fft2(g, axes=(0, 1)), axes=(0, 1)))
        return self._flat(psi, q)

    def lap_h(self, q):
        g = self._grid(q)
        out = (np.roll(g, 1, 0) + np.roll(g, -1, 0) + np.roll(g, 1, 1) + np.roll(g, -1, 1) - 4.0 * g)
        return self._flat(out / self.d ** 2, q)

    def jacobian(self, a, b):
        """Arakawa J_A(a, b) ~ a_x b_y - a_y b_x (x = axis 1, y = axis 0)."""
        A = self._grid(a)
        B = self._grid(b)
        sh = lambda f, dj, di: np.roll(np.roll(f, -dj, 0), -di, 1)   # f[j+dj, i+di]
        a_e, a_w, a_n, a_s = sh(A, 0, 1), sh(A, 0, -1), sh(A, 1, 0), sh(A, -1, 0)
        b_e, b_w, b_n, b_s = sh(B, 0, 1), sh(B, 0, -1), sh(B, 1, 0), sh(B, -1, 0)
        a_ne, a_nw, a_se, a_sw = sh(A, 1, 1), sh(A, 1, -1), sh(A, -1, 1), sh(A, -1, -1)
        b_ne, b_nw, b_se, b_sw = sh(B, 1, 1), sh(B, 1, -1), sh(B, -1, 1), sh(B, -1, -1)
        j_pp = (a_e - a_w) * (b_n - b_s) - (a_n - a_s) * (b_e - b_w)
        j_px = (a_e * (b_ne - b_se) - a_w * (b_nw - b_sw)
                - a_n * (b_ne - b_nw) + a_s * (b_se - b_sw))
        j_xp = (b_n * (a_ne - a_nw) - b_s * (a_se - a_sw)
                - b_e * (a_ne - a_se) + b_w * (a_nw - a_sw))
        out = (j_pp + j_px + j_xp) / (12.0 * self.d ** 2)
        return self._flat(out, a)

    def _b(self, U, like):
        return U if like.ndim == U.ndim else U[:, None] * np.ones((1, like.shape[1]))

    def rhs(self, q):
        psi = self.poisson(q)
        F = self.F.reshape(-1) if q.ndim == 1 else self.F.reshape(-1, 1)
        return -self.jacobian(psi, q) + self.nu * self.lap_h(q) + F

    def jvp(self, U, dq):
        Ub = self._b(U, dq)
        return (-self.jacobian(self.poisson(dq), Ub) - self.jacobian(self._b(self.poisson(U), dq), dq)
                + self.nu * self.lap_h(dq))

    def vjp(self, U, w):
        Ub = self._b(U, w)
        return (-self.poisson(self.jacobian(Ub, w)) + self.jacobian(self._b(self.poisson(U), w), w)
                + self.nu * self.lap_h(w))

    # -- dense forms (tiny grids) -----------------------------------------------
    def dense(self, op):
        return np.stack([op(e) for e in np.eye(self.n)], axis=1)


def inv_helmholtz_sqrt_symbol(N: int, c: float, ell: float) -> np.ndarray:
    """Fourier symbol of Gamma^{1/2} = c (I - ell^2 Lap)^{-1} (spectral Laplacian)."""
    k = np.fft.fftfreq(N, 1.0 / N)
    KY, KX = np.meshgrid(k, k, indexing="ij")
    return c / (1.0 + ell ** 2 * (KX ** 2 + KY ** 2))


def apply_symbol_2d(symbol, X, N):
    """real(ifft2(symbol * fft2(X))) for X of shape (N*N,) or (N*N, k)."""
    g = X.reshape((N, N) + X.shape[1:])
    s = symbol if g.ndim == 2 else symbol[:, :, None]
    out = np.real(np.fft.ifft2(s * np.fft.fft2(g, axes=(0, 1)), axes=(0, 1)))
    return out.reshape(X.shape)
