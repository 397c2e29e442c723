"""Viscous Burgers with homogeneous Dirichlet boundaries (oracle).

The Burgers set-up of Sec. 5.1: u_t + u u_x = nu u_xx on (0, 1) with
u(t, 0) = u(t, 1) = 0, second-order central differences on the n interior
points x_j = j dx, dx = 1/(n+1), j = 1..n (boundary values 0):

    f_j = -u_j (u_{j+1} - u_{j-1}) / (2 dx) + nu (u_{j+1} - 2 u_j + u_{j-1}) / dx^2.

With zero boundary values the central first difference D1 is skew-symmetric and
the second difference D2 symmetric, so F(u)^T w = -(D1 u) w + D1 (u w) + nu D2 w.
"""
from __future__ import annotations

import numpy as np


class BurgersDirichlet:
    def __init__(self, n: int, nu: float):
        self.n = int(n)
        self.nu = float(nu)
        self.dx = 1.0 / (self.n + 1)
        self.x = np.arange(1, self.n + 1) * self.dx

    def _pad(self, u):
        z = np.zeros((1,) + u.shape[1:])
        return np.concatenate([z, u, z], axis=0)

    def d1(self, u):
        p = self._pad(u)
        return (p[2:] - p[:-2]) / (2.0 * self.dx)

    def d2(self, u):
        p = self._pad(u)
        return (p[2:] - 2.0 * p[1:-1] + p[:-2]) / self.dx ** 2

    def _b(self, U, like):
        return U if like.ndim == U.ndim else U[:, None]

    def rhs(self, u):
        return -u * self.d1(u) + self.nu * self.d2(u)

    def jvp(self, U, d):
        Ub = self._b(U, d)
        return -(d * self._b(self.d1(U), d) + Ub * self.d1(d)) + self.nu * self.d2(d)

    def vjp(self, U, w):
        Ub = self._b(U, w)
        return -self._b(self.d1(U), w) * w + self.d1(Ub * w) + self.nu * self.d2(w)

    def jacobian_dense(self, U):
        return np.stack([self.jvp(U, e) for e in np.eye(self.n)], axis=1)


def dirichlet_laplacian(n: int) -> np.ndarray:
    """tridiag(1, -2, 1): the 3-point Dirichlet Laplacian stencil (unscaled)."""
    return -2.0 * np.eye(n) + np.eye(n, k=1) + np.eye(n, k=-1)


def inv_helmholtz_sqrt(n: int, a: float, b: float):
    """Gamma^{1/2} = (a I - b Delta*)^{-1} with Delta* = tridiag(1, -2, 1), so that
    Gamma = (a I - b Delta*)^{-2} (the Burgers prior of Sec. 5.1 with a = 0.5,
    b = 500). Applied by a banded solve."""
    from scipy.linalg import solve_banded
    ab = np.zeros((3, n))
    ab[0, 1:] = -b
    ab[1, :] = a + 2.0 * b
    ab[2, :-1] = -b
    return lambda X: solve_banded((1, 1), ab, X)
