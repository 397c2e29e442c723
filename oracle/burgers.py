"""Semi-discrete viscous Burgers model on a periodic grid (oracle).

Sec. 5.1 discretizes u_t + u u_x = nu u_xx with second-order central finite
differences. On the periodic grid x_j = j/n, dx = 1/n, with the advective form:

  f_j(u) = -u_j (u_{j+1} - u_{j-1}) / (2 dx) + nu (u_{j+1} - 2 u_j + u_{j-1}) / dx^2

Writing D1 for the central first difference and D2 for the three-point second
difference (both circulant, D1^T = -D1, D2^T = D2):

  Jacobian   F(u) d   = -(D1 u) o d - u o (D1 d) + nu D2 d
  transpose  F(u)^T w = -(D1 u) o w + D1 (u o w) + nu D2 w
"""
from __future__ import annotations

import numpy as np


def _col(u, like):
    return u if like.ndim == u.ndim else u[:, None]


class Burgers1D:
    def __init__(self, n: int, nu: float):
        self.n = int(n)
        self.nu = float(nu)
        self.dx = 1.0 / self.n

    def d1(self, u):
        return (np.roll(u, -1, axis=0) - np.roll(u, 1, axis=0)) / (2.0 * self.dx)

    def d2(self, u):
        return (np.roll(u, -1, axis=0) - 2.0 * u + np.roll(u, 1, axis=0)) / (self.dx * self.dx)

    def rhs(self, u):
        return -u * self.d1(u) + self.nu * self.d2(u)

    def jvp(self, U, d):
        Uc = _col(U, d)
        return -_col(self.d1(U), d) * d - Uc * self.d1(d) + self.nu * self.d2(d)

    def vjp(self, U, w):
        Uc = _col(U, w)
        return -_col(self.d1(U), w) * w + self.d1(Uc * w) + self.nu * self.d2(w)

    def jacobian_dense(self, U):
        """Explicit n x n Jacobian (tiny n only), assembled entry by entry."""
        n, dx, nu = self.n, self.dx, self.nu
        du = self.d1(U)
        J = np.zeros((n, n))
        for j in range(n):
            jp, jm = (j + 1) % n, (j - 1) % n
            J[j, j] += -du[j] - 2.0 * nu / dx ** 2
            J[j, jp] += -U[j] / (2.0 * dx) + nu / dx ** 2
            J[j, jm] += U[j] / (2.0 * dx) + nu / dx ** 2
        return J
