"""Wind-driven barotropic vorticity in a closed basin (oracle; test infrastructure).

The double-gyre set-up of Sec. 5.2 (non-dimensional form):

    omega_t = -J(psi, omega) + Ro^{-1} psi_x + Re^{-1} Lap omega + Ro^{-1} F,
    Lap psi = -omega,        F(x, y) = sin(pi y),

on (0, 1) x (-1, 1) with psi = omega = 0 on the boundary, J(a, b) = a_y b_x -
a_x b_y. Second-order central differences on the nx x ny interior points
x_i = i h, y_j = -1 + j h (i = 1..nx, j = 1..ny), h = 1/(nx + 1), ny = 2 nx + 1;
boundary values are zero. A field is stored row-major (y slow, x fast): entry
(j - 1) nx + (i - 1).

    D_x a = (a_{i+1,j} - a_{i-1,j}) / (2h),  D_y a = (a_{i,j+1} - a_{i,j-1}) / (2h),
    Lap_h a = (a_{i+1,j} + a_{i-1,j} + a_{i,j+1} + a_{i,j-1} - 4 a_{i,j}) / h^2,
    psi = P omega := h^2 L^{-1} omega,  L = -Delta* (the unscaled five-point matrix).

The Poisson solve is a sparse direct (LU) solve of the five-point matrix assembled
as a Kronecker sum. With zero boundary values D_x and D_y are skew-symmetric and
Lap_h and P symmetric, which gives the transpose of the Jacobian used by vjp:

    F(U)^T w = D_x(psi_y w) - D_y(psi_x w) + Re^{-1} Lap_h w
               + P [ D_y(omega_x w) - D_x(omega_y w) - Ro^{-1} D_x w ],

with omega = U, psi = P U and subscripts the central differences.
"""
from __future__ import annotations

import numpy as np


def dirichlet_laplacian_2d(nx: int, ny: int):
    """Delta*: the unscaled five-point Laplacian with zero boundary values on an
    nx x ny interior grid, row-major (y slow), as a scipy sparse matrix."""
    import scipy.sparse as sp
    tx = sp.diags([1.0, -2.0, 1.0], [-1, 0, 1], shape=(nx, nx))
    ty = sp.diags([1.0, -2.0, 1.0], [-1, 0, 1], shape=(ny, ny))
    return (sp.kron(sp.identity(ny), tx) + sp.kron(ty, sp.identity(nx))).tocsc()


class BVEGyre:
    def __init__(self, nx: int, re: float, ro: float):
        from scipy.sparse.linalg import splu
        self.nx = int(nx)
        self.ny = 2 * self.nx + 1
        self.n = self.nx * self.ny
        self.h = 1.0 / (self.nx + 1)
        self.re_inv = 1.0 / float(re)
        self.ro_inv = 1.0 / float(ro)
        self.x = np.arange(1, self.nx + 1) * self.h
        self.y = -1.0 + np.arange(1, self.ny + 1) * self.h
        self._L = splu(-dirichlet_laplacian_2d(self.nx, self.ny))
        # forcing on the grid, flattened row-major
        self.F = np.repeat(np.sin(np.pi * self.y), self.nx)

    # -- grid helpers -------------------------------------------------------
    def _grid(self, f):
        return f.reshape((self.ny, self.nx) + f.shape[1:])

    def _flat(self, g):
        return g.reshape((self.n,) + g.shape[2:])

    def _pad(self, f):
        g = self._grid(f)
        return np.pad(g, [(1, 1), (1, 1)] + [(0, 0)] * (g.ndim - 2))

    def dx(self, f):
        p = self._pad(f)
        return self._flat((p[1:-1, 2:] - p[1:-1, :-2]) / (2.0 * self.h))

    def dy(self, f):
        p = self._pad(f)
        return self._flat((p[2:, 1:-1] - p[:-2, 1:-1]) / (2.0 * self.h))

    def lap(self, f):
        p = self._pad(f)
        return self._flat((p[1:-1, 2:] + p[1:-1, :-2] + p[2:, 1:-1] + p[:-2, 1:-1]
                           - 4.0 * p[1:-1, 1:-1]) / self.h ** 2)

    def poisson(self, omega):
        """psi with Lap_h psi = -omega and psi = 0 on the boundary."""
        return self.h ** 2 * self._L.solve(np.asarray(omega, dtype=np.float64))

    def jac(self, a, b):
        """J(a, b) = a_y b_x - a_x b_y by central differences."""
        return self.dy(a) * self.dx(b) - self.dx(a) * self.dy(b)

    def _b(self, U, like):
        return U if like.ndim == U.ndim else U[:, None]

    # -- model interface (rk4 module) ----------------------------------------
    def rhs(self, omega):
        psi = self.poisson(omega)
        F = self.F if omega.ndim == 1 else self.F[:, None]
        return (-self.jac(psi, omega) + self.ro_inv * self.dx(psi) + self.re_inv * self.lap(omega)
                + self.ro_inv * F)

    def jvp(self, U, d):
        psi = self._b(self.poisson(U), d)
        Ub = self._b(U, d)
        dpsi = self.poisson(d)
        return (-(self.jac(dpsi, Ub) + self.jac(psi, d)) + self.ro_inv * self.dx(dpsi)
                + self.re_inv * self.lap(d))

    def vjp(self, U, w):
        psi = self.poisson(U)
        psx, psy = self._b(self.dx(psi), w), self._b(self.dy(psi), w)
        omx, omy = self._b(self.dx(U), w), self._b(self.dy(U), w)
        inner = self.dy(omx * w) - self.dx(omy * w) - self.ro_inv * self.dx(w)
        return self.dx(psy * w) - self.dy(psx * w) + self.re_inv * self.lap(w) + self.poisson(inner)

    def jacobian_dense(self, U):
        return np.stack([self.jvp(U, e) for e in np.eye(self.n)], axis=1)


def inv_helmholtz_sqrt_2d(nx: int, a: float, b: float):
    """Gamma^{1/2} = (a I - b Delta*)^{-1} with the five-point Delta* of an
    nx x (2 nx + 1) interior grid, so that Gamma = (a I - b Delta*)^{-2} (the
    prior of Sec. 5.2 with a = 0, b = 0.06). Applied by a sparse LU solve."""
    import scipy.sparse as sp
    from scipy.sparse.linalg import splu
    ny = 2 * nx + 1
    T = (a * sp.identity(nx * ny) - b * dirichlet_laplacian_2d(nx, ny)).tocsc()
    lu = splu(T)
    return lambda X: lu.solve(np.asarray(X, dtype=np.float64))
