"""Classic RK4 step, its tangent-linear step and its discrete adjoint (oracle).

The paper builds its TLM and ADJ as the discrete Runge-Kutta tangent-linear and
adjoint models of Sandu (cited in Sec. 2.1 and Sec. 5.1/5.2). For an explicit
RK method with coefficients a_ij, b_i applied to x' = f(x):

  stages   X_i = x + h sum_{j<i} a_ij k_j,   k_i = f(X_i),   x' = x + h sum_i b_i k_i
  TLM      dX_i = dx + h sum_{j<i} a_ij dk_j, dk_i = F_i dX_i, dx' = dx + h sum_i b_i dk_i
  ADJ      kappa_i = h b_i lam' + h sum_{j>i} a_ji theta_j,  theta_i = F_i^T kappa_i,
           lam = lam' + sum_i theta_i
with F_i = f'(X_i). The ADJ step is the exact transpose of the TLM step. The
default tableau is classic RK4: a21 = a32 = 1/2, a43 = 1, b = (1/6, 1/3, 1/3,
1/6). RK3_TVD is the third-order total-variation-diminishing scheme of the
paper's experiments (Sec. 5.1, 5.2; Gottlieb & Shu) in Butcher form: a21 = 1,
a31 = a32 = 1/4, b = (1/6, 1/6, 2/3).

``model`` is any object with rhs(u), jvp(U, d) and vjp(U, w); blocks of k
directions are (n, k) arrays and the base stage state U is (n,).
"""
from __future__ import annotations

import numpy as np

A = np.array([[0.0, 0.0, 0.0, 0.0],
              [0.5, 0.0, 0.0, 0.0],
              [0.0, 0.5, 0.0, 0.0],
              [0.0, 0.0, 1.0, 0.0]])
B = np.array([1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0])
S = 4
RK4 = (A, B)
RK3_TVD = (np.array([[0.0, 0.0, 0.0],
                     [1.0, 0.0, 0.0],
                     [0.25, 0.25, 0.0]]),
           np.array([1.0 / 6.0, 1.0 / 6.0, 2.0 / 3.0]))


def stages(model, x, h, tab=RK4):
    """Base stage states X_1..X_S and slopes k_1..k_S of one step from x."""
    A, B = tab
    S = len(B)
    X, K = [], []
    for i in range(S):
        Xi = x.copy()
        for j in range(i):
            if A[i, j] != 0.0:
                Xi = Xi + h * A[i, j] * K[j]
        X.append(Xi)
        K.append(model.rhs(Xi))
    return X, K


def fwd_step(model, x, h, tab=RK4):
    A, B = tab
    S = len(B)
    _, K = stages(model, x, h, tab)
    out = x.copy()
    for i in range(S):
        out = out + h * B[i] * K[i]
    return out


def tlm_step(model, x, dx, h, tab=RK4):
    A, B = tab
    S = len(B)
    X, _ = stages(model, x, h, tab)
    dK = []
    for i in range(S):
        dXi = dx.copy()
        for j in range(i):
            if A[i, j] != 0.0:
                dXi = dXi + h * A[i, j] * dK[j]
        dK.append(model.jvp(X[i], dXi))
    out = dx.copy()
    for i in range(S):
        out = out + h * B[i] * dK[i]
    return out


def adj_step(model, x, lam_next, h, tab=RK4):
    A, B = tab
    S = len(B)
    X, _ = stages(model, x, h, tab)
    theta = [None] * S
    for i in reversed(range(S)):
        kap = h * B[i] * lam_next
        for j in range(i + 1, S):
            if A[j, i] != 0.0:
                kap = kap + h * A[j, i] * theta[j]
        theta[i] = model.vjp(X[i], kap)
    out = lam_next.copy()
    for i in range(S):
        out = out + theta[i]
    return out
