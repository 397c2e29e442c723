"""Randomized low-rank approximations of the data-misfit Hessian H = A^T A (oracle).

Each routine follows the steps of the paper's algorithm in order, with numpy /
scipy dense routines (QR, SVD, Cholesky, triangular solve) as its steps. The
operators are callables on blocks: A_op (n,k)->(m,k), At_op (m,k)->(n,k),
H_op (n,k)->(n,k) (misfit part only), I_plus_H (n,)->(n,).

All return a LowRank with V (n x l, orthonormal columns) and lam (l,) >= 0 such
that  H_hat = V diag(lam) V^T, plus W (l x n) where the algorithm builds one.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.linalg as sla

from . import philox

EPS_FP64 = 2.0 ** -53     # unit roundoff of the precision that forms Y (Alg. 2, step 3)


@dataclasses.dataclass
class LowRank:
    V: np.ndarray
    lam: np.ndarray
    W: np.ndarray | None = None
    tlm: int = 0          # TLM applications spent (columns)
    adj: int = 0          # ADJ applications spent (columns)
    kappa_hist: list | None = None

    @property
    def rank(self) -> int:
        return len(self.lam)

    def H_hat(self):
        return (self.V * self.lam) @ self.V.T


def woodbury_apply(lr: LowRank, R):
    """(I + V Lam V^T)^{-1} R = R - V (Lam^{-1} + I)^{-1} V^T R   (Eq. woodbury)."""
    d = lr.lam / (1.0 + lr.lam)
    T = lr.V.T @ R
    T = (d * T.T).T if T.ndim == 2 else d * T
    return R - lr.V @ T


def woodbury_apply_W(W, R):
    """(I + W^T W)^{-1} R = R - W^T (I_l + W W^T)^{-1} W R   (Remark 1, Eq. randsvdsv)."""
    l = W.shape[0]
    G = np.eye(l) + W @ W.T
    c = sla.cho_factor(G, lower=True)
    return R - W.T @ sla.cho_solve(c, W @ R)


def thin_svd_lowrank(W, tlm=0, adj=0):
    """thin SVD W = U S V^T -> V, Lam = S^2 (the last step of Algs. 1, 3, 4, 5)."""
    _, s, Vt = np.linalg.svd(W, full_matrices=False)
    return LowRank(V=Vt.T, lam=s ** 2, W=W, tlm=tlm, adj=adj)


def kappa_estimate(I_plus_H, precond_apply, v):
    """|| (I + H)(I + H_hat)^{-1} v ||_2 with v a unit vector (Eqs. condtext, condtext2)."""
    return float(np.linalg.norm(I_plus_H(precond_apply(v))))


def unit_test_vector(seed, stream, n, index=0):
    w = philox.gaussian(seed, stream, n, 1, col0=index)[:, 0]
    return w / np.linalg.norm(w)


# --------------------------------------------------------------------------- Alg. 1
def randsvd(A_op, At_op, Omega):
    """Alg. 1 (RandSVD): Y = A Omega; Y = QR; W^T = A^T Q; W = U S V^T; Lam = S^2."""
    Y = A_op(Omega)
    Q, _ = np.linalg.qr(Y)
    Wt = At_op(Q)
    l = Omega.shape[1]
    return thin_svd_lowrank(Wt.T, tlm=l, adj=l)


# --------------------------------------------------------------------------- Alg. 2
def nystrom_core(Omega, Y, eps=EPS_FP64, n=None):
    """Steps 3-7 of Alg. 2 on a given sketch Y = H Omega."""
    n = Omega.shape[0] if n is None else n
    nu = np.sqrt(n) * eps * np.linalg.norm(Y, 2)
    Y = Y + nu * Omega
    C = Omega.T @ Y
    L = np.linalg.cholesky(0.5 * (C + C.T))
    W = sla.solve_triangular(L, Y.T, lower=True)          # L^{-1} Y^T
    _, s, Vt = np.linalg.svd(W, full_matrices=False)
    lam = np.maximum(0.0, s ** 2 - nu)
    return LowRank(V=Vt.T, lam=lam, W=None), nu


def nystrom(H_op, Omega, eps=EPS_FP64):
    """Alg. 2 (Nystrom, stabilized fixed-rank form; rank truncation r = l)."""
    Y = H_op(Omega)
    lr, _ = nystrom_core(Omega, Y, eps)
    l = Omega.shape[1]
    lr.tlm, lr.adj = l, l
    return lr


# --------------------------------------------------------------------------- Alg. 3
def pinv_upper(R, rtol=1e-12):
    """Pseudo-inverse of a square upper-triangular R (the R_M^dagger of Alg. 3)."""
    return np.linalg.pinv(R, rcond=rtol)


def singleview_W(QY, Psi, Z):
    """Steps 4-5 of Alg. 3: M = Psi^T Q_Y = Q_M R_M;  W = R_M^dagger (Z Q_M)^T."""
    M = Psi.T @ QY
    QM, RM = np.linalg.qr(M)
    return pinv_upper(RM) @ (Z @ QM).T


def singleview(A_op, At_op, Omega, Psi):
    """Alg. 3 (SingleView): Y = A Omega, Z = A^T Psi; QR of Y; W; thin SVD."""
    Y = A_op(Omega)
    Z = At_op(Psi)
    QY, _ = np.linalg.qr(Y)
    W = singleview_W(QY, Psi, Z)
    return thin_svd_lowrank(W, tlm=Omega.shape[1], adj=Psi.shape[1])


# --------------------------------------------------------------------------- Alg. 6
def qr_update(A1, A2, B1, B2, Q1, R1):
    """Alg. 6: QR of [A1; A2][B1 B2] given Q1 R1 = A1 B1 (B1, B2 orthonormal)."""
    Q2, R2 = np.linalg.qr(A2 @ B1)
    Q3, R3 = np.linalg.qr(np.vstack([R1, R2]))
    k1 = Q1.shape[1]
    blk = np.zeros((Q1.shape[0] + Q2.shape[0], k1 + Q2.shape[1]))
    blk[:Q1.shape[0], :k1] = Q1
    blk[Q1.shape[0]:, k1:] = Q2
    Q3 = blk @ Q3
    P1 = np.vstack([A1, A2]) @ B2
    T = Q3.T @ P1
    P2 = P1 - Q3 @ T
    Q4, R4 = np.linalg.qr(P2)
    Q5 = np.hstack([Q3, Q4])
    R5 = np.block([[R3, T], [np.zeros((R4.shape[0], R3.shape[1])), R4]])
    return Q5, R5


# --------------------------------------------------------------------------- Alg. 4
def cgs2(Q, Y):
    """Y - Q (Q^T Y), applied twice (the extra Gram-Schmidt pass of Algs. 4/5)."""
    for _ in range(2):
        Y = Y - Q @ (Q.T @ Y)
    return Y


def adaptive_randsvd(A_op, At_op, I_plus_H, draw_omega, l0, l_hat, eps_sk,
                     l_max, draw_v):
    """Alg. 4 (adaptive RandSVD); draw_omega(col0, cols) returns Omega columns,
    draw_v(t) the t-th unit test vector. kappa_sk uses Remark 1 with W."""
    Omega = draw_omega(0, l0)
    Y = A_op(Omega)
    Qh, _ = np.linalg.qr(Y)
    W = At_op(Qh).T
    Q = np.zeros((Y.shape[0], 0))
    l = l0
    tlm, adj = l0, l0
    kap = kappa_estimate(I_plus_H, lambda r: woodbury_apply_W(W, r), draw_v(0))
    hist = [(l, kap)]
    t = 1
    while kap > eps_sk and l + l_hat <= l_max:
        Q = np.hstack([Q, Qh])
        Omega_h = draw_omega(l, l_hat)
        Y = A_op(Omega_h)
        Y = cgs2(Q, Y)
        Qh, _ = np.linalg.qr(Y)
        Wh = At_op(Qh).T
        l += l_hat
        tlm += l_hat
        adj += l_hat
        W = np.vstack([W, Wh])
        kap = kappa_estimate(I_plus_H, lambda r: woodbury_apply_W(W, r), draw_v(t))
        hist.append((l, kap))
        t += 1
    lr = thin_svd_lowrank(W, tlm=tlm, adj=adj)
    lr.kappa_hist = hist
    return lr


# --------------------------------------------------------------------------- Alg. 5
def adaptive_singleview(A_op, At_op, I_plus_H, draw_omega, draw_psi, l1, l2,
                        l1_hat, l2_hat, eps_sk, l_max, draw_v):
    """Alg. 5 (adaptive SingleView). The new row-space sketch of each round is
    Z_hat = A^T Psi_hat, and the small QR of [Psi^T; Psi_hat^T][Q_Y Q_Y_hat] is
    recomputed directly."""
    Omega = draw_omega(0, l1)
    Psi = draw_psi(0, l2)
    Y = A_op(Omega)
    Z = At_op(Psi)
    QY, _ = np.linalg.qr(Y)
    W = singleview_W(QY, Psi, Z)
    tlm, adj = l1, l2
    kap = kappa_estimate(I_plus_H, lambda r: woodbury_apply_W(W, r), draw_v(0))
    hist = [(l1, kap)]
    t = 1
    while kap > eps_sk and l1 + l1_hat <= l_max:
        Omega_h = draw_omega(l1, l1_hat)
        Psi_h = draw_psi(l2, l2_hat)
        Y = A_op(Omega_h)
        Y = cgs2(QY, Y)
        QYh, _ = np.linalg.qr(Y)
        Zh = At_op(Psi_h)
        QY = np.hstack([QY, QYh])
        Psi = np.hstack([Psi, Psi_h])
        Z = np.hstack([Z, Zh])
        W = singleview_W(QY, Psi, Z)
        l1 += l1_hat
        l2 += l2_hat
        tlm += l1_hat
        adj += l2_hat
        kap = kappa_estimate(I_plus_H, lambda r: woodbury_apply_W(W, r), draw_v(t))
        hist.append((l1, kap))
        t += 1
    lr = thin_svd_lowrank(W, tlm=tlm, adj=adj)
    lr.kappa_hist = hist
    return lr


# ----------------------------------------------------------------- adaptive Nystrom
def adaptive_nystrom(H_op, I_plus_H, draw_omega, l0, l_hat, eps_sk, l_max, draw_v,
                     eps=EPS_FP64):
    """Adaptive Nystrom: grow the sketch Y = H Omega by l_hat columns and redo the
    Nystrom factorization (steps 3-7 of Alg. 2) on the whole sketch until
    kappa_sk <= eps_sk (the paper defers to Frangella et al. for this variant)."""
    Omega = draw_omega(0, l0)
    Y = H_op(Omega)
    lr, _ = nystrom_core(Omega, Y, eps)
    l = l0
    kap = kappa_estimate(I_plus_H, lambda r: woodbury_apply(lr, r), draw_v(0))
    hist = [(l, kap)]
    t = 1
    while kap > eps_sk and l + l_hat <= l_max:
        Om = draw_omega(l, l_hat)
        Omega = np.hstack([Omega, Om])
        Y = np.hstack([Y, H_op(Om)])
        l += l_hat
        lr, _ = nystrom_core(Omega, Y, eps)
        kap = kappa_estimate(I_plus_H, lambda r: woodbury_apply(lr, r), draw_v(t))
        hist.append((l, kap))
        t += 1
    lr.tlm, lr.adj = l, l
    lr.kappa_hist = hist
    return lr
