"""The SC-4DVAR problem in the control variable v (oracle).

Eq. 4dvar_cf:  J(x0) = 1/2 |x0 - xb|^2_{Gamma^-1} + 1/2 sum_i |O(x_i) - y_i|^2_{R_i^-1}
With x0 = xb + Gamma^{1/2} v and R_i = sigma^2 I this is
               J(v)  = 1/2 |v|^2 + 1/2 |d|^2,   d_i = (O x_i - y_i) / sigma.
Eq. Rhalf:     A = [R_i^{-1/2} O_i M_i Gamma^{1/2}]_{i=1..n_t}  (m x n),  H = A^T A.
Eq. 4dvar_gradient, mapped to v (g_v = Gamma^{1/2} grad_x J):
               g_v = v + A^T d
Eq. gniterf1 / pcgsystem: (I + H) dv = -g_v, and x0 <- x0 + Gamma^{1/2} dv.

Observation times are t_i = obs_steps[i] RK steps after t0 (t0 itself is not an
observation time: the sum in Eq. 4dvar_cf starts at i = 1). The observation
operator O_i selects grid points obs_idx[i, :]. Rows of A (and of W = A X) are
ordered time-major: row i * n_o + o.

The adjoint sweep runs t = N .. 1; at an observation step the forcing
O_i^T R_i^{-1/2} w_i is added to lambda_t before stepping back to t - 1.
"""
from __future__ import annotations

import numpy as np

from . import rk4


class FourDVar:
    def __init__(self, model, h, n_steps, obs_steps, obs_idx, sigma_obs,
                 prior_sqrt, xb=None, y=None, tableau=rk4.RK4):
        self.model = model
        self.tab = tableau
        self.h = float(h)
        self.N = int(n_steps)
        self.obs_steps = np.asarray(obs_steps, dtype=np.int64)
        self.obs_idx = np.asarray(obs_idx, dtype=np.int64)
        assert self.obs_idx.shape[0] == len(self.obs_steps)
        assert np.all(self.obs_steps >= 1) and np.all(self.obs_steps <= self.N)
        assert np.all(np.diff(self.obs_steps) > 0)
        self.sigma = float(sigma_obs)
        self.prior_sqrt = prior_sqrt           # callable: (n,) or (n,k) -> same
        self.n = model.n
        self.n_t, self.n_o = self.obs_idx.shape
        self.m = self.n_t * self.n_o
        self._obs_at = {int(s): i for i, s in enumerate(self.obs_steps)}
        self.xb = None if xb is None else np.asarray(xb, dtype=np.float64)
        self.y = None if y is None else np.asarray(y, dtype=np.float64).reshape(self.n_t, self.n_o)
        self.traj = None
        self.counters = {"fwd": 0, "tlm": 0, "adj": 0}

    # -- model runs ----------------------------------------------------------
    def forward(self, x0):
        """FWD sweep: the full trajectory x_0 .. x_N (list of (n,) arrays)."""
        xs = [np.array(x0, dtype=np.float64)]
        for _ in range(self.N):
            xs.append(rk4.fwd_step(self.model, xs[-1], self.h, self.tab))
        return xs

    def observe(self, traj):
        """O x_{t_i} for every observation time, shape (n_t, n_o)."""
        return np.stack([traj[int(s)][self.obs_idx[i]] for i, s in enumerate(self.obs_steps)])

    def set_iterate(self, v):
        """x0 = xb + Gamma^{1/2} v, then FWD; returns J(v)."""
        self.v = np.array(v, dtype=np.float64)
        self.x0 = self.xb + self.prior_sqrt(self.v)
        self.traj = self.forward(self.x0)
        self.counters["fwd"] += 1
        self.d = ((self.observe(self.traj) - self.y) / self.sigma).reshape(self.m)
        return self.cost()

    def cost(self):
        return 0.5 * float(self.v @ self.v) + 0.5 * float(np.sum(self.d * self.d))

    # -- linearized operators along the stored trajectory -------------------
    def tlm_obs(self, dx0):
        """R^{-1/2} O_i M_i dx0 for all i: the TLM sweep of a block (n, k) -> (m, k)."""
        dx = np.array(dx0, dtype=np.float64)
        out = np.zeros((self.n_t, self.n_o) + dx.shape[1:])
        for t in range(self.N):
            dx = rk4.tlm_step(self.model, self.traj[t], dx, self.h, self.tab)
            i = self._obs_at.get(t + 1)
            if i is not None:
                out[i] = dx[self.obs_idx[i]] / self.sigma
        return out.reshape((self.m,) + dx.shape[1:])

    def adj_obs(self, W):
        """sum_i M_i^T O_i^T R^{-1/2} w_i: the ADJ sweep of a block (m, k) -> (n, k)."""
        W = np.asarray(W, dtype=np.float64)
        Wt = W.reshape((self.n_t, self.n_o) + W.shape[1:])
        lam = np.zeros((self.n,) + W.shape[1:])
        for t in range(self.N, 0, -1):
            i = self._obs_at.get(t)
            if i is not None:
                np.add.at(lam, self.obs_idx[i], Wt[i] / self.sigma)
            lam = rk4.adj_step(self.model, self.traj[t - 1], lam, self.h, self.tab)
        return lam

    def A(self, X):
        """A X of Eq. Rhalf (block)."""
        self.counters["tlm"] += 1 if np.ndim(X) == 1 else np.shape(X)[1]
        return self.tlm_obs(self.prior_sqrt(X))

    def At(self, W):
        """A^T W of Eq. Rhalf (block)."""
        self.counters["adj"] += 1 if np.ndim(W) == 1 else np.shape(W)[1]
        return self.prior_sqrt(self.adj_obs(W))

    def misfit_hvp(self, X):
        """H X = A^T A X (the data-misfit part, Eq. Rhalf)."""
        return self.At(self.A(X))

    def hvp(self, X):
        """(I + H) X, the prior-preconditioned GN Hessian of Eq. gniterf1."""
        return X + self.misfit_hvp(X)

    def gradient(self):
        """g_v = v + A^T d (Eq. 4dvar_gradient in the control variable)."""
        return self.v + self.At(self.d)

    # -- dense forms (tiny problems only) -----------------------------------
    def A_dense(self):
        return np.stack([self.A(e) for e in np.eye(self.n)], axis=1)

    def At_dense(self):
        return np.stack([self.At(e) for e in np.eye(self.m)], axis=1)
