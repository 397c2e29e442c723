"""GB300 SC-4DVAR Gauss-Newton library: thin Python binding of include/sc4dvar.h.

Every numerical step runs in the CUDA kernels of libsc4dvar.so; this module only
turns torch tensors (device memory, streams) into pointers and sizes. Importing
it loads the library and raises if the library cannot be built or loaded: there
is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _abi
from ._abi import (DF64, FP32, FP64, GEMM_3XTF32, GEMM_BF16, GEMM_SIMT, GEMM_TF32,  # noqa: F401
                   MODEL_BURGERS1D, PRIOR_SE, PRIOR_SYMBOL, SKETCH_NONE, SKETCH_NYSTROM, SKETCH_RANDSVD,
                   SKETCH_SINGLEVIEW, STREAM_KAPPA, STREAM_PSI, STREAM_SKETCH, Sc4dvarError)

lib = _abi.load()
check = _abi.check

METHODS = {"none": SKETCH_NONE, "randsvd": SKETCH_RANDSVD, "nystrom": SKETCH_NYSTROM,
           "singleview": SKETCH_SINGLEVIEW}


def _torch():
    import torch
    return torch


def _ptr(t):
    if t is None:
        return None
    assert t.is_cuda and t.is_contiguous(), "device tensors must be contiguous CUDA tensors"
    return C.c_void_p(t.data_ptr())


def _stream(stream=None):
    torch = _torch()
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def _dtype(prec):
    torch = _torch()
    return torch.float32 if prec == FP32 else torch.float64


class Precond:
    """Low-rank H_hat = V diag(lam) V^T (Sec. 3.1); owns its device arrays."""

    def __init__(self, handle, n):
        self.h = handle
        self.n = n

    @property
    def rank(self):
        r = C.c_int()
        check(lib.sc4dvar_precond_info(self.h, C.byref(r), None, None))
        return r.value

    def arrays(self):
        r = self.rank
        lam = np.zeros(max(r, 1))
        V = np.zeros((max(r, 1), self.n))
        check(lib.sc4dvar_precond_info(self.h, None, lam.ctypes.data_as(C.c_void_p),
                                       V.ctypes.data_as(C.c_void_p)))
        return V[:r].T.copy(), lam[:r].copy()

    def apply(self, R, stream=None):
        """(I + H_hat)^{-1} R (Eq. woodbury); R is (n,) or (k, n) float64."""
        R2 = R.reshape(-1, self.n).contiguous()
        Z = _torch().empty_like(R2)
        check(lib.sc4dvar_precond_apply(self.h, _ptr(R2), self.n, R2.shape[0], _ptr(Z), self.n,
                                        _stream(stream)))
        return Z.reshape(R.shape)

    def sketchsolv(self, g, stream=None):
        """dv = -(I + H_hat)^{-1} g (Eq. dxsol in the control variable)."""
        dv = _torch().empty_like(g)
        check(lib.sc4dvar_sketchsolv(self.h, _ptr(g), _ptr(dv), _stream(stream)))
        return dv

    def close(self):
        if self.h:
            lib.sc4dvar_precond_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class GNCheckpoint:
    """Gauss-Newton state at an iteration boundary, for checkpoint and resume.

    v: the iterate (float64, (n,)). next_iter: the iterations completed, which is
    also the random-number state (the sketch draws and the kappa_re probe of
    iteration k are keyed by k). g0_inf: |g_0|_inf, the gtol reference. V, lam:
    the factors (n, l) and (l,) of the preconditioner held across the boundary, or
    None. sketch_iter: the iteration that built them (-1: none). counters: the
    problem's counters. record: the per-iteration records of the iterations done.
    save() and load() write and read one .npz file."""

    FORMAT = 1

    def __init__(self, v, next_iter, g0_inf, sketch_iter, V, lam, counters, record):
        self.v = np.asarray(v, dtype=np.float64)
        self.next_iter = int(next_iter)
        self.g0_inf = float(g0_inf)
        self.sketch_iter = int(sketch_iter)
        self.V = None if V is None else np.asarray(V, dtype=np.float64)
        self.lam = None if lam is None else np.asarray(lam, dtype=np.float64)
        self.counters = {k: int(x) for k, x in dict(counters).items()}
        self.record = [dict(r) for r in record]

    def save(self, path):
        import json
        has = self.V is not None
        np.savez(path, format=np.int64(self.FORMAT), v=self.v, next_iter=np.int64(self.next_iter),
                 g0_inf=np.float64(self.g0_inf), sketch_iter=np.int64(self.sketch_iter),
                 has_precond=np.int64(int(has)), V=self.V if has else np.zeros((self.v.shape[0], 0)),
                 lam=self.lam if has else np.zeros(0),
                 counters=np.array(json.dumps(self.counters)), record=np.array(json.dumps(self.record)))

    @classmethod
    def load(cls, path):
        import json
        with np.load(path, allow_pickle=False) as z:
            if int(z["format"]) != cls.FORMAT:
                raise ValueError(f"GN checkpoint format {int(z['format'])}, expected {cls.FORMAT}")
            has = bool(int(z["has_precond"]))
            return cls(z["v"], int(z["next_iter"]), float(z["g0_inf"]), int(z["sketch_iter"]),
                       z["V"] if has else None, z["lam"] if has else None,
                       json.loads(str(z["counters"])), json.loads(str(z["record"])))


class Problem:
    """One SC-4DVAR assimilation window (handle of sc4dvar_problem_create).

    Blocks are torch tensors of shape (k, n) / (k, m) whose rows are the columns
    of the column-major C blocks (so a contiguous (k, n) tensor is an n x k block
    with leading dimension n).
    """

    def __init__(self, *, n, nu, dt, n_steps, obs_steps, obs_idx, sigma_obs,
                 prior_sigma=None, prior_length=None, prior_symbol=None, model=MODEL_BURGERS1D,
                 grid=None, forcing_amp=0.0, forcing_k=0, n_checkpoints=0, integrator=0):
        obs_steps = np.ascontiguousarray(obs_steps, dtype=np.int32)
        obs_idx = np.ascontiguousarray(obs_idx, dtype=np.int32)
        d = _abi.ProblemDesc()
        d.model = model
        if model == _abi.MODEL_BVE2D:
            d.nx = d.ny = int(grid)
            d.forcing_amp, d.forcing_k = float(forcing_amp), int(forcing_k)
        elif model == _abi.MODEL_BVE_GYRE:
            d.nx, d.ny = int(grid), 2 * int(grid) + 1
            d.forcing_amp = float(forcing_amp)
        else:
            d.nx, d.ny = int(n), 1
        d.n_checkpoints = int(n_checkpoints)
        d.nu, d.dt, d.n_steps = float(nu), float(dt), int(n_steps)
        d.n_obs_times = int(obs_idx.shape[0])
        d.n_obs = int(obs_idx.shape[1])
        d.obs_steps = obs_steps.ctypes.data_as(C.POINTER(C.c_int))
        d.obs_idx = obs_idx.ctypes.data_as(C.POINTER(C.c_int))
        d.sigma_obs = float(sigma_obs)
        d.integrator = int(integrator)
        if model == _abi.MODEL_BVE2D:
            d.prior_kind = _abi.PRIOR_INV_HELMHOLTZ
            d.prior_sigma, d.prior_length = float(prior_sigma), float(prior_length)
        elif model in (_abi.MODEL_BURGERS1D_DIRICHLET, _abi.MODEL_BVE_GYRE):
            d.prior_kind = _abi.PRIOR_DIRICHLET_INV_HELMHOLTZ
            d.prior_sigma, d.prior_length = float(prior_sigma), float(prior_length)
        elif prior_symbol is not None:
            sym = np.ascontiguousarray(prior_symbol, dtype=np.float64)
            d.prior_kind = PRIOR_SYMBOL
            d.prior_symbol = sym.ctypes.data_as(C.POINTER(C.c_double))
        else:
            d.prior_kind = PRIOR_SE
            d.prior_sigma, d.prior_length = float(prior_sigma), float(prior_length)
        h = C.c_void_p()
        check(lib.sc4dvar_problem_create(C.byref(d), C.byref(h)))
        self.h = h
        nn, mm = C.c_int(), C.c_int()
        check(lib.sc4dvar_problem_dims(h, C.byref(nn), C.byref(mm)))
        self.n, self.m = nn.value, mm.value

    @classmethod
    def from_workload(cls, wl, obs_idx, **kw):
        return cls(n=wl.n, nu=wl.nu, dt=wl.dt, n_steps=wl.n_steps, obs_steps=wl.obs_steps,
                   obs_idx=obs_idx, sigma_obs=wl.sigma_obs, prior_sigma=wl.sigma_b,
                   prior_length=wl.length_b, **kw)

    @classmethod
    def from_bve_workload(cls, wl, draws, n_checkpoints=None):
        """Barotropic vorticity problem: N x N doubly periodic grid (fields of N*N,
        row-major, y slow), inverse-Helmholtz prior c (I - ell^2 Lap)^{-1}.
        n_checkpoints: None takes the workload's (0 = store every stage state)."""
        if n_checkpoints is None:
            n_checkpoints = getattr(wl, "n_checkpoints", 0)
        return cls(n_checkpoints=n_checkpoints, n=wl.n, nu=wl.nu, dt=wl.dt, n_steps=wl.n_steps, obs_steps=wl.obs_steps,
                   obs_idx=draws["obs_idx"], sigma_obs=draws["sigma_obs"],
                   prior_sigma=draws["prior_c"], prior_length=draws["prior_ell"],
                   model=_abi.MODEL_BVE2D, grid=wl.N, forcing_amp=wl.forcing_amp,
                   forcing_k=wl.forcing_k)

    @classmethod
    def from_paper_burgers_workload(cls, wl, draws):
        """The Burgers experiment of Sec. 5.1: Dirichlet boundaries, n interior
        points, RK3-TVD, prior Gamma^{1/2} = (a I - b Delta*)^{-1}."""
        return cls(n=wl.n, nu=wl.nu, dt=wl.dt, n_steps=wl.n_steps, obs_steps=wl.obs_steps,
                   obs_idx=draws["obs_idx"], sigma_obs=wl.sigma_obs, prior_sigma=wl.prior_a,
                   prior_length=wl.prior_b, model=_abi.MODEL_BURGERS1D_DIRICHLET,
                   integrator=_abi.RK3_TVD)

    @classmethod
    def from_gyre_workload(cls, wl, draws):
        """The barotropic vorticity experiment of Sec. 5.2: the double gyre in the
        closed basin (0, 1) x (-1, 1) on nx x (2 nx + 1) interior points, Re, Ro,
        RK3-TVD, prior Gamma^{1/2} = (a I - b Delta*)^{-1} (five-point Delta*)."""
        return cls(n=wl.n, nu=1.0 / wl.re, dt=wl.dt, n_steps=wl.n_steps, obs_steps=wl.obs_steps,
                   obs_idx=draws["obs_idx"], sigma_obs=wl.sigma_obs, prior_sigma=wl.prior_a,
                   prior_length=wl.prior_b, model=_abi.MODEL_BVE_GYRE, grid=wl.nx,
                   forcing_amp=1.0 / wl.ro, integrator=_abi.RK3_TVD)

    def close(self):
        if getattr(self, "h", None):
            lib.sc4dvar_problem_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- data -----------------------------------------------------------------
    def set_background(self, xb, stream=None):
        check(lib.sc4dvar_set_background(self.h, _ptr(xb), _stream(stream)))

    def set_observations(self, y, stream=None):
        check(lib.sc4dvar_set_observations(self.h, _ptr(y), _stream(stream)))

    def prior_symbol(self):
        s = np.zeros(self.n)
        check(lib.sc4dvar_prior_symbol(self.h, s.ctypes.data_as(C.c_void_p)))
        return s

    def prior_sqrt_apply(self, X, stream=None):
        """Gamma^{1/2} X for X of shape (n,) or (k, n), float64."""
        X2 = X.reshape(-1, self.n).contiguous()
        Y = _torch().empty_like(X2)
        check(lib.sc4dvar_prior_sqrt_apply(self.h, _ptr(X2), self.n, X2.shape[0], _ptr(Y), self.n,
                                           _stream(stream)))
        return Y.reshape(X.shape)

    def forecast(self, x0, stream=None):
        """O x_{t_i} for all observation times (m,), and the final state (n,)."""
        torch = _torch()
        obs = torch.empty(self.m, dtype=torch.float64, device=x0.device)
        xN = torch.empty(self.n, dtype=torch.float64, device=x0.device)
        check(lib.sc4dvar_forecast(self.h, _ptr(x0), _ptr(obs), _ptr(xN), _stream(stream)))
        return obs, xN

    # -- the path ---------------------------------------------------------------
    def fwd(self, v, want_d=False, stream=None):
        """x0 = xb + Gamma^{1/2} v, FWD sweep; returns J(v) (and d if asked)."""
        J = C.c_double()
        d = _torch().empty(self.m, dtype=_torch().float64, device=v.device) if want_d else None
        check(lib.sc4dvar_fwd(self.h, _ptr(v), C.byref(J), _ptr(d), _stream(stream)))
        self._fwd_gen = getattr(self, "_fwd_gen", 0) + 1
        return (J.value, d) if want_d else J.value

    def gradient(self, stream=None, out=None):
        g = out if out is not None else _torch().empty(self.n, dtype=_torch().float64, device="cuda")
        check(lib.sc4dvar_gradient(self.h, _ptr(g), _stream(stream)))
        return g

    def tlm_block(self, X, prec=FP64, stream=None, out=None):
        """A X (Eq. Rhalf). X: (k, n) -> (k, m)."""
        X2 = X.reshape(-1, self.n).contiguous()
        k = X2.shape[0]
        W = out if out is not None else _torch().empty((k, self.m), dtype=_dtype(prec), device=X.device)
        check(lib.sc4dvar_tlm_block(self.h, _ptr(X2), self.n, k, _ptr(W), self.m, prec, _stream(stream)))
        return W

    def adj_block(self, W, prec=FP64, stream=None, out=None):
        """A^T W (Eq. Rhalf). W: (k, m) -> (k, n)."""
        W2 = W.reshape(-1, self.m).contiguous()
        k = W2.shape[0]
        X = out if out is not None else _torch().empty((k, self.n), dtype=_dtype(prec), device=W.device)
        check(lib.sc4dvar_adj_block(self.h, _ptr(W2), self.m, k, _ptr(X), self.n, prec, _stream(stream)))
        return X

    def gn_hessian_apply_block(self, X, misfit_only=False, prec=FP64, stream=None, out=None):
        """(I + A^T A) X, or A^T A X. X: (k, n) -> (k, n)."""
        X2 = X.reshape(-1, self.n).contiguous()
        k = X2.shape[0]
        Y = out if out is not None else _torch().empty_like(X2)
        check(lib.sc4dvar_gn_hessian_apply_block(self.h, _ptr(X2), self.n, k, _ptr(Y), self.n,
                                                 int(misfit_only), prec, _stream(stream)))
        return Y.reshape(X.shape) if out is None else Y

    def build_precond(self, method="randsvd", l=20, l2=0, adaptive=False, l_hat=0, l_max=0,
                      eps_sk=1.01, seed=20240128, gn_iter=0, prec=FP64, Omega=None, Psi=None,
                      stream=None, gemm=0):
        """Sketch H at the stored iterate (Algs. 1-5). Omega: (l, n) float64 rows = columns.
        gemm: tall-product arithmetic of FP32 sketches (GEMM_3XTF32, GEMM_SIMT, ...)."""
        o = _abi.SketchOpts(METHODS[method], l, l2, int(adaptive), l_hat, l_max, eps_sk, seed,
                            gn_iter, prec, gemm)
        h = C.c_void_p()
        Om = None if Omega is None else Omega.contiguous()
        Ps = None if Psi is None else Psi.contiguous()
        check(lib.sc4dvar_build_precond(self.h, C.byref(o), _ptr(Om), _ptr(Ps), C.byref(h),
                                        _stream(stream)))
        return Precond(h, self.n)

    def kappa_estimate(self, precond=None, seed=20240128, stream_id=STREAM_KAPPA, column=0,
                       stream=None):
        k = C.c_double()
        check(lib.sc4dvar_kappa_estimate(self.h, None if precond is None else precond.h, seed,
                                         stream_id, column, C.byref(k), _stream(stream)))
        return k.value

    def pcg(self, b, precond=None, tol=1e-6, maxit=0, prec=FP64, refine=2, stream=None, x=None):
        x = _torch().empty_like(b) if x is None else x
        o = _abi.PcgOpts(tol, maxit, prec, refine)
        info = _abi.PcgInfo()
        check(lib.sc4dvar_pcg(self.h, None if precond is None else precond.h, _ptr(b), _ptr(x),
                              C.byref(o), C.byref(info), _stream(stream)))
        return x, {"iterations": info.iterations, "restarts": info.restarts,
                   "relres": info.relres, "status": info.status}

    def _gn_opts(self, iters, method, l, adaptive, l2, l_hat, l_max, eps_sk, eps_re, tol, maxit, prec,
                 refine, gtol, seed, line_search, ls_c1, ls_c2, ls_alpha1, solve, gemm):
        so = _abi.SketchOpts(METHODS[method], l, l2, int(adaptive), l_hat, l_max, eps_sk, seed, 0, prec,
                             gemm)
        return _abi.GnOpts(iters, gtol, so, eps_re, _abi.PcgOpts(tol, maxit, prec, refine),
                           int(line_search), ls_c1, ls_c2, ls_alpha1, {"pcg": 0, "sketchsolv": 1}[solve])

    @staticmethod
    def _gn_records(info, lo, hi):
        return [{"J": info.J[i], "g_inf": info.g_inf[i], "pcg_its": info.pcg_its[i],
                 "relres": info.relres[i], "sketched": bool(info.sketched[i]),
                 "rank": info.rank[i], "kappa_re": info.kappa_re[i], "alpha": info.alpha[i],
                 "ls_evals": info.ls_evals[i], "ls_status": info.ls_status[i]} for i in range(lo, hi)]

    def gauss_newton(self, v, iters=3, method="none", l=20, adaptive=False, l2=0, l_hat=0,
                     l_max=0, eps_sk=1.01, eps_re=10.0, tol=1e-6, maxit=0, prec=FP64, refine=2,
                     gtol=0.0, seed=20240128, line_search=False, ls_c1=1e-4, ls_c2=0.9,
                     ls_alpha1=1.0, solve="pcg", stream=None, gemm=0):
        """Gauss-Newton in place on v (float64, (n,)); returns the per-iteration record."""
        o = self._gn_opts(iters, method, l, adaptive, l2, l_hat, l_max, eps_sk, eps_re, tol, maxit, prec,
                          refine, gtol, seed, line_search, ls_c1, ls_c2, ls_alpha1, solve, gemm)
        info = _abi.GnInfo()
        check(lib.sc4dvar_gauss_newton(self.h, C.byref(o), _ptr(v), C.byref(info), _stream(stream)))
        return self._gn_records(info, 0, info.iters_done)

    def gauss_newton_resume(self, v, iters, checkpoint=None, method="none", l=20, adaptive=False, l2=0,
                            l_hat=0, l_max=0, eps_sk=1.01, eps_re=10.0, tol=1e-6, maxit=0, prec=FP64,
                            refine=2, gtol=0.0, seed=20240128, line_search=False, ls_c1=1e-4, ls_c2=0.9,
                            ls_alpha1=1.0, solve="pcg", stream=None, gemm=0):
        """Gauss-Newton iterations up to `iters` (counted from the start of the run),
        continuing from `checkpoint` (a GNCheckpoint; None starts a new run from v).
        v (float64, (n,), on the device) receives the checkpoint's iterate first and
        the final iterate on return. Returns (record of every iteration so far, the
        GNCheckpoint at the boundary where this call stopped). The options must be
        those of the interrupted run for the continuation to repeat it."""
        o = self._gn_opts(iters, method, l, adaptive, l2, l_hat, l_max, eps_sk, eps_re, tol, maxit, prec,
                          refine, gtol, seed, line_search, ls_c1, ls_c2, ls_alpha1, solve, gemm)
        torch = _torch()
        state = _abi.GnState(0, 0.0, -1)
        held = C.c_void_p()
        prev = []
        if checkpoint is not None:
            cp = checkpoint
            if cp.v.shape != (self.n,):
                raise ValueError(f"checkpoint of size {cp.v.shape}, problem of size {self.n}")
            v.copy_(torch.as_tensor(cp.v, dtype=torch.float64, device=v.device))
            state = _abi.GnState(cp.next_iter, cp.g0_inf, cp.sketch_iter)
            self.counters_set(cp.counters)
            if cp.V is not None:
                held = C.c_void_p(self._precond_import_handle(cp.V, cp.lam))
            prev = list(cp.record)[:cp.next_iter]
        k0 = state.next_iter
        info = _abi.GnInfo()
        rc = lib.sc4dvar_gauss_newton_resume(self.h, C.byref(o), _ptr(v), C.byref(state), C.byref(held),
                                             C.byref(info), _stream(stream))
        # the preconditioner handed back is ours in every case: wrap it at once
        held_pc = Precond(held.value, self.n) if held.value else None
        check(rc)
        record = prev + self._gn_records(info, k0, max(k0, info.iters_done))
        V = lam = None
        if held_pc is not None:
            V, lam = held_pc.arrays()
            held_pc.close()
        cp_out = GNCheckpoint(v.detach().cpu().numpy().copy(), state.next_iter, state.g0_inf,
                              state.sketch_iter if V is not None else -1, V, lam, self.counters(), record)
        return record, cp_out

    def _precond_import_handle(self, V, lam):
        V = np.asarray(V, dtype=np.float64)
        lam = np.ascontiguousarray(np.asarray(lam, dtype=np.float64))
        if V.ndim != 2 or V.shape[0] != self.n or V.shape[1] != lam.shape[0]:
            raise ValueError("V must be (n, l) and lam (l,)")
        Vc = np.ascontiguousarray(V.T)  # column-major n x l
        h = C.c_void_p()
        check(lib.sc4dvar_precond_import(self.h, lam.shape[0], lam.ctypes.data_as(C.c_void_p),
                                         Vc.ctypes.data_as(C.c_void_p), C.byref(h)))
        return h.value

    def precond_import(self, V, lam):
        """A Precond rebuilt from host factors V (n, l) and lam (l,), e.g. those of
        Precond.arrays() or of a GNCheckpoint."""
        return Precond(self._precond_import_handle(V, lam), self.n)

    def counters(self):
        c = _abi.Counters()
        check(lib.sc4dvar_counters(self.h, C.byref(c)))
        return {f: getattr(c, f) for f, _ in _abi.Counters._fields_}

    def counters_reset(self):
        check(lib.sc4dvar_counters_reset(self.h))

    def counters_set(self, counters):
        c = _abi.Counters(**{f: int(counters.get(f, 0)) for f, _ in _abi.Counters._fields_})
        check(lib.sc4dvar_counters_set(self.h, C.byref(c)))


class Batch:
    """Independent problems served together (graph-recorded batched operators)."""

    def __init__(self, problems):
        self.problems = list(problems)
        arr = (C.c_void_p * len(self.problems))(*[p.h for p in self.problems])
        h = C.c_void_p()
        check(lib.sc4dvar_batch_create(arr, len(self.problems), C.byref(h)))
        self.h = h
        self._keep = []

    def hessian_apply(self, Xs, Ys, misfit_only=False, prec=FP64, stream=None):
        """Ys[b] = (I + H_b) Xs[b] for tensors of shape (k_b, n_b)."""
        B = len(self.problems)
        X = (C.c_void_p * B)(*[x.data_ptr() for x in Xs])
        Y = (C.c_void_p * B)(*[y.data_ptr() for y in Ys])
        k = (C.c_int * B)(*[x.shape[0] for x in Xs])
        check(lib.sc4dvar_batch_hessian_apply(self.h, X, Y, k, int(misfit_only), prec, _stream(stream)))
        return Ys

    def pcg_start(self, rhs, preconds=None, tol=1e-6, prec=FP64, stream=None):
        B = len(self.problems)
        R = (C.c_void_p * B)(*[r.data_ptr() for r in rhs])
        Pc = None
        if preconds is not None:
            Pc = (C.c_void_p * B)(*[None if p is None else p.h for p in preconds])
        self._keep = [rhs, preconds]
        check(lib.sc4dvar_batch_pcg_start(self.h, Pc, R, tol, prec, _stream(stream)))

    def pcg_step(self, nsteps=1, stream=None):
        check(lib.sc4dvar_batch_pcg_step(self.h, nsteps, _stream(stream)))

    def pcg_status(self, stream=None):
        B = len(self.problems)
        rel, its, st = (C.c_double * B)(), (C.c_int * B)(), (C.c_int * B)()
        check(lib.sc4dvar_batch_pcg_status(self.h, rel, its, st, _stream(stream)))
        return list(rel), list(its), list(st)

    def pcg_solution(self, xs, stream=None):
        B = len(self.problems)
        X = (C.c_void_p * B)(*[x.data_ptr() for x in xs])
        check(lib.sc4dvar_batch_pcg_solution(self.h, X, _stream(stream)))
        return xs

    def close(self):
        if getattr(self, "h", None):
            lib.sc4dvar_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_COST_FN = None


def _cost_fn():
    global _COST_FN
    if _COST_FN is None:
        torch = _torch()

        class FourDVarCost(torch.autograd.Function):
            """J(v) = 1/2 |v|^2 + 1/2 sum_i |R_i^{-1/2}(O_i x_i - y_i)|^2, x0 = xb + Gamma^{1/2} v
            (Eq. 4dvar_cf in the control variable). forward: the FP64 FWD sweep,
            which leaves the trajectory (or, with checkpointing, the FP64
            checkpoints) and the residuals in the handle. backward: the discrete
            adjoint sweep (Eq. 4dvar_gradient), recomputing each checkpoint
            segment, g_v = v + A^T d, scaled by the incoming gradient."""

            @staticmethod
            def forward(ctx, v, problem):
                J = problem.fwd(v.detach().contiguous())
                ctx.problem = problem
                ctx.gen = problem._fwd_gen
                return v.new_tensor(J)

            @staticmethod
            def backward(ctx, gJ):
                pr = ctx.problem
                if getattr(pr, "_fwd_gen", None) != ctx.gen:
                    raise RuntimeError("the problem ran another FWD after this cost was evaluated; "
                                       "evaluate the cost again before calling backward")
                g = pr.gradient()
                return gJ.to(g.dtype) * g, None

        _COST_FN = FourDVarCost
    return _COST_FN


def cost(problem, v):
    """Differentiable 4D-Var cost J(v) (a 0-dim FP64 tensor on v's device):
    J.backward() runs the adjoint sweep of `problem` at the v of this call."""
    return _cost_fn().apply(v, problem)


def autotune(problem, k):
    """Pick the packed FP32 sweep's pairs per thread for this problem by timing."""
    c = C.c_int()
    check(lib.sc4dvar_autotune(problem.h, k, C.byref(c)))
    return c.value


def gaussian(seed, stream_id, rows, cols, col0=0, stream=None):
    """(cols, rows) float64 tensor: columns col0.. of the method's Philox stream."""
    torch = _torch()
    out = torch.empty((cols, rows), dtype=torch.float64, device="cuda")
    check(lib.sc4dvar_gaussian(seed, stream_id, rows, cols, col0, _ptr(out), _stream(stream)))
    return out


def tall_gemm(A, B, mode=GEMM_3XTF32, transB=False, alpha=1.0, beta=0.0, C=None, out_dtype=None,
              stream=None):
    """C = alpha A op(B) + beta C with the sketches' tall product. Column-major
    shapes as (cols, rows) row-major tensors: A (kk, rows) float32, B (c, kk)
    float64 (B (kk, c) when transB), C (c, rows) float32 or float64."""
    torch = _torch()
    kk, rows = A.shape
    c = B.shape[1] if transB else B.shape[0]
    assert (B.shape[0] if transB else B.shape[1]) == kk
    if C is None:
        C = torch.zeros((c, rows), dtype=out_dtype or torch.float32, device="cuda")
    cd = 1 if C.dtype == torch.float64 else 0
    check(lib.sc4dvar_tall_gemm(mode, rows, kk, c, alpha, _ptr(A), rows, _ptr(B), B.shape[1], int(transB),
                                beta, _ptr(C), cd, rows, _stream(stream)))
    return C


def qr_update(P, B, Q1, R1, r1, k1, stream=None):
    """Alg. 6: the thin QR of [A1; A2][B1 B2] from Q1 R1 = A1 B1, with
    A1 = P[:, :r1]^T, A2 = P[:, r1:]^T, B1 = B[:, :k1], B2 = B[:, k1:].
    P (m, r1 + r2) and B (m, k1 + k2) are float64 CUDA matrices in the usual
    (row, column) shape; returns Q (r1 + r2, k1 + k2) and R (k1 + k2, k1 + k2)."""
    torch = _torch()
    m, ra = P.shape
    kb = B.shape[1]
    r2, k2 = ra - r1, kb - k1
    Pc = P.t().contiguous()          # column-major m x ra
    Bc = B.t().contiguous()
    Qc = torch.zeros((kb, ra), dtype=torch.float64, device=P.device)   # column-major ra x kb
    Rc = torch.zeros((kb, kb), dtype=torch.float64, device=P.device)
    Qc[:k1, :r1] = Q1.t()
    Rc[:k1, :k1] = R1.t()
    check(lib.sc4dvar_qr_update(m, r1, r2, k1, k2, _ptr(Pc), m, _ptr(Bc), m, _ptr(Qc), ra,
                                _ptr(Rc), kb, _stream(stream)))
    return Qc.t(), Rc.t()
