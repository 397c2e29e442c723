"""PCG, SketchSolv and the Gauss-Newton loop with sketch reuse (oracle).

* pcg: conjugate gradients on (I + H) dv = -g_v (Eq. pcgsystem), preconditioned
  by (I + H_hat)^{-1} of Eq. woodbury when a sketch is given (SketchPrec,
  Sec. 2.2.2); with no sketch it is plain CG on the prior-preconditioned system
  (the paper's Prec_Gamma). x0 = 0; stop when the recurrence residual satisfies
  |r|_2 <= tol |b|_2; breakdown when p^T (I+H) p <= 0.
* sketchsolv_step: dv = -(I + H_hat)^{-1} g_v (Eq. dxsol, in v).
* gauss_newton: Sec. 3.2. Fixed sketch size: a new sketch at every GN iteration.
  SketchPrecA: adaptive sketch size (Algs. 4/5, adaptive Nystrom) and reuse of the
  last sketch while kappa_re of Eq. condtext2 stays below eps_re. Full GN steps
  (alpha = 1).

Random draws inside the loop (both sides use this convention with Philox4x32-10,
see oracle.philox.gaussian): at GN iteration k
  Omega columns  <- stream STREAM_SKETCH + k
  Psi columns    <- stream STREAM_SKETCH + k + STREAM_PSI
  kappa_re test  <- stream STREAM_KAPPA + k, column 0
  kappa_sk tests <- stream STREAM_KAPPA + k, columns 1, 2, ...
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import linesearch, philox, sketch

STREAM_SKETCH = 100
STREAM_KAPPA = 200
STREAM_PSI = 1000

# Same values as the library's status codes (SC4DVAR_ERR_BREAKDOWN = -4,
# SC4DVAR_ERR_NOT_CONVERGED = -5), so statuses compare directly.
OK, BREAKDOWN, NOT_CONVERGED = 0, -4, -5


def pcg(op, b, precond=None, tol=1e-6, maxit=None):
    n = b.shape[0]
    maxit = n if maxit is None else maxit
    P = (lambda r: r) if precond is None else precond
    x = np.zeros_like(b)
    bnorm = float(np.linalg.norm(b))
    if bnorm == 0.0:
        return x, 0, 0.0, OK
    r = b.copy()
    z = P(r)
    p = z.copy()
    rz = float(r @ z)
    relres = 1.0
    for it in range(1, maxit + 1):
        q = op(p)
        pq = float(p @ q)
        if not pq > 0.0:
            return x, it, relres, BREAKDOWN
        alpha = rz / pq
        x = x + alpha * p
        r = r - alpha * q
        relres = float(np.linalg.norm(r)) / bnorm
        if relres <= tol:
            return x, it, relres, OK
        z = P(r)
        rz_new = float(r @ z)
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, maxit, relres, NOT_CONVERGED


def sketchsolv_step(lr, g):
    """Eq. dxsol in the control variable: dv = -(I + H_hat)^{-1} g_v."""
    return -sketch.woodbury_apply(lr, g)


@dataclasses.dataclass
class GNOptions:
    iters: int = 3
    gtol: float = 0.0
    method: str = "none"          # none | randsvd | nystrom | singleview
    adaptive: bool = False        # SketchPrecA (adaptive size + reuse)
    solve: str = "pcg"            # pcg (SketchPrec) | sketchsolv
    l: int = 20                   # l, l_1 (initial size when adaptive)
    l2: int | None = None         # SingleView l_2 (default 2 l_1 + 1)
    l_hat: int | None = None      # adaptive increment (default l / 2)
    eps_sk: float = 1.01
    eps_re: float = 10.0
    l_max: int | None = None      # default min(8 l, n)
    pcg_tol: float = 1e-6
    pcg_maxit: int | None = None
    seed: int = 20240128
    line_search: bool = False     # strong-Wolfe step length instead of alpha = 1
    ls_c1: float = 1e-4
    ls_c2: float = 0.9
    ls_alpha1: float = 1.0        # first trial step


def build_sketch(prob, o: GNOptions, k: int):
    n, m = prob.n, prob.m
    s_om = STREAM_SKETCH + k
    s_ps = STREAM_SKETCH + k + STREAM_PSI
    s_ka = STREAM_KAPPA + k
    draw_omega = lambda c0, c: philox.gaussian(o.seed, s_om, n, c, col0=c0)
    draw_psi = lambda c0, c: philox.gaussian(o.seed, s_ps, m, c, col0=c0)
    draw_v = lambda t: sketch.unit_test_vector(o.seed, s_ka, n, index=1 + t)
    l = o.l
    l2 = 2 * l + 1 if o.l2 is None else o.l2
    if not o.adaptive:
        if o.method == "randsvd":
            return sketch.randsvd(prob.A, prob.At, draw_omega(0, l))
        if o.method == "nystrom":
            return sketch.nystrom(prob.misfit_hvp, draw_omega(0, l))
        if o.method == "singleview":
            return sketch.singleview(prob.A, prob.At, draw_omega(0, l), draw_psi(0, l2))
        raise ValueError(o.method)
    l_hat = max(1, l // 2) if o.l_hat is None else o.l_hat
    l_max = min(8 * l, n) if o.l_max is None else o.l_max
    if o.method == "randsvd":
        return sketch.adaptive_randsvd(prob.A, prob.At, prob.hvp, draw_omega, l, l_hat,
                                       o.eps_sk, l_max, draw_v)
    if o.method == "nystrom":
        return sketch.adaptive_nystrom(prob.misfit_hvp, prob.hvp, draw_omega, l, l_hat,
                                       o.eps_sk, l_max, draw_v)
    if o.method == "singleview":
        return sketch.adaptive_singleview(prob.A, prob.At, prob.hvp, draw_omega, draw_psi,
                                          l, l2, l_hat, 2 * l_hat, o.eps_sk, l_max, draw_v)
    raise ValueError(o.method)


def gauss_newton(prob, v0, o: GNOptions):
    """Returns (v, info): info is a list of per-iteration dicts."""
    v = np.array(v0, dtype=np.float64)
    info = []
    lr = None
    g0 = None
    carry = None   # (J, g) at v from the last line-search evaluation
    for k in range(o.iters):
        if carry is None:
            J = prob.set_iterate(v)
            g = prob.gradient()
        else:
            J, g = carry
            carry = None
        gn = float(np.max(np.abs(g)))
        g0 = gn if g0 is None else g0
        rec = {"k": k, "J": J, "g_inf": gn, "sketched": False, "l": 0,
               "kappa_re": None, "pcg_its": 0, "relres": 0.0, "status": OK,
               "tlm_off": 0, "adj_off": 0}
        if k > 0 and o.gtol > 0 and gn / g0 < o.gtol:
            info.append(rec)
            break
        if o.method != "none":
            need = lr is None or not o.adaptive
            if not need:
                vt = sketch.unit_test_vector(o.seed, STREAM_KAPPA + k, prob.n, index=0)
                kre = sketch.kappa_estimate(prob.hvp, lambda r: sketch.woodbury_apply(lr, r), vt)
                rec["kappa_re"] = kre
                need = not (kre < o.eps_re)
            if need:
                lr = build_sketch(prob, o, k)
                rec["sketched"] = True
                rec["tlm_off"], rec["adj_off"] = lr.tlm, lr.adj
            rec["l"] = lr.rank
        P = None if lr is None else (lambda r, lr=lr: sketch.woodbury_apply(lr, r))
        if o.solve == "sketchsolv":
            dv = sketchsolv_step(lr, g)
        else:
            dv, its, relres, st = pcg(prob.hvp, -g, P, o.pcg_tol, o.pcg_maxit)
            rec.update(pcg_its=its, relres=relres, status=st)
        alpha = 1.0
        if o.line_search:
            last = {}

            def phi(a, v=v, dv=dv):
                Ja = prob.set_iterate(v + a * dv)
                ga = prob.gradient()
                last["v"] = (a, Ja, ga)
                return Ja, float(ga @ dv)

            res = linesearch.strong_wolfe(phi, J, float(g @ dv), o.ls_alpha1, o.ls_c1, o.ls_c2)
            if res.status != linesearch.NOT_DESCENT:
                alpha = res.alpha
            rec.update(alpha=alpha, ls_evals=res.evals, ls_status=res.status)
            if res.last and "v" in last and last["v"][0] == alpha:
                carry = (last["v"][1], last["v"][2])
        v = v + alpha * dv
        info.append(rec)
    return v, info
