"""Parity of the CUDA sketches, PCG and Gauss-Newton with the FP64 oracle."""
import numpy as np
import pytest

import sc4dvar_inputs as si

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from test_gpu_burgers import make_pair, rel  # noqa: E402


@pytest.fixture(scope="module")
def small():
    wl = si.burgers_workload("burgers_n128")
    prob, ref = make_pair(wl)
    ref.set_iterate(np.zeros(wl.n))
    prob.fwd(torch.zeros(wl.n, dtype=torch.float64, device="cuda"))
    return wl, prob, ref


def hhat_action(V, lam, X):
    return V @ (lam[:, None] * (V.T @ X))


@pytest.mark.parametrize("method,l", [("randsvd", 20), ("nystrom", 20), ("singleview", 20),
                                      ("randsvd", 21), ("nystrom", 33)])
def test_sketch_matches_oracle_given_omega(small, method, l):
    """l = 20 is the workload's size; odd l exercises the padding pair of the
    parallel-order Jacobi eigen-solver of the thin SVD."""
    from oracle import philox, sketch
    wl, prob, ref = small
    Om = philox.gaussian(wl.seed, 100, wl.n, l)
    Ps = philox.gaussian(wl.seed, 1100, wl.m, 2 * l + 1)
    pc = prob.build_precond(method, l=l, Omega=torch.tensor(Om.T.copy(), device="cuda"),
                            Psi=torch.tensor(Ps.T.copy(), device="cuda"))
    V, lam = pc.arrays()
    if method == "randsvd":
        lr = sketch.randsvd(ref.A, ref.At, Om)
    elif method == "nystrom":
        lr = sketch.nystrom(ref.misfit_hvp, Om)
    else:
        lr = sketch.singleview(ref.A, ref.At, Om, Ps)
    X = np.random.default_rng(1).standard_normal((wl.n, 4))
    ref_act = hhat_action(lr.V, lr.lam, X)
    assert rel(hhat_action(V, lam, X), ref_act) <= 1e-8
    lam_ref = np.sort(lr.lam)[::-1]
    big = lam_ref > 1e-6 * lam_ref[0]
    assert np.allclose(lam[:big.sum()], lam_ref[big], rtol=1e-8)
    # V orthonormal
    assert np.max(np.abs(V.T @ V - np.eye(V.shape[1]))) <= 1e-8
    # the Woodbury apply inverts I + H_hat
    R = np.random.default_rng(2).standard_normal((3, wl.n))
    Z = pc.apply(torch.tensor(R, device="cuda")).cpu().numpy()
    back = Z.T + hhat_action(V, lam, Z.T)
    assert rel(back, R.T) <= 1e-10


@pytest.mark.parametrize("method,l", [("randsvd", 20), ("nystrom", 20), ("singleview", 20),
                                      ("randsvd", 21)])
def test_fp32_sketch_close_to_oracle(small, method, l):
    """FP32 sketches (FP32 sweeps, double-float Gram products, FP32 tall
    products) against the FP64 oracle given the same Omega / Psi: the action of
    H_hat to FP32 accuracy, V orthonormal to FP32 accuracy. The Nystrom shift
    uses the unit roundoff of the precision that forms Y (2^-24 here) on both
    sides."""
    import paper_2401_15758_gb300 as g
    from oracle import philox, sketch
    wl, prob, ref = small
    Om = philox.gaussian(wl.seed, 100, wl.n, l)
    Ps = philox.gaussian(wl.seed, 1100, wl.m, 2 * l + 1)
    pc = prob.build_precond(method, l=l, prec=g.FP32, Omega=torch.tensor(Om.T.copy(), device="cuda"),
                            Psi=torch.tensor(Ps.T.copy(), device="cuda"))
    V, lam = pc.arrays()
    if method == "randsvd":
        lr = sketch.randsvd(ref.A, ref.At, Om)
    elif method == "nystrom":
        lr = sketch.nystrom(ref.misfit_hvp, Om, eps=2.0 ** -24)
    else:
        lr = sketch.singleview(ref.A, ref.At, Om, Ps)
    X = np.random.default_rng(1).standard_normal((wl.n, 4))
    assert rel(hhat_action(V, lam, X), hhat_action(lr.V, lr.lam, X)) <= 1e-4
    assert np.max(np.abs(V.T @ V - np.eye(V.shape[1]))) <= 1e-5


def test_philox_drawn_sketch_equals_given_omega(small):
    from oracle import philox
    wl, prob, ref = small
    Om = philox.gaussian(wl.seed, 100 + 2, wl.n, 10)
    a = prob.build_precond("randsvd", l=10, gn_iter=2, seed=wl.seed)
    b = prob.build_precond("randsvd", l=10, Omega=torch.tensor(Om.T.copy(), device="cuda"))
    Va, la = a.arrays()
    Vb, lb = b.arrays()
    X = np.random.default_rng(4).standard_normal((wl.n, 2))
    assert rel(hhat_action(Va, la, X), hhat_action(Vb, lb, X)) <= 1e-12


@pytest.mark.parametrize("method", ["none", "randsvd"])
def test_pcg_matches_oracle(small, method):
    from oracle import philox, sketch, solvers
    wl, prob, ref = small
    b = np.random.default_rng(9).standard_normal(wl.n)
    pc = None
    P = None
    if method != "none":
        Om = philox.gaussian(wl.seed, 100, wl.n, wl.k)
        pc = prob.build_precond(method, l=wl.k, Omega=torch.tensor(Om.T.copy(), device="cuda"))
        lr = sketch.randsvd(ref.A, ref.At, Om)
        P = lambda r: sketch.woodbury_apply(lr, r)
    x, info = prob.pcg(torch.tensor(b, device="cuda"), pc, tol=1e-10)
    xr, its, relres, st = solvers.pcg(ref.hvp, b, P, tol=1e-10)
    assert info["status"] == 0 and st == 0
    # unpreconditioned CG on a rank-deficient I + H: the round-off of the Krylov
    # tail decides the last few iterations; a good preconditioner leaves none
    assert abs(info["iterations"] - its) <= (4 if method == "none" else 1)
    assert rel(x.cpu().numpy(), xr) <= 1e-9


@pytest.mark.parametrize("method", ["none", "randsvd", "nystrom", "singleview"])
def test_gauss_newton_matches_oracle(method):
    from oracle import solvers
    wl = si.burgers_workload("burgers_n128")
    prob, ref = make_pair(wl)
    v = torch.zeros(wl.n, dtype=torch.float64, device="cuda")
    rec = prob.gauss_newton(v, iters=3, method=method, l=wl.k, tol=1e-6)
    vr, info = solvers.gauss_newton(ref, np.zeros(wl.n),
                                    solvers.GNOptions(iters=3, method=method, l=wl.k, pcg_tol=1e-6))
    # iteration 0 is the same iterate: J to round-off. Later iterates differ by the
    # PCG stopping point (relative residual 1e-6): J to 1e-7, the iterate to 1e-5.
    assert abs(rec[0]["J"] - info[0]["J"]) <= 1e-11 * abs(info[0]["J"])
    for a, b in zip(rec, info):
        assert abs(a["J"] - b["J"]) <= 1e-7 * abs(b["J"])
        assert abs(a["pcg_its"] - b["pcg_its"]) <= (4 if method == "none" else 1)
    assert rel(v.cpu().numpy(), vr) <= 1e-5


def test_adaptive_reuse_gauss_newton_matches_oracle():
    from oracle import solvers
    wl = si.burgers_workload("burgers_n128")
    prob, ref = make_pair(wl)
    v = torch.zeros(wl.n, dtype=torch.float64, device="cuda")
    rec = prob.gauss_newton(v, iters=3, method="randsvd", l=8, adaptive=True, tol=1e-6)
    vr, info = solvers.gauss_newton(ref, np.zeros(wl.n),
                                    solvers.GNOptions(iters=3, method="randsvd", l=8, adaptive=True,
                                                      pcg_tol=1e-6))
    for a, b in zip(rec, info):
        assert a["sketched"] == b["sketched"]
        assert a["rank"] == b["l"]
        assert abs(a["J"] - b["J"]) <= 1e-9 * abs(b["J"])
        if b["kappa_re"] is not None:
            assert abs(a["kappa_re"] - b["kappa_re"]) <= 1e-8 * b["kappa_re"]


@pytest.mark.parametrize("alpha1", [1.0, 3.0])
def test_gauss_newton_line_search_matches_oracle(alpha1):
    """Strong-Wolfe GN steps (alpha1 = 3 overshoots, so the bracketing and
    zoom phases run): cost, step length and trial count per iteration and the
    final iterate against the oracle's line search."""
    from oracle import solvers
    wl = si.burgers_workload("burgers_n128")
    prob, ref = make_pair(wl)
    v = torch.zeros(wl.n, dtype=torch.float64, device="cuda")
    rec = prob.gauss_newton(v, iters=3, method="randsvd", l=20, tol=1e-10, line_search=True,
                            ls_alpha1=alpha1)
    vr, info = solvers.gauss_newton(ref, np.zeros(wl.n),
                                    solvers.GNOptions(iters=3, method="randsvd", l=20, pcg_tol=1e-10,
                                                      line_search=True, ls_alpha1=alpha1))
    for a, b in zip(rec, info):
        assert abs(a["J"] - b["J"]) <= 1e-9 * abs(b["J"])
        assert a["ls_evals"] == b["ls_evals"] and a["ls_status"] == b["ls_status"]
        assert abs(a["alpha"] - b["alpha"]) <= 1e-8 * abs(b["alpha"])
    if alpha1 != 1.0:
        assert rec[0]["ls_evals"] > 1
    assert rel(v.cpu().numpy(), vr) <= 1e-7


@pytest.mark.parametrize("method", ["randsvd", "nystrom", "singleview"])
def test_gauss_newton_sketchsolv_matches_oracle(method):
    """SketchSolv GN steps (Eq. dxsol): no PCG, the sketch's Woodbury inverse
    applied to the gradient; costs and the final iterate against the oracle,
    and the online counts (no TLM, one ADJ per gradient)."""
    from oracle import solvers
    wl = si.burgers_workload("burgers_n128")
    prob, ref = make_pair(wl)
    prob.counters_reset()
    v = torch.zeros(wl.n, dtype=torch.float64, device="cuda")
    rec = prob.gauss_newton(v, iters=3, method=method, l=20, solve="sketchsolv")
    vr, info = solvers.gauss_newton(ref, np.zeros(wl.n),
                                    solvers.GNOptions(iters=3, method=method, l=20, solve="sketchsolv"))
    for a, b in zip(rec, info):
        assert abs(a["J"] - b["J"]) <= 1e-9 * abs(b["J"]) and a["pcg_its"] == 0
    assert rel(v.cpu().numpy(), vr) <= 1e-8
    c = prob.counters()
    assert c["tlm_online"] == 0 and c["adj_online"] == 3
