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
    assert rel(hhat_action(V, lam, X), ref_act) <= 1e-12
    # eigenvalues: CholeskyQR2 + a Jacobi eigen-solve of the Gram matrix against
    # Householder QR + SVD; both carry an absolute error of order u lambda_1 in
    # every eigenvalue, so they are compared on the scale of lambda_1
    lam_ref = np.sort(lr.lam)[::-1]
    big = lam_ref > 1e-6 * lam_ref[0]
    assert np.max(np.abs(lam[:big.sum()] - lam_ref[big])) <= 1e-10 * lam_ref[0]
    # V orthonormal
    assert np.max(np.abs(V.T @ V - np.eye(V.shape[1]))) <= 1e-12
    # the Woodbury apply inverts I + H_hat
    R = np.random.default_rng(2).standard_normal((3, wl.n))
    Z = pc.apply(torch.tensor(R, device="cuda")).cpu().numpy()
    back = Z.T + hhat_action(V, lam, Z.T)
    assert rel(back, R.T) <= 1e-12


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
    assert rel(hhat_action(V, lam, X), hhat_action(lr.V, lr.lam, X)) <= 1e-5
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


def _reuse_pair(wl, eps_re):
    from oracle import solvers
    prob, ref = make_pair(wl)
    v = torch.zeros(wl.n, dtype=torch.float64, device="cuda")
    rec = prob.gauss_newton(v, iters=3, method="randsvd", l=8, adaptive=True, eps_re=eps_re,
                            tol=1e-6)
    vr, info = solvers.gauss_newton(ref, np.zeros(wl.n),
                                    solvers.GNOptions(iters=3, method="randsvd", l=8, adaptive=True,
                                                      eps_re=eps_re, pcg_tol=1e-6))
    for a, b in zip(rec, info):
        assert a["sketched"] == b["sketched"]
        assert a["rank"] == b["l"]
        assert abs(a["J"] - b["J"]) <= 1e-9 * abs(b["J"])
        if b["kappa_re"] is not None:
            assert abs(a["kappa_re"] - b["kappa_re"]) <= 1e-8 * b["kappa_re"]
    return rec, info


def test_adaptive_reuse_gauss_newton_matches_oracle():
    """The reuse rule of Sec. 3.2 (Eq. condtext2) on both sides: with the
    paper's eps_re = 10 the later GN iterations keep the first sketch; with
    eps_re just below the kappa_re of iteration 1 that iteration re-sketches."""
    wl = si.burgers_workload("burgers_n128")
    rec, info = _reuse_pair(wl, 10.0)
    assert rec[0]["sketched"] and any(not r["sketched"] for r in rec[1:])
    k1 = info[1]["kappa_re"]
    assert k1 is not None and k1 < 10.0
    rec2, info2 = _reuse_pair(wl, k1 * (1 - 1e-4))
    assert rec2[1]["sketched"] and info2[1]["sketched"]


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


@pytest.mark.parametrize("m,r1,r2,k1,k2", [
    (300, 41, 20, 20, 10),    # A2 B1 wide (r2 < k1 + ...), the usual growth round
    (257, 17, 16, 8, 8),      # r2 = 2 k2 as in Alg. 5 with l2 = 2 l1 + 1
    (500, 33, 40, 16, 20),    # A2 B1 tall (r2 > k1)
    (128, 25, 0, 12, 6),      # no new rows: only steps 4-7
    (128, 25, 10, 12, 0),     # no new columns: only steps 1-3
])
def test_qr_update_matches_oracle(m, r1, r2, k1, k2):
    """Alg. 6 through the C ABI against the oracle's restatement: R up to the
    signs of its rows (Q up to the same column signs), Q R = [A1; A2][B1 B2]
    and Q orthonormal."""
    import paper_2401_15758_gb300 as g
    from oracle import sketch
    rng = np.random.default_rng(m + r1 + r2 + k1 + k2)
    P = rng.standard_normal((m, r1 + r2))
    B, _ = np.linalg.qr(rng.standard_normal((m, k1 + k2)))
    A1, A2, B1, B2 = P[:, :r1].T, P[:, r1:].T, B[:, :k1], B[:, k1:]
    Q1, R1 = np.linalg.qr(A1 @ B1)
    dev = lambda a: torch.tensor(np.ascontiguousarray(a), device="cuda")
    Q, R = g.qr_update(dev(P), dev(B), dev(Q1), dev(R1), r1, k1)
    Q, R = Q.cpu().numpy(), R.cpu().numpy()
    Qo, Ro = sketch.qr_update(A1, A2, B1, B2, Q1, R1)
    assert np.all(np.tril(R, -1) == 0.0)
    D = np.sign(np.diag(R)) * np.sign(np.diag(Ro))
    scale = np.abs(Ro).max()
    assert np.abs(D[:, None] * R - Ro).max() <= 1e-12 * scale
    assert np.abs(Q * D - Qo).max() <= 1e-12 * max(1.0, scale / np.abs(np.diag(Ro)).min())
    assert np.abs(Q @ R - P.T @ B).max() <= 1e-12 * scale
    assert np.abs(Q.T @ Q - np.eye(k1 + k2)).max() <= 1e-13


def test_qr_update_rejects_bad_sizes():
    import paper_2401_15758_gb300 as g
    z = torch.zeros((8, 8), dtype=torch.float64, device="cuda")
    with pytest.raises(g.Sc4dvarError) as e:     # r1 < k1: no thin QR of A1 B1
        g.check(g.lib.sc4dvar_qr_update(8, 2, 2, 3, 1, g._ptr(z), 8, g._ptr(z), 8, g._ptr(z), 8,
                                        g._ptr(z), 8, None))
    assert e.value.code == g._abi.ERR_INVALID_ARG


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_adaptive_singleview_matches_oracle(small, prec):
    """Alg. 5 with the Alg. 6 QR update on the GPU against the oracle's Alg. 5
    (direct QR of each grown M), growing 8 -> 24 columns (l_hat = 4, l2 = 2 l + 1
    growing by 2 l_hat): the action of H_hat, the rank and the PDE-solve counts."""
    import paper_2401_15758_gb300 as g
    from oracle import solvers
    wl, prob, ref = small
    o = solvers.GNOptions(method="singleview", adaptive=True, l=8, l_hat=4, eps_sk=0.5, l_max=24,
                          seed=wl.seed)
    lr = solvers.build_sketch(ref, o, 0)
    prob.counters_reset()
    pc = prob.build_precond("singleview", l=8, adaptive=True, l_hat=4, eps_sk=0.5, l_max=24,
                            seed=wl.seed, prec=g.FP64 if prec == "fp64" else g.FP32)
    c = prob.counters()
    V, lam = pc.arrays()
    X = np.random.default_rng(11).standard_normal((wl.n, 4))
    tol = 1e-10 if prec == "fp64" else 1e-5
    assert rel(hhat_action(V, lam, X), hhat_action(lr.V, lr.lam, X)) <= tol
    assert (c["tlm_offline"], c["adj_offline"]) == (lr.tlm, lr.adj) == (24, 49)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_adaptive_nystrom_matches_oracle(small, prec):
    """Adaptive Nystrom (Alg. 2 steps 3-7 redone on the grown sketch; the paper
    defers this variant to Frangella et al., Sec. 3.1.2) against the oracle,
    growing 8 -> 24 columns (l_hat = 4): the action of H_hat, the kappa_sk
    history's final size and the PDE-solve counts. The FP32 sketch shifts with
    u = 2^-24 and is compared with the oracle run at that u."""
    import paper_2401_15758_gb300 as g
    from oracle import philox, sketch, solvers
    wl, prob, ref = small
    eps = 2.0 ** -53 if prec == "fp64" else 2.0 ** -24
    n = wl.n
    draw_omega = lambda c0, c: philox.gaussian(wl.seed, solvers.STREAM_SKETCH, n, c, col0=c0)
    draw_v = lambda t: sketch.unit_test_vector(wl.seed, solvers.STREAM_KAPPA, n, index=1 + t)
    lr = sketch.adaptive_nystrom(ref.misfit_hvp, ref.hvp, draw_omega, 8, 4, 0.5, 24, draw_v, eps=eps)
    prob.counters_reset()
    pc = prob.build_precond("nystrom", l=8, adaptive=True, l_hat=4, eps_sk=0.5, l_max=24,
                            seed=wl.seed, prec=g.FP64 if prec == "fp64" else g.FP32)
    c = prob.counters()
    V, lam = pc.arrays()
    X = np.random.default_rng(12).standard_normal((n, 4))
    tol = 1e-10 if prec == "fp64" else 1e-5
    assert rel(hhat_action(V, lam, X), hhat_action(lr.V, lr.lam, X)) <= tol
    assert lr.kappa_hist[-1][0] == 24
    assert (c["tlm_offline"], c["adj_offline"]) == (lr.tlm, lr.adj) == (24, 24)


def test_shifted_cholqr_retry_on_a_rank_deficient_sketch(small):
    """A RandSVD sketch of l = 64 columns of an operator of numerical rank 43
    (the prior's square root keeps 43 modes): the Gram matrix Y^T Y of the
    CholeskyQR2 is singular, its Cholesky factorization fails and is redone
    with a diagonal shift (shifted CholeskyQR3). The result still matches the
    oracle's Householder-QR RandSVD on the action of H_hat and on the leading
    eigenvalues, and keeps at most 43 of them."""
    from oracle import philox, sketch
    wl, prob, ref = small
    l = 64
    Om = philox.gaussian(wl.seed, 100, wl.n, l)
    prob.counters_reset()
    pc = prob.build_precond("randsvd", l=l, Omega=torch.tensor(Om.T.copy(), device="cuda"))
    assert prob.counters()["qr_shifted"] >= 1
    V, lam = pc.arrays()
    lr = sketch.randsvd(ref.A, ref.At, Om)
    X = np.random.default_rng(13).standard_normal((wl.n, 4))
    assert rel(hhat_action(V, lam, X), hhat_action(lr.V, lr.lam, X)) <= 1e-10
    lam_ref = np.sort(lr.lam)[::-1]
    big = lam_ref > 1e-6 * lam_ref[0]
    assert len(lam) <= 43
    assert np.max(np.abs(lam[:big.sum()] - lam_ref[big])) <= 1e-10 * lam_ref[0]


@pytest.mark.parametrize("gemm,tol", [(2, 5e-3), (3, 5e-2), (1, 1e-5)])
def test_fp32_sketch_with_other_tall_product_arithmetic(small, gemm, tol):
    """FP32 RandSVD with the tall products in TF32 (gemm = 2) or BF16 (3) on the
    tensor cores, or on the CUDA cores (1): the action of H_hat against the FP64
    oracle within the accuracy of that arithmetic, and PCG preconditioned by it
    still converges in a handful of iterations."""
    import paper_2401_15758_gb300 as g
    from oracle import philox, sketch
    wl, prob, ref = small
    Om = philox.gaussian(wl.seed, 100, wl.n, 20)
    pc = prob.build_precond("randsvd", l=20, prec=g.FP32, gemm=gemm,
                            Omega=torch.tensor(Om.T.copy(), device="cuda"))
    V, lam = pc.arrays()
    lr = sketch.randsvd(ref.A, ref.At, Om)
    X = np.random.default_rng(1).standard_normal((wl.n, 4))
    assert rel(hhat_action(V, lam, X), hhat_action(lr.V, lr.lam, X)) <= tol
    b = torch.tensor(np.random.default_rng(2).standard_normal(wl.n), device="cuda")
    x, info = prob.pcg(b, pc, tol=1e-8)
    assert info["status"] == 0 and info["iterations"] <= 12


@pytest.mark.parametrize("method", ["randsvd", "nystrom", "singleview"])
def test_sketchsolv_step_within_the_thm4_bound(small, method):
    """Thm. 4 on the GPU's SketchSolv step: |dv - dv_hat| / |dv| <= |H - H_hat|_2
    (the Gamma^{-1} norm of the paper is the 2-norm in v). H is the dense misfit
    Hessian from the FP64 block product of the identity, dv the dense solve of
    (I + H) dv = -g, H_hat = V diag(lam) V^T from the GPU sketch."""
    wl, prob, _ = small
    n = wl.n
    H = prob.gn_hessian_apply_block(torch.eye(n, dtype=torch.float64, device="cuda"),
                                    misfit_only=True).cpu().numpy()
    H = 0.5 * (H + H.T)
    P = prob.build_precond(method, l=12, l2=25)
    V, lam = P.arrays()
    normE = np.linalg.norm(H - (V * lam) @ V.T, 2)
    g = np.random.default_rng(11).standard_normal(n)
    dvh = P.sketchsolv(torch.tensor(g, device="cuda")).cpu().numpy()
    dv = -np.linalg.solve(np.eye(n) + H, g)
    err = np.linalg.norm(dv - dvh) / np.linalg.norm(dv)
    assert 0.0 < normE
    assert err <= normE * (1 + 1e-9) + 1e-12
