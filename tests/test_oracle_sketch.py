"""Pins of the oracle's sketching and solver layer.

Checks exact identities (Woodbury, Remark 1, Alg. 6), exactness when the sketch
size reaches the rank, the structural bounds of Thms. 4 and 5 (which must hold on
every instance), E = H - H_hat >= 0 for RandSVD and Nystrom (Sec. 4.3 proofs), the
expectation bounds of Thms. 1-3 by Monte Carlo, PCG against a dense solve and the
paper's cost accounting (Tables 3 and 4).
"""
import os

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import philox, sketch, solvers

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def synthetic_operator(n, m, lam, seed):
    """A = U diag(sqrt(lam)) V^T with random orthonormal U (m x r), V (n x r)."""
    rng = np.random.default_rng(seed)
    r = len(lam)
    U, _ = np.linalg.qr(rng.standard_normal((m, r)))
    V, _ = np.linalg.qr(rng.standard_normal((n, r)))
    return (U * np.sqrt(lam)) @ V.T


def ops(A):
    n = A.shape[1]
    return (lambda X: A @ X, lambda W: A.T @ W, lambda X: A.T @ (A @ X),
            lambda x: x + A.T @ (A @ x), np.eye(n) + A.T @ A)


def precond_kappa(Hfull, Hhat):
    w = sla.eigh(Hfull, np.eye(Hfull.shape[0]) + Hhat, eigvals_only=True)
    return w.max() / w.min()


def test_woodbury_and_remark1_identities():
    rng = np.random.default_rng(0)
    n, l = 30, 7
    V, _ = np.linalg.qr(rng.standard_normal((n, l)))
    lam = rng.uniform(0, 50, l)
    lr = sketch.LowRank(V=V, lam=lam)
    x = rng.standard_normal((n, 3))
    assert np.allclose((np.eye(n) + lr.H_hat()) @ sketch.woodbury_apply(lr, x), x, atol=1e-13)
    W = rng.standard_normal((l, n))
    assert np.allclose((np.eye(n) + W.T @ W) @ sketch.woodbury_apply_W(W, x), x, atol=1e-12)


@pytest.mark.parametrize("method", ["randsvd", "nystrom", "singleview"])
def test_sketch_exact_when_l_reaches_rank(method):
    n, m, r = 40, 30, 6
    A = synthetic_operator(n, m, np.geomspace(100, 0.1, r), 1)
    Aop, Atop, Hop, _, Hf = ops(A)
    H = A.T @ A
    Om = philox.gaussian(3, 100, n, 9)
    if method == "randsvd":
        lr = sketch.randsvd(Aop, Atop, Om)
    elif method == "nystrom":
        lr = sketch.nystrom(Hop, Om)
    else:
        lr = sketch.singleview(Aop, Atop, Om, philox.gaussian(3, 1100, m, 19))
    assert np.max(np.abs(lr.H_hat() - H)) < 1e-10 * np.abs(H).max()
    assert precond_kappa(Hf, lr.H_hat()) < 1 + 1e-9
    x, its, rel, st = solvers.pcg(lambda v: Hf @ v, np.ones(n),
                                  lambda r_: sketch.woodbury_apply(lr, r_), tol=1e-10)
    assert st == solvers.OK and its == 1


@pytest.mark.parametrize("method", ["randsvd", "nystrom", "singleview"])
@pytest.mark.parametrize("decay", ["poly", "exp"])
def test_structural_bounds_thm4_thm5(method, decay):
    n, m = 60, 45
    j = np.arange(1, 41)
    lam = 200.0 * (j ** -2.0 if decay == "poly" else np.exp(-0.5 * j))
    A = synthetic_operator(n, m, lam, 2)
    Aop, Atop, Hop, _, Hf = ops(A)
    H = A.T @ A
    for seed in range(5):
        Om = philox.gaussian(seed, 100, n, 8)
        if method == "randsvd":
            lr = sketch.randsvd(Aop, Atop, Om)
        elif method == "nystrom":
            lr = sketch.nystrom(Hop, Om)
        else:
            lr = sketch.singleview(Aop, Atop, Om, philox.gaussian(seed, 1100, m, 17))
        E = H - lr.H_hat()
        normE = np.linalg.norm(E, 2)
        kap = precond_kappa(Hf, lr.H_hat())
        if method in ("randsvd", "nystrom"):
            # E >= 0 (proofs of Thms. 1, 2) and the tighter Thm. 5 bound
            assert np.linalg.eigvalsh(0.5 * (E + E.T)).min() >= -1e-10 * np.abs(H).max()
            assert kap <= 1 + normE + 1e-9
        assert kap <= (1 + normE) ** 2 + 1e-9
        # Thm. 4: SketchSolv step error in the Gamma^{-1} norm (= 2-norm in v)
        g = np.random.default_rng(seed).standard_normal(n)
        dv = -np.linalg.solve(Hf, g)
        dvh = solvers.sketchsolv_step(lr, g)
        assert np.linalg.norm(dv - dvh) / np.linalg.norm(dv) <= normE + 1e-12


def _psi_bound(lam, r, p):
    tail = lam[r:].sum()
    return lam[r] + r / (p - 1) * tail


@pytest.mark.parametrize("decay", ["poly", "exp"])
def test_expectation_bounds_thm1_thm2_thm3(decay):
    """Monte-Carlo means over 200 seeds stay below the Thm. 1 / Thm. 2 bound
    1 + Psi_H(r, p) and the Thm. 3 bound on E[sqrt(kappa)]."""
    n, m = 50, 40
    j = np.arange(1, 41)
    lam = 30.0 * (j ** -2.0 if decay == "poly" else np.exp(-0.5 * j))
    A = synthetic_operator(n, m, lam, 5)
    Aop, Atop, Hop, _, Hf = ops(A)
    r, p = 4, 4
    l = r + p
    ks = {"randsvd": [], "nystrom": [], "singleview": []}
    for s in range(200):
        Om = philox.gaussian(s, 100, n, l)
        ks["randsvd"].append(precond_kappa(Hf, sketch.randsvd(Aop, Atop, Om).H_hat()))
        ks["nystrom"].append(precond_kappa(Hf, sketch.nystrom(Hop, Om).H_hat()))
        l1, l2 = 2 * r + 1, 4 * r + 3
        sv = sketch.singleview(Aop, Atop, philox.gaussian(s, 100, n, l1),
                               philox.gaussian(s, 1100, m, l2))
        ks["singleview"].append(np.sqrt(precond_kappa(Hf, sv.H_hat())))
    bound = 1 + _psi_bound(lam, r, p)
    assert np.mean(ks["randsvd"]) <= bound
    assert np.mean(ks["nystrom"]) <= bound
    theta = 4 * np.sqrt(lam[0] * lam[r:].sum()) + 4 * lam[r:].sum()
    assert np.mean(ks["singleview"]) <= 1 + theta


def test_intrinsic_dimension_closed_forms():
    """Sec. 4.2. Severely ill-posed (e^{-alpha j}): id_r = 1/(1 - e^{-alpha}) for every r.
    Moderately ill-posed (j^{-alpha}): id_r = (r+1)^alpha zeta(alpha, r+1) (Hurwitz
    zeta); the printed bound zeta(alpha) is attained at r = 0 and is exceeded for
    r >= 1 (a reading recorded with the design notes)."""
    from scipy.special import zeta
    j = np.arange(1, 200001, dtype=np.float64)
    for alpha in (1.5, 2.0, 3.0):
        lam = j ** -alpha
        for r in (0, 1, 5, 20):
            idr = lam[r:].sum() / lam[r]
            exact = (r + 1) ** alpha * zeta(alpha, r + 1)
            assert abs(idr - exact) <= 2e-2 * exact      # truncated tail of the sum
        assert abs(lam.sum() - zeta(alpha)) <= 1e-2
    for alpha in (0.2, 0.5, 1.0):
        lam = np.exp(-alpha * j[:2000])
        for r in (1, 5, 20):
            assert abs(lam[r:].sum() / lam[r] - 1 / (1 - np.exp(-alpha))) <= 1e-10


def test_qr_update_alg6_equals_direct_qr():
    rng = np.random.default_rng(7)
    A1, A2 = rng.standard_normal((13, 40)), rng.standard_normal((9, 40))
    B, _ = np.linalg.qr(rng.standard_normal((40, 10)))
    B1, B2 = B[:, :6], B[:, 6:]
    Q1, R1 = np.linalg.qr(A1 @ B1)
    Q5, R5 = sketch.qr_update(A1, A2, B1, B2, Q1, R1)
    M = np.vstack([A1, A2]) @ B
    assert np.allclose(Q5 @ R5, M, atol=1e-12)
    assert np.allclose(Q5.T @ Q5, np.eye(10), atol=1e-12)
    assert np.allclose(np.tril(R5, -1), 0, atol=1e-12)
    _, Rd = np.linalg.qr(M)
    assert np.allclose(np.abs(np.diag(R5)), np.abs(np.diag(Rd)), rtol=1e-10)


@pytest.mark.parametrize("method", ["randsvd", "nystrom", "singleview"])
def test_adaptive_sketch_meets_eps_sk(method):
    n, m = 80, 60
    j = np.arange(1, 61)
    A = synthetic_operator(n, m, 500.0 * np.exp(-0.3 * j), 9)
    Aop, Atop, Hop, Ipf, Hf = ops(A)
    draw_om = lambda c0, c: philox.gaussian(11, 100, n, c, col0=c0)
    draw_ps = lambda c0, c: philox.gaussian(11, 1100, m, c, col0=c0)
    draw_v = lambda t: sketch.unit_test_vector(11, 200, n, index=1 + t)
    if method == "randsvd":
        lr = sketch.adaptive_randsvd(Aop, Atop, Ipf, draw_om, 4, 4, 1.01, 60, draw_v)
    elif method == "nystrom":
        lr = sketch.adaptive_nystrom(Hop, Ipf, draw_om, 4, 4, 1.01, 60, draw_v)
    else:
        lr = sketch.adaptive_singleview(Aop, Atop, Ipf, draw_om, draw_ps, 4, 9, 4, 8, 1.01, 60, draw_v)
    hist = lr.kappa_hist
    assert hist[-1][1] <= 1.01 and all(k > 1.01 for _, k in hist[:-1])
    assert len(hist) > 1                      # it had to grow
    assert lr.tlm == hist[-1][0]
    if method == "singleview":
        assert lr.adj == 2 * lr.tlm + 1       # l2 = 2 l1 + 1 kept while growing
    # the estimate is a lower bound on the true preconditioned norm ratio
    P = np.eye(n) - (lr.V * (lr.lam / (1 + lr.lam))) @ lr.V.T
    assert hist[-1][1] <= np.linalg.norm(Hf @ P, 2) + 1e-12
    # Alg. 4's appended RandSVD basis gives the same H_hat as one batch of that size
    if method == "randsvd":
        one = sketch.randsvd(Aop, Atop, draw_om(0, lr.tlm))
        assert np.allclose(one.H_hat(), lr.H_hat(), atol=1e-8 * np.abs(lr.H_hat()).max())


def test_pcg_matches_dense_solve(tiny_prob, tiny_dense):
    p = tiny_prob
    Hf = np.eye(p.n) + tiny_dense["H"]
    rng = np.random.default_rng(8)
    b = rng.standard_normal(p.n)
    x, its, rel, st = solvers.pcg(p.hvp, b, tol=1e-13)
    xd = sla.cho_solve(sla.cho_factor(Hf), b)
    assert st == solvers.OK and its <= p.n
    assert np.linalg.norm(x - xd) <= 1e-10 * np.linalg.norm(xd)
    assert rel <= 1e-13
    # a breakdown is reported, not hidden
    x, its, rel, st = solvers.pcg(lambda v: -v, b, tol=1e-10)
    assert st == solvers.BREAKDOWN


def test_gn_step_equals_dense_normal_equations(tiny_wl, tiny_prob, tiny_dense):
    import sc4dvar_inputs as si
    from oracle import workload
    prob = workload.burgers_problem(tiny_wl, si.burgers_draws(tiny_wl))
    o = solvers.GNOptions(iters=1, method="randsvd", l=8, pcg_tol=1e-13)
    v1, info = solvers.gauss_newton(prob, np.zeros(tiny_wl.n), o)
    prob.set_iterate(np.zeros(tiny_wl.n))
    g = prob.gradient()
    dv = -np.linalg.solve(np.eye(tiny_wl.n) + tiny_dense["H"], g)
    assert np.linalg.norm(v1 - dv) <= 1e-10 * np.linalg.norm(dv)
    assert info[0]["sketched"] and info[0]["tlm_off"] == 8 and info[0]["adj_off"] == 8


def _paper_rows():
    rows = []
    with open(os.path.join(GOLDEN, "paper_counts.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                t, meth, *vals = line.split()
                rows.append((t, meth, [None if v == "-" else int(v) for v in vals]))
    return rows


def test_paper_count_identities():
    """The accounting the library's counters follow (Tables 3, 4): online ADJ =
    PCG iterations + one gradient per GN iteration; online TLM = PCG iterations;
    SingleView offline ADJ = sum over sketches of (2 l1 + 1)."""
    gn = {"T3": 3, "T4": 25}
    for t, meth, (pcg, tlm_off, adj_off, fwd, tlm_on, adj_on) in _paper_rows():
        if meth.startswith("SketchSolv"):
            assert tlm_on == 0 and adj_on == gn[t]
            continue
        if meth.endswith("Lanczos"):
            continue
        assert tlm_on == pcg
        extra = adj_on - pcg
        # the paper's SketchPrecA RandSVD row prints one more gradient than the rest
        assert extra == gn[t] or (t, meth) == ("T4", "SketchPrecA_RandSVD")
        if meth == "SketchPrec_SingleView":
            n_sk = gn[t]
            l1 = tlm_off // n_sk
            assert adj_off == n_sk * (2 * l1 + 1)
    sv = [r for r in _paper_rows() if r[1] == "SketchPrecA_SingleView"][0][2]
    # adaptive SingleView sketched 4 times with l1 in {1536, 1408, 1536, 1408} (Sec. 5.2)
    assert sv[1] == 1536 + 1408 + 1536 + 1408 and sv[2] == sv[1] * 2 + 4


def test_oracle_gn_counters_follow_paper_accounting(tiny_wl):
    import sc4dvar_inputs as si
    from oracle import workload
    prob = workload.burgers_problem(tiny_wl, si.burgers_draws(tiny_wl))
    o = solvers.GNOptions(iters=3, method="singleview", l=5, pcg_tol=1e-8)
    prob.counters = {"fwd": 0, "tlm": 0, "adj": 0}
    v, info = solvers.gauss_newton(prob, np.zeros(tiny_wl.n), o)
    pcg = sum(r["pcg_its"] for r in info)
    off_t = sum(r["tlm_off"] for r in info)
    off_a = sum(r["adj_off"] for r in info)
    assert off_t == 3 * 5 and off_a == 3 * 11
    assert prob.counters["tlm"] == pcg + off_t
    assert prob.counters["adj"] == pcg + 3 + off_a
    assert prob.counters["fwd"] == 3


# --------------------------------------------------------------------------- Alg. 2 shift
def test_nystrom_shift_closed_form_on_an_invariant_subspace():
    """Alg. 2 steps 3-7 with Omega spanning the leading eigenvectors of H:
    Y = H Omega = Q_l D_l, so |Y|_2 = d_1 and the shift is nu = sqrt(n) eps d_1
    (step 3); the Nystrom approximation of H + nu I on that subspace is exact,
    so sigma^2 = d_i + nu and Lam_hat = d_i, V_hat = Q_l up to signs. A dropped
    '- nu', a wrong norm or a wrong constant in nu breaks one of these."""
    n, l = 40, 6
    rng = np.random.default_rng(21)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    d = 50.0 * 0.3 ** np.arange(n)
    H = (Q * d) @ Q.T
    Om = Q[:, :l]
    eps = 1e-3                                 # large, so nu is visible (nu / d_l ~ 2.6)
    lr, nu = sketch.nystrom_core(Om, H @ Om, eps)
    assert nu == pytest.approx(np.sqrt(n) * eps * d[0], rel=1e-13)
    assert nu > d[l - 1]                       # the shift is not negligible here
    assert np.allclose(lr.lam, d[:l], rtol=1e-11, atol=0)
    assert np.allclose(np.abs(lr.V.T @ Q[:, :l]), np.eye(l), atol=1e-10)
    # the planted mistake (no '- nu' in Lam_hat) fails the same check
    assert not np.allclose(lr.lam + nu, d[:l], rtol=1e-6, atol=0)


def _nystrom_shifted_dense(H, Om, nu, l):
    """The stabilized Nystrom approximation from its definition: the Nystrom
    approximation of H + nu I, (H + nu I) Om (Om^T (H + nu I) Om)^+ ((H + nu I) Om)^T,
    eigen-decomposed, its l leading eigenvalues shifted back by nu and clamped at 0."""
    n = H.shape[0]
    Hn = H + nu * np.eye(n)
    Yn = Hn @ Om
    Hhat_nu = Yn @ np.linalg.pinv(Om.T @ Yn) @ Yn.T
    mu, U = np.linalg.eigh(0.5 * (Hhat_nu + Hhat_nu.T))
    mu, U = mu[::-1][:l], U[:, ::-1][:, :l]
    lam = np.maximum(0.0, mu - nu)
    return lam, (U * lam) @ U.T


@pytest.mark.parametrize("eps", [2.0 ** -24, 1e-4])
def test_nystrom_shift_matches_dense_definition_and_interlacing(eps):
    """Alg. 2 with a Gaussian Omega at a reduced-precision unit roundoff (and a
    larger one) against the definition evaluated densely; and, since the Nystrom
    approximation of the PSD matrix H + nu I is dominated by it, every Lam_hat_i
    is at most lambda_i(H)."""
    n, m = 60, 45
    j = np.arange(1, 41)
    A = synthetic_operator(n, m, 300.0 * np.exp(-0.7 * j), 4)
    H = A.T @ A
    Om = philox.gaussian(7, 100, n, 10)
    lr, nu = sketch.nystrom_core(Om, H @ Om, eps)
    lam_d, Hhat_d = _nystrom_shifted_dense(H, Om, nu, 10)
    scale = np.abs(H).max()
    assert np.allclose(lr.lam, lam_d, rtol=0, atol=1e-9 * scale)
    assert np.max(np.abs(lr.H_hat() - Hhat_d)) <= 1e-9 * scale
    lamH = np.sort(np.linalg.eigvalsh(H))[::-1][:10]
    assert np.all(lr.lam <= lamH + 1e-10 * scale)
    if eps == 1e-4:
        # nu is large enough here that the planted mistake (no '- nu') breaks
        # both the dense definition and the interlacing bound
        bad = lr.lam + nu
        assert not np.allclose(bad, lam_d, rtol=0, atol=1e-9 * scale)
        assert np.any(bad > lamH + 1e-10 * scale)


# ------------------------------------------------------------------ reuse rule (Sec. 3.2)
def _reuse_run(wl, eps_re, iters=3):
    import sc4dvar_inputs as si
    from oracle import workload
    prob = workload.burgers_problem(wl, si.burgers_draws(wl))
    o = solvers.GNOptions(iters=iters, method="randsvd", adaptive=True, l=4, eps_re=eps_re,
                          pcg_tol=1e-10)
    prob.counters = {"fwd": 0, "tlm": 0, "adj": 0}
    v, info = solvers.gauss_newton(prob, np.zeros(wl.n), o)
    return prob, o, v, info


def test_gn_reuse_rule_follows_kappa_re_in_both_directions(tiny_wl):
    """Eq. condtext2: at GN iteration k > 0 the last sketch is kept while
    kappa_re = |(I + H^(k)) (I + H_hat^(k-i))^{-1} v|_2 < eps_re and recomputed
    otherwise; iteration 0 always sketches. kappa_re is checked against a dense
    evaluation of that definition (assembled H at the new iterate, dense solve
    with the previous sketch), eps_re is then set just above and just below it,
    and the per-iteration flags and PDE-solve counters follow."""
    # eps_re huge: sketch once, then reuse
    prob, o, v, info = _reuse_run(tiny_wl, 1e30)
    assert info[0]["sketched"] and info[0]["kappa_re"] is None
    assert [r["sketched"] for r in info[1:]] == [False, False]
    for r in info[1:]:
        assert r["tlm_off"] == 0 and r["adj_off"] == 0 and r["l"] == info[0]["l"]
    # counters: one HVP per PCG iteration, per kappa_sk test of the adaptive
    # sketch and per kappa_re test, plus the sketch columns and one gradient per
    # GN iteration
    from oracle import workload
    import sc4dvar_inputs as si
    p0 = workload.burgers_problem(tiny_wl, si.burgers_draws(tiny_wl))
    p0.set_iterate(np.zeros(tiny_wl.n))
    lr0 = solvers.build_sketch(p0, o, 0)
    n_ksk = len(lr0.kappa_hist)
    pcg = sum(r["pcg_its"] for r in info)
    assert prob.counters["tlm"] == pcg + lr0.tlm + n_ksk + 2
    assert prob.counters["adj"] == pcg + lr0.adj + n_ksk + 2 + 3

    # kappa_re at iteration 1 from its definition
    _, _, v1, _ = _reuse_run(tiny_wl, 1e30, iters=1)
    p0.set_iterate(v1)
    A1 = p0.A_dense()
    Ip = np.eye(tiny_wl.n) + A1.T @ A1
    vt = sketch.unit_test_vector(o.seed, solvers.STREAM_KAPPA + 1, tiny_wl.n, index=0)
    k_dense = float(np.linalg.norm(Ip @ np.linalg.solve(np.eye(tiny_wl.n) + lr0.H_hat(), vt)))
    k1 = info[1]["kappa_re"]
    assert k1 == pytest.approx(k_dense, rel=1e-10)
    assert k1 > 1.0 + 1e-6               # the Hessian moved: the rule has something to decide

    # eps_re just above kappa_re: reuse; just below: re-sketch (kappa_re >= eps_re)
    _, _, _, above = _reuse_run(tiny_wl, k1 * (1 + 1e-7), iters=2)
    _, _, _, below = _reuse_run(tiny_wl, k1 * (1 - 1e-7), iters=2)
    assert above[1]["kappa_re"] == pytest.approx(k1, rel=1e-12)
    assert below[1]["kappa_re"] == pytest.approx(k1, rel=1e-12)
    assert not above[1]["sketched"] and above[1]["tlm_off"] == 0
    assert below[1]["sketched"] and below[1]["tlm_off"] > 0 and below[1]["adj_off"] > 0
    assert above[0]["sketched"] and below[0]["sketched"]
