"""Parity of the CUDA path (through the C ABI) with the FP64 oracle: Burgers model.

Tolerances: FP64 path 1e-10 relative, FP32 sweeps 1e-5 relative on Hessian
products (both stated for this method). Inputs come from sc4dvar_inputs; the
expected values from oracle/ only.
"""
import numpy as np
import pytest

import sc4dvar_inputs as si

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def make_pair(wl):
    import paper_2401_15758_gb300 as g
    from oracle import workload
    draws = si.burgers_draws(wl)
    ref = workload.burgers_problem(wl, draws)
    prob = g.Problem.from_workload(wl, draws["obs_idx"])
    prob.set_background(torch.tensor(ref.xb, device="cuda"))
    prob.set_observations(torch.tensor(ref.y.reshape(-1), device="cuda"))
    return prob, ref


@pytest.fixture(scope="module")
def small():
    wl = si.burgers_workload("burgers_n128")
    prob, ref = make_pair(wl)
    v = 0.3 * np.random.default_rng(11).standard_normal(wl.n)
    Jr = ref.set_iterate(v)
    Jg = prob.fwd(torch.tensor(v, device="cuda"))
    return wl, prob, ref, v, Jr, Jg


def test_philox_draws_match_oracle():
    import paper_2401_15758_gb300 as g
    from oracle import philox
    for rows, cols, col0 in ((37, 5, 0), (1000, 3, 7)):
        a = g.gaussian(20240128, 105, rows, cols, col0).cpu().numpy().T
        b = philox.gaussian(20240128, 105, rows, cols, col0=col0)
        assert np.max(np.abs(a - b)) <= 1e-13 * max(1.0, np.max(np.abs(b)))


@pytest.mark.parametrize("n", [16, 128, 2048, 8192])
def test_prior_symbol_and_apply(n):
    import paper_2401_15758_gb300 as g
    from oracle import prior
    wl = si.burgers_workload("burgers_n128", n=n)
    prob = g.Problem.from_workload(wl, si.burgers_obs_idx(wl))
    sym_ref = prior.se_sqrt_symbol(n, wl.sigma_b, wl.length_b)
    sym = prob.prior_symbol()
    assert np.max(np.abs(sym - sym_ref)) <= 1e-12 * sym_ref.max()
    X = np.random.default_rng(n).standard_normal((5, n))
    Y = prob.prior_sqrt_apply(torch.tensor(X, device="cuda")).cpu().numpy()
    Yr = prior.apply_symbol(sym_ref, X.T).T
    assert rel(Y, Yr) <= 1e-12


def test_forecast_matches_oracle(small):
    wl, prob, ref, v, Jr, Jg = small
    obs, xN = prob.forecast(torch.tensor(ref.x_true_traj[0], device="cuda"))
    assert rel(obs.cpu().numpy(), ref.observe(ref.x_true_traj).reshape(-1)) <= 1e-12
    assert rel(xN.cpu().numpy(), ref.x_true_traj[-1]) <= 1e-12


def test_cost_and_gradient_match_oracle(small):
    wl, prob, ref, v, Jr, Jg = small
    assert abs(Jg - Jr) <= 1e-11 * abs(Jr)
    g_ = prob.gradient().cpu().numpy()
    assert rel(g_, ref.gradient()) <= 1e-10


@pytest.mark.parametrize("k", [1, 5, 20])
def test_fp64_blocks_match_oracle(small, k):
    wl, prob, ref, v, Jr, Jg = small
    rng = np.random.default_rng(100 + k)
    X = rng.standard_normal((k, wl.n))
    Wm = rng.standard_normal((k, wl.m))
    Xd = torch.tensor(X, device="cuda")
    A = prob.tlm_block(Xd).cpu().numpy()
    assert rel(A, ref.A(X.T).T) <= 1e-10
    At = prob.adj_block(torch.tensor(Wm, device="cuda")).cpu().numpy()
    assert rel(At, ref.At(Wm.T).T) <= 1e-10
    H = prob.gn_hessian_apply_block(Xd).cpu().numpy()
    assert rel(H, ref.hvp(X.T).T) <= 1e-10
    Hm = prob.gn_hessian_apply_block(Xd, misfit_only=True).cpu().numpy()
    assert rel(Hm, ref.misfit_hvp(X.T).T) <= 1e-10


def test_fp32_hessian_within_1e5(small):
    import paper_2401_15758_gb300 as g
    wl, prob, ref, v, Jr, Jg = small
    X = np.random.default_rng(3).standard_normal((7, wl.n))
    H = prob.gn_hessian_apply_block(torch.tensor(X, device="cuda", dtype=torch.float32),
                                    prec=g.FP32).cpu().numpy()
    Hr = ref.hvp(X.T).T
    for j in range(7):
        assert rel(H[j], Hr[j]) <= 1e-5


def test_adjoint_dot_test_on_gpu(small):
    wl, prob, ref, v, Jr, Jg = small
    rng = np.random.default_rng(5)
    X = torch.tensor(rng.standard_normal((3, wl.n)), device="cuda")
    W = torch.tensor(rng.standard_normal((3, wl.m)), device="cuda")
    a = torch.sum(prob.tlm_block(X) * W).item()
    b = torch.sum(X * prob.adj_block(W)).item()
    assert abs(a - b) <= 1e-12 * abs(a)


def test_errors_are_status_codes():
    import paper_2401_15758_gb300 as g
    wl = si.burgers_workload("burgers_n128")
    with pytest.raises(g.Sc4dvarError) as e:
        g.Problem.from_workload(si.burgers_workload("burgers_n128", n=100), si.burgers_obs_idx(wl))
    assert e.value.code == g._abi.ERR_INVALID_ARG
    bad = si.burgers_obs_idx(wl).copy()
    bad[0, 0] = wl.n
    with pytest.raises(g.Sc4dvarError):
        g.Problem.from_workload(wl, bad)
    prob = g.Problem.from_workload(wl, si.burgers_obs_idx(wl))
    with pytest.raises(g.Sc4dvarError) as e:
        prob.gradient()
    assert e.value.code == g._abi.ERR_STATE
    # empty block is a no-op
    prob.fwd(torch.zeros(wl.n, dtype=torch.float64, device="cuda"))
    out = prob.gn_hessian_apply_block(torch.zeros((0, wl.n), dtype=torch.float64, device="cuda"))
    assert out.shape == (0, wl.n)


# Larger grids run the register-resident kernels (contiguous points per thread,
# shuffle halos) with and without thread-block clusters; short windows keep the
# oracle fast while the launch shapes are the ones of the full workloads.
V2_CASES = [
    # (n, output steps, k, precision)
    (8192, 20, 6, "fp32"),   # packed FP32x2, 8 pairs per thread, one CTA per direction
    (8192, 20, 3, "fp32"),   # packed FP32x2, few directions: one CTA each (the cluster form is
                             # rerun under SC4DVAR_FEW_CLUSTER=8 by test_gpu_cluster_knob.py)
    (512, 20, 5, "fp32"),    # scalar register-resident kernels
    (8192, 20, 2, "fp64"),   # 16-CTA cluster, 512 points per CTA (few directions)
    (2048, 20, 5, "fp64"),   # 2 points per thread, odd k (FFT pair tail)
    (1024, 20, 1, "fp32"),   # one direction, one CTA (a 2-CTA cluster under the knob)
]


@pytest.mark.parametrize("n,n_out,k,prec", V2_CASES)
def test_register_resident_sweeps_match_oracle(n, n_out, k, prec):
    import paper_2401_15758_gb300 as g
    wl = si.burgers_workload("burgers_n8192", n=n, n_out=n_out)
    prob, ref = make_pair(wl)
    v = 0.2 * np.random.default_rng(n).standard_normal(wl.n)
    Jr = ref.set_iterate(v)
    Jg = prob.fwd(torch.tensor(v, device="cuda"))
    assert abs(Jg - Jr) <= 1e-10 * abs(Jr)
    p = g.FP64 if prec == "fp64" else g.FP32
    dt = torch.float64 if prec == "fp64" else torch.float32
    tol = 1e-10 if prec == "fp64" else 1e-5
    rng = np.random.default_rng(7 + n + k)
    X = rng.standard_normal((k, wl.n))
    Wm = rng.standard_normal((k, wl.m))
    A = prob.tlm_block(torch.tensor(X, device="cuda", dtype=dt), prec=p).double().cpu().numpy()
    At = prob.adj_block(torch.tensor(Wm, device="cuda", dtype=dt), prec=p).double().cpu().numpy()
    H = prob.gn_hessian_apply_block(torch.tensor(X, device="cuda", dtype=dt),
                                    prec=p).double().cpu().numpy()
    Ar, Atr, Hr = ref.A(X.T).T, ref.At(Wm.T).T, ref.hvp(X.T).T
    for j in range(k):
        assert rel(A[j], Ar[j]) <= tol
        assert rel(At[j], Atr[j]) <= tol
        assert rel(H[j], Hr[j]) <= tol
    g_ = prob.gradient().cpu().numpy()
    assert rel(g_, ref.gradient()) <= 1e-10


# Double-float sweeps: double blocks in and out, the TLM / ADJ sweeps on (hi, lo)
# float pairs (about 48 significant bits), held to the FP64 tolerance.
DF64_CASES = [
    # (n, output steps, k)
    (128, None, 1),     # the small window, one direction
    (128, None, 6),     # several directions, one CTA each
    (8192, 20, 2),      # 16-CTA cluster, 512 points per CTA
    (2048, 20, 5),      # 2 points per thread, odd k
]


@pytest.mark.parametrize("n,n_out,k", DF64_CASES)
def test_df64_hessian_matches_oracle(n, n_out, k):
    import paper_2401_15758_gb300 as g
    kw = {} if n_out is None else {"n": n, "n_out": n_out}
    wl = si.burgers_workload("burgers_n128" if n == 128 else "burgers_n8192", **kw)
    prob, ref = make_pair(wl)
    v = 0.2 * np.random.default_rng(n + 1).standard_normal(wl.n)
    ref.set_iterate(v)
    prob.fwd(torch.tensor(v, device="cuda"))
    X = np.random.default_rng(40 + k).standard_normal((k, wl.n))
    Xd = torch.tensor(X, device="cuda")
    H = prob.gn_hessian_apply_block(Xd, prec=g.DF64).cpu().numpy()
    Hm = prob.gn_hessian_apply_block(Xd, misfit_only=True, prec=g.DF64).cpu().numpy()
    Hr, Hmr = ref.hvp(X.T).T, ref.misfit_hvp(X.T).T
    for j in range(k):
        assert rel(H[j], Hr[j]) <= 1e-10
        assert rel(Hm[j], Hmr[j]) <= 1e-10
    # a new FWD refreshes the double-float trajectory
    v2 = v + 0.1
    ref.set_iterate(v2)
    prob.fwd(torch.tensor(v2, device="cuda"))
    H2 = prob.gn_hessian_apply_block(Xd[:1], prec=g.DF64).cpu().numpy()
    assert rel(H2[0], ref.hvp(X[:1].T).T[0]) <= 1e-10
