"""Parity of the CUDA barotropic vorticity path (through the C ABI) with the
FP64 oracle: prior multiplier, FWD, cost and gradient, TLM/ADJ/Hessian blocks
(FP64 1e-10, FP32 1e-5), the adjoint dot test and a Gauss-Newton run."""
import numpy as np
import pytest

import sc4dvar_inputs as si

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from test_gpu_burgers import rel  # noqa: E402


def make_bve(N, n_steps, obs_every):
    import paper_2401_15758_gb300 as g
    from oracle import workload
    wl = si.bve_workload("bve_n256", N=N, n_steps=n_steps, obs_every=obs_every)
    draws = si.bve_draws(wl)
    ref = workload.bve_problem(wl, draws)
    prob = g.Problem.from_bve_workload(wl, draws)
    prob.set_background(torch.tensor(ref.xb, device="cuda"))
    prob.set_observations(torch.tensor(ref.y.reshape(-1), device="cuda"))
    return wl, prob, ref


CASES = [(16, 10, 5), (32, 20, 5), (64, 12, 4), (128, 6, 3), (256, 4, 2), (512, 2, 1)]


@pytest.fixture(scope="module", params=CASES, ids=lambda c: f"N{c[0]}")
def bve_pair(request):
    N, steps, every = request.param
    wl, prob, ref = make_bve(N, steps, every)
    v = 0.3 * np.random.default_rng(N).standard_normal(wl.n)
    Jr = ref.set_iterate(v)
    Jg = prob.fwd(torch.tensor(v, device="cuda"))
    return wl, prob, ref, v, Jr, Jg


def test_prior_multiplier(bve_pair):
    wl, prob, ref, *_ = bve_pair
    from oracle import bve
    X = np.random.default_rng(1).standard_normal((3, wl.n))
    Y = prob.prior_sqrt_apply(torch.tensor(X, device="cuda")).cpu().numpy()
    assert rel(Y, bve.apply_symbol_2d(ref.symbol, X.T, wl.N).T) <= 1e-12
    assert np.allclose(prob.prior_symbol().reshape(wl.N, wl.N), ref.symbol, rtol=1e-14, atol=0)


def test_forecast_cost_gradient(bve_pair):
    wl, prob, ref, v, Jr, Jg = bve_pair
    obs, xN = prob.forecast(torch.tensor(ref.x_true_traj[0], device="cuda"))
    assert rel(obs.cpu().numpy(), ref.observe(ref.x_true_traj).reshape(-1)) <= 1e-11
    assert rel(xN.cpu().numpy(), ref.x_true_traj[-1]) <= 1e-11
    assert abs(Jg - Jr) <= 1e-10 * abs(Jr)
    assert rel(prob.gradient().cpu().numpy(), ref.gradient()) <= 1e-10


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_blocks_match_oracle(bve_pair, prec):
    import paper_2401_15758_gb300 as g
    wl, prob, ref, *_ = bve_pair
    p = g.FP64 if prec == "fp64" else g.FP32
    dt = torch.float64 if prec == "fp64" else torch.float32
    tol = 1e-10 if prec == "fp64" else 1e-5
    k = 3
    rng = np.random.default_rng(5)
    X = rng.standard_normal((k, wl.n))
    Wm = rng.standard_normal((k, wl.m))
    A = prob.tlm_block(torch.tensor(X, device="cuda", dtype=dt), prec=p).double().cpu().numpy()
    At = prob.adj_block(torch.tensor(Wm, device="cuda", dtype=dt), prec=p).double().cpu().numpy()
    H = prob.gn_hessian_apply_block(torch.tensor(X, device="cuda", dtype=dt), prec=p).double().cpu().numpy()
    Ar, Atr, Hr = ref.A(X.T).T, ref.At(Wm.T).T, ref.hvp(X.T).T
    for j in range(k):
        assert rel(A[j], Ar[j]) <= tol
        assert rel(At[j], Atr[j]) <= tol
        assert rel(H[j], Hr[j]) <= tol


def test_dot_test_on_gpu(bve_pair):
    wl, prob, *_ = bve_pair
    rng = np.random.default_rng(6)
    X = torch.tensor(rng.standard_normal((2, wl.n)), device="cuda")
    W = torch.tensor(rng.standard_normal((2, wl.m)), device="cuda")
    a = torch.sum(prob.tlm_block(X) * W).item()
    b = torch.sum(X * prob.adj_block(W)).item()
    assert abs(a - b) <= 1e-12 * abs(a)


def test_bve_gauss_newton_matches_oracle():
    from oracle import solvers
    wl, prob, ref = make_bve(32, 20, 5)
    v = torch.zeros(wl.n, dtype=torch.float64, device="cuda")
    rec = prob.gauss_newton(v, iters=2, method="randsvd", l=40, tol=1e-8)
    vr, info = solvers.gauss_newton(ref, np.zeros(wl.n),
                                    solvers.GNOptions(iters=2, method="randsvd", l=40, pcg_tol=1e-8))
    assert abs(rec[0]["J"] - info[0]["J"]) <= 1e-11 * abs(info[0]["J"])
    assert abs(rec[1]["J"] - info[1]["J"]) <= 1e-9 * abs(info[1]["J"])
    assert abs(rec[0]["pcg_its"] - info[0]["pcg_its"]) <= 1
    assert rel(v.cpu().numpy(), vr) <= 1e-6


@pytest.mark.parametrize("N", [16, 32, 64, 128, 256, 512, 1024])
def test_prior_multiplier_every_grid(N):
    """The 2D multiplier of every grid size (each size is its own kernel
    instantiation) against numpy's FFT, on an odd number of fields."""
    import paper_2401_15758_gb300 as g
    from oracle import bve
    wl = si.bve_workload("bve_n256", N=N, n_steps=2, obs_every=1)
    draws = si.bve_draws(wl)
    prob = g.Problem.from_bve_workload(wl, draws)
    sym = bve.inv_helmholtz_sqrt_symbol(N, draws["prior_c"], draws["prior_ell"])
    X = np.random.default_rng(N).standard_normal((3, wl.n))
    Y = prob.prior_sqrt_apply(torch.tensor(X, device="cuda")).cpu().numpy()
    assert rel(Y, bve.apply_symbol_2d(sym, X.T, N).T) <= 1e-12


def test_full_window_256_sampled_columns():
    """bve_n256 at full size (256^2, 200 RK4 steps, m = 131 080) in the launch
    configuration the benchmark times (one FP32 block of k = 256 directions):
    two sampled columns (the first; the second lane of the last direction pair)
    against the oracle's FP64 Hessian product of the same columns."""
    import paper_2401_15758_gb300 as g
    from oracle import workload
    wl = si.bve_workload("bve_n256")
    assert (wl.N, wl.n_steps, wl.k) == (256, 200, 256)
    draws = si.bve_draws(wl)
    ref = workload.bve_problem(wl, draws)
    prob = g.Problem.from_bve_workload(wl, draws)
    prob.set_background(torch.tensor(ref.xb, device="cuda"))
    prob.set_observations(torch.tensor(ref.y.reshape(-1), device="cuda"))
    prob.fwd(torch.zeros(wl.n, dtype=torch.float64, device="cuda"))
    ref.set_iterate(np.zeros(wl.n))
    X = si.gaussian_matrix(wl.seed, wl.k, wl.n, stream=23)
    H = prob.gn_hessian_apply_block(torch.tensor(X, device="cuda", dtype=torch.float32), prec=g.FP32)
    cols = [0, wl.k - 1]
    Hr = ref.hvp(X[cols].T).T
    for j, c in enumerate(cols):
        err = rel(H[c].double().cpu().numpy(), Hr[j])
        print(f"column {c}: relative error {err:.3e}")
        assert err <= 1e-5
