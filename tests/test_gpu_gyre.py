"""Parity of the CUDA double-gyre barotropic vorticity path (the experiment of
Sec. 5.2) with the FP64 oracle, through the C ABI: prior, forecast, cost,
gradient, TLM / ADJ / Hessian blocks (FP64 1e-10, FP32 1e-5), the dot test, the
full 128 x 257 grid on sampled columns of blocks large enough for the tiled
sine transform, the paper's 40-step window with l = 384 directions, and a
Gauss-Newton run with sketched PCG."""
import numpy as np
import pytest

import sc4dvar_inputs as si

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from test_gpu_burgers import rel  # noqa: E402


def make(wl):
    import paper_2401_15758_gb300 as g
    from oracle import workload
    draws = si.gyre_draws(wl)
    ref = workload.gyre_problem(wl, draws)
    prob = g.Problem.from_gyre_workload(wl, draws)
    prob.set_background(torch.tensor(ref.xb, device="cuda"))
    prob.set_observations(torch.tensor(ref.y.reshape(-1), device="cuda"))
    return prob, ref


SMALL = si.gyre_workload(nx=16, obs_every=2, n_obs_times=3, n_sensors=4, spin_steps=50)


@pytest.fixture(scope="module")
def small():
    prob, ref = make(SMALL)
    v = 0.3 * np.random.default_rng(3).standard_normal(SMALL.n)
    Jr = ref.set_iterate(v)
    Jg = prob.fwd(torch.tensor(v, device="cuda"))
    return prob, ref, v, Jr, Jg


def test_prior_forecast_cost_gradient(small):
    prob, ref, v, Jr, Jg = small
    X = np.random.default_rng(1).standard_normal((3, SMALL.n))
    assert rel(prob.prior_sqrt_apply(torch.tensor(X, device="cuda")).cpu().numpy(), ref.prior_sqrt(X.T).T) <= 1e-12
    obs, xN = prob.forecast(torch.tensor(ref.x_true_traj[0], device="cuda"))
    assert rel(obs.cpu().numpy(), ref.observe(ref.x_true_traj).reshape(-1)) <= 1e-11
    assert rel(xN.cpu().numpy(), ref.x_true_traj[-1]) <= 1e-11
    assert abs(Jg - Jr) <= 1e-11 * abs(Jr)
    assert rel(prob.gradient().cpu().numpy(), ref.gradient()) <= 1e-10


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_blocks_match_oracle(small, prec):
    import paper_2401_15758_gb300 as g
    prob, ref, *_ = small
    p = g.FP64 if prec == "fp64" else g.FP32
    dt = torch.float64 if prec == "fp64" else torch.float32
    tol = 1e-10 if prec == "fp64" else 1e-5
    rng = np.random.default_rng(5)
    X = rng.standard_normal((3, SMALL.n))
    Wm = rng.standard_normal((3, SMALL.m))
    A = prob.tlm_block(torch.tensor(X, device="cuda", dtype=dt), prec=p).double().cpu().numpy()
    At = prob.adj_block(torch.tensor(Wm, device="cuda", dtype=dt), prec=p).double().cpu().numpy()
    H = prob.gn_hessian_apply_block(torch.tensor(X, device="cuda", dtype=dt), prec=p).double().cpu().numpy()
    Hm = prob.gn_hessian_apply_block(torch.tensor(X, device="cuda", dtype=dt), misfit_only=True,
                                     prec=p).double().cpu().numpy()
    Ar, Atr, Hr, Hmr = ref.A(X.T).T, ref.At(Wm.T).T, ref.hvp(X.T).T, ref.misfit_hvp(X.T).T
    for j in range(3):
        assert rel(A[j], Ar[j]) <= tol
        assert rel(At[j], Atr[j]) <= tol
        assert rel(H[j], Hr[j]) <= tol
        assert rel(Hm[j], Hmr[j]) <= tol


def test_dot_test_and_errors(small):
    import paper_2401_15758_gb300 as g
    prob, *_ = small
    rng = np.random.default_rng(6)
    X = torch.tensor(rng.standard_normal((2, SMALL.n)), device="cuda")
    W = torch.tensor(rng.standard_normal((2, SMALL.m)), device="cuda")
    a = torch.sum(prob.tlm_block(X) * W).item()
    b = torch.sum(X * prob.adj_block(W)).item()
    assert abs(a - b) <= 1e-12 * abs(a)
    with pytest.raises(g.Sc4dvarError) as e:
        prob.gn_hessian_apply_block(X, prec=g.DF64)
    assert e.value.code == g._abi.ERR_INVALID_ARG
    with pytest.raises(g.Sc4dvarError) as e:   # ny must be 2 nx + 1, nx a power of two
        g.Problem.from_gyre_workload(si.gyre_workload(nx=24), si.gyre_draws(si.gyre_workload(nx=24)))
    assert e.value.code == g._abi.ERR_INVALID_ARG


@pytest.mark.parametrize("nx,n_obs_times,k", [
    (128, 2, 48),    # full grid, 4 steps, tiled transform (48 x 257 rows > 152 CTAs)
    (64, 2, 160),    # tiled transform with 128-row tiles, two Thomas slabs in FP64
])
def test_tiled_blocks_sampled_columns(nx, n_obs_times, k):
    import paper_2401_15758_gb300 as g
    wl = si.gyre_workload(nx=nx, obs_every=2, n_obs_times=n_obs_times, spin_steps=20)
    prob, ref = make(wl)
    v = 0.2 * np.random.default_rng(nx).standard_normal(wl.n)
    Jr = ref.set_iterate(v)
    Jg = prob.fwd(torch.tensor(v, device="cuda"))
    assert abs(Jg - Jr) <= 1e-11 * abs(Jr)
    X = si.gaussian_matrix(wl.seed, k, wl.n, stream=31)
    H64 = prob.gn_hessian_apply_block(torch.tensor(X, device="cuda"), prec=g.FP64).cpu().numpy()
    H32 = prob.gn_hessian_apply_block(torch.tensor(X, device="cuda", dtype=torch.float32),
                                      prec=g.FP32).double().cpu().numpy()
    P64 = prob.prior_sqrt_apply(torch.tensor(X, device="cuda")).cpu().numpy()
    cols = [0, k // 2, k - 1]
    Hr = ref.hvp(X[cols].T).T
    Pr = ref.prior_sqrt(X[cols].T).T
    for j, c in enumerate(cols):
        assert rel(H64[c], Hr[j]) <= 1e-10
        assert rel(H32[c], Hr[j]) <= 1e-5
        assert rel(P64[c], Pr[j]) <= 1e-12


def test_paper_window_sampled_columns():
    """128 x 257 grid, 40 RK3 steps, 8 observation times of 256 sensors: two
    Hessian-product columns of an l = 384 block (the paper's sketch size) in FP64
    and FP32 against the oracle, and three FP32 blocks bitwise equal."""
    import paper_2401_15758_gb300 as g
    wl = si.gyre_workload()
    prob, ref = make(wl)
    prob.fwd(torch.zeros(wl.n, dtype=torch.float64, device="cuda"))
    ref.set_iterate(np.zeros(wl.n))
    X = si.gaussian_matrix(wl.seed, wl.k, wl.n, stream=29)
    H64 = prob.gn_hessian_apply_block(torch.tensor(X, device="cuda"), prec=g.FP64).cpu().numpy()
    X32 = torch.tensor(X, device="cuda", dtype=torch.float32)
    H32 = prob.gn_hessian_apply_block(X32, prec=g.FP32).double().cpu().numpy()
    # the pipelined tensor-core row transform is free of races: repeated FP32
    # blocks are bitwise identical (a slot released before its reads completed
    # showed up here as run-to-run differences in the later tiles' fields)
    for _ in range(2):
        assert np.array_equal(prob.gn_hessian_apply_block(X32, prec=g.FP32).double().cpu().numpy(), H32)
    cols = [0, wl.k - 1]
    Hr = ref.hvp(X[cols].T).T
    for j, c in enumerate(cols):
        assert rel(H64[c], Hr[j]) <= 1e-10
        assert rel(H32[c], Hr[j]) <= 1e-5


def test_gauss_newton_matches_oracle():
    """RandSVD (l = 24) sketched PCG over two GN iterations on a 32 x 65 basin."""
    from oracle import solvers
    wl = si.gyre_workload(nx=32, obs_every=2, n_obs_times=4, n_sensors=8, spin_steps=50)
    prob, ref = make(wl)
    v = torch.zeros(wl.n, dtype=torch.float64, device="cuda")
    rec = prob.gauss_newton(v, iters=2, method="randsvd", l=24, tol=1e-9)
    vr, info = solvers.gauss_newton(ref, np.zeros(wl.n),
                                    solvers.GNOptions(iters=2, method="randsvd", l=24, pcg_tol=1e-9))
    for a, b in zip(rec, info):
        assert abs(a["J"] - b["J"]) <= 1e-9 * abs(b["J"])
        assert abs(a["pcg_its"] - b["pcg_its"]) <= 1
    assert rel(v.cpu().numpy(), vr) <= 1e-7
