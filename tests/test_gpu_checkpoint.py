"""Checkpointed barotropic vorticity sweeps and the autograd cost.

With n_checkpoints = c the FWD keeps only the FP64 state every L = ceil(N / c)
steps and every sweep recomputes one segment of stage states at a time. FP64
sweeps recompute with the FWD's kernels in the FWD's order, so their results
must be bit-identical to the stored-trajectory run; FP32 sweeps recompute in
FP32 from the rounded checkpoint and agree to FP32 accuracy (and stay exact
transposes of each other: the FP32 dot test). The autograd cost (forward = FWD,
backward = the adjoint sweep, Eq. 4dvar_gradient) is checked against the FP64
oracle at 64^2 and, at the 1024^2 / 256-step / 16-checkpoint size, against
central differences of J and the adjoint dot test (the oracle is too slow there)."""
import numpy as np
import pytest

import sc4dvar_inputs as si

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from test_gpu_burgers import rel  # noqa: E402


def make(wl, draws, c, background=None, observations=None):
    import paper_2401_15758_gb300 as g
    prob = g.Problem.from_bve_workload(wl, draws, n_checkpoints=c)
    if background is None:
        xt = torch.tensor(draws["x_true0"], device="cuda")
        obs, _ = prob.forecast(xt)
        observations = obs + draws["sigma_obs"] * torch.tensor(draws["xi_o"].reshape(-1), device="cuda")
        background = xt + prob.prior_sqrt_apply(torch.tensor(draws["xi_b"], device="cuda"))
    prob.set_background(background)
    prob.set_observations(observations)
    return prob, background, observations


SMALL = si.bve_workload("bve_n256", N=64, n_steps=40, obs_every=10)


@pytest.fixture(scope="module")
def small():
    draws = si.bve_draws(SMALL)
    full, xb, y = make(SMALL, draws, 0)
    v = torch.tensor(0.3 * np.random.default_rng(5).standard_normal(SMALL.n), device="cuda")
    return draws, full, xb, y, v


@pytest.mark.parametrize("c", [1, 3, 7, 40])
def test_checkpointed_equals_full(small, c):
    import paper_2401_15758_gb300 as g
    draws, full, xb, y, v = small
    ck, _, _ = make(SMALL, draws, c, xb, y)
    J0, d0 = full.fwd(v, want_d=True)
    J1, d1 = ck.fwd(v, want_d=True)
    assert J0 == J1 and torch.equal(d0, d1)
    assert torch.equal(full.gradient(), ck.gradient())
    X = torch.tensor(np.random.default_rng(c).standard_normal((3, SMALL.n)), device="cuda")
    assert torch.equal(full.tlm_block(X, prec=g.FP64), ck.tlm_block(X, prec=g.FP64))
    assert torch.equal(full.gn_hessian_apply_block(X, prec=g.FP64), ck.gn_hessian_apply_block(X, prec=g.FP64))
    Xf = X.float()
    for fn in (lambda p: p.tlm_block(Xf, prec=g.FP32), lambda p: p.gn_hessian_apply_block(Xf, prec=g.FP32)):
        a, b = fn(full).double().cpu().numpy(), fn(ck).double().cpu().numpy()
        assert rel(b, a) <= 1e-5
    # the recomputed FP32 states are shared by the TLM and the ADJ: exact transposes
    W = torch.tensor(np.random.default_rng(c + 1).standard_normal((2, SMALL.m)), device="cuda").float()
    V = Xf[:2]
    lhs = torch.sum(ck.tlm_block(V, prec=g.FP32).double() * W.double()).item()
    rhs = torch.sum(V.double() * ck.adj_block(W, prec=g.FP32).double()).item()
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)


def test_autograd_matches_oracle_and_differences(small):
    import paper_2401_15758_gb300 as g
    from oracle import workload
    draws, _, xb, y, v = small
    ck, _, _ = make(SMALL, draws, 6, xb, y)
    ref = workload.bve_problem(SMALL, draws)
    vv = v.clone().requires_grad_(True)
    J = g.cost(ck, vv)
    J.backward()
    Jr = ref.set_iterate(v.cpu().numpy())
    assert abs(J.item() - Jr) <= 1e-10 * abs(Jr)
    assert rel(vv.grad.cpu().numpy(), ref.gradient()) <= 1e-10
    # central differences of J along a random direction (FP64 FWD runs)
    p = torch.tensor(np.random.default_rng(11).standard_normal(SMALL.n), device="cuda")
    eps = 1e-4
    fd = (ck.fwd(v + eps * p) - ck.fwd(v - eps * p)) / (2 * eps)
    assert abs(fd - torch.dot(vv.grad, p).item()) <= 1e-7 * abs(fd)


def test_backward_after_another_fwd_raises(small):
    import paper_2401_15758_gb300 as g
    draws, _, xb, y, v = small
    ck, _, _ = make(SMALL, draws, 4, xb, y)
    vv = v.clone().requires_grad_(True)
    J = g.cost(ck, vv)
    ck.fwd(2 * v)
    with pytest.raises(RuntimeError):
        J.backward()


def test_full_size_1024_checkpointed():
    """bve_n1024 (N = 1024, 256 RK4 steps, 16 checkpoints): gradient of the
    autograd cost against central differences, the adjoint dot test in FP64,
    the FP32 block against the FP64 block, and the checkpointed gradient
    bit-identical to the stored-trajectory one."""
    import paper_2401_15758_gb300 as g
    wl = si.bve_workload("bve_n1024")
    assert wl.n_checkpoints == 16 and wl.N == 1024 and wl.n_steps == 256
    draws = si.bve_draws(wl)
    ck, xb, y = make(wl, draws, wl.n_checkpoints)
    rng = np.random.default_rng(3)
    v = torch.tensor(0.3 * rng.standard_normal(wl.n), device="cuda")
    vv = v.clone().requires_grad_(True)
    J = g.cost(ck, vv)
    J.backward()
    grad = vv.grad.clone()
    p = torch.tensor(rng.standard_normal(wl.n), device="cuda")
    eps = 1e-4
    fd = (ck.fwd(v + eps * p) - ck.fwd(v - eps * p)) / (2 * eps)
    assert abs(fd - torch.dot(grad, p).item()) <= 1e-6 * abs(fd)
    ck.fwd(v)
    x = torch.tensor(rng.standard_normal((1, wl.n)), device="cuda")
    w = torch.tensor(rng.standard_normal((1, wl.m)), device="cuda")
    lhs = torch.dot(ck.tlm_block(x, prec=g.FP64)[0], w[0]).item()
    rhs = torch.dot(x[0], ck.adj_block(w, prec=g.FP64)[0]).item()
    assert abs(lhs - rhs) <= 1e-10 * max(abs(lhs), abs(rhs))
    X = torch.tensor(rng.standard_normal((4, wl.n)), device="cuda")
    H64 = ck.gn_hessian_apply_block(X, prec=g.FP64)
    H32 = ck.gn_hessian_apply_block(X.float(), prec=g.FP32).double()
    assert rel(H32.cpu().numpy(), H64.cpu().numpy()) <= 1e-4
    g_ck = ck.gradient()
    del ck
    full, _, _ = make(wl, draws, 0, xb, y)
    full.fwd(v)
    assert torch.equal(full.gradient(), g_ck)
