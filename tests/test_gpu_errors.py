"""Status codes of the C ABI: argument and state errors are reported as
negative codes with a message, and the handle stays usable afterwards. Every
case is rejected by host-side checks before any kernel is launched."""
import numpy as np
import pytest

import sc4dvar_inputs as si

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

OK, INVALID_ARG, NOT_CONVERGED, STATE = 0, -1, -5, -8


def burgers_problem():
    import paper_2401_15758_gb300 as g
    wl = si.burgers_workload("burgers_n128")
    d = si.burgers_draws(wl)
    return wl, g.Problem.from_workload(wl, d["obs_idx"])


def code_of(fn):
    import paper_2401_15758_gb300 as g
    with pytest.raises(g.Sc4dvarError) as e:
        fn()
    assert str(e.value)  # carries the library's message
    return e.value.code


def test_state_errors_before_fwd():
    import paper_2401_15758_gb300 as g
    wl, prob = burgers_problem()
    X = torch.zeros((2, wl.n), dtype=torch.float64, device="cuda")
    assert code_of(lambda: prob.gradient()) == STATE
    assert code_of(lambda: prob.tlm_block(X)) == STATE
    assert code_of(lambda: prob.gn_hessian_apply_block(X)) == STATE
    assert code_of(lambda: prob.build_precond("randsvd", l=4)) == STATE
    # after a FWD the same calls succeed on the same handle
    prob.fwd(torch.zeros(wl.n, dtype=torch.float64, device="cuda"))
    assert prob.gn_hessian_apply_block(X).shape == X.shape
    assert prob.counters()["fwd"] == 1


def test_invalid_arguments():
    import ctypes as C
    import paper_2401_15758_gb300 as g
    wl, prob = burgers_problem()
    prob.fwd(torch.zeros(wl.n, dtype=torch.float64, device="cuda"))
    X = torch.zeros((1, wl.n), dtype=torch.float64, device="cuda")
    Y = torch.empty_like(X)
    lib = g.lib
    # leading dimension below n, negative k, unknown precision, sketch size out of range
    assert lib.sc4dvar_gn_hessian_apply_block(prob.h, C.c_void_p(X.data_ptr()), wl.n - 1, 1,
                                              C.c_void_p(Y.data_ptr()), wl.n, 0, 0, None) == INVALID_ARG
    assert lib.sc4dvar_gn_hessian_apply_block(prob.h, C.c_void_p(X.data_ptr()), wl.n, -1,
                                              C.c_void_p(Y.data_ptr()), wl.n, 0, 0, None) == INVALID_ARG
    assert lib.sc4dvar_gn_hessian_apply_block(prob.h, C.c_void_p(X.data_ptr()), wl.n, 1,
                                              C.c_void_p(Y.data_ptr()), wl.n, 0, 7, None) == INVALID_ARG
    assert lib.sc4dvar_last_error()
    assert code_of(lambda: prob.build_precond("randsvd", l=wl.n + 1)) == INVALID_ARG
    # the handle still works
    out = prob.gn_hessian_apply_block(X)
    assert torch.isfinite(out).all()


def test_unsupported_grids_rejected():
    import paper_2401_15758_gb300 as g
    wl = si.burgers_workload("burgers_n128")
    d = si.burgers_draws(wl)
    for n in (96, 16384):  # not a power of two; above the largest grid
        assert code_of(lambda: g.Problem(n=n, nu=wl.nu, dt=wl.dt, n_steps=wl.n_steps,
                                         obs_steps=wl.obs_steps, obs_idx=np.zeros_like(d["obs_idx"]),
                                         sigma_obs=wl.sigma_obs, prior_sigma=wl.sigma_b,
                                         prior_length=wl.length_b)) == INVALID_ARG
    bw = si.bve_workload("bve_n256", N=32, n_steps=4, obs_every=2)
    bd = si.bve_draws(bw)
    # checkpointing is a vorticity option; more checkpoints than steps is rejected
    assert code_of(lambda: g.Problem.from_bve_workload(bw, bd, n_checkpoints=5)) == INVALID_ARG
    assert code_of(lambda: g.Problem(n=wl.n, nu=wl.nu, dt=wl.dt, n_steps=wl.n_steps,
                                     obs_steps=wl.obs_steps, obs_idx=d["obs_idx"], sigma_obs=wl.sigma_obs,
                                     prior_sigma=wl.sigma_b, prior_length=wl.length_b,
                                     n_checkpoints=2)) == INVALID_ARG


def test_pcg_reports_not_converged():
    """maxit below what the solve needs: NOT_CONVERGED in the info record, the
    iterate returned and the residual reported (not an exception)."""
    wl, prob = burgers_problem()
    prob.fwd(torch.zeros(wl.n, dtype=torch.float64, device="cuda"))
    b = torch.tensor(np.random.default_rng(4).standard_normal(wl.n), device="cuda")
    x, info = prob.pcg(b, None, tol=1e-12, maxit=2)
    assert info["status"] == NOT_CONVERGED and info["iterations"] == 2
    # CG minimises the energy norm of the error, so two steps may leave a
    # residual above |b|; it is finite and above the tolerance
    assert np.isfinite(info["relres"]) and info["relres"] > 1e-12 and torch.isfinite(x).all()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_pcg_nonfinite_rhs_is_a_breakdown(prec):
    """A right-hand side with a NaN (made on the host) ends the solve at once
    with status SC4DVAR_ERR_BREAKDOWN and no iterations; the handle stays
    usable for the next, finite solve."""
    import paper_2401_15758_gb300 as g
    wl, prob = burgers_problem()
    prob.fwd(torch.zeros(wl.n, dtype=torch.float64, device="cuda"))
    p = g.FP64 if prec == "fp64" else g.FP32
    b = np.random.default_rng(3).standard_normal(wl.n)
    b[17] = np.nan
    x, info = prob.pcg(torch.tensor(b, device="cuda"), None, tol=1e-6, prec=p)
    assert info["status"] == g._abi.ERR_BREAKDOWN and info["iterations"] == 0
    b[17] = 0.0
    x, info = prob.pcg(torch.tensor(b, device="cuda"), None, tol=1e-6, prec=p)
    assert info["status"] == OK and np.all(np.isfinite(x.cpu().numpy()))
