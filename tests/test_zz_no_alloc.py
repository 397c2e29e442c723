"""The allocation-free block Hessian product (sc4dvar_gn_hessian_apply_block_noalloc).

Callers that cannot allocate device memory during a call (graph capture, an
external pool allocator owning all device memory, allocator-free real-time
loops) use this entry point; it must give the same product as
sc4dvar_gn_hessian_apply_block. The file is named to be collected last.
"""
import ctypes as C

import numpy as np
import pytest

import sc4dvar_inputs as si

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _problem():
    import paper_2401_15758_gb300 as g
    from oracle import workload
    wl = si.burgers_workload("burgers_n128")
    draws = si.burgers_draws(wl)
    ref = workload.burgers_problem(wl, draws)
    prob = g.Problem.from_workload(wl, draws["obs_idx"])
    prob.set_background(torch.tensor(ref.xb, device="cuda"))
    prob.set_observations(torch.tensor(ref.y.reshape(-1), device="cuda"))
    prob.fwd(torch.zeros(wl.n, dtype=torch.float64, device="cuda"))
    return g, wl, prob


def _noalloc(g, prob, X, misfit_only, prec):
    Y = torch.empty_like(X)
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = g.lib.sc4dvar_gn_hessian_apply_block_noalloc(
        prob.h, C.c_void_p(X.data_ptr()), prob.n, X.shape[0], C.c_void_p(Y.data_ptr()), prob.n,
        int(misfit_only), prec, s)
    g.check(rc)
    return Y


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_noalloc_matches_allocating_entry_point_twice(prec):
    g, wl, prob = _problem()
    p = g.FP64 if prec == "fp64" else g.FP32
    dt = torch.float64 if prec == "fp64" else torch.float32
    tol = 1e-12 if prec == "fp64" else 1e-5
    rng = np.random.default_rng(42)
    for call, (k, misfit) in enumerate(((7, False), (3, True))):
        X = torch.tensor(rng.standard_normal((k, wl.n)), device="cuda", dtype=dt)
        want = prob.gn_hessian_apply_block(X, misfit_only=misfit, prec=p).double().cpu().numpy()
        got = _noalloc(g, prob, X, misfit, p).double().cpu().numpy()
        err = np.linalg.norm(got - want) / np.linalg.norm(want)
        assert err <= tol, (call, err)


def test_noalloc_rejects_k_beyond_fixed_scratch():
    g, wl, prob = _problem()
    k = (32 << 20) // ((2 * wl.n + wl.m) * 8) + 1
    X = torch.zeros((k, wl.n), dtype=torch.float64, device="cuda")
    with pytest.raises(g.Sc4dvarError) as e:
        _noalloc(g, prob, X, False, g.FP64)
    assert e.value.code == g._abi.ERR_INVALID_ARG
    assert "scratch" in str(e.value)
