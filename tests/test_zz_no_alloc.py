"""The allocation-free block Hessian product (sc4dvar_gn_hessian_apply_block_noalloc).

Callers that cannot allocate device memory during a call (an external pool
allocator owning all device memory, allocator-free real-time loops) use this
entry point; it must give the same product as sc4dvar_gn_hessian_apply_block and
as the oracle. The cases cover each sweep variant the product dispatches to:
the scalar kernels (n = 128), the packed FP32x2 sweeps with one CTA per direction
(n = 8192, k = 6) and over a CTA cluster (k = 3), and the FP64 cluster sweeps
(n = 8192, k = 2). The file is named to be collected last.
"""
import ctypes as C

import numpy as np
import pytest

import sc4dvar_inputs as si

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _problem(n=None, n_out=None):
    import paper_2401_15758_gb300 as g
    from oracle import workload
    if n is None:
        wl = si.burgers_workload("burgers_n128")
    else:
        wl = si.burgers_workload("burgers_n8192", n=n, n_out=n_out)
    draws = si.burgers_draws(wl)
    ref = workload.burgers_problem(wl, draws)
    prob = g.Problem.from_workload(wl, draws["obs_idx"])
    prob.set_background(torch.tensor(ref.xb, device="cuda"))
    prob.set_observations(torch.tensor(ref.y.reshape(-1), device="cuda"))
    v = 0.2 * np.random.default_rng(wl.n + 3).standard_normal(wl.n)
    ref.set_iterate(v)
    prob.fwd(torch.tensor(v, device="cuda"))
    return g, wl, prob, ref


def _noalloc(g, prob, X, misfit_only, prec):
    Y = torch.empty_like(X)
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = g.lib.sc4dvar_gn_hessian_apply_block_noalloc(
        prob.h, C.c_void_p(X.data_ptr()), prob.n, X.shape[0], C.c_void_p(Y.data_ptr()), prob.n,
        int(misfit_only), prec, s)
    g.check(rc)
    return Y


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


CASES = [
    # (n, output steps, precision, block widths of the two calls in a row)
    (None, None, "fp64", (7, 3)),
    (None, None, "fp32", (7, 3)),
    (8192, 20, "fp32", (6, 6)),     # packed FP32x2, one CTA per direction
    (8192, 20, "fp32", (3, 3)),     # packed FP32x2 over a CTA cluster
    (8192, 20, "fp64", (2, 2)),     # FP64 cluster sweeps
]


@pytest.mark.parametrize("n,n_out,prec,ks", CASES)
def test_noalloc_matches_allocating_entry_point_and_oracle_twice(n, n_out, prec, ks):
    g, wl, prob, ref = _problem(n, n_out)
    p = g.FP64 if prec == "fp64" else g.FP32
    dt = torch.float64 if prec == "fp64" else torch.float32
    tol_same = 1e-12 if prec == "fp64" else 1e-5
    tol_oracle = 1e-10 if prec == "fp64" else 1e-5
    rng = np.random.default_rng(42 + wl.n)
    for call, (k, misfit) in enumerate(zip(ks, (False, True))):
        X = torch.tensor(rng.standard_normal((k, wl.n)), device="cuda", dtype=dt)
        want = prob.gn_hessian_apply_block(X, misfit_only=misfit, prec=p).double().cpu().numpy()
        got = _noalloc(g, prob, X, misfit, p).double().cpu().numpy()
        assert _rel(got, want) <= tol_same, (call, _rel(got, want))
        Xr = X.double().cpu().numpy().T
        ora = (ref.misfit_hvp(Xr) if misfit else ref.hvp(Xr)).T
        for j in range(k):
            assert _rel(got[j], ora[j]) <= tol_oracle, (call, j)


def test_noalloc_rejects_k_beyond_fixed_scratch():
    g, wl, prob, ref = _problem()
    k = (32 << 20) // ((2 * wl.n + wl.m) * 8) + 1
    X = torch.zeros((k, wl.n), dtype=torch.float64, device="cuda")
    with pytest.raises(g.Sc4dvarError) as e:
        _noalloc(g, prob, X, False, g.FP64)
    assert e.value.code == g._abi.ERR_INVALID_ARG
    assert "scratch" in str(e.value)
