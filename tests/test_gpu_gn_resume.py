"""GN-level checkpoint and resume through the C ABI (sc4dvar_gauss_newton_resume,
sc4dvar_precond_import, sc4dvar_counters_set): a run stopped at an iteration
boundary, written to a file, and continued by a fresh problem handle repeats the
uninterrupted run bit for bit. The continuation must reuse the imported
preconditioner under the reuse rule of Sec. 3.2 exactly where the uninterrupted
run reused its own. The sketch draws and kappa_re probes are keyed by the
iteration index, so resuming at iteration k draws what the uninterrupted run drew
there."""
import numpy as np
import pytest

import sc4dvar_inputs as si

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from test_gpu_burgers import make_pair  # noqa: E402

OPTS = dict(method="randsvd", l=8, adaptive=True, eps_re=10.0, tol=1e-6)


@pytest.mark.parametrize("stop,opts", [
    (1, OPTS),                                        # the held sketch is reused after the boundary
    (2, OPTS),
    (2, dict(OPTS, adaptive=False)),                  # a fixed sketch: re-sketched every iteration
    (1, dict(method="nystrom", l=8, adaptive=True, eps_re=10.0, tol=1e-6, prec="fp32")),  # FP32 operator
])
def test_resumed_run_repeats_the_uninterrupted_one(tmp_path, stop, opts):
    import paper_2401_15758_gb300 as g
    if opts.get("prec") == "fp32":
        opts = dict(opts, prec=g.FP32)
    wl = si.burgers_workload("burgers_n128")
    iters = 4
    prob, _ = make_pair(wl)
    v = torch.zeros(wl.n, dtype=torch.float64, device="cuda")
    rec_full = prob.gauss_newton(v, iters=iters, **opts)
    v_full = v.cpu().numpy()
    c_full = prob.counters()
    assert any(not r["sketched"] for r in rec_full) == bool(opts.get("adaptive"))

    # the same run through the resumable call, stopped at the boundary `stop`
    prob2, _ = make_pair(wl)
    v2 = torch.zeros(wl.n, dtype=torch.float64, device="cuda")
    rec_a, cp = prob2.gauss_newton_resume(v2, stop, **opts)
    assert cp.next_iter == stop and len(rec_a) == stop
    assert (cp.V is None) == (cp.sketch_iter < 0)
    path = tmp_path / "gn.npz"
    cp.save(path)
    del prob2

    # a fresh handle continues from the file
    prob3, _ = make_pair(wl)
    v3 = torch.zeros(wl.n, dtype=torch.float64, device="cuda")
    rec_b, cp2 = prob3.gauss_newton_resume(v3, iters, checkpoint=g.GNCheckpoint.load(path), **opts)
    assert cp2.next_iter == iters and len(rec_b) == iters
    assert np.array_equal(v3.cpu().numpy(), v_full)
    assert np.array_equal(cp2.v, v_full)
    for a, b in zip(rec_b, rec_full):
        assert a == b
    assert prob3.counters() == c_full


def test_precond_import_applies_like_the_original():
    import paper_2401_15758_gb300 as g
    wl = si.burgers_workload("burgers_n128")
    prob, _ = make_pair(wl)
    prob.fwd(torch.zeros(wl.n, dtype=torch.float64, device="cuda"))
    P = prob.build_precond("randsvd", l=12)
    V, lam = P.arrays()
    Q = prob.precond_import(V, lam)
    assert Q.rank == P.rank
    R = torch.tensor(si.gaussian_matrix(7, 3, wl.n, stream=5), device="cuda")
    assert torch.equal(Q.apply(R), P.apply(R))
    k1 = prob.kappa_estimate(P)
    k2 = prob.kappa_estimate(Q)
    assert k1 == k2
    # the empty preconditioner and bad factors
    E = prob.precond_import(np.zeros((wl.n, 0)), np.zeros(0))
    assert E.rank == 0
    assert torch.equal(E.apply(R), R)
    with pytest.raises(g.Sc4dvarError):
        prob.precond_import(V, -lam)
    with pytest.raises(g.Sc4dvarError):
        prob.precond_import(V, np.where(np.arange(lam.size) == 0, np.nan, lam))


def test_resume_rejects_inconsistent_state():
    import paper_2401_15758_gb300 as g
    wl = si.burgers_workload("burgers_n128")
    prob, _ = make_pair(wl)
    v = torch.zeros(wl.n, dtype=torch.float64, device="cuda")
    _, cp = prob.gauss_newton_resume(v, 1, **OPTS)
    bad = g.GNCheckpoint(cp.v, 5, cp.g0_inf, cp.sketch_iter, cp.V, cp.lam, cp.counters, cp.record)
    with pytest.raises(g.Sc4dvarError):
        prob.gauss_newton_resume(v, 3, checkpoint=bad, **OPTS)        # next_iter beyond iters
    with pytest.raises(g.Sc4dvarError):                                 # a held sketch with method none
        prob.gauss_newton_resume(v, 3, checkpoint=cp, **dict(OPTS, method="none"))
    wrong_size = g.GNCheckpoint(np.zeros(wl.n + 1), 1, 1.0, -1, None, None, {}, [])
    with pytest.raises(ValueError):
        prob.gauss_newton_resume(v, 3, checkpoint=wrong_size, **OPTS)
