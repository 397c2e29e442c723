"""Batched serving of uneven Burgers problems (graph-recorded batched Hessian
products and PCG steps) against the per-problem entry points."""
import dataclasses

import numpy as np
import pytest

import sc4dvar_inputs as si

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from test_gpu_burgers import rel  # noqa: E402


@pytest.fixture(scope="module")
def batch():
    import paper_2401_15758_gb300 as g
    items = si.burgers_batch(6)
    probs, wls = [], []
    for wl, d in items:
        wl = dataclasses.replace(wl, n_out=20)          # short windows keep the test quick
        d = si.burgers_draws(wl)
        p = g.Problem.from_workload(wl, d["obs_idx"])
        p.set_background(torch.tensor(d["x_true0"], device="cuda"))
        p.set_observations(torch.zeros(wl.m, dtype=torch.float64, device="cuda"))
        p.fwd(torch.zeros(wl.n, dtype=torch.float64, device="cuda"))
        probs.append(p)
        wls.append(wl)
    return g, wls, probs


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_batched_hessian_matches_per_problem(batch, prec):
    g, wls, probs = batch
    p = g.FP64 if prec == "fp64" else g.FP32
    dt = torch.float64 if prec == "fp64" else torch.float32
    tol = 1e-12 if prec == "fp64" else 1e-6
    b = g.Batch(probs)
    rng = np.random.default_rng(3)
    Xs = [torch.tensor(rng.standard_normal((min(wl.k, 8), wl.n)), device="cuda", dtype=dt) for wl in wls]
    Ys = [torch.empty_like(x) for x in Xs]
    for call in range(3):           # first call records the graph, later calls replay it
        for x in Xs:
            x.copy_(torch.randn_like(x))
        b.hessian_apply(Xs, Ys, prec=p)
        torch.cuda.synchronize()
        for pr, x, y in zip(probs, Xs, Ys):
            want = pr.gn_hessian_apply_block(x, prec=p)
            assert rel(y.double().cpu().numpy(), want.double().cpu().numpy()) <= tol, call
    b.close()


@pytest.mark.parametrize("precond", [False, True])
def test_batched_pcg_matches_per_problem(batch, precond):
    g, wls, probs = batch
    rng = np.random.default_rng(4)
    rhs = [torch.tensor(rng.standard_normal(wl.n), device="cuda") for wl in wls]
    pcs = [pr.build_precond("randsvd", l=8) for pr in probs] if precond else None
    b = g.Batch(probs)
    b.pcg_start(rhs, preconds=pcs, tol=1e-8)
    for _ in range(40):
        b.pcg_step(5)
        rel_, its, st = b.pcg_status()
        if max(rel_) <= 1e-8:
            break
    assert all(s == 0 for s in st) and max(rel_) <= 1e-8
    xs = b.pcg_solution([torch.empty_like(r) for r in rhs])
    for i, (pr, r) in enumerate(zip(probs, rhs)):
        x1, info = pr.pcg(r, None if pcs is None else pcs[i], tol=1e-8)
        assert abs(info["iterations"] - its[i]) <= 2
        assert rel(xs[i].cpu().numpy(), x1.cpu().numpy()) <= 1e-6
        res = r - pr.gn_hessian_apply_block(xs[i].reshape(1, -1)).reshape(-1)
        assert (torch.linalg.norm(res) / torch.linalg.norm(r)).item() <= 2e-8
    b.close()


def test_autotune_picks_a_valid_shape(batch):
    g, wls, probs = batch
    for wl, pr in zip(wls, probs):
        c = g.autotune(pr, 8)
        if wl.n >= 1024:
            assert c in (1, 2, 4, 8)
        else:
            assert c == 0
        x = torch.randn((3, wl.n), device="cuda", dtype=torch.float32)
        y = pr.gn_hessian_apply_block(x, prec=g.FP32)
        assert torch.isfinite(y).all()


# Problems of the 64-problem batch that cover its shapes: n from 512 to 8192,
# k from 16 to 64, one to 32 RK4 substeps per output step. Windows shortened to
# 20 output steps (up to 640 RK4 steps) so that the oracle keeps up.
C4_PICK = [27, 0, 7, 1, 4, 2, 10, 16]


@pytest.fixture(scope="module")
def c4():
    import paper_2401_15758_gb300 as g
    from oracle import workload
    items = si.burgers_batch(64)
    out = []
    for i in C4_PICK:
        wl0, d0 = items[i]
        wl = dataclasses.replace(wl0, n_out=20)
        d = si.burgers_draws(wl)
        d["obs_idx"] = ((d["obs_idx"] + int(d0["obs_idx"][0, 0]) % 8) % wl.n).astype(np.int32)
        ref = workload.burgers_problem(wl, d)
        p = g.Problem.from_workload(wl, d["obs_idx"])
        p.set_background(torch.tensor(ref.xb, device="cuda"))
        p.set_observations(torch.tensor(ref.y.reshape(-1), device="cuda"))
        v = 0.2 * np.random.default_rng(i).standard_normal(wl.n)
        ref.set_iterate(v)
        p.fwd(torch.tensor(v, device="cuda"))
        out.append((wl, p, ref))
    shapes = {(wl.n, wl.k, wl.substeps) for wl, _, _ in out}
    assert {n for n, _, _ in shapes} == {512, 1024, 2048, 4096, 8192}
    assert {k for _, k, _ in shapes} == {16, 32, 64}
    return g, out


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_batched_hessian_matches_oracle_at_batch_shapes(c4, prec):
    """The graph-replayed batched block product (each problem at its own block
    width k) against the oracle's (I + H) X on the first and last column of
    every problem: 1e-5 per column with FP32 sweeps, 1e-10 with FP64."""
    g, probs = c4
    p = g.FP64 if prec == "fp64" else g.FP32
    dt = torch.float64 if prec == "fp64" else torch.float32
    tol = 1e-10 if prec == "fp64" else 1e-5
    b = g.Batch([pr for _, pr, _ in probs])
    rng = np.random.default_rng(5)
    Xs = [torch.tensor(rng.standard_normal((wl.k, wl.n)), device="cuda", dtype=dt) for wl, _, _ in probs]
    Ys = [torch.empty_like(x) for x in Xs]
    for call in range(2):             # the first call records the graph, the second replays it
        b.hessian_apply(Xs, Ys, prec=p)
        torch.cuda.synchronize()
    for (wl, pr, ref), x, y in zip(probs, Xs, Ys):
        cols = [0, wl.k - 1]
        xs = x[cols].double().cpu().numpy()
        want = ref.hvp(xs.T).T
        got = y[cols].double().cpu().numpy()
        for j in range(2):
            assert rel(got[j], want[j]) <= tol, (wl.n, wl.k, cols[j], rel(got[j], want[j]))
    b.close()


def test_batched_pcg_solutions_meet_the_oracle_residual(c4):
    """Batched PCG (one graph launch advances every problem by an iteration;
    FP64 operator) to 1e-9: each solution's residual b - (I + H) x, evaluated with
    the oracle's Hessian product, is below 1e-8 |b|."""
    g, probs = c4
    rng = np.random.default_rng(6)
    rhs = [rng.standard_normal(wl.n) for wl, _, _ in probs]
    b = g.Batch([pr for _, pr, _ in probs])
    b.pcg_start([torch.tensor(r, device="cuda") for r in rhs], None, tol=1e-9)
    for _ in range(60):
        b.pcg_step(5)
        rel_, its, st = b.pcg_status()
        if max(rel_) <= 1e-9:
            break
    assert all(s == 0 for s in st) and max(rel_) <= 1e-9
    xs = b.pcg_solution([torch.empty(wl.n, dtype=torch.float64, device="cuda") for wl, _, _ in probs])
    for (wl, pr, ref), r, x in zip(probs, rhs, xs):
        res = r - ref.hvp(x.cpu().numpy())
        assert np.linalg.norm(res) <= 1e-8 * np.linalg.norm(r), wl.n
    b.close()
