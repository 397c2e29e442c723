"""Parity of the benchmarked Burgers block with the FP64 oracle over the whole
window: n = 8192, 400 output steps of 32 RK4 substeps (12 800 RK4 steps),
m = 40 960 observations, a block of k = 128 FP32 directions in the launch
configuration of the timed step (the bench's X, one CTA per direction, packed
FP32x2 sweeps). The oracle computes two sampled columns (the first and the
last CTA of the launch); FP32 results are held to 1e-5 relative per column,
and one column through the FP64 and the double-float (DF64) paths to 1e-10.
"""
import numpy as np
import pytest

import sc4dvar_inputs as si

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from test_gpu_burgers import make_pair, rel  # noqa: E402

K = 128
COLS = [0, K - 1]


@pytest.fixture(scope="module")
def full():
    wl = si.burgers_workload("burgers_n8192")
    assert wl.n == 8192 and wl.n_steps == 12800 and wl.m == 40960
    prob, ref = make_pair(wl)
    Jr = ref.set_iterate(np.zeros(wl.n))
    Jg = prob.fwd(torch.zeros(wl.n, dtype=torch.float64, device="cuda"))
    X = si.gaussian_matrix(wl.seed, K, wl.n, stream=21)       # the timed step's directions
    Xs = X[COLS].T.astype(np.float32).astype(np.float64)      # the FP32 inputs, exactly
    Wr = ref.A(Xs)                                             # A X       (m, 2)
    Zr = ref.At(Wr)                                            # A^T A X   (n, 2)
    gr = ref.gradient()
    return wl, prob, ref, X, Wr, Zr, Jr, Jg, gr


def test_full_window_cost_and_gradient(full):
    wl, prob, ref, X, Wr, Zr, Jr, Jg, gr = full
    assert abs(Jg - Jr) <= 1e-10 * abs(Jr)
    assert rel(prob.gradient().cpu().numpy(), gr) <= 1e-10


def test_full_window_fp32_block_k128(full):
    import paper_2401_15758_gb300 as g
    wl, prob, ref, X, Wr, Zr, Jr, Jg, gr = full
    X32 = torch.tensor(X, device="cuda", dtype=torch.float32)
    A = prob.tlm_block(X32, prec=g.FP32)
    # A^T W in the same k = 128 launch: the sampled rows carry the oracle's A X
    Win = A.clone()
    Win[COLS] = torch.tensor(Wr.T, device="cuda", dtype=torch.float32)
    At = prob.adj_block(Win, prec=g.FP32).double().cpu().numpy()
    H = prob.gn_hessian_apply_block(X32, prec=g.FP32).double().cpu().numpy()
    A = A.double().cpu().numpy()
    Xs = X[COLS].T.astype(np.float32).astype(np.float64)
    for j, c in enumerate(COLS):
        ea = rel(A[c], Wr[:, j])
        et = rel(At[c], Zr[:, j])
        eh = rel(H[c], Xs[:, j] + Zr[:, j])
        assert ea <= 1e-5, (c, ea)
        assert et <= 1e-5, (c, et)
        assert eh <= 1e-5, (c, eh)


@pytest.mark.parametrize("prec", ["fp64", "df64"])
def test_full_window_fp64_class_column(full, prec):
    import paper_2401_15758_gb300 as g
    wl, prob, ref, X, Wr, Zr, Jr, Jg, gr = full
    p = g.FP64 if prec == "fp64" else g.DF64
    x = X[COLS[0]].astype(np.float32).astype(np.float64)
    H = prob.gn_hessian_apply_block(torch.tensor(x[None, :], device="cuda"), prec=p).cpu().numpy()
    assert rel(H[0], x + Zr[:, 0]) <= 1e-10
