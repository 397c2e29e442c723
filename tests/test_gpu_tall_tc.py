"""The sketches' tall product C = alpha A op(B) + beta C on the tensor cores
(tcgen05 MMAs accumulating in tensor memory) against numpy FP64, through the C
ABI: ragged sizes (rows not a multiple of the 128-row tile, K not a multiple of
the 32-wide chunk, columns not a multiple of 16 and more than one 256-column
tile), the transposed factor, beta != 0 and FP64 output. Tolerances follow the
arithmetic: 3xTF32 and CUDA-core FP32 at FP32 accuracy, TF32 and BF16 at the
accuracy of their input roundings (2^-11 and 2^-8, growing like sqrt(K))."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = {0: 2e-6, 1: 2e-6, 2: 2e-3, 3: 2e-2}   # GEMM_3XTF32, GEMM_SIMT, GEMM_TF32, GEMM_BF16


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("mode", [0, 1, 2, 3])
@pytest.mark.parametrize("rows,kk,c,transB,beta,out64", [
    (300, 40, 24, False, 0.0, False),     # ragged in every dimension, one column tile
    (1000, 128, 300, True, 0.0, False),   # two column tiles, transposed factor
    (257, 7, 17, False, -1.0, False),     # K below one instruction, beta = -1 (a Gram-Schmidt update)
    (513, 96, 64, False, 0.0, True),      # FP64 output (the thin SVD's V)
])
def test_tall_product_matches_fp64(mode, rows, kk, c, transB, beta, out64):
    import paper_2401_15758_gb300 as g
    rng = np.random.default_rng(rows + kk + c)
    A = rng.standard_normal((kk, rows)).astype(np.float32)          # column-major rows x kk
    B = rng.standard_normal((kk, c) if transB else (c, kk))         # op(B) = kk x c
    C0 = rng.standard_normal((c, rows))
    dt = torch.float64 if out64 else torch.float32
    Cd = torch.tensor(C0, device="cuda", dtype=dt)
    out = g.tall_gemm(torch.tensor(A, device="cuda"), torch.tensor(B, device="cuda"), mode=mode,
                      transB=transB, alpha=1.5, beta=beta, C=Cd)
    opB = B if transB else B.T                                       # kk x c
    c_in = C0 if out64 else C0.astype(np.float32).astype(np.float64)  # C as the device held it
    want = 1.5 * (A.T.astype(np.float64) @ opB) + beta * c_in.T
    assert rel(out.double().cpu().numpy().T, want) <= TOL[mode]


def test_tall_product_at_the_sketch_shape():
    """Q = Y R^{-1} of the n = 8192 workload's sketch: 40 960 x 128 times 128 x 128."""
    import paper_2401_15758_gb300 as g
    rng = np.random.default_rng(9)
    Y = rng.standard_normal((128, 40960)).astype(np.float32)
    R = np.triu(rng.standard_normal((128, 128))) + 10 * np.eye(128)
    out = g.tall_gemm(torch.tensor(Y, device="cuda"), torch.tensor(R, device="cuda"), mode=g.GEMM_3XTF32)
    want = Y.T.astype(np.float64) @ R.T
    assert rel(out.double().cpu().numpy().T, want) <= 2e-6


def test_tall_product_rejects_a_bad_mode():
    import paper_2401_15758_gb300 as g
    z = torch.zeros((4, 8), dtype=torch.float32, device="cuda")
    b = torch.zeros((4, 4), dtype=torch.float64, device="cuda")
    with pytest.raises(g.Sc4dvarError) as e:
        g.tall_gemm(z, b, mode=7)
    assert e.value.code == g._abi.ERR_INVALID_ARG
