"""Pins of the oracle's model layer: Philox, RK4, Burgers, prior, A / A^T, gradient.

Every check compares the oracle with something other than itself: published
test vectors, closed-form RK4 amplification factors, dense matrices assembled
entry by entry, finite differences, or conservation laws of the discretization.
"""
import os

import numpy as np
import pytest

from oracle import burgers, philox, prior, rk4

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _kat_rows():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([int(w, 16) for w in line.split()])
    return rows


@pytest.mark.parametrize("row", _kat_rows())
def test_philox_known_answers(row):
    ctr, key, want = row[:4], row[4:6], row[6:]
    got = philox.philox4x32_10(np.array(ctr, dtype=np.uint64), key)
    assert [int(x) for x in got] == want


def test_gaussian_stream_layout_and_moments():
    g = philox.gaussian(7, 123, 1001, 40)
    # columns are a window of one infinite column-major stream
    g2 = philox.gaussian(7, 123, 1001, 15, col0=25)
    assert np.array_equal(g[:, 25:], g2)
    # distinct streams and seeds differ
    assert not np.allclose(philox.gaussian(7, 124, 1001, 1), g[:, :1])
    assert not np.allclose(philox.gaussian(8, 123, 1001, 1), g[:, :1])
    x = g.ravel()
    assert abs(x.mean()) < 4.0 / np.sqrt(x.size)
    assert abs(x.var() - 1.0) < 6.0 * np.sqrt(2.0 / x.size)
    from scipy import stats
    assert stats.kstest(x, "norm").pvalue > 1e-3


class _Linear:
    """x' = L x, a linear test model (rhs = jvp = L, vjp = L^T)."""

    def __init__(self, L):
        self.L = L
        self.n = L.shape[0]

    def rhs(self, u):
        return self.L @ u

    def jvp(self, U, d):
        return self.L @ d

    def vjp(self, U, w):
        return self.L.T @ w


def test_rk4_tableau_matches_taylor_polynomial():
    rng = np.random.default_rng(1)
    L = rng.standard_normal((6, 6))
    h = 0.07
    x = rng.standard_normal(6)
    Z = h * L
    G = np.eye(6) + Z + Z @ Z / 2 + Z @ Z @ Z / 6 + Z @ Z @ Z @ Z / 24
    m = _Linear(L)
    assert np.allclose(rk4.fwd_step(m, x, h), G @ x, rtol=1e-14, atol=1e-14)
    assert np.allclose(rk4.tlm_step(m, x, x, h), G @ x, rtol=1e-14, atol=1e-14)
    assert np.allclose(rk4.adj_step(m, x, x, h), G.T @ x, rtol=1e-14, atol=1e-14)


def test_burgers_jacobian_dense_is_fd_of_rhs():
    n = 12
    m = burgers.Burgers1D(n, 0.03)
    rng = np.random.default_rng(2)
    U = rng.standard_normal(n)
    J = m.jacobian_dense(U)
    eps = 1e-6
    Jfd = np.stack([(m.rhs(U + eps * e) - m.rhs(U - eps * e)) / (2 * eps) for e in np.eye(n)], axis=1)
    assert np.max(np.abs(J - Jfd)) < 1e-6 * np.max(np.abs(J))
    d = rng.standard_normal((n, 3))
    assert np.allclose(m.jvp(U, d), J @ d, rtol=1e-13, atol=1e-12)
    assert np.allclose(m.vjp(U, d), J.T @ d, rtol=1e-13, atol=1e-12)


def test_burgers_rhs_second_order_consistent():
    nu = 0.02
    errs = []
    for n in (64, 128, 256):
        m = burgers.Burgers1D(n, nu)
        x = np.arange(n) / n
        u = np.sin(2 * np.pi * x)
        exact = -u * 2 * np.pi * np.cos(2 * np.pi * x) - nu * 4 * np.pi ** 2 * u
        errs.append(np.max(np.abs(m.rhs(u) - exact)))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 1.9) and np.all(rates < 2.1)


def test_burgers_conserves_mean_and_constants():
    m = burgers.Burgers1D(64, 0.01)
    rng = np.random.default_rng(3)
    u = np.sin(2 * np.pi * np.arange(64) / 64) + 0.3 * rng.standard_normal(64)
    assert abs(np.sum(m.rhs(u))) < 1e-12 * np.sum(np.abs(m.rhs(u)))
    u1 = rk4.fwd_step(m, u, 1e-3)
    assert abs(u1.sum() - u.sum()) < 1e-12
    c = np.full(64, 0.7)
    assert np.array_equal(rk4.fwd_step(m, c, 1e-3), c)


@pytest.mark.parametrize("kappa", [1, 3, 7])
def test_tlm_about_constant_state_is_exact_advection_diffusion(kappa):
    """Linearized about a constant U the TLM is RK4 applied to -U D1 + nu D2; on a
    Fourier mode the step multiplies by G(z), z = h(-i U sin(2 pi k/n)/dx - 4 nu
    sin^2(pi k/n)/dx^2), G(z) = 1 + z + z^2/2 + z^3/6 + z^4/24. This fixes the sign
    and size of both the advection and the diffusion terms."""
    n, nu, U, h, N = 32, 0.02, 0.8, 2e-3, 25
    m = burgers.Burgers1D(n, nu)
    dx = 1.0 / n
    j = np.arange(n)
    lam = -1j * U * np.sin(2 * np.pi * kappa / n) / dx - 4 * nu * np.sin(np.pi * kappa / n) ** 2 / dx ** 2
    z = h * lam
    G = 1 + z + z ** 2 / 2 + z ** 3 / 6 + z ** 4 / 24
    phi = np.exp(2j * np.pi * kappa * j / n)
    base = np.full(n, U)
    d = np.real(phi)
    for _ in range(N):
        d = rk4.tlm_step(m, base, d, h)
    assert np.allclose(d, np.real(G ** N * phi), rtol=0, atol=1e-13)


def test_se_prior_square_root_squares_to_covariance():
    """(Gamma^{1/2})^2 equals the dense SE covariance (its PSD part, with the same
    relative clamp, obtained through a dense symmetric eigensolver, not the FFT)."""
    for n, L in ((64, 0.05), (96, 0.1), (128, 0.05)):
        sym = prior.se_sqrt_symbol(n, 0.1, L)
        S = prior.apply_symbol(sym, np.eye(n))
        C = prior.se_covariance_dense(n, 0.1, L)
        w, Q = np.linalg.eigh(C)
        w = np.where(w < prior.CLAMP_REL * w.max(), 0.0, w)
        Cp = (Q * w) @ Q.T
        assert np.allclose(S, S.T, atol=1e-15)
        assert np.max(np.abs(S @ S - Cp)) < 1e-12 * np.max(np.abs(C))
        if L == 0.05:      # wrap-around negligible: the kernel itself is PSD to round-off
            assert np.max(np.abs(S @ S - C)) < 1e-9 * np.max(np.abs(C))


def test_tlm_matches_central_differences_of_fwd(tiny_prob):
    p = tiny_prob
    rng = np.random.default_rng(4)
    dx = rng.standard_normal(p.n)
    x0 = p.x0
    tl = p.tlm_obs(dx)
    errs = []
    epss = [1e-2, 1e-3, 1e-4, 1e-5]
    for eps in epss:
        fp = p.observe(p.forward(x0 + eps * dx)).reshape(-1) / p.sigma
        fm = p.observe(p.forward(x0 - eps * dx)).reshape(-1) / p.sigma
        errs.append(np.linalg.norm((fp - fm) / (2 * eps) - tl) / np.linalg.norm(tl))
    slopes = np.log10(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(slopes > 1.8), (errs, slopes)
    assert errs[-1] < 1e-8


def test_adjoint_dot_product(tiny_prob):
    p = tiny_prob
    rng = np.random.default_rng(5)
    X = rng.standard_normal((p.n, 4))
    W = rng.standard_normal((p.m, 4))
    a = np.sum(p.A(X) * W)
    b = np.sum(X * p.At(W))
    assert abs(a - b) <= 1e-12 * abs(a)


def test_assembled_adjoint_is_transpose(tiny_dense):
    A, At = tiny_dense["A"], tiny_dense["At"]
    assert A.shape == At.T.shape
    assert np.max(np.abs(At - A.T)) <= 1e-12 * np.max(np.abs(A))


def test_hessian_symmetric_spd(tiny_prob, tiny_dense):
    p = tiny_prob
    Hx = np.stack([p.hvp(e) for e in np.eye(p.n)], axis=1)
    assert np.max(np.abs(Hx - Hx.T)) <= 1e-12 * np.max(np.abs(Hx))
    assert np.allclose(Hx, np.eye(p.n) + tiny_dense["H"], rtol=1e-12, atol=1e-12)
    assert np.linalg.eigvalsh(0.5 * (Hx + Hx.T)).min() >= 1.0 - 1e-10


def test_gradient_matches_finite_differences(tiny_prob):
    p = tiny_prob
    rng = np.random.default_rng(6)
    v = 0.1 * rng.standard_normal(p.n)
    p.set_iterate(v)
    g = p.gradient()
    for _ in range(3):
        dvec = rng.standard_normal(p.n)
        eps = 1e-5
        Jp = p.set_iterate(v + eps * dvec)
        Jm = p.set_iterate(v - eps * dvec)
        fd = (Jp - Jm) / (2 * eps)
        assert abs(fd - g @ dvec) <= 1e-7 * max(1.0, abs(fd))
    p.set_iterate(np.zeros(p.n))
