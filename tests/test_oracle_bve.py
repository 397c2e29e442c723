"""Pins of the oracle's barotropic vorticity model (closed forms, invariants,
dense transposes, finite differences)."""
import numpy as np
import pytest

from oracle import bve, rk4


def mode(N, kx, ky, phase=0.3):
    d = 2 * np.pi / N
    x = np.arange(N) * d
    X, Y = np.meshgrid(x, x, indexing="xy")   # X[j, i] = x_i, Y[j, i] = y_j
    return np.cos(kx * X + ky * Y + phase).reshape(-1)


@pytest.mark.parametrize("kx,ky", [(1, 0), (2, 3), (-4, 5), (7, 7)])
def test_poisson_exact_on_fourier_modes(kx, ky):
    m = bve.BVE2D(32, 1e-3)
    q = mode(32, kx, ky)
    assert np.allclose(m.poisson(q), -q / (kx ** 2 + ky ** 2), atol=1e-13)
    assert np.allclose(m.poisson(np.ones(m.n)), 0.0, atol=1e-14)   # mean mode removed


@pytest.mark.parametrize("kx,ky", [(1, 2), (5, -3)])
def test_five_point_laplacian_eigenvalue(kx, ky):
    N = 24
    m = bve.BVE2D(N, 1e-3)
    q = mode(N, kx, ky)
    d = m.d
    lam = -(4 / d ** 2) * (np.sin(kx * d / 2) ** 2 + np.sin(ky * d / 2) ** 2)
    assert np.allclose(m.lap_h(q), lam * q, atol=1e-10)


def test_arakawa_invariants():
    m = bve.BVE2D(20, 1e-3)
    rng = np.random.default_rng(0)
    a, b = rng.standard_normal(m.n), rng.standard_normal(m.n)
    J = m.jacobian(a, b)
    s = np.abs(J).sum()
    assert np.allclose(J, -m.jacobian(b, a), atol=1e-12 * s)      # antisymmetry
    assert abs(J.sum()) < 1e-12 * s                               # vorticity
    assert abs(a @ J) < 1e-11 * s * np.abs(a).max()               # energy
    assert abs(b @ J) < 1e-11 * s * np.abs(b).max()               # enstrophy
    assert np.allclose(m.jacobian(a, 2.5 * a), 0.0, atol=1e-12 * s)


def test_arakawa_second_order_convergence():
    errs = []
    for N in (32, 64, 128):
        m = bve.BVE2D(N, 0.0)
        d = m.d
        x = np.arange(N) * d
        X, Y = np.meshgrid(x, x, indexing="xy")
        a = np.sin(X) * np.cos(2 * Y)
        b = np.cos(3 * X + Y)
        ax, ay = np.cos(X) * np.cos(2 * Y), -2 * np.sin(X) * np.sin(2 * Y)
        bx, by = -3 * np.sin(3 * X + Y), -np.sin(3 * X + Y)
        exact = ax * by - ay * bx
        errs.append(np.max(np.abs(m.jacobian(a.reshape(-1), b.reshape(-1)) - exact.reshape(-1))))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 1.9) and np.all(rates < 2.2), rates


def test_forced_single_mode_is_exact_rk4():
    """q = A sin(4y): psi is proportional to q so J_A(psi, q) = 0 and the model reduces
    to the affine ODE A' = -nu lam A + 1 per step; RK4's step on it is
    A' = G(z) A + h P(z), z = -nu lam h, G = 1+z+z^2/2+z^3/6+z^4/24, P = 1+z/2+z^2/6+z^3/24."""
    N, nu, h = 32, 0.05, 0.01
    m = bve.BVE2D(N, nu, forcing_amp=1.0, forcing_k=4)
    d = m.d
    y = (np.arange(N) * d)[:, None] * np.ones((1, N))
    s4 = np.sin(4 * y).reshape(-1)
    lam = (4 / d ** 2) * np.sin(4 * d / 2) ** 2
    z = -nu * lam * h
    G = 1 + z + z ** 2 / 2 + z ** 3 / 6 + z ** 4 / 24
    Pz = 1 + z / 2 + z ** 2 / 6 + z ** 3 / 24
    A = 0.3
    q = A * s4
    for _ in range(15):
        q = rk4.fwd_step(m, q, h)
        A = G * A + h * Pz
    assert np.allclose(q, A * s4, atol=1e-13)


def test_jacobian_dense_matches_fd_and_transpose():
    N = 8
    m = bve.BVE2D(N, 0.02)
    rng = np.random.default_rng(1)
    U = rng.standard_normal(m.n)
    Jd = m.dense(lambda e: m.jvp(U, e))
    eps = 1e-6
    Jfd = m.dense(lambda e: (m.rhs(U + eps * e) - m.rhs(U - eps * e)) / (2 * eps))
    assert np.max(np.abs(Jd - Jfd)) < 1e-7 * np.max(np.abs(Jd))
    JTd = m.dense(lambda e: m.vjp(U, e))
    assert np.max(np.abs(JTd - Jd.T)) < 1e-12 * np.max(np.abs(Jd))
    X = rng.standard_normal((m.n, 3))
    assert np.allclose(m.jvp(U, X), Jd @ X, atol=1e-11)
    assert np.allclose(m.vjp(U, X), Jd.T @ X, atol=1e-11)


def test_inv_helmholtz_prior_symbol():
    N = 16
    c, ell = 0.2, 0.5
    sym = bve.inv_helmholtz_sqrt_symbol(N, c, ell)
    S = bve.apply_symbol_2d(sym, np.eye(N * N), N)
    assert np.allclose(S, S.T, atol=1e-15)
    # (I - ell^2 Lap) S = c I with the spectral Laplacian (Lap of a mode = -|kappa|^2)
    m = bve.BVE2D(N, 0.0)
    lap_spec = lambda X: -bve.apply_symbol_2d(m.K2, X, N)
    assert np.allclose(S - ell ** 2 * lap_spec(S), c * np.eye(N * N), atol=1e-12)


def test_bve_problem_adjoint_and_fd():
    import sc4dvar_inputs as si
    from oracle import workload
    wl = si.bve_workload("bve_n256", N=16, n_steps=12, obs_every=4)
    p = workload.bve_problem(wl, si.bve_draws(wl))
    p.set_iterate(np.zeros(wl.n))
    rng = np.random.default_rng(2)
    X = rng.standard_normal((wl.n, 2))
    W = rng.standard_normal((wl.m, 2))
    a, b = np.sum(p.A(X) * W), np.sum(X * p.At(W))
    assert abs(a - b) <= 1e-12 * abs(a)
    dx = rng.standard_normal(wl.n)
    tl = p.tlm_obs(dx)
    errs = []
    for eps in (1e-2, 1e-3, 1e-4):
        fp = p.observe(p.forward(p.x0 + eps * dx)).reshape(-1) / p.sigma
        fm = p.observe(p.forward(p.x0 - eps * dx)).reshape(-1) / p.sigma
        errs.append(np.linalg.norm((fp - fm) / (2 * eps) - tl) / np.linalg.norm(tl))
    assert errs[1] / errs[2] > 50 and errs[2] < 1e-7, errs
