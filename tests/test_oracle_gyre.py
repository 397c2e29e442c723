"""Pins of the oracle's double-gyre barotropic vorticity set-up (Sec. 5.2).

* Sine modes sin(p pi i/(nx+1)) sin(q pi j/(ny+1)) are eigenvectors of the
  five-point Delta* with eigenvalue -4 sin^2(p pi/(2(nx+1))) - 4 sin^2(q pi/(2(ny+1))):
  the Laplacian, the Poisson solve and the prior (a I - b Delta*)^{-1} must act on
  them by exactly those numbers.
* The discrete right-hand side converges at second order to the continuous
  -J(psi, omega) + Ro^{-1} psi_x + Re^{-1} Lap omega + Ro^{-1} sin(pi y) for a
  stream function psi = sin(pi x) sin(pi y) + 0.4 sin(2 pi x) sin(3 pi y) with
  omega = -Lap psi (both vanish on the boundary); the continuous value is
  written out by hand from the derivatives of the two modes. Two distinct modes
  make J(psi, omega) nonzero, so a flipped sign or swapped argument of J, a
  wrong sign of the beta term or of the Poisson solve fails.
* The Jacobian matches central differences of the rhs; vjp is its transpose.
* The 4D-Var problem: adjoint dot test and the gradient against differences of J.
"""
import numpy as np
import pytest

from oracle import bve_gyre, fourdvar, rk4


def _mode(m, p, q):
    gx = np.sin(p * np.pi * np.arange(1, m.nx + 1) / (m.nx + 1))
    gy = np.sin(q * np.pi * np.arange(1, m.ny + 1) / (m.ny + 1))
    return (gy[:, None] * gx[None, :]).reshape(-1)


def _mu(m, p, q):
    return 4 * np.sin(p * np.pi / (2 * (m.nx + 1))) ** 2 + 4 * np.sin(q * np.pi / (2 * (m.ny + 1))) ** 2


@pytest.mark.parametrize("p,q", [(1, 1), (3, 7), (8, 17)])
def test_sine_modes_laplacian_poisson_prior(p, q):
    m = bve_gyre.BVEGyre(8, 200.0, 0.0016)
    f = _mode(m, p, q)
    mu = _mu(m, p, q)
    assert np.allclose(m.lap(f), -mu / m.h ** 2 * f, rtol=1e-12, atol=1e-9)
    assert np.allclose(m.poisson(f), m.h ** 2 / mu * f, rtol=1e-12, atol=1e-14)
    a, b = 0.3, 0.06
    psq = bve_gyre.inv_helmholtz_sqrt_2d(8, a, b)
    assert np.allclose(psq(f), f / (a + b * mu), rtol=1e-12, atol=1e-12)


def test_prior_matches_dense_definition():
    nx, ny = 4, 9
    L = bve_gyre.dirichlet_laplacian_2d(nx, ny).toarray()
    # the dense five-point matrix written entry by entry
    D = np.zeros((nx * ny, nx * ny))
    for j in range(ny):
        for i in range(nx):
            r = j * nx + i
            D[r, r] = -4.0
            for di, dj in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                ii, jj = i + di, j + dj
                if 0 <= ii < nx and 0 <= jj < ny:
                    D[r, jj * nx + ii] = 1.0
    assert np.array_equal(L, D)
    X = np.random.default_rng(2).standard_normal((nx * ny, 3))
    psq = bve_gyre.inv_helmholtz_sqrt_2d(nx, 0.0, 0.06)
    assert np.allclose(psq(X), np.linalg.solve(-0.06 * D, X), rtol=1e-12, atol=1e-12)


def _continuous_rhs(x, y, re, ro):
    """-J(psi, omega) + psi_x / ro + Lap omega / re + sin(pi y) / ro for
    psi = s1 + c s2, s1 = sin(pi x) sin(pi y), s2 = sin(2 pi x) sin(3 pi y),
    omega = -Lap psi = 2 pi^2 s1 + 13 pi^2 c s2."""
    c, pi = 0.4, np.pi
    s1 = np.sin(pi * x) * np.sin(pi * y)
    s1x = pi * np.cos(pi * x) * np.sin(pi * y)
    s1y = pi * np.sin(pi * x) * np.cos(pi * y)
    s2 = np.sin(2 * pi * x) * np.sin(3 * pi * y)
    s2x = 2 * pi * np.cos(2 * pi * x) * np.sin(3 * pi * y)
    s2y = 3 * pi * np.sin(2 * pi * x) * np.cos(3 * pi * y)
    psi_x, psi_y = s1x + c * s2x, s1y + c * s2y
    om_x = 2 * pi ** 2 * s1x + 13 * pi ** 2 * c * s2x
    om_y = 2 * pi ** 2 * s1y + 13 * pi ** 2 * c * s2y
    lap_om = -(2 * pi ** 2) ** 2 * s1 - (13 * pi ** 2) ** 2 * c * s2
    J = psi_y * om_x - psi_x * om_y
    omega = 2 * pi ** 2 * s1 + 13 * pi ** 2 * c * s2
    return omega, -J + psi_x / ro + lap_om / re + np.sin(pi * y) / ro


def test_rhs_second_order_consistency():
    errs = []
    for nx in (16, 32, 64):
        m = bve_gyre.BVEGyre(nx, 200.0, 0.0016)
        X, Y = np.meshgrid(m.x, m.y)
        omega, exact = _continuous_rhs(X.reshape(-1), Y.reshape(-1), 200.0, 0.0016)
        errs.append(np.max(np.abs(m.rhs(omega) - exact)) / np.max(np.abs(exact)))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert errs[-1] < 1e-2
    assert np.all(rates > 1.8), (errs, rates)


def test_jacobian_and_transpose():
    m = bve_gyre.BVEGyre(4, 200.0, 0.0016)
    rng = np.random.default_rng(4)
    U = 50.0 * rng.standard_normal(m.n)
    Jd = m.jacobian_dense(U)
    eps = 1e-4
    fd = np.stack([(m.rhs(U + eps * e) - m.rhs(U - eps * e)) / (2 * eps) for e in np.eye(m.n)], axis=1)
    assert np.max(np.abs(Jd - fd)) <= 1e-6 * np.max(np.abs(Jd))
    W = rng.standard_normal((m.n, 3))
    assert np.allclose(m.vjp(U, W), Jd.T @ W, rtol=1e-11, atol=1e-9 * np.max(np.abs(Jd)))
    assert np.allclose(m.jvp(U, W), Jd @ W, rtol=1e-11, atol=1e-9 * np.max(np.abs(Jd)))


@pytest.fixture(scope="module")
def small_gyre():
    import sc4dvar_inputs as si
    from oracle import workload
    wl = si.gyre_workload(nx=8, obs_every=2, n_obs_times=3, n_sensors=3, spin_steps=50)
    return wl, workload.gyre_problem(wl, si.gyre_draws(wl))


def test_gyre_dot_test_and_gradient(small_gyre):
    wl, prob = small_gyre
    rng = np.random.default_rng(7)
    v = 0.5 * rng.standard_normal(wl.n)
    J = prob.set_iterate(v)
    x = rng.standard_normal((wl.n, 2))
    w = rng.standard_normal((wl.m, 2))
    lhs = np.sum(prob.A(x) * w)
    rhs = np.sum(x * prob.At(w))
    assert abs(lhs - rhs) <= 1e-11 * abs(lhs)
    g = prob.gradient()
    p = rng.standard_normal(wl.n)
    eps = 1e-5
    fd = (prob.set_iterate(v + eps * p) - prob.set_iterate(v - eps * p)) / (2 * eps)
    assert abs(fd - g @ p) <= 1e-6 * abs(fd)
    assert J > 0


def test_gyre_rk3_steps_are_transposes(small_gyre):
    wl, prob = small_gyre
    m = prob.model
    rng = np.random.default_rng(9)
    x = 50.0 * rng.standard_normal(wl.n)
    d = rng.standard_normal(wl.n)
    lam = rng.standard_normal(wl.n)
    a = lam @ rk4.tlm_step(m, x, d, wl.dt, rk4.RK3_TVD)
    b = d @ rk4.adj_step(m, x, lam, wl.dt, rk4.RK3_TVD)
    assert abs(a - b) <= 1e-12 * max(abs(a), 1.0)


def test_gyre_workload_shape():
    import sc4dvar_inputs as si
    wl = si.gyre_workload()
    d = si.gyre_draws(wl)
    assert (wl.nx, wl.ny, wl.n, wl.m, wl.n_steps) == (128, 257, 32896, 2048, 40)
    assert abs(wl.h - 0.0078) < 1e-4                      # the paper's grid spacing
    assert abs(wl.obs_every * wl.dt - 0.001225) < 1e-12    # six-hour observation interval
    sites = d["obs_idx"][0]
    assert len(set(sites.tolist())) == 256
    # the sensor grid is symmetric about the basin centre
    jy, ix = sites // wl.nx, sites % wl.nx
    assert set((wl.ny - 1 - jy).tolist()) == set(jy.tolist())
    assert set((wl.nx - 1 - ix).tolist()) == set(ix.tolist())
