"""Pins of the oracle's Dirichlet / RK3-TVD Burgers set-up (Sec. 5.1).

* RK3-TVD tableau: on a linear model one step is exactly the cubic Taylor
  polynomial of hL; its TLM step is the same matrix and its ADJ step the
  transpose.
* About the zero state the Dirichlet model is nu D2, whose eigenvectors are the
  sine modes sin(k pi x_j) with eigenvalue -4 sin^2(k pi / (2 (n+1))) / dx^2, so
  one TLM step multiplies a mode by exactly 1 + z + z^2/2 + z^3/6.
* The rhs is second-order consistent with -u u_x + nu u_xx on sin(pi x).
* The Jacobian assembled entry by entry matches central differences of the rhs,
  and vjp is its transpose.
* The prior (a I - b Delta*)^{-1} has the sine modes as eigenvectors with
  eigenvalue 1 / (a + 4 b sin^2(k pi / (2 (n+1)))).
* The 4D-Var problem: adjoint dot test and the gradient against differences of J.
"""
import numpy as np
import pytest

from oracle import burgers_dirichlet as bd
from oracle import rk4


class _Linear:
    def __init__(self, L):
        self.L = L
        self.n = L.shape[0]

    def rhs(self, u):
        return self.L @ u

    def jvp(self, U, d):
        return self.L @ d

    def vjp(self, U, w):
        return self.L.T @ w


def test_rk3_tvd_is_cubic_taylor():
    rng = np.random.default_rng(2)
    L = rng.standard_normal((5, 5))
    h = 0.05
    Z = h * L
    G = np.eye(5) + Z + Z @ Z / 2 + Z @ Z @ Z / 6
    x = rng.standard_normal(5)
    m = _Linear(L)
    tab = rk4.RK3_TVD
    assert np.allclose(rk4.fwd_step(m, x, h, tab), G @ x, rtol=1e-14, atol=1e-14)
    assert np.allclose(rk4.tlm_step(m, x, x, h, tab), G @ x, rtol=1e-14, atol=1e-14)
    assert np.allclose(rk4.adj_step(m, x, x, h, tab), G.T @ x, rtol=1e-14, atol=1e-14)


@pytest.mark.parametrize("k", [1, 3, 10])
def test_sine_mode_amplification(k):
    n, nu, h = 63, 0.1, 2.5e-5 * 4
    m = bd.BurgersDirichlet(n, nu)
    mode = np.sin(k * np.pi * m.x)
    z = h * nu * (-4.0 * np.sin(k * np.pi / (2 * (n + 1))) ** 2 / m.dx ** 2)
    G = 1 + z + z * z / 2 + z ** 3 / 6
    out = rk4.tlm_step(m, np.zeros(n), mode, h, rk4.RK3_TVD)
    assert np.allclose(out, G * mode, rtol=1e-13, atol=1e-15)


def test_rhs_second_order_consistency():
    errs = []
    for n in (63, 127, 255):
        m = bd.BurgersDirichlet(n, 0.1)
        u = np.sin(np.pi * m.x)
        exact = -u * np.pi * np.cos(np.pi * m.x) - 0.1 * np.pi ** 2 * u
        errs.append(np.max(np.abs(m.rhs(u) - exact)))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 1.9)


def test_jacobian_and_transpose():
    m = bd.BurgersDirichlet(15, 0.1)
    rng = np.random.default_rng(4)
    U = rng.standard_normal(15)
    Jd = m.jacobian_dense(U)
    eps = 1e-6
    fd = np.stack([(m.rhs(U + eps * e) - m.rhs(U - eps * e)) / (2 * eps) for e in np.eye(15)], axis=1)
    assert np.max(np.abs(Jd - fd)) <= 1e-6 * np.max(np.abs(Jd))
    W = rng.standard_normal((15, 3))
    assert np.allclose(m.vjp(U, W), Jd.T @ W, rtol=1e-12, atol=1e-12)
    assert np.allclose(m.jvp(U, W), Jd @ W, rtol=1e-12, atol=1e-12)


def test_prior_sine_mode_eigenvalues():
    n, a, b = 40, 0.5, 500.0
    psq = bd.inv_helmholtz_sqrt(n, a, b)
    x = np.arange(1, n + 1) / (n + 1)
    for k in (1, 7, 40):
        mode = np.sin(k * np.pi * x)
        lam = 1.0 / (a + 4.0 * b * np.sin(k * np.pi / (2 * (n + 1))) ** 2)
        assert np.allclose(psq(mode), lam * mode, rtol=1e-12, atol=1e-14)
    # the dense definition
    T = a * np.eye(n) - b * bd.dirichlet_laplacian(n)
    X = np.random.default_rng(1).standard_normal((n, 3))
    assert np.allclose(psq(X), np.linalg.solve(T, X), rtol=1e-12, atol=1e-14)


@pytest.fixture(scope="module")
def small_paper():
    import sc4dvar_inputs as si
    from oracle import workload
    wl = si.paper_burgers_workload(n=31, obs_every=20, n_obs_times=5, n_obs=7)
    prob = workload.paper_burgers_problem(wl, si.paper_burgers_draws(wl))
    return wl, prob


def test_paper_burgers_dot_test_and_gradient(small_paper):
    wl, prob = small_paper
    rng = np.random.default_rng(7)
    v = 0.5 * rng.standard_normal(wl.n)
    J = prob.set_iterate(v)
    x = rng.standard_normal((wl.n, 2))
    w = rng.standard_normal((wl.m, 2))
    lhs = np.sum(prob.A(x) * w)
    rhs = np.sum(x * prob.At(w))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    g = prob.gradient()
    p = rng.standard_normal(wl.n)
    eps = 1e-5
    fd = (prob.set_iterate(v + eps * p) - prob.set_iterate(v - eps * p)) / (2 * eps)
    assert abs(fd - g @ p) <= 1e-7 * abs(fd)
    assert J > 0


def test_paper_workload_shape():
    import sc4dvar_inputs as si
    wl = si.paper_burgers_workload()
    d = si.paper_burgers_draws(wl)
    assert (wl.n, wl.n_steps, wl.m) == (399, 8000, 300)
    assert np.allclose(wl.nu * wl.dt * (wl.n + 1) ** 2, 0.4)      # diffusive number, RK3-stable
    assert list(d["obs_idx"][0]) == [25 * (i + 1) - 1 for i in range(15)]
    assert np.allclose(d["x_true0"], np.sin(np.pi * wl.x))
