"""Pins of the oracle's strong-Wolfe line search and of its use in the GN loop.

The one-dimensional test functions are those of Moré and Thuente's line-search
paper (ACM TOMS 20, 1994), restated from their formulas; for every start step
the returned step must satisfy the strong Wolfe conditions it was asked for.
A quadratic has a known minimiser; the linear (advection-free) 4D-Var problem
has an exactly quadratic cost, so its GN step is the minimiser and the search
must accept alpha = 1 at the first evaluation."""
import math

import numpy as np
import pytest

from oracle import linesearch as ls


def f1(a, b=2.0):
    return -a / (a * a + b), (a * a - b) / (a * a + b) ** 2


def f2(a, b=0.004):
    return (a + b) ** 5 - 2.0 * (a + b) ** 4, 5.0 * (a + b) ** 4 - 8.0 * (a + b) ** 3


def f3(a, b=0.01, l=39):
    if a <= 1.0 - b:
        p0, d0 = 1.0 - a, -1.0
    elif a >= 1.0 + b:
        p0, d0 = a - 1.0, 1.0
    else:
        p0, d0 = (a - 1.0) ** 2 / (2.0 * b) + b / 2.0, (a - 1.0) / b
    w = l * math.pi / 2.0
    return p0 + 2.0 * (1.0 - b) / (l * math.pi) * math.sin(w * a), d0 + (1.0 - b) * math.cos(w * a)


CASES = [(f1, 1e-3, 0.1), (f2, 0.1, 0.1), (f3, 0.1, 0.1)]


@pytest.mark.parametrize("fn,c1,c2", CASES)
@pytest.mark.parametrize("alpha1", [1e-3, 1e-1, 1e1, 1e3])
def test_strong_wolfe_on_test_functions(fn, c1, c2, alpha1):
    f0, d0 = fn(0.0)
    res = ls.strong_wolfe(fn, f0, d0, alpha1=alpha1, c1=c1, c2=c2, alpha_max=1e4, max_evals=60)
    assert res.status == ls.OK
    fa, da = fn(res.alpha)
    assert fa <= f0 + c1 * res.alpha * d0 + 1e-15
    assert abs(da) <= c2 * abs(d0) + 1e-15
    assert (fa, da) == (res.phi, res.dphi)


def test_quadratic_minimiser():
    a, b = 3.0, -2.0                      # phi = a x^2 / 2 + b x, minimiser 2/3
    q = lambda x: (0.5 * a * x * x + b * x, a * x + b)
    res = ls.strong_wolfe(q, 0.0, b, alpha1=1.0, c1=1e-4, c2=1e-3)
    assert abs(res.alpha - 2.0 / 3.0) <= 1e-3 * 2.0 / 3.0
    # started at the minimiser: accepted at once
    res = ls.strong_wolfe(q, 0.0, b, alpha1=2.0 / 3.0, c1=1e-4, c2=1e-3)
    assert res.evals == 1 and res.alpha == 2.0 / 3.0


def test_cubic_interpolant_exact_on_cubics():
    c = lambda x: (x ** 3 - 3 * x, 3 * x * x - 3)   # local minimiser at 1
    fa, da = c(0.2)
    fb, db = c(1.7)
    assert abs(ls.cubic_min(0.2, fa, da, 1.7, fb, db) - 1.0) <= 1e-12


def test_not_descent_is_reported():
    res = ls.strong_wolfe(lambda x: (x, 1.0), 0.0, 1.0)
    assert res.status == ls.NOT_DESCENT and res.evals == 0


class _Heat:
    """Periodic heat equation x' = nu D2 x (the Burgers model without advection)."""

    def __init__(self, n, nu):
        self.n = n
        D2 = -2.0 * np.eye(n) + np.roll(np.eye(n), 1, 0) + np.roll(np.eye(n), -1, 0)
        self.L = nu * n * n * D2

    def rhs(self, u):
        return self.L @ u

    def jvp(self, U, d):
        return self.L @ d

    def vjp(self, U, w):
        return self.L.T @ w


def test_linear_problem_accepts_the_full_step(tiny_wl):
    """A linear model: J(v) is quadratic, the GN step is its minimiser,
    phi'(1) = 0 and the search accepts alpha = 1 at the first evaluation."""
    from oracle import fourdvar, prior, solvers
    import sc4dvar_inputs as si
    wl = tiny_wl
    draws = si.burgers_draws(wl)
    sym = prior.se_sqrt_symbol(wl.n, wl.sigma_b, wl.length_b)
    psq = lambda X: prior.apply_symbol(sym, X)
    prob = fourdvar.FourDVar(_Heat(wl.n, wl.nu), wl.dt, wl.n_steps, wl.obs_steps, draws["obs_idx"],
                             wl.sigma_obs, psq)
    prob.y = prob.observe(prob.forward(draws["x_true0"])) + wl.sigma_obs * draws["xi_o"]
    prob.xb = draws["x_true0"] + psq(draws["xi_b"])
    o = solvers.GNOptions(iters=2, method="none", pcg_tol=1e-12, line_search=True)
    v, info = solvers.gauss_newton(prob, np.zeros(wl.n), o)
    assert info[0]["alpha"] == 1.0 and info[0]["ls_evals"] == 1 and info[0]["ls_status"] == ls.OK
    # the second iteration starts at the minimiser: gradient ~ 0
    assert info[1]["g_inf"] <= 1e-8 * info[0]["g_inf"]


def test_gn_with_line_search_decreases_the_cost(tiny_wl):
    from oracle import solvers, workload
    import sc4dvar_inputs as si
    wl = tiny_wl
    prob = workload.burgers_problem(wl, si.burgers_draws(wl))
    o = solvers.GNOptions(iters=4, method="randsvd", l=8, pcg_tol=1e-10, line_search=True)
    v, info = solvers.gauss_newton(prob, np.zeros(wl.n), o)
    J = [r["J"] for r in info]
    assert all(J[i + 1] < J[i] for i in range(len(J) - 1))
    assert all(0.0 < r["alpha"] for r in info)
