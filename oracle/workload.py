"""Twin-experiment assembly of a Burgers problem from seeded draws (oracle side).

xb = x_true0 + Gamma^{1/2} xi_b and y_i = O(x_true(t_i)) + sigma_obs xi_o,i, the
standard synthetic set-up of Sec. 5.1 (background = truth + prior-distributed
error, observations = observed truth + observation error).
"""
from __future__ import annotations

import numpy as np

from . import burgers, burgers_dirichlet, bve_gyre, fourdvar, prior, rk4


def burgers_problem(wl, draws):
    model = burgers.Burgers1D(wl.n, wl.nu)
    sym = prior.se_sqrt_symbol(wl.n, wl.sigma_b, wl.length_b)
    psq = lambda X: prior.apply_symbol(sym, X)
    prob = fourdvar.FourDVar(model, wl.dt, wl.n_steps, wl.obs_steps, draws["obs_idx"],
                             wl.sigma_obs, psq)
    truth = prob.forward(draws["x_true0"])
    prob.x_true_traj = truth
    prob.y = prob.observe(truth) + wl.sigma_obs * draws["xi_o"]
    prob.xb = draws["x_true0"] + psq(draws["xi_b"])
    prob.symbol = sym
    return prob


def bve_problem(wl, draws):
    """Twin experiment for the barotropic vorticity workload (Sec. 5.2 set-up on a
    doubly periodic grid): same construction as burgers_problem."""
    from . import bve
    model = bve.BVE2D(wl.N, wl.nu, wl.forcing_amp, wl.forcing_k)
    sym = bve.inv_helmholtz_sqrt_symbol(wl.N, draws["prior_c"], draws["prior_ell"])
    psq = lambda X: bve.apply_symbol_2d(sym, X, wl.N)
    prob = fourdvar.FourDVar(model, wl.dt, wl.n_steps, wl.obs_steps, draws["obs_idx"],
                             draws["sigma_obs"], psq)
    truth = prob.forward(draws["x_true0"])
    prob.x_true_traj = truth
    prob.y = prob.observe(truth) + draws["sigma_obs"] * draws["xi_o"]
    prob.xb = draws["x_true0"] + psq(draws["xi_b"])
    prob.symbol = sym
    return prob


def paper_burgers_problem(wl, draws):
    """The Dirichlet / RK3-TVD Burgers experiment of Sec. 5.1 (same twin
    construction as burgers_problem)."""
    model = burgers_dirichlet.BurgersDirichlet(wl.n, wl.nu)
    psq = burgers_dirichlet.inv_helmholtz_sqrt(wl.n, wl.prior_a, wl.prior_b)
    prob = fourdvar.FourDVar(model, wl.dt, wl.n_steps, wl.obs_steps, draws["obs_idx"],
                             wl.sigma_obs, psq, tableau=rk4.RK3_TVD)
    truth = prob.forward(draws["x_true0"])
    prob.x_true_traj = truth
    prob.y = prob.observe(truth) + wl.sigma_obs * draws["xi_o"]
    prob.xb = draws["x_true0"] + psq(draws["xi_b"])
    return prob


def gyre_truth0(wl, draws, model=None, psq=None):
    """Spun-up truth of the double-gyre workload: init_scale Gamma^{1/2} xi_init
    advanced spin_steps RK3-TVD steps."""
    model = model or bve_gyre.BVEGyre(wl.nx, wl.re, wl.ro)
    psq = psq or bve_gyre.inv_helmholtz_sqrt_2d(wl.nx, wl.prior_a, wl.prior_b)
    x = wl.init_scale * psq(draws["xi_init"])
    for _ in range(wl.spin_steps):
        x = rk4.fwd_step(model, x, wl.dt, rk4.RK3_TVD)
    return x


def gyre_problem(wl, draws):
    """The double-gyre barotropic vorticity experiment of Sec. 5.2 (same twin
    construction as burgers_problem, truth from gyre_truth0)."""
    model = bve_gyre.BVEGyre(wl.nx, wl.re, wl.ro)
    psq = bve_gyre.inv_helmholtz_sqrt_2d(wl.nx, wl.prior_a, wl.prior_b)
    prob = fourdvar.FourDVar(model, wl.dt, wl.n_steps, wl.obs_steps, draws["obs_idx"],
                             wl.sigma_obs, psq, tableau=rk4.RK3_TVD)
    x0 = gyre_truth0(wl, draws, model, psq)
    truth = prob.forward(x0)
    prob.x_true_traj = truth
    prob.y = prob.observe(truth) + wl.sigma_obs * draws["xi_o"]
    prob.xb = x0 + psq(draws["xi_b"])
    return prob
