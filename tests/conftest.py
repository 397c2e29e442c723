import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built library")


@pytest.fixture(scope="session")
def tiny_wl():
    import sc4dvar_inputs as si
    # n = 16, 20 RK steps, 4 observation times of 8 sites (m = 32 > n):
    # small enough to assemble A, A^T and H densely.
    return si.BurgersWorkload(name="tiny", n=16, nu=0.01, dt_out=0.01, n_out=20,
                              obs_every=5, obs_stride=2, sigma_obs=0.05, length_b=0.2, k=8)


@pytest.fixture(scope="session")
def tiny_prob(tiny_wl):
    import sc4dvar_inputs as si
    from oracle import workload
    prob = workload.burgers_problem(tiny_wl, si.burgers_draws(tiny_wl))
    prob.set_iterate(np.zeros(tiny_wl.n))
    return prob


@pytest.fixture(scope="session")
def tiny_dense(tiny_prob):
    A = tiny_prob.A_dense()
    return {"A": A, "At": tiny_prob.At_dense(), "H": A.T @ A}
