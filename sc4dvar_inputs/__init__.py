"""Seeded synthetic workloads for the SC-4DVAR Gauss-Newton hot path.

This module only *draws* inputs and states workload shapes. It performs none of
the method's arithmetic: no model step, no prior square root, no observation of a
trajectory, no solver. The CPU oracle (``oracle/``) and the CUDA library both take
their inputs from here, so that a parity test feeds both sides the same numbers.

What is drawn here (all with numpy's PCG64 ``default_rng`` from a fixed seed):

* the raw truth field of the 1D Burgers workloads (a sine plus a Gaussian-smoothed
  white-noise field, Sec. 5.1 uses a sine for the truth; the smoothing recipe is
  the workload's own),
* the standard-normal vectors that become the background error (xi_b) and the
  observation error (xi_o) once a caller applies the prior square root and the
  observation noise level,
* observation site indices,
* dense Gaussian test matrices for tests that pass Omega/Psi explicitly.

The random matrices that the method itself draws inside a Gauss-Newton run
(Omega, Psi, the kappa test vectors) are NOT drawn here: each side implements the
Philox4x32-10 counter-based generator from its published definition instead.
"""
from __future__ import annotations

import dataclasses

import numpy as np

DEFAULT_SEED = 20240128

# Stream offsets for the seeded draws (added to the workload seed).
STREAM_TRUTH = 0
STREAM_BACKGROUND = 1
STREAM_OBS_NOISE = 2
STREAM_OBS_SITES = 3
# Stream ids used by the method's own Philox draws (passed to both sides).
STREAM_SKETCH_BASE = 100
STREAM_KAPPA_BASE = 200
STREAM_PSI_OFFSET = 1000


@dataclasses.dataclass(frozen=True)
class BurgersWorkload:
    """Shape of a periodic 1D viscous Burgers assimilation window.

    ``dt_out`` is the model output step of the workload description; the RK4
    step is ``dt_out / substeps`` (see :func:`burgers_substeps`).
    Observations are taken every ``obs_every`` output steps (t0 excluded) at the
    grid points j with j % obs_stride == 0.
    """
    name: str
    n: int
    nu: float
    dt_out: float
    n_out: int
    obs_every: int
    obs_stride: int
    sigma_obs: float
    sigma_b: float = 0.1
    length_b: float = 0.05
    k: int = 20
    gn_iters: int = 3
    pcg_tol: float = 1e-6
    seed: int = DEFAULT_SEED
    substeps_override: int | None = None

    @property
    def dx(self) -> float:
        return 1.0 / self.n

    @property
    def substeps(self) -> int:
        if self.substeps_override is not None:
            return self.substeps_override
        return burgers_substeps(self.n, self.nu, self.dt_out)

    @property
    def dt(self) -> float:
        return self.dt_out / self.substeps

    @property
    def n_steps(self) -> int:
        return self.n_out * self.substeps

    @property
    def obs_steps(self) -> np.ndarray:
        """RK step index of every observation time (1-based, t0 excluded)."""
        t = np.arange(self.obs_every, self.n_out + 1, self.obs_every, dtype=np.int64)
        return (t * self.substeps).astype(np.int32)

    @property
    def n_obs_times(self) -> int:
        return len(self.obs_steps)

    @property
    def n_obs(self) -> int:
        return len(range(0, self.n, self.obs_stride))

    @property
    def m(self) -> int:
        return self.n_obs_times * self.n_obs


def burgers_substeps(n: int, nu: float, dt_out: float, limit: float = 0.6) -> int:
    """Smallest power of two s with nu*(dt_out/s)/dx^2 <= limit (explicit RK4
    diffusive stability; the workload's output step is kept as the
    observation clock)."""
    dx = 1.0 / n
    s = 1
    while nu * (dt_out / s) / (dx * dx) > limit:
        s *= 2
    return s


BURGERS_WORKLOADS = {
    # Plain FP64 method, small.
    "burgers_n128": BurgersWorkload(
        name="burgers_n128", n=128, nu=0.01, dt_out=1e-3, n_out=50, obs_every=5,
        obs_stride=4, sigma_obs=0.05, k=20, gn_iters=3),
    # Burgers at scale (block of k=128 sketch vectors).
    "burgers_n8192": BurgersWorkload(
        name="burgers_n8192", n=8192, nu=0.005, dt_out=5e-5, n_out=400, obs_every=10,
        obs_stride=8, sigma_obs=0.05, k=128, gn_iters=3),
}


def burgers_workload(name: str, **overrides) -> BurgersWorkload:
    base = BURGERS_WORKLOADS[name]
    return dataclasses.replace(base, **overrides) if overrides else base


def _rng(seed: int, stream: int) -> np.random.Generator:
    return np.random.default_rng([seed, stream])


def periodic_gaussian_weights(n: int, width: float) -> np.ndarray:
    """Unit-sum periodic Gaussian weights of standard deviation ``width`` on the
    grid x_j = j/n (used only to smooth the raw truth noise)."""
    j = np.arange(n)
    d = np.minimum(j, n - j) / n
    w = np.exp(-0.5 * (d / width) ** 2)
    return w / w.sum()


def burgers_truth(wl: BurgersWorkload) -> np.ndarray:
    """x_true(t0) = sin(2 pi x) + G * (0.1 xi), G the unit-sum periodic Gaussian
    of width 0.05 (a circular convolution, evaluated with numpy.fft)."""
    n = wl.n
    x = np.arange(n) / n
    xi = 0.1 * _rng(wl.seed, STREAM_TRUTH).standard_normal(n)
    w = periodic_gaussian_weights(n, 0.05)
    # circular convolution via FFT of two real sequences (input smoothing only)
    smooth = np.real(np.fft.ifft(np.fft.fft(w) * np.fft.fft(xi)))
    return np.sin(2.0 * np.pi * x) + smooth


def burgers_obs_idx(wl: BurgersWorkload) -> np.ndarray:
    """Observation sites, shape (n_t, n_o): every obs_stride-th point at every time."""
    sites = np.arange(0, wl.n, wl.obs_stride, dtype=np.int32)
    return np.tile(sites, (wl.n_obs_times, 1))


def burgers_draws(wl: BurgersWorkload) -> dict:
    """All seeded random inputs of one Burgers workload."""
    return {
        "x_true0": burgers_truth(wl),
        "xi_b": _rng(wl.seed, STREAM_BACKGROUND).standard_normal(wl.n),
        "xi_o": _rng(wl.seed, STREAM_OBS_NOISE).standard_normal((wl.n_obs_times, wl.n_obs)),
        "obs_idx": burgers_obs_idx(wl),
    }


def gaussian_matrix(seed: int, rows: int, cols: int, stream: int = 7) -> np.ndarray:
    """Dense standard-normal test matrix (column-major use; float64)."""
    return _rng(seed, stream).standard_normal((rows, cols))


def se_prior_params(wl: BurgersWorkload) -> dict:
    return {"sigma_b": wl.sigma_b, "length": wl.length_b}


def describe(wl: BurgersWorkload) -> dict:
    return {
        "workload": wl.name, "n": wl.n, "nu": wl.nu, "dt_out": wl.dt_out,
        "substeps": wl.substeps, "rk_steps": wl.n_steps, "n_t": wl.n_obs_times,
        "n_o": wl.n_obs, "m": wl.m, "k": wl.k,
    }



# ---------------------------------------------------------------------------- BVE
@dataclasses.dataclass(frozen=True)
class BVEWorkload:
    """Doubly periodic barotropic vorticity window on [0, 2 pi)^2 with N x N points.

    The truth is normalized to max |grad^perp psi| = 1 and the RK4 step is
    cfl * d (d = 2 pi / N). Observations: a fraction obs_frac of the grid points,
    drawn once without replacement, observed every obs_every steps (t0 excluded).
    Prior Gamma^{1/2} = c (I - ell^2 Lap)^{-1} with ell = ell_cells * d and
    c = prior_frac * std(q_true0); sigma_obs = sigma_frac * max |q_true0|.
    """
    name: str
    N: int
    nu: float
    n_steps: int
    obs_every: int
    obs_frac: float = 0.1
    forcing_amp: float = 1.0
    forcing_k: int = 4
    k: int = 256
    seed: int = DEFAULT_SEED
    cfl: float = 0.2
    ell_cells: float = 4.0
    prior_frac: float = 0.1
    sigma_frac: float = 0.02
    n_checkpoints: int = 0

    @property
    def n(self) -> int:
        return self.N * self.N

    @property
    def d(self) -> float:
        return 2.0 * np.pi / self.N

    @property
    def dt(self) -> float:
        return self.cfl * self.d

    @property
    def obs_steps(self) -> np.ndarray:
        return np.arange(self.obs_every, self.n_steps + 1, self.obs_every, dtype=np.int32)

    @property
    def n_obs_times(self) -> int:
        return len(self.obs_steps)

    @property
    def n_obs(self) -> int:
        return int(round(self.obs_frac * self.n))

    @property
    def m(self) -> int:
        return self.n_obs_times * self.n_obs


BVE_WORKLOADS = {
    "bve_n256": BVEWorkload(name="bve_n256", N=256, nu=1e-4, n_steps=200, obs_every=10, k=256),
    "bve_n1024": BVEWorkload(name="bve_n1024", N=1024, nu=1e-4, n_steps=256, obs_every=10, k=512,
                             n_checkpoints=16),
}


def bve_workload(name: str, **overrides) -> BVEWorkload:
    base = BVE_WORKLOADS[name]
    return dataclasses.replace(base, **overrides) if overrides else base


def _wavenumbers(N):
    k = np.fft.fftfreq(N, 1.0 / N)
    KY, KX = np.meshgrid(k, k, indexing="ij")
    return KX, KY


def bve_truth(wl: BVEWorkload) -> np.ndarray:
    """Random vorticity with energy spectrum ~ |kappa|^-3 (amplitude of q ~ |kappa|^-1)
    on 1 <= |kappa| <= N/3, normalized so that the velocity grad^perp psi has
    maximum 1 (psi = Lap^{-1} q evaluated spectrally, for the normalization only)."""
    N = wl.N
    rng = _rng(wl.seed, STREAM_TRUTH)
    KX, KY = _wavenumbers(N)
    K = np.sqrt(KX ** 2 + KY ** 2)
    band = (K >= 1.0) & (K <= N / 3.0)
    amp = np.where(band, 1.0 / np.where(K > 0, K, 1.0), 0.0)
    qh = amp * (rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N)))
    q = np.real(np.fft.ifft2(qh))
    qh = np.fft.fft2(q)
    K2 = np.where(K > 0, K ** 2, 1.0)
    psih = np.where(K > 0, -qh / K2, 0.0)
    u = np.real(np.fft.ifft2(-1j * KY * psih))
    v = np.real(np.fft.ifft2(1j * KX * psih))
    umax = np.max(np.sqrt(u ** 2 + v ** 2))
    return (q / umax).reshape(-1)


def bve_draws(wl: BVEWorkload) -> dict:
    q0 = bve_truth(wl)
    sites = np.sort(_rng(wl.seed, STREAM_OBS_SITES).choice(wl.n, size=wl.n_obs, replace=False))
    return {
        "x_true0": q0,
        "xi_b": _rng(wl.seed, STREAM_BACKGROUND).standard_normal(wl.n),
        "xi_o": _rng(wl.seed, STREAM_OBS_NOISE).standard_normal((wl.n_obs_times, wl.n_obs)),
        "obs_idx": np.tile(sites.astype(np.int32), (wl.n_obs_times, 1)),
        "prior_c": wl.prior_frac * float(np.std(q0)),
        "prior_ell": wl.ell_cells * wl.d,
        "sigma_obs": wl.sigma_frac * float(np.max(np.abs(q0))),
    }


@dataclasses.dataclass(frozen=True)
class PaperBurgersWorkload:
    """The Burgers experiment of Sec. 5.1 (Experiments 1.1 / 1.2): Dirichlet
    boundaries on (0, 1), n interior points, nu = 0.1, RK3-TVD step 2.5e-5,
    n_t = 20 observation times 0.01 apart (400 steps), n_o = 15 observed states,
    R = 0.01 I, Gamma = (0.5 I - 500 Delta*)^{-2}, truth sin(pi x), l = 15."""
    name: str = "burgers_paper"
    n: int = 399
    nu: float = 0.1
    dt: float = 2.5e-5
    obs_every: int = 400
    n_obs_times: int = 20
    n_obs: int = 15
    sigma_obs: float = 0.1
    prior_a: float = 0.5
    prior_b: float = 500.0
    k: int = 15
    gn_iters: int = 3
    pcg_tol: float = 1e-9
    seed: int = DEFAULT_SEED

    @property
    def n_steps(self) -> int:
        return self.obs_every * self.n_obs_times

    @property
    def obs_steps(self) -> np.ndarray:
        return np.arange(1, self.n_obs_times + 1, dtype=np.int32) * self.obs_every

    @property
    def m(self) -> int:
        return self.n_obs_times * self.n_obs

    @property
    def x(self) -> np.ndarray:
        return np.arange(1, self.n + 1) / (self.n + 1)


def paper_burgers_workload(**overrides) -> PaperBurgersWorkload:
    base = PaperBurgersWorkload()
    return dataclasses.replace(base, **overrides) if overrides else base


def paper_burgers_draws(wl: PaperBurgersWorkload) -> dict:
    """Truth sin(pi x); n_o sites evenly spaced over the interior (index
    round((i + 1)(n + 1)/(n_o + 1)) - 1, the same at every time); background and
    observation noise from the seeded streams."""
    sites = np.array([int(round((i + 1) * (wl.n + 1) / (wl.n_obs + 1))) - 1 for i in range(wl.n_obs)],
                     dtype=np.int32)
    return {
        "x_true0": np.sin(np.pi * wl.x),
        "xi_b": _rng(wl.seed, STREAM_BACKGROUND).standard_normal(wl.n),
        "xi_o": _rng(wl.seed, STREAM_OBS_NOISE).standard_normal((wl.n_obs_times, wl.n_obs)),
        "obs_idx": np.tile(sites, (wl.n_obs_times, 1)),
    }


@dataclasses.dataclass(frozen=True)
class GyreWorkload:
    """The barotropic vorticity experiment of Sec. 5.2: a wind-driven double gyre
    on (0, 1) x (-1, 1) with psi = omega = 0 on the boundary, Re = 200,
    Ro = 0.0016, F = sin(pi y). nx x ny interior points, h = 1/(nx + 1),
    ny = 2 nx + 1 (128 x 257 = 32896 states, h = 0.00775). RK3-TVD step
    2.45e-4; n_t = 8 observation times 5 steps (about six hours) apart; a
    16 x 16 sensor grid; R = 361 I; Gamma = (-0.06 Delta*)^{-2}; l = 384.

    The truth is a spun-up state: a small random vorticity field (prior-shaped,
    init_scale Gamma^{1/2} xi_init) run spin_steps RK3 steps forward by each
    side's own model."""
    name: str = "bve_gyre"
    nx: int = 128
    re: float = 200.0
    ro: float = 0.0016
    dt: float = 2.45e-4
    obs_every: int = 5
    n_obs_times: int = 8
    n_sensors: int = 16          # per dimension
    sigma_obs: float = 19.0
    prior_a: float = 0.0
    prior_b: float = 0.06
    init_scale: float = 1e-3
    spin_steps: int = 400
    k: int = 384
    pcg_tol: float = 1e-9
    seed: int = DEFAULT_SEED

    @property
    def ny(self) -> int:
        return 2 * self.nx + 1

    @property
    def n(self) -> int:
        return self.nx * self.ny

    @property
    def h(self) -> float:
        return 1.0 / (self.nx + 1)

    @property
    def n_steps(self) -> int:
        return self.obs_every * self.n_obs_times

    @property
    def obs_steps(self) -> np.ndarray:
        return np.arange(1, self.n_obs_times + 1, dtype=np.int32) * self.obs_every

    @property
    def n_obs(self) -> int:
        return self.n_sensors * self.n_sensors

    @property
    def m(self) -> int:
        return self.n_obs_times * self.n_obs


def gyre_workload(**overrides) -> GyreWorkload:
    base = GyreWorkload()
    return dataclasses.replace(base, **overrides) if overrides else base


def gyre_sensor_index(wl: GyreWorkload) -> np.ndarray:
    """Sensor sites of an equally spaced s x s grid: along each axis of m
    interior points the 1-based indices round((2a + 1)(m + 1) / (2 s)),
    a = 0..s-1 (symmetric about the centre); flattened row-major (y slow)."""
    s = wl.n_sensors

    def axis(m):
        idx = np.array([int(np.floor((2 * a + 1) * (m + 1) / (2.0 * s) + 0.5)) for a in range(s)]) - 1
        assert np.all(np.diff(idx) > 0) and idx[0] >= 0 and idx[-1] < m
        return idx
    ix, iy = axis(wl.nx), axis(wl.ny)
    return (iy[:, None] * wl.nx + ix[None, :]).reshape(-1).astype(np.int32)


def gyre_draws(wl: GyreWorkload) -> dict:
    """xi_init (shape of the spin-up's initial field), xi_b, xi_o and the sensor
    sites (the same at every observation time)."""
    sites = gyre_sensor_index(wl)
    return {
        "xi_init": _rng(wl.seed, STREAM_TRUTH).standard_normal(wl.n),
        "xi_b": _rng(wl.seed, STREAM_BACKGROUND).standard_normal(wl.n),
        "xi_o": _rng(wl.seed, STREAM_OBS_NOISE).standard_normal((wl.n_obs_times, wl.n_obs)),
        "obs_idx": np.tile(sites, (wl.n_obs_times, 1)),
    }


def burgers_batch(count: int = 64, seed: int = DEFAULT_SEED):
    """Uneven batch of Burgers windows: n from {512, ..., 8192}, N_out from
    {100, 200, 400} and k from {16, 32, 64}, drawn per problem from seed + p;
    dt_out = 5e-5, nu = 0.005, observations every 10 output steps at every 8th
    point (each problem its own pattern: a random offset of the 8-point comb)."""
    out = []
    for p in range(count):
        rng = _rng(seed + p, 50)
        n = int(rng.choice([512, 1024, 2048, 4096, 8192]))
        n_out = int(rng.choice([100, 200, 400]))
        k = int(rng.choice([16, 32, 64]))
        wl = BurgersWorkload(name=f"batch{p}", n=n, nu=0.005, dt_out=5e-5, n_out=n_out, obs_every=10,
                             obs_stride=8, sigma_obs=0.05, k=k, seed=seed + p)
        offset = int(rng.integers(0, 8))
        draws = burgers_draws(wl)
        draws["obs_idx"] = ((draws["obs_idx"] + offset) % n).astype(np.int32)
        out.append((wl, draws))
    return out
