"""Seeded synthetic inputs for the LBM-LETKF experiments.

This module is shared by the CUDA path's callers (tests, bench) and by the
FP64 oracle's callers.  It holds none of the method's arithmetic: it only
draws or writes down *inputs* -- initial velocity fields, body-force fields,
observation networks, observation-error variances and noise.  Turning a
velocity field into distribution functions (the equilibrium), the LBM step,
the observation operator, localization and the LETKF analysis all live on
each side separately (``oracle/`` in NumPy FP64, the library in CUDA).

Every random draw goes through ``numpy.random.Generator(PCG64(seed))`` so a
seed fixes the input bit for bit on any host.

The workloads mirror the paper's OSSE (Sec. V): a 2D periodic D2Q9 flow, a
nature run that produces noisy observations of the velocity at a regular or
clustered set of observation points, and an ensemble started from perturbed
copies of the truth.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "generator", "taylor_green_velocity", "kolmogorov_force", "band_limited_force",
    "regular_obs_network", "clustered_obs_network", "gaussian", "Workload", "WORKLOADS",
    "loc_cutoff2", "poisson_requests",
]


def generator(seed: int) -> np.random.Generator:
    """PCG64 stream for ``seed`` (identical on x86 and Arm hosts)."""
    return np.random.Generator(np.random.PCG64(int(seed)))


def gaussian(shape, sigma: float, seed: int) -> np.ndarray:
    """Independent N(0, sigma^2) draws, float64."""
    return sigma * generator(seed).standard_normal(shape)


def taylor_green_velocity(nx: int, ny: int, u0: float):
    """Taylor-Green vortex velocity on the periodic nx x ny lattice.

    u_x = -u0 cos(kx x) sin(ky y),  u_y = u0 (kx/ky) sin(kx x) cos(ky y),
    kx = 2 pi / nx, ky = 2 pi / ny (divergence free).  Arrays are [ny][nx].
    """
    x = np.arange(nx, dtype=np.float64)[None, :]
    y = np.arange(ny, dtype=np.float64)[:, None]
    kx = 2.0 * math.pi / nx
    ky = 2.0 * math.pi / ny
    ux = -u0 * np.cos(kx * x) * np.sin(ky * y)
    uy = u0 * (kx / ky) * np.sin(kx * x) * np.cos(ky * y)
    return ux, uy


def kolmogorov_force(nx: int, ny: int, amp: float, n: int):
    """Kolmogorov body force F_x = amp sin(2 pi n y / ny), F_y = 0 ([ny][nx])."""
    y = np.arange(ny, dtype=np.float64)[:, None]
    fx = amp * np.sin(2.0 * math.pi * n * y / ny) * np.ones((1, nx))
    return fx, np.zeros((ny, nx))


def band_limited_force(nx: int, ny: int, kmin: float, kmax: float, rms: float, seed: int):
    """Frozen, divergence-free random body force with wavenumbers in [kmin, kmax].

    A streamfunction psi = sum_k cos(2 pi (a x/nx + b y/ny) + phi_k) over the
    integer wavevectors k = (a, b) of one half plane with kmin <= |k| <= kmax
    and seeded phases phi_k; F = (d psi/dy, -d psi/dx) is rescaled so that
    sqrt(mean(Fx^2 + Fy^2)) = rms.  Every mode has zero mean, so the force
    adds no net momentum.
    """
    rng = generator(seed)
    x = np.arange(nx, dtype=np.float64)[None, :]
    y = np.arange(ny, dtype=np.float64)[:, None]
    fx = np.zeros((ny, nx))
    fy = np.zeros((ny, nx))
    kmax_i = int(math.floor(kmax))
    for a in range(0, kmax_i + 1):
        for b in range(-kmax_i, kmax_i + 1):
            if a == 0 and b <= 0:
                continue  # half plane: (a, b) and (-a, -b) are the same mode
            kk = math.hypot(a, b)
            if kk < kmin or kk > kmax:
                continue
            phi = rng.uniform(0.0, 2.0 * math.pi)
            arg = 2.0 * math.pi * (a * x / nx + b * y / ny) + phi
            s = np.sin(arg)
            fx += -(2.0 * math.pi * b / ny) * s
            fy += (2.0 * math.pi * a / nx) * s
    norm = math.sqrt(float(np.mean(fx * fx + fy * fy)))
    if norm > 0.0:
        fx *= rms / norm
        fy *= rms / norm
    return fx, fy


def regular_obs_network(nx: int, ny: int, stride: int, offset: int = 0) -> np.ndarray:
    """Observation points every ``stride`` cells in x and y, int32 [L][2] as (x, y).

    Ordered row by row (y outer, x inner).
    """
    xs = np.arange(offset, nx, stride, dtype=np.int32)
    ys = np.arange(offset, ny, stride, dtype=np.int32)
    gy, gx = np.meshgrid(ys, xs, indexing="ij")
    return np.stack([gx.ravel(), gy.ravel()], axis=1).astype(np.int32)


def clustered_obs_network(nx: int, ny: int, dense_stride: int, sparse_stride: int,
                          patch: tuple, empty_band: tuple) -> np.ndarray:
    """Clustered network: a dense patch inside a sparse background, with a void.

    patch = (x0, y0, w, h): observed every ``dense_stride`` cells inside.
    empty_band = (y0, h): rows [y0, y0 + h) carry no observation at all.
    Elsewhere every ``sparse_stride`` cells.  int32 [L][2] as (x, y), sorted
    by (y, x) and free of duplicates.
    """
    px, py, pw, ph = patch
    by, bh = empty_band
    pts = set()
    for y in range(0, ny, sparse_stride):
        for x in range(0, nx, sparse_stride):
            pts.add((x, y))
    for y in range(py, py + ph, dense_stride):
        for x in range(px, px + pw, dense_stride):
            pts.add((x % nx, y % ny))
    pts = [(x, y) for (x, y) in pts if not (by <= y < by + bh)]
    pts.sort(key=lambda p: (p[1], p[0]))
    return np.asarray(pts, dtype=np.int32).reshape(-1, 2)


def loc_cutoff2(radius: float) -> float:
    """Squared cutoff (2 sqrt(10/3) r)^2 = (40/3) r^2 of the truncated Gaussian."""
    return 40.0 * radius * radius / 3.0


@dataclass
class Workload:
    """One synthetic LBM-LETKF workload (sizes, seeds, noise levels)."""
    name: str
    nx: int
    ny: int
    k: int
    tau: float
    obs_stride: int
    obs_sigma: float
    loc_radius: float
    steps_per_cycle: int
    cycles: int
    init: str                 # "taylor_green" or "turbulence"
    u0: float = 0.01          # Taylor-Green amplitude
    truth_noise: float = 1e-3 # N(0, .) added to the truth's initial velocity
    member_sigma: float = 5e-3
    kolmogorov_amp: float = 0.0
    kolmogorov_n: int = 4
    random_band: tuple = (4.0, 6.0)
    random_rms: float = 0.0
    spinup: int = 0
    seed: int = 20230803
    obs_vars: tuple = ("u", "v")
    extra: dict = field(default_factory=dict)

    @property
    def n_points(self) -> int:
        return self.nx * self.ny

    def obs_network(self) -> np.ndarray:
        return regular_obs_network(self.nx, self.ny, self.obs_stride)

    def force(self):
        """Total body force (Kolmogorov + frozen band-limited random), float64 [ny][nx]."""
        fx = np.zeros((self.ny, self.nx))
        fy = np.zeros((self.ny, self.nx))
        if self.kolmogorov_amp:
            kx, ky = kolmogorov_force(self.nx, self.ny, self.kolmogorov_amp, self.kolmogorov_n)
            fx += kx
            fy += ky
        if self.random_rms:
            rx, ry = band_limited_force(self.nx, self.ny, self.random_band[0], self.random_band[1],
                                        self.random_rms, self.seed + 1)
            fx += rx
            fy += ry
        return fx, fy

    def truth_velocity(self):
        """Initial truth velocity (before any spin-up), float64 [ny][nx] each."""
        if self.init == "taylor_green":
            ux, uy = taylor_green_velocity(self.nx, self.ny, self.u0)
        else:
            ux = np.zeros((self.ny, self.nx))
            uy = np.zeros((self.ny, self.nx))
        if self.truth_noise:
            ux = ux + gaussian((self.ny, self.nx), self.truth_noise, self.seed + 2)
            uy = uy + gaussian((self.ny, self.nx), self.truth_noise, self.seed + 3)
        return ux, uy

    def member_perturbations(self):
        """Velocity perturbations of the k members, float64 [k][ny][nx] each."""
        shp = (self.k, self.ny, self.nx)
        return (gaussian(shp, self.member_sigma, self.seed + 4),
                gaussian(shp, self.member_sigma, self.seed + 5))

    def obs_noise(self, cycle: int, n_scalars: int) -> np.ndarray:
        """Observation noise of one analysis cycle, N(0, obs_sigma^2) per scalar."""
        return gaussian((n_scalars,), self.obs_sigma, self.seed + 1000 + cycle)

    def obs_error_var(self, n_scalars: int) -> np.ndarray:
        """Diagonal of R: obs_sigma^2 for every observed scalar."""
        return np.full(n_scalars, self.obs_sigma ** 2)


WORKLOADS = {
    # Single-cycle, FP64-checkable case: Taylor-Green truth on 32x32.
    "tgv32_k8": Workload(
        name="tgv32_k8", nx=32, ny=32, k=8, tau=0.6, obs_stride=4, obs_sigma=0.01,
        loc_radius=3.0, steps_per_cycle=50, cycles=1, init="taylor_green"),
    # Forced 2D turbulence, plain FP32 form.
    "turb256_k32": Workload(
        name="turb256_k32", nx=256, ny=256, k=32, tau=0.52, obs_stride=8, obs_sigma=0.01,
        loc_radius=8.0, steps_per_cycle=100, cycles=50, init="turbulence", truth_noise=1e-3,
        kolmogorov_amp=1e-5, kolmogorov_n=4, random_rms=1e-5, spinup=20000),
    # The analysis shape of the 1024^2 case (k = 64, obs every 4th point, r = 12) on a 256^2
    # grid: a small stand-in for profiling its kernels.
    "turb256_k64": Workload(
        name="turb256_k64", nx=256, ny=256, k=64, tau=0.52, obs_stride=4, obs_sigma=0.01,
        loc_radius=12.0, steps_per_cycle=100, cycles=50, init="turbulence", truth_noise=1e-3,
        kolmogorov_amp=1e-5, kolmogorov_n=4, random_rms=1e-5, spinup=20000),
    # Same turbulence at scale (FP32 and mixed forms).  "Same" is read as the same forced flow
    # in lattice units: with the forcing wavenumbers fixed in domain periods, the steady
    # Kolmogorov amplitude F / (nu kappa^2) grows with N^2, so both forcing amplitudes are
    # scaled by (256 / 1024)^2.  With the 256^2 amplitudes the amplitude would be ~2.5
    # lattice units (Mach > 1) and BGK at tau = 0.52 overflows during the spin-up.
    "turb1024_k64": Workload(
        name="turb1024_k64", nx=1024, ny=1024, k=64, tau=0.52, obs_stride=4, obs_sigma=0.01,
        loc_radius=12.0, steps_per_cycle=100, cycles=50, init="turbulence", truth_noise=1e-3,
        kolmogorov_amp=1e-5 / 16, kolmogorov_n=4, random_rms=1e-5 / 16, spinup=20000),
}


def poisson_requests(n: int, rate_hz: float, seed: int, grids=(128, 256, 512, 1024),
                     ks=(16, 32, 64, 128), cycles=(10, 100), strides=(4, 8)) -> list:
    """A seeded stream of independent DA experiments: Poisson arrivals at rate_hz, grid edge,
    ensemble size and observation stride drawn uniformly from the given sets, cycle counts
    uniform in [cycles[0], cycles[1]].  Returns dicts (rid, arrival_s, nx, ny, k, obs_stride,
    cycles, seed) in arrival order."""
    rng = generator(seed)
    t = 0.0
    out = []
    for i in range(n):
        t += float(rng.exponential(1.0 / rate_hz))
        g = int(rng.choice(grids))
        out.append(dict(rid=i, arrival_s=t, nx=g, ny=g, k=int(rng.choice(ks)),
                        obs_stride=int(rng.choice(strides)),
                        cycles=int(rng.integers(cycles[0], cycles[1] + 1)),
                        seed=seed * 100003 + i))
    return out
