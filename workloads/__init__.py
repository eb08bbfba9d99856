"""Seeded synthetic inputs for the coupled LB step (shared by oracle tests,
GPU tests and bench.py).

This module holds NO arithmetic of the LB method: only initial fields
(diffuse-interface profiles, the analytic two-layer channel profile used as a
start field and as the analytic target), solid masks, the counter-based
random numbers that perturb them, and the request trace of the serving
workload.  Everything is deterministic in the seed.

Random numbers: splitmix64 (Steele, Lea, Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) applied to (seed XOR site
index), mapped to U(-1, 1) from the top 53 bits.

Shapes: fields are numpy arrays [nz, ny, nx] (x fastest); velocity fields are
[3, nz, ny, nx].  The initial interface profile is the equilibrium profile
phi = 1/2 + 1/2 tanh(2 d / W) of the conservative Allen-Cahn equation with the
theta of Sec. II, d = signed distance, positive inside the heavy phase.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

DEFAULT_SEED = 251201027

_M64 = (1 << 64) - 1


def splitmix64(x: np.ndarray) -> np.ndarray:
    """splitmix64 finaliser of uint64 counters (vectorised)."""
    z = np.asarray(x, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = z + np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform_pm1(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """U(-1, 1) for counters offset..offset+n-1: splitmix64(seed ^ index)."""
    idx = np.arange(offset, offset + n, dtype=np.uint64)
    z = splitmix64(idx ^ np.uint64(seed & _M64))
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 / 9007199254740992.0) - 1.0


def tanh_profile(d: np.ndarray, W: float) -> np.ndarray:
    """phi = 1/2 + 1/2 tanh(2 d / W)."""
    return 0.5 + 0.5 * np.tanh(2.0 * d / W)


def grid_coords(nx: int, ny: int, nz: int = 1):
    z, y, x = np.meshgrid(np.arange(nz, dtype=np.float64), np.arange(ny, dtype=np.float64),
                          np.arange(nx, dtype=np.float64), indexing="ij")
    return x, y, z


@dataclass
class Case:
    """A fully specified synthetic workload (fields + parameters)."""

    name: str
    lattice: str
    shape: tuple  # (nx, ny, nz)
    params: dict
    phi0: np.ndarray
    P0: np.ndarray
    u0: np.ndarray
    periodic: tuple = (1, 1, 1)
    solid: np.ndarray | None = None
    steps: int = 0
    meta: dict = field(default_factory=dict)

    @property
    def N(self) -> int:
        nx, ny, nz = self.shape
        return nx * ny * nz


def base_params(**kw) -> dict:
    """The paper's global parameters (Sec. III): rho_ratio = 1000, M = 0.166,
    W = 4; lambda_b = 1/6 and the delta-theta constants of Sec. II."""
    d = dict(rho_w=1.0, rho_a=1e-3, nu_w=0.0167, nu_a=0.167, sigma=1e-3, M=0.166, W=4.0,
             lambda_b=1.0 / 6.0, gamma=-22.5, phi_n=0.8, phi_m=0.2, D=1e-4, eps=1e-10,
             g_ext=(0.0, 0.0, 0.0), clamp_phi_props=1)
    d.update(kw)
    return d


# ---------------------------------------------------------------------------
# 2D static droplet (Laplace law; mass conservation; spurious currents)

def droplet_2d(n: int = 64, R: float = 16.0, center=None, W: float = 4.0, ux: float = 0.0,
               P0: float = 0.0, steps: int = 2000, **pkw) -> Case:
    """n x n periodic D2Q9 domain, one heavy droplet of radius R.
    Default centre ((n-1)/2, (n-1)/2) keeps the data mirror-symmetric."""
    cx, cy = center if center is not None else ((n - 1) / 2.0, (n - 1) / 2.0)
    x, y, _ = grid_coords(n, n, 1)
    d = R - np.sqrt((x - cx) ** 2 + (y - cy) ** 2)
    phi = tanh_profile(d, W)
    u = np.zeros((3,) + phi.shape)
    u[0] = ux
    params = base_params(W=W, **pkw)
    return Case(f"droplet2d_n{n}_R{R:g}", "D2Q9", (n, n, 1), params, phi,
                np.full(phi.shape, float(P0)), u, (1, 1, 1), None, steps,
                dict(R=R, center=(cx, cy)))


# ---------------------------------------------------------------------------
# 2D rising bubble (Sec. III.D, Table tab_bubblerise)

# (rho_1, mu_1, mu_2, sigma) of the two cases of the table; the bubble's
# density rho_2 = 0.22, R = 50 at (100, 100) in a 200 x 400 domain, gravity
# g = 1.36e-8 in -y (Sec. III.D).
BUBBLE_CASES = {1: (2.2, 7.3e-3, 7.3e-4, 3.0e-5), 2: (220.0, 7.3e-1, 7.3e-3, 2.4e-4)}


def rising_bubble_2d(case: int = 1, nx: int = 200, ny: int = 400, R: float = 50.0, center=(100.0, 100.0),
                     g: float = 1.36e-8, W: float = 4.0, steps: int = 20000) -> Case:
    """A light bubble (phi = 0, density 0.22) in a heavier liquid column
    (phi = 1), gravity in -y.  The boundaries are not given in the paper:
    periodic in x, solid rows at y = 0 and y = ny - 1 (halfway bounce-back).
    Kinematic viscosities are the table's dynamic ones over the densities."""
    rho1, mu1, mu2, sigma = BUBBLE_CASES[case]
    rho2 = 0.22
    x, y, _ = grid_coords(nx, ny, 1)
    d = np.sqrt((x - center[0]) ** 2 + (y - center[1]) ** 2) - R   # positive in the liquid
    phi = tanh_profile(d, W)
    solid = np.zeros(phi.shape, np.uint8)
    solid[:, 0, :] = 1
    solid[:, -1, :] = 1
    phi = np.where(solid.astype(bool), 0.0, phi)
    params = base_params(rho_w=rho1, rho_a=rho2, nu_w=mu1 / rho1, nu_a=mu2 / rho2, sigma=sigma, W=W,
                         g_ext=(0.0, -g, 0.0))
    return Case(f"bubble2d_case{case}_{nx}x{ny}", "D2Q9", (nx, ny, 1), params, phi, np.zeros(phi.shape),
                np.zeros((3,) + phi.shape), (1, 0, 1), solid, steps,
                dict(R=R, center=center, rho1=rho1, rho2=rho2, g=g))


# ---------------------------------------------------------------------------
# 2D layered two-phase Poiseuille flow

def two_layer_poiseuille_profile(y: np.ndarray, y_wall_lo: float, y_int: float, y_wall_hi: float,
                                 rho1: float, mu1: float, rho2: float, mu2: float,
                                 g: float) -> np.ndarray:
    """Sharp-interface steady solution of mu_k u'' = -rho_k g with u = 0 at
    both walls and continuous u and mu u' at the interface (heavy layer 1
    between y_wall_lo and y_int, light layer 2 above)."""
    h1 = y_int - y_wall_lo
    h2 = y_wall_hi - y_int
    k1 = rho1 * g / (2.0 * mu1)
    k2 = rho2 * g / (2.0 * mu2)
    A = np.array([[h1, -h2], [mu1, mu2]], dtype=np.float64)
    b = np.array([k1 * h1 * h1 - k2 * h2 * h2, g * (rho1 * h1 + rho2 * h2)])
    A1, A2 = np.linalg.solve(A, b)
    y = np.asarray(y, dtype=np.float64)
    u1 = -k1 * (y - y_wall_lo) ** 2 + A1 * (y - y_wall_lo)
    u2 = -k2 * (y_wall_hi - y) ** 2 + A2 * (y_wall_hi - y)
    u = np.where(y <= y_int, u1, u2)
    return np.where((y < y_wall_lo) | (y > y_wall_hi), 0.0, u)


def poiseuille_2d(nx: int = 128, ny: int = 256, g: float = 1e-7, nu_w: float = 8.35e-3,
                  nu_a: float = 0.167, start_analytic: bool = True, steps: int = 20000,
                  **pkw) -> Case:
    """Channel with solid rows y = 0 and y = ny-1, periodic in x, heavy layer
    below y_int = (ny-1)/2, body acceleration g along x."""
    params = base_params(nu_w=nu_w, nu_a=nu_a, g_ext=(g, 0.0, 0.0), **pkw)
    W = params["W"]
    x, y, _ = grid_coords(nx, ny, 1)
    y_int = (ny - 1) / 2.0
    phi = tanh_profile(y_int - y, W)
    solid = np.zeros(phi.shape, dtype=np.uint8)
    solid[:, 0, :] = 1
    solid[:, ny - 1, :] = 1
    u = np.zeros((3,) + phi.shape)
    ylo, yhi = 0.5, ny - 1.5
    prof = two_layer_poiseuille_profile(np.arange(ny, dtype=np.float64), ylo, y_int, yhi,
                                        params["rho_w"], params["rho_w"] * nu_w,
                                        params["rho_a"], params["rho_a"] * nu_a, g)
    if start_analytic:
        u[0] = prof[None, :, None]
    u[:, solid.astype(bool)] = 0.0
    phi = np.where(solid.astype(bool), 0.0, phi)
    return Case(f"poiseuille2d_{nx}x{ny}", "D2Q9", (nx, ny, 1), params, phi, np.zeros(phi.shape),
                u, (1, 0, 1), solid, steps,
                dict(y_wall_lo=ylo, y_int=y_int, y_wall_hi=yhi, analytic=prof))


# ---------------------------------------------------------------------------
# 3D droplet impact on a liquid film (D3Q27)

def droplet_film_3d(n: int = 256, R: float = 32.0, film: float = 32.0, gap: float | None = None,
                    uz: float = -0.05, noise: float = 1e-4, seed: int = DEFAULT_SEED,
                    steps: int = 2000, lattice: str = "D3Q27", nz: int | None = None,
                    **pkw) -> Case:
    """n x n x nz box, periodic in x and y, solid planes z = 0 and z = nz-1.
    Liquid film phi = 1 for z <= film (interface at film + 1/2); droplet of
    radius R centred at ((n-1)/2, (n-1)/2, film + 1/2 + gap + R), gap = 2W by
    default, moving with u_z = uz; phi perturbed by noise * xi * 4 phi (1-phi)
    with xi = U(-1,1) from splitmix64(seed ^ site)."""
    params = base_params(**pkw)
    W = params["W"]
    nz = n if nz is None else nz
    gap = 2.0 * W if gap is None else gap
    x, y, z = grid_coords(n, n, nz)
    zi = film + 0.5
    c = ((n - 1) / 2.0, (n - 1) / 2.0, zi + gap + R)
    phi_film = tanh_profile(zi - z, W)
    phi_drop = tanh_profile(R - np.sqrt((x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2), W)
    phi = np.maximum(phi_film, phi_drop)
    xi = uniform_pm1(seed, phi.size).reshape(phi.shape)
    phi = phi + noise * xi * 4.0 * phi * (1.0 - phi)
    solid = np.zeros(phi.shape, dtype=np.uint8)
    solid[0] = 1
    solid[nz - 1] = 1
    u = np.zeros((3,) + phi.shape)
    u[2] = uz * phi_drop
    sb = solid.astype(bool)
    u[:, sb] = 0.0
    phi = np.where(sb, 0.0, phi)
    return Case(f"drop_film3d_{n}", lattice, (n, n, nz), params, phi, np.zeros(phi.shape), u,
                (1, 1, 0), solid, steps, dict(R=R, film=film, gap=gap, center=c))


def droplet_3d(n: int = 32, R: float | None = None, axes=(1.1, None, None), W: float = 4.0,
               lattice: str = "D3Q27", steps: int = 500, **pkw) -> Case:
    """Periodic n^3 box with an ellipsoidal droplet (axes R*a, R/sqrt(a), R/sqrt(a))
    centred in the box (oscillating-droplet request of the serving workload)."""
    params = base_params(W=W, **pkw)
    R = 0.3 * n if R is None else R
    a = axes[0]
    ax = (R * a, R / math.sqrt(a), R / math.sqrt(a))
    x, y, z = grid_coords(n, n, n)
    c = (n - 1) / 2.0
    r = np.sqrt(((x - c) / ax[0]) ** 2 + ((y - c) / ax[1]) ** 2 + ((z - c) / ax[2]) ** 2)
    phi = tanh_profile(R * (1.0 - r), W)
    return Case(f"droplet3d_{n}", lattice, (n, n, n), params, phi, np.zeros(phi.shape),
                np.zeros((3,) + phi.shape), (1, 1, 1), None, steps, dict(R=R, axes=ax))


# ---------------------------------------------------------------------------
# Serving trace

@dataclass
class Request:
    rid: int
    arrival: float
    edge: int
    R: float
    ratio: float
    sigma: float
    steps: int

    def case(self) -> Case:
        return droplet_3d(n=self.edge, R=self.R, rho_a=1.0 / self.ratio, sigma=self.sigma,
                          steps=self.steps)


def request_trace(n: int = 2000, seed: int = DEFAULT_SEED, rate: float = 1.0,
                  edges=(32, 48, 64, 96, 128), steps_range=(500, 5000)) -> list:
    """Poisson arrivals (exponential gaps of mean 1/rate seconds); edge uniform
    over `edges`; R = U(0.25, 0.35) edge; density ratio log-uniform in
    [10, 1000]; sigma = U(5e-4, 2e-3); steps uniform integer in steps_range."""
    k = 7
    u = (uniform_pm1(seed ^ 0x5E5E, n * k).reshape(n, k) + 1.0) * 0.5  # U(0,1)
    gaps = -np.log(np.clip(1.0 - u[:, 0], 1e-300, 1.0)) / rate
    t = np.cumsum(gaps) - gaps[0]
    out = []
    for i in range(n):
        edge = int(edges[min(int(u[i, 1] * len(edges)), len(edges) - 1)])
        R = (0.25 + 0.10 * u[i, 2]) * edge
        ratio = 10.0 ** (1.0 + 2.0 * u[i, 3])
        sigma = 5e-4 + 1.5e-3 * u[i, 4]
        lo, hi = steps_range
        steps = int(lo + min(int(u[i, 5] * (hi - lo + 1)), hi - lo))
        out.append(Request(i, float(t[i]), edge, float(R), float(ratio), float(sigma), steps))
    return out
