"""Seeded synthetic inputs shared by the oracle tests, the CUDA-path tests and the benchmark.

This module holds the input recipe only: grid faces, workload shapes and
parameters, and seeded random fields. It performs none of the solver's
arithmetic (no divergence, no transform, no tridiagonal solve, no time step),
so the oracle and the CUDA path stay independent of each other while being fed
bit-identical inputs.

All random numbers are drawn on the host with numpy's PCG64 generator; nothing
is generated on the device.

Array layout (C order, x fastest):
  u, v, p   [nz][ny][nx]     cell-z (u at x-faces, v at y-faces, p at centres)
  w, T      [nz+1][ny][nx]   z-faces; planes 0 and nz are the walls
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, asdict

import numpy as np


def tanh_faces(nz: int, stretch: float) -> np.ndarray:
    """Wall-normal face coordinates z_0=0 < ... < z_nz=1, clustered at both walls.

    The paper uses a non-uniform wall-normal grid clustered near the walls
    (Sec. 2.1) without printing the law; the workloads use the symmetric
    hyperbolic-tangent map z_k = (1 + tanh(s(2k/nz - 1))/tanh(s)) / 2.
    stretch == 0 gives the uniform grid.
    """
    k = np.arange(nz + 1, dtype=np.float64)
    if stretch == 0.0:
        z = k / nz
    else:
        z = 0.5 * (1.0 + np.tanh(stretch * (2.0 * k / nz - 1.0)) / math.tanh(stretch))
    z[0] = 0.0
    z[-1] = 1.0
    return z


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


@dataclass
class Workload:
    """Grid and physical parameters of one synthetic workload."""
    name: str
    nx: int
    ny: int
    nz: int
    lx: float
    ly: float
    stretch: float
    nu: float = 0.0
    kappa: float = 0.0
    buoyancy: float = 0.0
    u_bot: float = 0.0
    u_top: float = 0.0
    T_bot: float = 0.0
    T_top: float = 0.0
    cfl: float = 0.7
    dt_max: float = 1e-2
    has_T: bool = True
    steps: int = 1
    extra: dict = field(default_factory=dict)

    @property
    def points(self) -> int:
        return self.nx * self.ny * self.nz

    def faces(self) -> np.ndarray:
        return tanh_faces(self.nz, self.stretch)

    def as_dict(self) -> dict:
        return asdict(self)


def rb_params(ra: float, pr: float) -> tuple[float, float]:
    """Free-fall units for Rayleigh-Benard: nu = sqrt(Pr/Ra), kappa = 1/sqrt(Ra Pr)."""
    return math.sqrt(pr / ra), 1.0 / math.sqrt(ra * pr)


def workload(name: str, **over) -> Workload:
    """The named synthetic workloads (shapes of the paper's RB / Couette runs)."""
    if name == "pc64":  # plain FP64 pressure correction, 64^3
        w = Workload("pc64", 64, 64, 64, 1.0, 1.0, 1.5)
    elif name == "rb512":  # Rayleigh-Benard Ra=1e8 Pr=1 Gamma=1, 512x512x384
        nu, ka = rb_params(1e8, 1.0)
        w = Workload("rb512", 512, 512, 384, 1.0, 1.0, 1.5, nu=nu, kappa=ka, buoyancy=1.0,
                     T_bot=1.0, T_top=0.0, cfl=0.7, dt_max=5e-3, steps=100,
                     extra={"Ra": 1e8, "Pr": 1.0})
    elif name == "couette1024":  # plane Couette Re_w=4000, 4pi x 2pi x 1, 1024x512x256
        w = Workload("couette1024", 1024, 512, 256, 4 * math.pi, 2 * math.pi, 1.5,
                     nu=0.5 / 4000.0, u_bot=-1.0, u_top=1.0, cfl=0.7, dt_max=2e-2,
                     has_T=False, steps=50, extra={"Re_w": 4000.0})
    elif name == "poisson2048":  # large mixed-precision Poisson solve
        w = Workload("poisson2048", 2048, 2048, 1024, 1.0, 1.0, 1.5)
    elif name == "adj256":  # adjoint RB Ra=1e7, 256x256x128
        nu, ka = rb_params(1e7, 1.0)
        w = Workload("adj256", 256, 256, 128, 1.0, 1.0, 1.5, nu=nu, kappa=ka, buoyancy=1.0,
                     T_bot=1.0, T_top=0.0, cfl=0.7, dt_max=5e-3, steps=20,
                     extra={"Ra": 1e7, "Pr": 1.0, "checkpoint_every": 5})
    else:
        raise KeyError(name)
    for k, v in over.items():
        setattr(w, k, v)
    return w


def velocity_noise(w: Workload, seed: int, sigma: float = 1.0):
    """u, v, w ~ iid N(0, sigma^2); w is zero on the two wall planes."""
    g = rng(seed)
    nx, ny, nz = w.nx, w.ny, w.nz
    u = g.standard_normal((nz, ny, nx)) * sigma
    v = g.standard_normal((nz, ny, nx)) * sigma
    ww = g.standard_normal((nz + 1, ny, nx)) * sigma
    ww[0] = 0.0
    ww[-1] = 0.0
    return u, v, ww


def rb_initial(w: Workload, seed: int, amp: float = 1e-3):
    """Rayleigh-Benard start: conduction profile T = 1 - z on faces plus U(-amp, amp)
    noise on the interior faces; velocity and pressure zero."""
    g = rng(seed)
    nx, ny, nz = w.nx, w.ny, w.nz
    zf = w.faces()
    T = np.empty((nz + 1, ny, nx))
    T[:] = (w.T_bot + (w.T_top - w.T_bot) * zf)[:, None, None]
    T[1:-1] += g.uniform(-amp, amp, size=(nz - 1, ny, nx))
    u = np.zeros((nz, ny, nx))
    v = np.zeros((nz, ny, nx))
    ww = np.zeros((nz + 1, ny, nx))
    p = np.zeros((nz, ny, nx))
    return u, v, ww, T, p


def conduction_temperature(zf, ny: int, nx: int, T_bot: float, T_top: float, seed: int,
                           amp: float = 1e-3) -> np.ndarray:
    """Conduction profile T = T_bot + (T_top - T_bot) z on the given face
    coordinates zf (nz+1 of them, any grid, e.g. a refined temperature grid)
    plus U(-amp, amp) noise on the interior faces: [nz+1][ny][nx]."""
    g = rng(seed)
    zf = np.asarray(zf, dtype=np.float64)
    T = np.empty((len(zf), ny, nx))
    T[:] = (T_bot + (T_top - T_bot) * zf)[:, None, None]
    if amp != 0.0:
        T[1:-1] += g.uniform(-amp, amp, size=(len(zf) - 2, ny, nx))
    return T


def couette_initial(w: Workload, seed: int, sigma: float = 0.05):
    """Plane Couette start: laminar u = u_bot + (u_top-u_bot) zc plus N(0, sigma^2) on
    u, v, w (w zero on the walls); pressure zero."""
    g = rng(seed)
    nx, ny, nz = w.nx, w.ny, w.nz
    zf = w.faces()
    zc = 0.5 * (zf[1:] + zf[:-1])
    u = (w.u_bot + (w.u_top - w.u_bot) * zc)[:, None, None] + g.standard_normal((nz, ny, nx)) * sigma
    v = g.standard_normal((nz, ny, nx)) * sigma
    ww = g.standard_normal((nz + 1, ny, nx)) * sigma
    ww[0] = 0.0
    ww[-1] = 0.0
    p = np.zeros((nz, ny, nx))
    return u, v, ww, p


def manufactured_modes(seed: int, count: int = 8, amax: int = 16, mmax: int = 16):
    """(a, b, m) integer triples for cos(2 pi a x/Lx) cos(2 pi b y/Ly) cos(pi m z) modes."""
    g = rng(seed)
    out = []
    for _ in range(count):
        out.append((int(g.integers(0, amax + 1)), int(g.integers(0, amax + 1)),
                    int(g.integers(1, mmax + 1))))
    return out


def noise(shape, seed: int, sigma: float = 1.0) -> np.ndarray:
    return rng(seed).standard_normal(shape) * sigma


def uniform(shape, seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    return rng(seed).uniform(lo, hi, size=shape)


def manufactured_rhs(w: Workload, seed: int, noise_sigma: float = 1.0, modes=None, out=None):
    """Right-hand side of the large Poisson workload: N(0, sigma^2) noise plus the
    manufactured modes cos(2 pi a x/Lx) cos(2 pi b y/Ly) cos(pi m z) sampled at
    cell centres (unit amplitude), built one z-slab at a time into `out`
    ([nz][ny][nx] float64, allocated if None). noise_sigma = 0 gives the modes
    only. Returns (out, modes)."""
    nx, ny, nz = w.nx, w.ny, w.nz
    if modes is None:
        modes = manufactured_modes(seed + 1000)
    if out is None:
        out = np.empty((nz, ny, nx))
    zf = w.faces()
    zc = 0.5 * (zf[1:] + zf[:-1])
    xc = (np.arange(nx) + 0.5) * (w.lx / nx)
    yc = (np.arange(ny) + 0.5) * (w.ly / ny)
    g = rng(seed)
    cx = {a: np.cos(2 * np.pi * a * xc / w.lx) for a, _, _ in modes}
    cy = {b: np.cos(2 * np.pi * b * yc / w.ly) for _, b, _ in modes}
    slab = max(1, (1 << 26) // (nx * ny))
    for k0 in range(0, nz, slab):
        k1 = min(nz, k0 + slab)
        blk = out[k0:k1]
        if noise_sigma:
            blk[:] = g.standard_normal(blk.shape)
            if noise_sigma != 1.0:
                blk *= noise_sigma
        else:
            blk[:] = 0.0
        for a, b, m in modes:
            cz = np.cos(np.pi * m * zc[k0:k1])
            blk += cz[:, None, None] * np.outer(cy[b], cx[a])[None]
    return out, modes
