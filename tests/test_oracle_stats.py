"""Pins of the wall-normal statistics of the oracle (oracle/stats.py) against
exact states and independent formulas: the conduction profile (Nu = 1 at
both walls and in the volume), the laminar Couette profile (wall shear stress
2 nu exactly with the half-cell wall distance), horizontal means that remove
Fourier modes exactly, the volume Nusselt number of the existing oracle
(a different summation), and the mean square of a cosine."""
import math

import numpy as np
import pytest
import torch

import synth
from oracle import Grid, stats, timestep as ts


def grid(nx, ny, nz, stretch=1.5, lx=1.0, ly=1.0):
    return Grid(nx, ny, nz, lx, ly, synth.tanh_faces(nz, stretch))


def zeros(g, faces=False):
    return torch.zeros(g.face_shape() if faces else g.cell_shape(), dtype=torch.float64)


def test_conduction_profile_nusselt_is_one():
    g = grid(8, 6, 11)
    zf = g.zf.double()
    T = (1.0 - zf)[:, None, None].expand(g.face_shape()).clone()
    prof = stats.plane_means(g, zeros(g), zeros(g), zeros(g, True), T)
    s = stats.scalars(g, prof, nu=1e-3, kappa=1e-3, u_bot=0.0, u_top=0.0, T_bot=1.0, T_top=0.0)
    for key in ("nu_volume", "nu_bottom", "nu_top"):
        assert abs(s[key] - 1.0) < 1e-13, (key, s[key])
    assert s["ke"] == 0.0 and s["tau_bottom"] == 0.0 and s["re_tau"] == 0.0


def test_laminar_couette_wall_shear():
    g = grid(8, 4, 13, stretch=2.0)
    nu = 1.25e-4
    u = (2.0 * g.zc.double() - 1.0)[:, None, None].expand(g.cell_shape()).clone()
    prof = stats.plane_means(g, u, zeros(g), zeros(g, True))
    s = stats.scalars(g, prof, nu=nu, kappa=0.0, u_bot=-1.0, u_top=1.0, T_bot=0.0, T_top=0.0)
    assert abs(s["tau_bottom"] - 2.0 * nu) < 1e-15 and abs(s["tau_top"] - 2.0 * nu) < 1e-15
    assert abs(s["re_tau"] - 0.5 * math.sqrt(2.0 * nu) / nu) < 1e-9


def test_horizontal_means_remove_fourier_modes():
    g = grid(16, 12, 7, lx=2.0, ly=0.5)
    x = (torch.arange(g.nx, dtype=torch.float64) + 0.5) * g.dx
    y = (torch.arange(g.ny, dtype=torch.float64) + 0.5) * g.dy
    prof_z = torch.as_tensor(synth.noise((g.nz,), seed=3))
    f = prof_z[:, None, None] + torch.cos(2 * math.pi * 3 * x / g.lx)[None, None, :] \
        * torch.sin(2 * math.pi * 2 * y / g.ly)[None, :, None] * 5.0
    prof = stats.plane_means(g, f, zeros(g), zeros(g, True))
    assert float((prof[:g.nz, 0] - prof_z).abs().max()) < 1e-14


def test_volume_nusselt_matches_face_weighted_sum():
    g = grid(12, 8, 9)
    w = torch.as_tensor(synth.noise(g.face_shape(), seed=5))
    w[0] = 0.0
    w[-1] = 0.0
    T = torch.as_tensor(synth.noise(g.face_shape(), seed=6))
    ra, pr = 1e7, 1.0
    prof = stats.plane_means(g, zeros(g), zeros(g), w, T)
    s = stats.scalars(g, prof, nu=math.sqrt(pr / ra), kappa=1.0 / math.sqrt(ra * pr), u_bot=0.0,
                      u_top=0.0, T_bot=1.0, T_top=0.0)
    ref = float(ts.nusselt(g, w, T, ra, pr))
    assert abs(s["nu_volume"] - ref) < 1e-12 * abs(ref)


def test_kinetic_energy_of_a_cosine():
    g = grid(16, 8, 5)
    x = (torch.arange(g.nx, dtype=torch.float64) + 0.5) * g.dx
    A = 0.7
    u = (A * torch.cos(2 * math.pi * x / g.lx))[None, None, :].expand(g.cell_shape()).clone()
    prof = stats.plane_means(g, u, zeros(g), zeros(g, True))
    s = stats.scalars(g, prof, nu=1.0, kappa=1.0, u_bot=0.0, u_top=0.0, T_bot=1.0, T_top=0.0)
    assert abs(s["ke"] - A * A / 4.0) < 1e-15
