"""Sampled-mode Poisson oracle for grids too large for the full oracle.

TEST INFRASTRUCTURE ONLY (see the package header).

The solve of Sec. 2.2 decouples into one wall-normal system per wavenumber pair
(kx, ky). For a chosen set of pairs this module computes the right-hand side's
Fourier coefficients by a direct FP64 discrete Fourier transform,
    bhat(kx, ky, z) = sum_j sum_i b[z, j, i] exp(-2 pi i (kx i / nx + ky j / ny)),
(a matrix product along x, then a weighted sum along y), removes the
cell-volume-weighted mean from the (0,0) column (solvability), and solves each
column with the oracle's own Thomas routine and exact zero-mode integration,
then applies the zero-weighted-mean gauge to the (0,0) column. The result is
the unnormalised Fourier coefficient of the full solve's phi at those pairs.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from .grid import Grid
from . import poisson


def mode_columns(g: Grid, f, pairs):
    """Direct FP64 DFT of the field f ([nz][ny][nx], numpy or torch) at the
    (kx, ky) pairs: {(kx, ky): complex128 array [nz]}."""
    f = f.detach().cpu().numpy() if isinstance(f, torch.Tensor) else np.asarray(f)
    nz, ny, nx = f.shape
    kxs = sorted({kx for kx, _ in pairs})
    ang = 2.0 * np.pi * np.outer(np.arange(nx), kxs) / nx           # [nx, nkx]
    flat = f.reshape(-1, nx)
    # real matrix products (no complex copy of f): sum_x f e^{-i ang}
    A = (flat @ np.cos(ang) - 1j * (flat @ np.sin(ang))).reshape(nz, ny, len(kxs))
    j = np.arange(ny)
    out = {}
    for kx, ky in pairs:
        ey = np.exp(-2j * np.pi * j * ky / ny)
        out[(kx, ky)] = A[:, :, kxs.index(kx)] @ ey                  # sum over y
    return out


def solve_modes(g: Grid, b, pairs):
    """Unnormalised Fourier coefficients of phi = solve(b) at the pairs."""
    cols = mode_columns(g, b, pairs)
    lx, ly = poisson.modified_wavenumbers(g)
    a, c = poisson.z_coefficients(g)
    dzc = g.dzc.numpy()
    out = {}
    for (kx, ky), bh in cols.items():
        if kx == 0 and ky == 0:
            bh = bh - (dzc * bh).sum() / dzc.sum()              # solvability
            ph = poisson.zero_mode(g, torch.as_tensor(bh)).numpy()
            ph = ph - (dzc * ph).sum() / dzc.sum()              # gauge
        else:
            kyh = min(ky, g.ny - ky)
            lam = float(lx[kx]) + float(ly[kyh])
            diag = (-a - c - lam)[:, None]
            ph = poisson.thomas(a, diag, c, torch.as_tensor(bh)[:, None]).numpy()[:, 0]
        out[(kx, ky)] = ph
    return out


def default_pairs(g: Grid, seed: int = 0, count: int = 16):
    """(0,0), the lowest pairs, the Nyquist edges and seeded others."""
    base = [(0, 0), (1, 0), (0, 1), (1, 1), (g.nx // 2, 0), (0, g.ny // 2), (g.nx // 2, g.ny // 2),
            (2, g.ny - 1)]
    rng = np.random.Generator(np.random.PCG64(seed))
    while len(base) < count:
        p = (int(rng.integers(0, g.nx // 2 + 1)), int(rng.integers(0, g.ny)))
        if p not in base:
            base.append(p)
    return base
