"""Direct Fourier-Thomas solve of the pressure-correction Poisson equation (Sec. 2.2).

The paper reduces the Poisson equation by a two-dimensional FFT in the
periodic directions to one tridiagonal system per wavenumber pair along the
wall-normal direction, solved by the Thomas algorithm, using modified
wavenumbers (the eigenvalues of the discrete second difference) instead of
the exact ones. Its twelve-step listing interleaves those transforms with
pencil transposes; on one address space the transposes carry no arithmetic
and are dropped, leaving: forward real-to-complex transform, forward complex
transform, tridiagonal solves, inverse complex transform, inverse
complex-to-real transform.

Readings where the paper is silent:
* modified wavenumber lambda = 4 sin^2(pi k / N) / Delta^2 (the exact
  eigenvalue of the 3-point operator; written with sin^2 rather than 2 - 2cos
  to keep relative accuracy at small k);
* the (0,0) Fourier mode is singular under zero-flux walls; the right-hand
  side's cell-volume-weighted mean is removed first (solvability), the mode is
  then integrated exactly as a 1-D flux problem (prefix sums), and the gauge is
  a zero cell-volume-weighted mean of the solution.
The FFT itself is a library primitive (torch.fft, unnormalised forward,
1/(nx ny) on the inverse).
"""
from __future__ import annotations

import math

import torch

from .grid import Grid


def modified_wavenumbers(g: Grid):
    """lambda_x(kx), kx = 0..nx/2 and lambda_y(ky), ky = 0..ny-1 (Sec. 2.2)."""
    kx = torch.arange(g.nx // 2 + 1, dtype=torch.float64)
    ky = torch.arange(g.ny, dtype=torch.float64)
    lx = (2.0 * torch.sin(math.pi * kx / g.nx) / g.dx) ** 2
    ly = (2.0 * torch.sin(math.pi * ky / g.ny) / g.dy) ** 2
    return lx, ly


def z_coefficients(g: Grid):
    """Off-diagonals of the wall-normal operator at cell k:
    a_k = 1/(dzc_k dzf_k) (0 at k = 0), c_k = 1/(dzc_k dzf_{k+1}) (0 at k = nz-1)."""
    a = torch.zeros(g.nz, dtype=torch.float64)
    c = torch.zeros(g.nz, dtype=torch.float64)
    a[1:] = 1.0 / (g.dzc[1:] * g.dzf[1:-1])
    c[:-1] = 1.0 / (g.dzc[:-1] * g.dzf[1:-1])
    return a, c


def thomas(a, b, c, d):
    """Thomas algorithm for a_k x_{k-1} + b_k x_k + c_k x_{k+1} = d_k, k = 0..n-1.

    a, c: [n] (shared by all systems); b: [n, *batch]; d: [n, *batch] (real or
    complex). Forward elimination k = 0 -> n-1, back substitution n-1 -> 0.
    Written with Python lists so that automatic differentiation can run through it.
    """
    n = d.shape[0]
    cp = [c[0] / b[0]]
    dp = [d[0] / b[0]]
    for k in range(1, n):
        den = b[k] - a[k] * cp[k - 1]
        cp.append(c[k] / den)
        dp.append((d[k] - a[k] * dp[k - 1]) / den)
    x = [None] * n
    x[n - 1] = dp[n - 1]
    for k in range(n - 2, -1, -1):
        x[k] = dp[k] - cp[k] * x[k + 1]
    return torch.stack(x)


def zero_mode(g: Grid, bhat):
    """Exact solution of the singular (kx, ky) = (0, 0) system.

    Multiplying row k by dzc_k turns it into F_{k+1} - F_k = dzc_k bhat_k for the
    face fluxes F_k = (phi_k - phi_{k-1})/dzf_k with F_0 = F_nz = 0. Hence
    F_k = sum_{m<k} dzc_m bhat_m and phi_k = phi_{k-1} + dzf_k F_k, phi_0 = 0.
    """
    nz = g.nz
    F = [bhat[0] * 0.0]
    for k in range(1, nz):
        F.append(F[k - 1] + g.dzc[k - 1] * bhat[k - 1])
    phi = [bhat[0] * 0.0]
    for k in range(1, nz):
        phi.append(phi[k - 1] + g.dzf[k] * F[k])
    return torch.stack(phi)


def weighted_mean(g: Grid, f):
    """Cell-volume-weighted mean sum(W_c f)/sum(W_c) (a 0-d tensor)."""
    w = g.dzc[:, None, None]
    return (w * f).sum() / (w.sum() * g.nx * g.ny)


def solve(g: Grid, b, return_mean: bool = False):
    """phi with L phi = b - mean_W(b) and mean_W(phi) = 0."""
    mb = weighted_mean(g, b)
    b = b - mb
    bh = torch.fft.rfft2(b)                           # [nz][ny][nx/2+1]
    lx, ly = modified_wavenumbers(g)
    lam = ly[:, None] + lx[None, :]                   # [ny][nx/2+1]
    a, c = z_coefficients(g)
    diag = (-a - c)[:, None, None] - lam[None]        # [nz][ny][nx/2+1]
    diag[:, 0, 0] = 1.0                               # placeholder, replaced below
    ph = thomas(a, diag, c, bh).clone()
    ph[:, 0, 0] = zero_mode(g, bh[:, 0, 0])
    phi = torch.fft.irfft2(ph, s=(g.ny, g.nx))
    phi = phi - weighted_mean(g, phi)
    if return_mean:
        return phi, mb
    return phi
