"""Pins of the oracle's operators and Poisson solve against facts fixed by the
mathematics, not by the oracle's own code: closed-form discrete eigenpairs,
a dense brute-force solve assembled from the face/cell geometry, summation by
parts, manufactured solutions and second-order convergence to the continuum."""
import math

import numpy as np
import pytest
import torch

import synth
from oracle import Grid, operators as op, poisson


def grid(nx, ny, nz, stretch=1.5, lx=1.0, ly=1.0):
    return Grid(nx, ny, nz, lx, ly, synth.tanh_faces(nz, stretch))


def t(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64)


def test_faces():
    for s in (0.0, 1.5, 2.5):
        z = synth.tanh_faces(24, s)
        assert z[0] == 0.0 and z[-1] == 1.0
        assert np.all(np.diff(z) > 0)
        np.testing.assert_allclose(z + z[::-1], 1.0, atol=1e-15)   # symmetric
    np.testing.assert_allclose(np.diff(synth.tanh_faces(10, 0.0)), 0.1, atol=1e-15)
    g = grid(4, 4, 12)
    # centre spacings add up to the distance between the wall planes
    assert abs(float(g.dzf.sum()) - 1.0) < 1e-15


def dense_operators(g):
    """Divergence (cells x faces) and gradient (faces x cells) matrices assembled
    face by face from the geometry: unknown ordering z-major, x fastest."""
    nx, ny, nz = g.nx, g.ny, g.nz
    dzc = g.dzc.numpy()
    zf = g.zf.numpy()
    zc = 0.5 * (zf[1:] + zf[:-1])
    nc = nx * ny * nz
    cell = lambda i, j, k: (k * ny + j % ny) * nx + i % nx
    # face lists: x-faces (i,j,k), y-faces, interior z-faces (k = 1..nz-1)
    faces = []
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                faces.append(("x", i, j, k))
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                faces.append(("y", i, j, k))
    for k in range(1, nz):
        for j in range(ny):
            for i in range(nx):
                faces.append(("z", i, j, k))
    nf = len(faces)
    Dm = np.zeros((nc, nf))
    Gm = np.zeros((nf, nc))
    for f, (d, i, j, k) in enumerate(faces):
        if d == "x":   # face between cells (i-1) and i, area dy dz, normal +x
            lo, hi, h, area = cell(i - 1, j, k), cell(i, j, k), g.dx, g.dy * dzc[k]
        elif d == "y":
            lo, hi, h, area = cell(i, j - 1, k), cell(i, j, k), g.dy, g.dx * dzc[k]
        else:
            lo, hi, h, area = cell(i, j, k - 1), cell(i, j, k), zc[k] - zc[k - 1], g.dx * g.dy
        Gm[f, hi] += 1.0 / h
        Gm[f, lo] -= 1.0 / h
        # outward flux of cell lo is +area*q, of cell hi is -area*q; divide by volume
        vol_lo = g.dx * g.dy * dzc[k - 1 if d == "z" else k]
        vol_hi = g.dx * g.dy * dzc[k]
        Dm[lo, f] += area / vol_lo
        Dm[hi, f] -= area / vol_hi
    return Dm, Gm, faces


def test_dense_laplacian_matches_stencil():
    g = grid(4, 6, 5)
    Dm, Gm, _ = dense_operators(g)
    L = Dm @ Gm
    phi = synth.noise(g.cell_shape(), seed=3)
    ref = (L @ phi.reshape(-1)).reshape(g.cell_shape())
    got = op.laplacian(g, t(phi)).numpy()
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-10 * np.abs(ref).max())


@pytest.mark.parametrize("shape", [(8, 8, 8), (8, 4, 6)])
def test_dense_bruteforce_solve(shape):
    """8^3 dense LU with one row replaced by the gauge (zero weighted mean)."""
    nx, ny, nz = shape
    g = grid(nx, ny, nz)
    Dm, Gm, _ = dense_operators(g)
    L = Dm @ Gm
    wc = np.repeat(g.dzc.numpy(), nx * ny)
    b = synth.noise(g.cell_shape(), seed=1).reshape(-1)
    b = b - (wc * b).sum() / wc.sum()
    A = L.copy()
    rhs = b.copy()
    A[0, :] = wc
    rhs[0] = 0.0
    ref = np.linalg.solve(A, rhs).reshape(g.cell_shape())
    got = poisson.solve(g, t(b.reshape(g.cell_shape()))).numpy()
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err < 1e-12, err


def test_summation_by_parts():
    """sum_cells W_c phi D(u) = -sum_faces W_f u . G phi when w vanishes on the walls."""
    g = grid(6, 5, 7)
    u, v, w = (t(a) for a in synth.velocity_noise(synth.workload("pc64", nx=6, ny=5, nz=7), 4))
    phi = t(synth.noise(g.cell_shape(), seed=5))
    lhs = float((g.w_cell() * phi * op.divergence(g, u, v, w)).sum())
    gu, gv, gw = op.gradient(g, phi)
    rhs = -float((g.w_cell() * (u * gu + v * gv)).sum() + (g.w_face() * w * gw).sum())
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def closed_form_mode(g, a, b, m):
    xc = (np.arange(g.nx) + 0.5) * g.dx
    yc = (np.arange(g.ny) + 0.5) * g.dy
    zc = g.zc.numpy()
    f = (np.cos(np.pi * m * zc)[:, None, None] * np.cos(2 * np.pi * b * yc / g.ly)[None, :, None]
         * np.cos(2 * np.pi * a * xc / g.lx)[None, None, :])
    dz = 1.0 / g.nz
    lam = (4 * math.sin(math.pi * a / g.nx) ** 2 / g.dx**2
           + 4 * math.sin(math.pi * b / g.ny) ** 2 / g.dy**2
           + 4 * math.sin(math.pi * m / (2 * g.nz)) ** 2 / dz**2)
    return f, lam


@pytest.mark.parametrize("abm", [(1, 0, 0), (0, 2, 1), (3, 1, 2), (4, 4, 7), (0, 0, 3), (2, 3, 0)])
def test_closed_form_eigenpairs_uniform(abm):
    """On a uniform wall-normal grid cos(2pi a x)cos(2pi b y)cos(pi m z) sampled at
    centres is an exact eigenvector of L with eigenvalue
    -(4sin^2(pi a/Nx)/dx^2 + 4sin^2(pi b/Ny)/dy^2 + 4sin^2(pi m/(2Nz))/dz^2)."""
    g = grid(8, 8, 8, stretch=0.0, lx=2.0, ly=1.5)
    f, lam = closed_form_mode(g, *abm)
    Lf = op.laplacian(g, t(f)).numpy()
    np.testing.assert_allclose(Lf, -lam * f, atol=1e-11 * max(lam, 1.0))
    if lam > 0:
        phi = poisson.solve(g, t(f)).numpy()
        np.testing.assert_allclose(phi, -f / lam, atol=1e-13 * np.abs(f).max() / lam + 1e-16)


def test_manufactured_stretched():
    g = grid(16, 8, 12, stretch=2.0, lx=2 * math.pi, ly=math.pi)
    phi = t(synth.noise(g.cell_shape(), seed=7))
    phi = phi - poisson.weighted_mean(g, phi)
    b = op.laplacian(g, phi)
    got = poisson.solve(g, b)
    err = float((got - phi).norm() / phi.norm())
    assert err < 1e-12, err


def test_zero_mode_prefix_matches_dense():
    g = grid(1, 1, 9, stretch=1.5)
    a, c = poisson.z_coefficients(g)
    n = g.nz
    M = np.diag((-a - c).numpy()) + np.diag(a[1:].numpy(), -1) + np.diag(c[:-1].numpy(), 1)
    b = synth.noise(n, seed=11)
    dzc = g.dzc.numpy()
    b = b - (dzc * b).sum() / dzc.sum()
    A = M.copy()
    rhs = b.copy()
    A[0] = 0.0
    A[0, 0] = 1.0
    rhs[0] = 0.0            # phi_0 = 0, the prefix-sum gauge
    ref = np.linalg.solve(A, rhs)
    got = poisson.zero_mode(g, t(b)).numpy()
    np.testing.assert_allclose(got, ref, atol=1e-12 * np.abs(ref).max())


def test_second_order_convergence_to_continuum():
    """Continuum solution of lap phi = b with b = cos(2pi x)cos(2pi y)cos(pi z):
    phi = -b / (8 pi^2 + pi^2); the discrete error falls ~4x per refinement."""
    errs = []
    for n in (8, 16, 32):
        g = grid(n, n, n, stretch=1.5)
        xc = (np.arange(n) + 0.5) / n
        zc = g.zc.numpy()
        b = (np.cos(np.pi * zc)[:, None, None] * np.cos(2 * np.pi * xc)[None, :, None]
             * np.cos(2 * np.pi * xc)[None, None, :])
        exact = -b / (9 * np.pi**2)
        phi = poisson.solve(g, t(b)).numpy()
        errs.append(np.abs(phi - exact).max())
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(1.8 < r < 2.3 for r in rates), (errs, rates)


def test_mean_removal_and_gauge():
    g = grid(8, 8, 6)
    b = t(synth.noise(g.cell_shape(), seed=2)) + 3.0
    phi, mb = poisson.solve(g, b, return_mean=True)
    assert abs(float(mb) - 3.0) < 0.5
    assert abs(float(poisson.weighted_mean(g, phi))) < 1e-15
    r = op.laplacian(g, phi) - (b - mb)
    assert float(r.abs().max()) < 1e-11 * float(b.abs().max())


def test_sampled_mode_oracle_matches_full_solve():
    """The sampled-mode oracle (direct DFT + the same column solves) against the
    FFT of the full oracle solve, and its direct DFT against the library FFT."""
    from oracle import sampled
    g = grid(32, 16, 11, stretch=1.5, lx=1.3, ly=0.7)
    b = t(synth.noise(g.cell_shape(), seed=4)) + 0.2
    pairs = sampled.default_pairs(g, count=12)
    bh = torch.fft.rfft2(b).numpy()
    cols = sampled.mode_columns(g, b, pairs)
    for (kx, ky), v in cols.items():
        np.testing.assert_allclose(v, bh[:, ky, kx], atol=1e-12 * np.abs(bh).max())
    ph = torch.fft.rfft2(poisson.solve(g, b)).numpy()
    got = sampled.solve_modes(g, b, pairs)
    scale = np.abs(ph).max()
    for (kx, ky), v in got.items():
        np.testing.assert_allclose(v, ph[:, ky, kx], atol=1e-12 * scale)
