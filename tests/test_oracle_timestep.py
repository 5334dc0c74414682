"""Pins of the oracle's projection, advection, Crank-Nicolson solves, RK3
integrator, CFL and Nusselt number against properties fixed by the paper or by
the mathematics: solenoidal projection to round-off (Sec. 2.2), projector
identities, energy conservation of the advection operator (Sec. 2.1), exact
steady states (conduction, laminar Couette), Runge-Kutta order conditions and
the sqrt(3) stability limit (Sec. 2.1), and the Listing 1 CFL formula."""
import json
import math
import os

import numpy as np
import pytest
import torch

import synth
from oracle import Grid, operators as op, poisson, timestep as ts

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))


def t(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64)


def grid(nx, ny, nz, stretch=1.5, lx=1.0, ly=1.0):
    return Grid(nx, ny, nz, lx, ly, synth.tanh_faces(nz, stretch))


def random_velocity(g, seed):
    w = synth.workload("pc64", nx=g.nx, ny=g.ny, nz=g.nz)
    return tuple(t(a) for a in synth.velocity_noise(w, seed))


def solenoidal(g, seed):
    u, v, w = random_velocity(g, seed)
    p = torch.zeros(g.cell_shape(), dtype=torch.float64)
    u, v, w, _, _ = ts.pressure_correction(g, u, v, w, p)
    return u, v, w


# projection ---------------------------------------------------------------------
def test_projection_divergence_roundoff():
    g = grid(16, 12, 10)
    u, v, w = random_velocity(g, 0)
    p = torch.zeros(g.cell_shape(), dtype=torch.float64)
    d0 = float(op.divergence(g, u, v, w).abs().max())
    u2, v2, w2, p2, phi = ts.pressure_correction(g, u, v, w, p)
    d1 = float(op.divergence(g, u2, v2, w2).abs().max())
    # Sec. 2.2: residual divergence O(1e-13) in double precision
    assert d1 < GOLD["residual_divergence_fp64"]["value"] * 10 * max(1.0, d0 / 100), (d0, d1)
    assert float(w2[0].abs().max()) == 0.0 and float(w2[-1].abs().max()) == 0.0


def test_projection_is_weighted_orthogonal_projector():
    g = grid(8, 8, 6)
    z = torch.zeros(g.cell_shape(), dtype=torch.float64)
    P = lambda a: ts.pressure_correction(g, *a, z)[:3]
    a = random_velocity(g, 1)
    b = random_velocity(g, 2)
    Pa, Pb = P(a), P(b)
    PPa = P(Pa)
    for x, y in zip(Pa, PPa):                      # idempotent
        assert float((x - y).abs().max()) < 1e-12
    ip = lambda x, y: float((g.w_cell() * (x[0] * y[0] + x[1] * y[1])).sum()
                            + (g.w_face() * x[2] * y[2]).sum())
    assert abs(ip(Pa, b) - ip(a, Pb)) < 1e-12 * abs(ip(a, b) + 1.0)   # W_f-symmetric
    assert ip(Pa, Pa) <= ip(a, a)                                       # energy never grows


# advection ----------------------------------------------------------------------
def test_advection_energy_conservation():
    """sum W q A(q) vanishes for a discretely solenoidal field (Sec. 2.1)."""
    g = grid(12, 10, 9, stretch=2.0, lx=2.0, ly=1.3)
    u, v, w = solenoidal(g, 3)
    Au = op.adv_u(g, u, v, w)
    Av = op.adv_v(g, u, v, w)
    Aw = op.adv_face(g, u, v, w, w)
    T = t(synth.noise(g.face_shape(), seed=9))
    T[0] = 0.0
    T[-1] = 0.0
    AT = op.adv_face(g, u, v, w, T)
    scale = float((g.w_cell() * u * u).sum())
    for q, A, W in ((u, Au, g.w_cell()), (v, Av, g.w_cell()), (w, Aw, g.w_face()), (T, AT, g.w_face())):
        assert abs(float((W * q * A).sum())) < 1e-12 * scale * 100
    # and it is not trivially zero
    assert float(Au.abs().max()) > 1e-3


# Crank-Nicolson solves -----------------------------------------------------------
def test_cn_solves_against_operator():
    g = grid(5, 4, 11, stretch=2.0)
    beta = 0.37
    R = t(synth.noise(g.cell_shape(), seed=4))
    dq = ts.cn_solve_cell(g, beta, R)
    back = dq - beta * op.dzz_cell_dirichlet(g, dq, 0.0, 0.0)
    assert float((back - R).abs().max()) < 1e-12
    Rf = t(synth.noise(g.face_shape(), seed=5))
    Rf[0] = 0.0
    Rf[-1] = 0.0
    dqf = ts.cn_solve_face(g, beta, Rf)
    backf = dqf - beta * op.dzz_face(g, dqf)
    assert float((backf - Rf).abs().max()) < 1e-12


def test_dzz_exact_for_linear_profiles():
    g = grid(3, 3, 13, stretch=2.0)
    zc = g.zc[:, None, None].expand(g.cell_shape())
    q = 2.0 * zc - 1.0
    assert float(op.dzz_cell_dirichlet(g, q, -1.0, 1.0).abs().max()) < 1e-10
    zf = g.zf[:, None, None].expand(g.face_shape())
    assert float(op.dzz_face(g, 1.0 - zf).abs().max()) < 1e-10


# RK3 ------------------------------------------------------------------------------
def test_rk3_order_conditions():
    """Equivalent Butcher tableau of the low-storage scheme satisfies the
    third-order conditions."""
    G, R = ts.GAMMA, ts.RHO
    a21, a31, a32 = G[0], G[0] + R[1], G[1]
    b = (G[0] + R[1], G[1] + R[2], G[2])
    c = (0.0, a21, a31 + a32)
    assert abs(sum(b) - 1) < 1e-15
    assert abs(sum(bi * ci for bi, ci in zip(b, c)) - 0.5) < 1e-15
    assert abs(sum(bi * ci * ci for bi, ci in zip(b, c)) - 1 / 3) < 1e-15
    assert abs(b[2] * a32 * c[1] - 1 / 6) < 1e-15
    assert abs(sum(ts.ALPHA) - 1.0) < 1e-15


def scalar_step(y, dt, le, li):
    """One RK3/CN step of y' = le*y (explicit) + li*y (implicit) through the
    oracle's own substep building blocks."""
    Hp = None
    for l in range(3):
        H = le * y
        R = ts.rk3_rhs(l, dt, H, Hp, li * y)
        y = y + R / (1.0 - ts.cn_beta(l, dt, 1.0) * li)
        Hp = H
    return y


@pytest.mark.parametrize("le,li,order", [(-1.3 + 2.0j, 0.0, 3), (0.0, -2.0, 2), (-0.5 + 1j, -1.0, 2)])
def test_rk3_cn_temporal_order(le, li, order):
    errs = []
    for n in (20, 40, 80):
        dt = 1.0 / n
        y = 1.0 + 0j
        for _ in range(n):
            y = scalar_step(y, dt, le, li)
        errs.append(abs(y - np.exp(le + li)))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(abs(r - order) < 0.25 for r in rates), rates


def test_rk3_stability_limit_sqrt3():
    """Sec. 2.1: the RK3 stability limit on the imaginary axis is CFL sqrt(3)."""
    lim = GOLD["rk3_stability_limit_cfl"]["value"]
    amp = lambda w: abs(scalar_step(1.0 + 0j, 1.0, 1j * w, 0.0))
    assert amp(lim * 0.999) <= 1.0
    assert amp(lim * 1.01) > 1.0


# steady states ----------------------------------------------------------------------
def test_rb_conduction_is_steady():
    wl = synth.workload("rb512", nx=8, ny=8, nz=10)
    g = Grid(wl.nx, wl.ny, wl.nz, wl.lx, wl.ly, wl.faces())
    ph = ts.Phys(nu=1e-2, kappa=1e-2, buoyancy=1.0, T_bot=1.0, T_top=0.0)
    u, v, w, T, p = (t(a) for a in synth.rb_initial(wl, 0, amp=0.0))
    T0 = T.clone()
    state, H = (u, v, w, T, p), None
    for _ in range(3):
        state, H = ts.step(g, ph, 1e-2, state, H)
    u, v, w, T, p = state
    assert max(float(x.abs().max()) for x in (u, v, w)) < 1e-13
    assert float((T - T0).abs().max()) < 1e-13
    # hydrostatic balance: dp/dz = T on interior faces
    gw = op.gradient(g, p)[2]
    assert float((gw[1:-1] - T[1:-1]).abs().max()) < 1e-11
    assert abs(float(ts.nusselt(g, w, T, 1e8, 1.0)) - 1.0) < 1e-9


def test_laminar_couette_is_steady():
    wl = synth.workload("couette1024", nx=8, ny=6, nz=12)
    g = Grid(wl.nx, wl.ny, wl.nz, wl.lx, wl.ly, wl.faces())
    ph = ts.Phys(nu=wl.nu, u_bot=-1.0, u_top=1.0)
    u, v, w, p = (t(a) for a in synth.couette_initial(wl, 0, sigma=0.0))
    u0 = u.clone()
    state, H = (u, v, w, None, p), None
    for _ in range(3):
        state, H = ts.step(g, ph, 0.05, state, H)
    u, v, w, _, p = state
    assert float((u - u0).abs().max()) < 1e-13
    assert max(float(v.abs().max()), float(w.abs().max()), float(p.abs().max())) < 1e-13


# CFL (Listing 1) ------------------------------------------------------------------------
def test_cfl_listing1():
    g = grid(5, 4, 6, stretch=1.5, lx=2.0, ly=3.0)
    u, v, w = random_velocity(g, 8)
    un, vn, wn = u.numpy(), v.numpy(), w.numpy()
    dzc = g.dzc.numpy()
    best = GOLD["cfl_floor"]["value"]
    for k in range(g.nz):          # the listing's triple loop, one cell at a time
        for j in range(g.ny):
            for i in range(g.nx):
                ip, jp = (i + 1) % g.nx, (j + 1) % g.ny
                q = (abs((un[k, j, i] + un[k, j, ip]) / g.dx) + abs((vn[k, j, i] + vn[k, jp, i]) / g.dy)
                     + abs((wn[k, j, i] + wn[k + 1, j, i]) / dzc[k]))
                best = max(best, 0.5 * q)
    assert abs(op.cfl_number(g, u, v, w) - best) < 1e-14 * best
    z = torch.zeros_like(u)
    assert op.cfl_number(g, z, z, torch.zeros_like(w)) == GOLD["cfl_floor"]["value"]
    assert op.cfl_dt(g, z, z, torch.zeros_like(w), 0.7, 5e-3) == 5e-3


# explicit terms: closed forms of single Fourier modes ---------------------------------
# Sec. 2.1 fixes the discretisation as central, second-order and conservative on the
# staggered grid. For a single Fourier mode on the periodic directions the central
# differences have closed forms: the second difference of cos(theta_j) is
# -4 sin^2(dtheta/2) cos(theta_j), and the centred first difference of sin(theta_j)
# over two spacings is cos(theta_j) sin(dtheta). The fields below make every other
# term of H vanish exactly, so a dropped factor 1/2, a wrong sign or a wrong spacing
# in the horizontal diffusion or in the horizontal advection fluxes fails. Together
# with the energy identity above (the x, y and z contributions of sum W q A(q) only
# cancel with the right relative sign and scale), they pin the z fluxes too.
def _xy(g):
    """x at x-faces and centres, y at y-faces and centres, shaped for broadcasting."""
    i = torch.arange(g.nx, dtype=torch.float64)
    j = torch.arange(g.ny, dtype=torch.float64)
    return (i * g.dx)[None, None, :], ((i + 0.5) * g.dx)[None, None, :], \
        (j * g.dy)[None, :, None], ((j + 0.5) * g.dy)[None, :, None]


def _zero(g, face=False):
    return torch.zeros(g.face_shape() if face else g.cell_shape(), dtype=torch.float64)


def _rel(a, ref, scale):
    return float((a - ref).abs().max()) / scale


EXPLICIT_GRID = dict(nx=16, ny=12, nz=9, stretch=1.7, lx=2.3, ly=1.1)


def test_explicit_horizontal_diffusion_closed_form():
    """nu (dxx + dyy) of cos modes: Hu = -nu 4 sin^2(pi b/ny)/dy^2 u for
    u = cos(2 pi b y/ly), Hv = -nu 4 sin^2(pi a/nx)/dx^2 v for v = cos(2 pi a x/lx),
    and HT = -kappa (4 sin^2(pi a/nx)/dx^2 + 4 sin^2(pi b/ny)/dy^2) T; with the
    velocity zero, Hw = buoyancy T on the interior faces."""
    g = grid(**EXPLICIT_GRID)
    xf, xc, yf, yc = _xy(g)
    a, b = 3, 2
    nu, kappa, bu = 0.013, 0.021, 0.7
    ph = ts.Phys(nu=nu, kappa=kappa, buoyancy=bu)
    lamx = 4.0 * math.sin(math.pi * a / g.nx) ** 2 / g.dx ** 2
    lamy = 4.0 * math.sin(math.pi * b / g.ny) ** 2 / g.dy ** 2
    # u varies along y only (u sits at y-centres)
    u = torch.cos(2 * math.pi * b * yc / g.ly).expand(g.cell_shape()).clone()
    Hu, Hv, Hw, _ = ts.explicit_terms(g, ph, u, _zero(g), _zero(g, True), None)
    assert _rel(Hu, -nu * lamy * u, nu * lamy) < 1e-13
    assert float(Hv.abs().max()) == 0.0 and float(Hw.abs().max()) == 0.0
    # v varies along x only (v sits at x-centres)
    v = torch.cos(2 * math.pi * a * xc / g.lx).expand(g.cell_shape()).clone()
    Hu, Hv, Hw, _ = ts.explicit_terms(g, ph, _zero(g), v, _zero(g, True), None)
    assert _rel(Hv, -nu * lamx * v, nu * lamx) < 1e-13
    assert float(Hu.abs().max()) == 0.0 and float(Hw.abs().max()) == 0.0
    # T on faces, a 2-D mode times a z profile, walls held at T_bot, T_top = 0
    hz = torch.sin(math.pi * g.zf)[:, None, None]
    T = hz * torch.cos(2 * math.pi * a * xc / g.lx) * torch.cos(2 * math.pi * b * yc / g.ly)
    T[0] = 0.0
    T[-1] = 0.0
    Hu, Hv, Hw, HT = ts.explicit_terms(g, ph, _zero(g), _zero(g), _zero(g, True), T)
    lam = lamx + lamy
    assert _rel(HT[1:-1], -kappa * lam * T[1:-1], kappa * lam) < 1e-13
    assert float(HT[0].abs().max()) == 0.0 and float(HT[-1].abs().max()) == 0.0
    assert _rel(Hw[1:-1], bu * T[1:-1], bu) < 1e-15
    assert float(Hu.abs().max()) == 0.0 and float(Hv.abs().max()) == 0.0


def test_explicit_advection_of_v_by_uniform_u():
    """v = eps sin(2 pi a x/lx) carried by a uniform u = U (w = 0, solenoidal):
    Hv = -U (v_{i+1} - v_{i-1})/(2 dx) = -U eps cos(2 pi a x/lx) sin(2 pi a/nx)/dx,
    and Hu = 0 (u is uniform, v does not vary along y)."""
    g = grid(**EXPLICIT_GRID)
    xf, xc, yf, yc = _xy(g)
    a, U, eps = 3, 0.8, 0.05
    ph = ts.Phys()
    v = (eps * torch.sin(2 * math.pi * a * xc / g.lx)).expand(g.cell_shape()).clone()
    u = torch.full(g.cell_shape(), U, dtype=torch.float64)
    Hu, Hv, Hw, _ = ts.explicit_terms(g, ph, u, v, _zero(g, True), None)
    ref = -U * eps * torch.cos(2 * math.pi * a * xc / g.lx) * math.sin(2 * math.pi * a / g.nx) / g.dx
    scale = U * eps / g.dx
    assert _rel(Hv, ref.expand(g.cell_shape()), scale) < 1e-13
    assert float(Hu.abs().max()) < 1e-15 * scale
    assert float(Hw.abs().max()) == 0.0
    # the closed form is not trivially small
    assert float(ref.abs().max()) > 0.5 * U * eps * math.sin(2 * math.pi * a / g.nx) / g.dx


def test_explicit_advection_of_u_by_uniform_v():
    """u = eps sin(2 pi b y/ly) carried by a uniform v = V (w = 0, solenoidal):
    Hu = -V (u_{j+1} - u_{j-1})/(2 dy) = -V eps cos(2 pi b y/ly) sin(2 pi b/ny)/dy,
    and Hv = 0."""
    g = grid(**EXPLICIT_GRID)
    xf, xc, yf, yc = _xy(g)
    b, V, eps = 2, -0.6, 0.05
    ph = ts.Phys()
    u = (eps * torch.sin(2 * math.pi * b * yc / g.ly)).expand(g.cell_shape()).clone()
    v = torch.full(g.cell_shape(), V, dtype=torch.float64)
    Hu, Hv, Hw, _ = ts.explicit_terms(g, ph, u, v, _zero(g, True), None)
    ref = -V * eps * torch.cos(2 * math.pi * b * yc / g.ly) * math.sin(2 * math.pi * b / g.ny) / g.dy
    scale = abs(V) * eps / g.dy
    assert _rel(Hu, ref.expand(g.cell_shape()), scale) < 1e-13
    assert float(Hv.abs().max()) < 1e-15 * scale
    assert float(Hw.abs().max()) == 0.0


def test_explicit_advection_of_face_scalar_by_uniform_flow():
    """T = eps h(z) sin(theta), theta = 2 pi (a x/lx + b y/ly), carried by a
    uniform (U, V) (w = 0): the volume-weighted interpolation reproduces U and V
    on the z-faces, so HT = -eps h(z) cos(theta) (U sin(2 pi a/nx)/dx
    + V sin(2 pi b/ny)/dy) on the interior faces, zero on the walls; the same
    horizontal fluxes serve w."""
    g = grid(**EXPLICIT_GRID)
    xf, xc, yf, yc = _xy(g)
    a, b, U, V, eps = 2, 3, 0.8, -0.6, 0.05
    ph = ts.Phys()
    hz = (1.0 + g.zf)[:, None, None]
    th = 2 * math.pi * (a * xc / g.lx + b * yc / g.ly)
    T = eps * hz * torch.sin(th)
    T[0] = 0.0
    T[-1] = 0.0
    u = torch.full(g.cell_shape(), U, dtype=torch.float64)
    v = torch.full(g.cell_shape(), V, dtype=torch.float64)
    _, _, _, HT = ts.explicit_terms(g, ph, u, v, _zero(g, True), T)
    ref = -eps * hz * torch.cos(th) * (U * math.sin(2 * math.pi * a / g.nx) / g.dx
                                       + V * math.sin(2 * math.pi * b / g.ny) / g.dy)
    scale = eps * (abs(U) / g.dx + abs(V) / g.dy) * 2.0
    assert _rel(HT[1:-1], ref[1:-1], scale) < 1e-13
    assert float(HT[0].abs().max()) == 0.0 and float(HT[-1].abs().max()) == 0.0
