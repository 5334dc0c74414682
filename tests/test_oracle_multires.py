"""Pins of the oracle's multiple-resolution temperature grid (Sec. 6, refined
temperature grid with its own time step) against what the mathematics fixes:
nesting of the fine grid, a library interpolator (scipy's RegularGridInterpolator
on periodically padded coordinates), exactness for the laminar Couette and
conduction profiles, reduction to the single-grid temperature update at
refinement 1, the closed-form amplification of a Fourier mode advected by a
uniform velocity under the three-stage third-order Runge-Kutta scheme, and the
conduction steady state of a full coupled step."""
import math

import numpy as np
import pytest
import torch

import synth
from oracle import Grid, timestep as ts, multires as mr

si = pytest.importorskip("scipy.interpolate")


def grid(nx, ny, nz, stretch=1.5, lx=1.0, ly=1.0):
    return Grid(nx, ny, nz, lx, ly, synth.tanh_faces(nz, stretch))


def rnd(shape, seed):
    return torch.as_tensor(synth.noise(shape, seed), dtype=torch.float64)


@pytest.mark.parametrize("r", [(1, 1, 1), (2, 2, 2), (3, 2, 1), (1, 1, 4)])
def test_fine_grid_nests_coarse(r):
    g = grid(8, 8, 6)
    gf = mr.fine_grid(g, *r)
    assert (gf.nx, gf.ny, gf.nz) == (r[0] * 8, r[1] * 8, r[2] * 6)
    assert torch.equal(gf.zf[:: r[2]], g.zf)  # coarse face k is fine face rz k, exactly
    dz = gf.dzc.reshape(g.nz, r[2])
    assert torch.allclose(dz, (g.dzc / r[2])[:, None].expand(-1, r[2]), rtol=1e-13, atol=0)
    assert abs(gf.dx * r[0] - g.dx) < 1e-15 and abs(gf.dy * r[1] - g.dy) < 1e-15


def test_prolong_identity_at_refinement_one():
    g = grid(8, 6, 5)
    gf = mr.fine_grid(g, 1, 1, 1)
    u, v = rnd((5, 6, 8), 1), rnd((5, 6, 8), 2)
    w = rnd((6, 6, 8), 3)
    w[0] = 0.0
    w[-1] = 0.0
    uf, vf, wf = mr.prolong(g, gf, (1, 1, 1), u, v, w, 0.3, -0.7)
    assert torch.equal(uf, u) and torch.equal(vf, v) and torch.equal(wf, w)


def _padded_interp(xs_c, period, vals_axis, q, axis):
    """Periodic padding of axis `axis` of q by one sample on each side."""
    first = np.take(q, [0], axis=axis)
    last = np.take(q, [-1], axis=axis)
    return np.concatenate([xs_c[-1:] - period, xs_c, xs_c[:1] + period]), np.concatenate([last, q, first], axis=axis)


@pytest.mark.parametrize("r", [(2, 2, 2), (3, 1, 2), (2, 3, 3)])
def test_prolong_matches_library_interpolator(r):
    """Trilinear interpolation = scipy's linear RegularGridInterpolator on the
    coarse staggered coordinates (x, y padded periodically, z extended by the
    wall values for u, v), evaluated at the fine staggered coordinates."""
    g = grid(8, 6, 5, lx=2.0, ly=1.5)
    gf = mr.fine_grid(g, *r)
    u, v = rnd((5, 6, 8), 11), rnd((5, 6, 8), 12)
    w = rnd((6, 6, 8), 13)
    w[0] = 0.0
    w[-1] = 0.0
    ub, ut = 0.25, -1.0
    uf, vf, wf = mr.prolong(g, gf, r, u, v, w, ub, ut)

    xf_c, xc_c = np.arange(g.nx) * g.dx, (np.arange(g.nx) + 0.5) * g.dx
    yf_c, yc_c = np.arange(g.ny) * g.dy, (np.arange(g.ny) + 0.5) * g.dy
    Xf, Xc = np.arange(gf.nx) * gf.dx, (np.arange(gf.nx) + 0.5) * gf.dx
    Yf, Yc = np.arange(gf.ny) * gf.dy, (np.arange(gf.ny) + 0.5) * gf.dy
    zc = np.concatenate([[0.0], g.zc.numpy(), [1.0]])

    def ref(q, zs, xs, ys, Zq, Yq, Xq, bot=None, top=None):
        q = q.numpy()
        if bot is not None:
            q = np.concatenate([np.full((1,) + q.shape[1:], bot), q, np.full((1,) + q.shape[1:], top)])
        xs2, q = _padded_interp(xs, g.lx, None, q, 2)
        ys2, q = _padded_interp(ys, g.ly, None, q, 1)
        f = si.RegularGridInterpolator((zs, ys2, xs2), q, method="linear")
        Z, Y, X = np.meshgrid(Zq, Yq, Xq, indexing="ij")
        return torch.as_tensor(f(np.stack([Z, Y, X], axis=-1)))

    ru = ref(u, zc, xf_c, yc_c, gf.zc.numpy(), Yc, Xf, ub, ut)
    rv = ref(v, zc, xc_c, yf_c, gf.zc.numpy(), Yf, Xc, 0.0, 0.0)
    rw = ref(w, g.zf.numpy(), xc_c, yc_c, gf.zf.numpy(), Yc, Xc)
    assert float((uf - ru).abs().max()) < 1e-13
    assert float((vf - rv).abs().max()) < 1e-13
    assert float((wf - rw).abs().max()) < 1e-13


def test_prolong_exact_for_couette_profile():
    """The laminar Couette velocity (linear in z, wall values +-1) is linear
    along z through the wall points, so its interpolant is exact on the
    stretched fine grid: a distance-weighted, not volume-weighted, rule."""
    g = grid(16, 8, 7, stretch=2.0)
    gf = mr.fine_grid(g, 2, 2, 3)
    prof = lambda z: -1.0 + 2.0 * z
    u = prof(g.zc)[:, None, None].expand(g.nz, g.ny, g.nx).clone()
    z = torch.zeros(g.cell_shape(), dtype=torch.float64)
    wz = torch.zeros(g.face_shape(), dtype=torch.float64)
    uf, vf, wf = mr.prolong(g, gf, (2, 2, 3), u, z, wz, -1.0, 1.0)
    exact = prof(gf.zc)[:, None, None].expand_as(uf)
    assert float((uf - exact).abs().max()) < 1e-15
    assert float(vf.abs().max()) == 0.0 and float(wf.abs().max()) == 0.0


def test_restrict_exact_cases():
    g = grid(8, 6, 5)
    r = (2, 3, 2)
    gf = mr.fine_grid(g, *r)
    # conduction profile T = 1 - z, sampled on fine faces: restriction = coarse samples
    Tf = (1.0 - gf.zf)[:, None, None].expand(gf.nz + 1, gf.ny, gf.nx).clone()
    Tc = mr.restrict(r, Tf)
    Tc_exact = (1.0 - g.zf)[:, None, None].expand(g.nz + 1, g.ny, g.nx)
    assert float((Tc - Tc_exact).abs().max()) < 1e-15  # a mean of equal values, up to its rounding
    # a field constant over each coarse cell's fine columns restricts to that constant
    c = rnd((g.nz + 1, g.ny, g.nx), 4)
    Tf = c.repeat_interleave(r[1], dim=1).repeat_interleave(r[0], dim=2)
    Tf = torch.cat([torch.cat([Tf[k:k + 1]] + [rnd((1, gf.ny, gf.nx), 100 + k)] * (r[2] - 1))
                    for k in range(g.nz)] + [Tf[-1:]])
    assert Tf.shape == (gf.nz + 1, gf.ny, gf.nx)
    assert float((mr.restrict(r, Tf) - c).abs().max()) < 1e-15
    # block mean: one non-zero fine value weighs 1 / (rx ry)
    Tf = torch.zeros(gf.nz + 1, gf.ny, gf.nx, dtype=torch.float64)
    Tf[2 * r[2], 4, 5] = 6.0
    Tc = mr.restrict(r, Tf)
    assert float(Tc[2, 4 // r[1], 5 // r[0]]) == pytest.approx(1.0, abs=1e-15)
    assert float(Tc.abs().sum()) == pytest.approx(1.0, abs=1e-15)


@pytest.mark.parametrize("l", [0, 1, 2])
def test_scalar_substep_reduces_to_single_grid(l):
    """Refinement 1: the fine temperature substep is the temperature part of the
    single-grid substep (same equation, same velocity)."""
    g = grid(8, 8, 6)
    w_ = synth.workload("pc64", nx=8, ny=8, nz=6)
    u, v, w = (torch.as_tensor(a, dtype=torch.float64) for a in synth.velocity_noise(w_, 5))
    T = rnd((7, 8, 8), 6)
    p = rnd((6, 8, 8), 7)
    Hprev = tuple(rnd(s, 20 + i) for i, s in enumerate([(6, 8, 8), (6, 8, 8), (7, 8, 8), (7, 8, 8)]))
    ph = ts.Phys(nu=0.01, kappa=0.02, buoyancy=1.0, T_bot=1.0, T_top=0.0)
    dt = 3e-3
    (_, _, _, Tn, _), (_, _, _, HT) = ts.substep(g, ph, l, dt, (u, v, w, T, p), Hprev)
    gf = mr.fine_grid(g, 1, 1, 1)
    velf = mr.prolong(g, gf, (1, 1, 1), u, v, w, ph.u_bot, ph.u_top)
    Tm, HTm = mr.scalar_substep(gf, ph, l, dt, velf, T, Hprev[3] if l > 0 else None)
    assert float((Tm - Tn).abs().max()) < 1e-15
    assert float((HTm - HT).abs().max()) < 1e-15


@pytest.mark.parametrize("r,n_sub", [((2, 2, 1), 1), ((2, 1, 2), 2), ((3, 2, 2), 3)])
def test_scalar_advance_fourier_mode_closed_form(r, n_sub):
    """Uniform velocity (U, V, 0), no diffusion: a horizontal Fourier mode on
    the fine grid obeys dT/dt = lambda T with lambda = -i (U sin(kx dx)/dx +
    V sin(ky dy)/dy) (central average-difference advection), and every
    three-stage third-order Runge-Kutta step multiplies it by
    1 + z + z^2/2 + z^3/6, z = lambda dt / n_sub. Wall planes stay fixed."""
    g = grid(8, 8, 4, lx=2.0, ly=1.0)
    gf = mr.fine_grid(g, *r)
    U, V = 0.7, -0.4
    ph = ts.Phys(nu=0.0, kappa=0.0, u_bot=U, u_top=U)
    u = torch.full(g.cell_shape(), U, dtype=torch.float64)
    v = torch.full(g.cell_shape(), V, dtype=torch.float64)
    w = torch.zeros(g.face_shape(), dtype=torch.float64)
    a, b = 3, 2
    kx, ky = 2 * math.pi * a / gf.lx, 2 * math.pi * b / gf.ly
    X = (torch.arange(gf.nx, dtype=torch.float64) + 0.5) * gf.dx
    Y = (torch.arange(gf.ny, dtype=torch.float64) + 0.5) * gf.dy
    phase = kx * X[None, :] + ky * Y[:, None]
    Tf = torch.cos(phase)[None].expand(gf.nz + 1, -1, -1).clone()
    Tf[0] = 1.0
    Tf[-1] = 0.0
    dt = 0.05
    out = mr.scalar_advance(g, gf, r, ph, dt, n_sub, (u, v, w), (u, v, w), Tf)
    lam = -1j * (U * math.sin(kx * gf.dx) / gf.dx + V * math.sin(ky * gf.dy) / gf.dy)
    z = lam * dt / n_sub
    G = (1 + z + z * z / 2 + z ** 3 / 6) ** n_sub
    exact = (G * torch.exp(1j * phase)).real
    # v is zero on the walls (no slip), so with rz > 1 the fine cells between a
    # wall and the first coarse centre see a sheared v: check the face planes
    # rz .. nzf - rz, whose neighbouring fine centres lie between coarse centres
    rz = r[2]
    inner = out[rz:gf.nz - rz + 1] if rz > 1 else out[1:-1]
    assert float((inner - exact[None]).abs().max()) < 1e-13
    assert float(out[0].sub(1.0).abs().max()) == 0.0 and float(out[-1].abs().max()) == 0.0


def test_step_keeps_conduction_state():
    """Rayleigh-Benard conduction state: no velocity and T linear in z on the
    fine grid is steady; the buoyancy (a function of z alone) is absorbed by
    the pressure, so the velocity stays zero to round-off."""
    g = grid(8, 8, 6)
    r = (2, 2, 2)
    gf = mr.fine_grid(g, *r)
    ph = ts.Phys(nu=1e-2, kappa=1e-2, buoyancy=1.0, T_bot=1.0, T_top=0.0)
    zero_c = torch.zeros(g.cell_shape(), dtype=torch.float64)
    state = (zero_c, zero_c.clone(), torch.zeros(g.face_shape(), dtype=torch.float64), zero_c.clone())
    Tf = (1.0 - gf.zf)[:, None, None].expand(gf.nz + 1, gf.ny, gf.nx).clone()
    (u, v, w, p), T2 = mr.step(g, gf, r, ph, 0.05, 2, state, Tf)
    assert float((T2 - Tf).abs().max()) < 1e-14
    assert max(float(u.abs().max()), float(v.abs().max()), float(w.abs().max())) < 1e-13
    assert float(p.abs().max()) > 1e-3  # the hydrostatic pressure built up


def test_scalar_advance_time_interpolation_third_order():
    """Velocity varying linearly in time between the two coarse states: the
    refined steps must evaluate it at their substep start times for the
    scheme to stay third order. A Fourier mode advected by a uniform U(t)
    has the exact amplification exp(-i s int U dt), s = sin(kx dx)/dx; the
    error must fall by about 2^3 each time n_sub doubles (a substep that used
    the wrong time would leave a first-order error, falling by 2)."""
    g = grid(16, 8, 4)
    r = (2, 1, 1)
    gf = mr.fine_grid(g, *r)
    U0, U1 = 0.3, 1.1
    ph = ts.Phys(nu=0.0, kappa=0.0)
    vel = []
    for U in (U0, U1):
        ph_u = torch.full(g.cell_shape(), U, dtype=torch.float64)
        vel.append((ph_u, torch.zeros(g.cell_shape(), dtype=torch.float64),
                    torch.zeros(g.face_shape(), dtype=torch.float64)))
    a = 5
    kx = 2 * math.pi * a / gf.lx
    X = (torch.arange(gf.nx, dtype=torch.float64) + 0.5) * gf.dx
    phase = (kx * X)[None, :].expand(gf.ny, -1)
    Tf = torch.cos(phase)[None].expand(gf.nz + 1, -1, -1).clone()
    s = math.sin(kx * gf.dx) / gf.dx
    dt = 0.6 / (s * U1)  # |lambda| dt / n_sub <= 0.3: the asymptotic range of the scheme
    errs = []
    for n_sub in (2, 4, 8):
        ph_w = ts.Phys(nu=0.0, kappa=0.0, u_bot=U0, u_top=U0)  # wall values only matter for rz > 1
        res = mr.scalar_advance(g, gf, r, ph_w, dt, n_sub, vel[0], vel[1], Tf)
        exact = (torch.exp(1j * phase) * complex(math.cos(-s * dt * (U0 + U1) / 2),
                                                 math.sin(-s * dt * (U0 + U1) / 2))).real
        errs.append(float((res[1:-1] - exact[None]).abs().max()))
    assert errs[0] / errs[1] > 6.5 and errs[1] / errs[2] > 7.0, errs
