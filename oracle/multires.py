"""Multiple-resolution temperature grid with a refined temperature time step
(Sec. 6, conclusions and future plans: the temperature lives on a grid finer
than that of the momentum and is integrated with its own, smaller time step;
the paper defers the details to a cited paper on the multiple-resolution
strategy).

TEST INFRASTRUCTURE ONLY (see the package header).

The paper fixes only the idea, so every step below is a reading:

* Fine grid: every coarse cell is split into rx x ry x rz equal cells. The
  fine z-faces nest the coarse ones: zf_fine[rz k + m] = zf[k] + m (zf[k+1] -
  zf[k]) / rz, so coarse face k is fine face rz k.
* Velocity onto the fine grid: each component is interpolated linearly along
  each direction, from its own coarse staggered positions to its own fine
  staggered positions (trilinear). x, y are periodic. Along z a cell-centred
  component (u, v) is taken to its Dirichlet wall value (u_bot / u_top for u,
  0 for v) on the wall plane, half a cell below the first centre and above the
  last; w, on z-faces, is linear between coarse faces (zero on the walls).
* Time: in a coarse step t -> t + dt the momentum takes its three RK3/CN
  substeps with the buoyancy of the restricted temperature at t, held fixed;
  the fine temperature then takes n_sub RK3/CN steps of dt / n_sub, each
  substep using the velocity at its own start time, linear in time between
  the coarse velocities at t and t + dt (substep starts at fractions 0, 8/15
  and 2/3 of a fine step: the partial sums of alpha).
* Fine temperature equation: exactly the single-grid one (explicit advection in
  divergence form and horizontal diffusion, Crank-Nicolson wall-normal
  diffusion, Dirichlet wall values) written on the fine grid with the fine
  velocity.
* Restriction (fine T -> coarse T, for the buoyancy and for statistics): the
  mean of the rx x ry fine values over a coarse cell's horizontal extent, on
  the coincident face plane rz k.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np
import torch

from .grid import Grid
from . import operators as op
from . import timestep as ts

# substep start times within one RK3 step, as fractions of the step
STAGE_START = (0.0, ts.ALPHA[0], ts.ALPHA[0] + ts.ALPHA[1])


def fine_grid(g: Grid, rx: int, ry: int, rz: int) -> Grid:
    """The refined grid: rx nx x ry ny cells, each coarse z-cell split in rz."""
    zf = g.zf.tolist()
    out = []
    for k in range(g.nz):
        for m in range(rz):
            out.append(zf[k] + (zf[k + 1] - zf[k]) * m / rz)
    out.append(zf[g.nz])
    return Grid(rx * g.nx, ry * g.ny, rz * g.nz, g.lx, g.ly, out)


# one-dimensional linear interpolation matrices ---------------------------------
def periodic_matrix(n: int, r: int, centred: bool) -> np.ndarray:
    """[r n][n]: coarse samples at (i + o) h -> fine positions (I + o) h / r,
    o = 1/2 for cell centres and 0 for faces, periodic with period n h."""
    o = Fraction(1, 2) if centred else Fraction(0)
    M = np.zeros((r * n, n))
    for I in range(r * n):
        s = (I + o) / r - o  # fine position in coarse index units
        i0 = s.numerator // s.denominator
        t = s - i0
        M[I, i0 % n] += float(1 - t)
        M[I, (i0 + 1) % n] += float(t)
    return M


def bracket_matrix(xc, xf) -> np.ndarray:
    """[len(xf)][len(xc)]: piecewise-linear interpolation from the increasing
    positions xc to the positions xf (all inside [xc[0], xc[-1]])."""
    xc = np.asarray(xc, dtype=np.float64)
    xf = np.asarray(xf, dtype=np.float64)
    M = np.zeros((len(xf), len(xc)))
    for K, z in enumerate(xf):
        a = int(np.searchsorted(xc, z, side="right")) - 1
        a = min(max(a, 0), len(xc) - 2)
        t = (z - xc[a]) / (xc[a + 1] - xc[a])
        M[K, a] += 1.0 - t
        M[K, a + 1] += t
    return M


def _apply(Mz, My, Mx, q):
    """out[K][J][I] = sum Mz[K,k] My[J,j] Mx[I,i] q[k][j][i], one axis at a time."""
    Mz, My, Mx = (torch.as_tensor(m, dtype=torch.float64) for m in (Mz, My, Mx))
    q = torch.einsum("Ii,kji->kjI", Mx, q)
    q = torch.einsum("Jj,kjI->kJI", My, q)
    return torch.einsum("Kk,kJI->KJI", Mz, q)


def prolong(g: Grid, gf: Grid, r, u, v, w, u_bot: float, u_top: float):
    """Coarse (u, v, w) -> fine (u, v, w), trilinear on the staggered grids."""
    rx, ry, rz = r
    zc_ext = [float(g.zf[0])] + g.zc.tolist() + [float(g.zf[-1])]
    Mz_c = bracket_matrix(zc_ext, gf.zc.tolist())
    Mz_f = bracket_matrix(g.zf.tolist(), gf.zf.tolist())
    X_face, X_cen = periodic_matrix(g.nx, rx, False), periodic_matrix(g.nx, rx, True)
    Y_face, Y_cen = periodic_matrix(g.ny, ry, False), periodic_matrix(g.ny, ry, True)

    def ext(q, bot, top):
        lo = torch.full((1,) + tuple(q.shape[1:]), bot, dtype=torch.float64)
        hi = torch.full((1,) + tuple(q.shape[1:]), top, dtype=torch.float64)
        return torch.cat([lo, q, hi], dim=0)

    uf = _apply(Mz_c, Y_cen, X_face, ext(u, u_bot, u_top))
    vf = _apply(Mz_c, Y_face, X_cen, ext(v, 0.0, 0.0))
    wf = _apply(Mz_f, Y_cen, X_cen, w)
    return uf, vf, wf


def restrict(r, Tf):
    """Fine face field [rz nz + 1][ry ny][rx nx] -> coarse face field: the mean
    over each coarse cell's rx x ry fine columns on face plane rz k."""
    rx, ry, rz = r
    planes = Tf[::rz]
    nzp, nyf, nxf = planes.shape
    return planes.reshape(nzp, nyf // ry, ry, nxf // rx, rx).mean(dim=(2, 4))


# the fine temperature ------------------------------------------------------------
def scalar_substep(gf: Grid, ph: ts.Phys, l: int, dt: float, vel, T, HTprev):
    """RK3/CN substep l of the temperature alone on grid gf with the velocity
    vel = (u, v, w) of that grid; the same equation as the single-grid substep.
    Returns (T_new, HT)."""
    u, v, w = vel
    HT = ts._zero_walls(-op.adv_face(gf, u, v, w, T) + ph.kappa * op.lap_h(gf, T))
    RT = ts.rk3_rhs(l, dt, HT, HTprev, ph.kappa * op.dzz_face(gf, T))
    return T + ts.cn_solve_face(gf, ts.cn_beta(l, dt, ph.kappa), RT), HT


def velocity_at(g, gf, r, ph, vel0, vel1, theta: float):
    """Fine velocity at t + theta dt: the coarse states linear in time, then
    prolonged."""
    lerp = [a + theta * (b - a) for a, b in zip(vel0, vel1)]
    return prolong(g, gf, r, *lerp, ph.u_bot, ph.u_top)


def scalar_advance(g: Grid, gf: Grid, r, ph: ts.Phys, dt: float, n_sub: int, vel0, vel1, Tf):
    """Fine temperature from t to t + dt in n_sub RK3/CN steps of dt / n_sub."""
    dts = dt / n_sub
    for m in range(n_sub):
        HT = None
        for l in range(3):
            theta = (m + STAGE_START[l]) / n_sub
            velf = velocity_at(g, gf, r, ph, vel0, vel1, theta)
            Tf, HT = scalar_substep(gf, ph, l, dts, velf, Tf, HT)
    return Tf


def step(g: Grid, gf: Grid, r, ph: ts.Phys, dt: float, n_sub: int, state, Tf):
    """One coarse step: state = (u, v, w, p) on g, Tf on gf. Returns
    ((u, v, w, p), Tf)."""
    u, v, w, p = state
    Tc = restrict(r, Tf)
    vel0 = (u, v, w)
    H = None
    for l in range(3):
        (u, v, w, _, p), H = ts.substep(g, ph, l, dt, (u, v, w, Tc, p), H, advance_scalar=False)
    Tf = scalar_advance(g, gf, r, ph, dt, n_sub, vel0, (u, v, w), Tf)
    return (u, v, w, p), Tf
