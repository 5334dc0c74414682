"""Conservative central second-order finite differences on the staggered grid.

Sec. 2.1 fixes the discretisation family (conservative, central, second-order,
staggered, energy-conserving as dt -> 0) without printing the stencils; the
readings used here are the standard ones for that family:

* divergence at cell centres, gradient at faces, their composition the
  7-point Laplacian with zero wall-normal flux at the walls;
* advection in divergence form with arithmetic face averages, and
  volume-weighted interpolation of the horizontal velocities onto z-faces,
  which is what makes sum_W q A(q) vanish for a discretely solenoidal field;
* horizontal viscous terms explicit, wall-normal second differences kept
  separate because they are treated implicitly (Sec. 2.1, Sec. 2.2 first
  paragraph);
* CFL number exactly as in Listing 1.

Shapes: u, v, p, phi [nz][ny][nx]; w, T [nz+1][ny][nx] (walls at 0 and nz).
"""
from __future__ import annotations

import torch

from .grid import Grid


# periodic neighbours ---------------------------------------------------------
def xp(a):  # value at i+1
    return torch.roll(a, -1, dims=2)


def xm(a):  # value at i-1
    return torch.roll(a, 1, dims=2)


def yp(a):
    return torch.roll(a, -1, dims=1)


def ym(a):
    return torch.roll(a, 1, dims=1)


def col(v):
    return v[:, None, None]


# divergence / gradient / Laplacian (Sec. 2.2 step 1; the Poisson operator) ----
def divergence(g: Grid, u, v, w):
    """D at cell centres: (u_{i+1}-u_i)/dx + (v_{j+1}-v_j)/dy + (w_{k+1}-w_k)/dzc_k."""
    return (xp(u) - u) / g.dx + (yp(v) - v) / g.dy + (w[1:] - w[:-1]) / col(g.dzc)


def gradient(g: Grid, phi):
    """G of a cell field: x-faces, y-faces, and interior z-faces (zero on the walls)."""
    gu = (phi - xm(phi)) / g.dx
    gv = (phi - ym(phi)) / g.dy
    gw = torch.zeros(g.face_shape(), dtype=phi.dtype)
    gw[1:-1] = (phi[1:] - phi[:-1]) / col(g.dzf[1:-1])
    return gu, gv, gw


def laplacian(g: Grid, phi):
    """L = D o G: the 7-point Laplacian, periodic in x, y, zero flux at the walls."""
    return divergence(g, *gradient(g, phi))


def dzz_cell_neumann(g: Grid, phi):
    """Wall-normal part of L at cell centres (zero flux through the walls)."""
    flux = torch.zeros(g.face_shape(), dtype=phi.dtype)
    flux[1:-1] = (phi[1:] - phi[:-1]) / col(g.dzf[1:-1])
    return (flux[1:] - flux[:-1]) / col(g.dzc)


def dzz_cell_dirichlet(g: Grid, q, q_bot: float, q_top: float):
    """Wall-normal second difference of a cell field with Dirichlet wall values.

    The wall value sits on the wall, half a cell (dzf[0] = dzc[0]/2) from the
    first centre, so a linear profile is differenced exactly.
    """
    flux = torch.empty(g.face_shape(), dtype=q.dtype)
    flux[1:-1] = (q[1:] - q[:-1]) / col(g.dzf[1:-1])
    flux[0] = (q[0] - q_bot) / g.dzf[0]
    flux[-1] = (q_top - q[-1]) / g.dzf[-1]
    return (flux[1:] - flux[:-1]) / col(g.dzc)


def dzz_face(g: Grid, q):
    """Wall-normal second difference on interior z-faces; q[0], q[nz] are the wall
    values. Returns a face-shaped array that is zero on the walls."""
    flux = (q[1:] - q[:-1]) / col(g.dzc)  # at cell centres
    out = torch.zeros_like(q)
    out[1:-1] = (flux[1:] - flux[:-1]) / col(g.dzf[1:-1])
    return out


def lap_h(g: Grid, q):
    """Horizontal (periodic, uniform) Laplacian, treated explicitly (Sec. 2.2)."""
    return (xp(q) - 2.0 * q + xm(q)) / g.dx**2 + (yp(q) - 2.0 * q + ym(q)) / g.dy**2


# advection, conservative divergence form (Sec. 2.1) --------------------------
def z_to_face(g: Grid, q):
    """Volume-weighted interpolation of a cell field onto interior z-faces:
    (dzc_{k-1} q_{k-1} + dzc_k q_k) / (2 dzf_k), face-shaped, zero on the walls."""
    out = torch.zeros((g.nz + 1,) + tuple(q.shape[1:]), dtype=q.dtype)
    out[1:-1] = (col(g.dzc[:-1]) * q[:-1] + col(g.dzc[1:]) * q[1:]) / (2.0 * col(g.dzf[1:-1]))
    return out


def adv_u(g: Grid, u, v, w):
    """Advection of u at x-face i (cell-z k)."""
    ucc = 0.5 * (u + xp(u))                      # at cell centre i
    ax = (ucc * ucc - xm(ucc * ucc)) / g.dx
    corner = 0.5 * (xm(v) + v) * 0.5 * (ym(u) + u)  # at (x-face i, y-face j)
    ay = (yp(corner) - corner) / g.dy
    fz = torch.zeros(g.face_shape(), dtype=u.dtype)  # at (x-face i, z-face k)
    fz[1:-1] = 0.5 * (xm(w[1:-1]) + w[1:-1]) * 0.5 * (u[:-1] + u[1:])
    az = (fz[1:] - fz[:-1]) / col(g.dzc)
    return ax + ay + az


def adv_v(g: Grid, u, v, w):
    """Advection of v at y-face j (cell-z k)."""
    corner = 0.5 * (ym(u) + u) * 0.5 * (xm(v) + v)  # at (x-face i, y-face j)
    ax = (xp(corner) - corner) / g.dx
    vcc = 0.5 * (v + yp(v))
    ay = (vcc * vcc - ym(vcc * vcc)) / g.dy
    fz = torch.zeros(g.face_shape(), dtype=v.dtype)
    fz[1:-1] = 0.5 * (ym(w[1:-1]) + w[1:-1]) * 0.5 * (v[:-1] + v[1:])
    az = (fz[1:] - fz[:-1]) / col(g.dzc)
    return ax + ay + az


def adv_face(g: Grid, u, v, w, q):
    """Advection of a z-face quantity q (w itself or the collocated T) on interior
    faces; q[0], q[nz] are its wall values. Face-shaped, zero on the walls."""
    uf = z_to_face(g, u)                          # u at (x-face i, z-face k)
    vf = z_to_face(g, v)
    fx = uf * 0.5 * (xm(q) + q)
    fy = vf * 0.5 * (ym(q) + q)
    wc = 0.5 * (w[:-1] + w[1:])                   # w at cell centres
    fz = wc * 0.5 * (q[:-1] + q[1:])              # at cell centres k = 0..nz-1
    out = torch.zeros_like(q)
    out[1:-1] = ((xp(fx) - fx) / g.dx + (yp(fy) - fy) / g.dy)[1:-1] \
        + (fz[1:] - fz[:-1]) / col(g.dzf[1:-1])
    return out


# CFL (Listing 1) --------------------------------------------------------------
def cfl_number(g: Grid, u, v, w):
    """Listing 1: max over cells of 0.5(|u_i+u_{i+1}|/dx + |v_j+v_{j+1}|/dy
    + |w_k+w_{k+1}|/dzc_k), floored at 1e-8."""
    q = (torch.abs(u + xp(u)) / g.dx + torch.abs(v + yp(v)) / g.dy
         + torch.abs(w[:-1] + w[1:]) / col(g.dzc))
    return max(1e-8, float(0.5 * q.max()))


def cfl_dt(g: Grid, u, v, w, cfl: float, dt_max: float) -> float:
    return min(cfl / cfl_number(g, u, v, w), dt_max)
