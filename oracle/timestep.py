"""Fractional-step pressure correction and the low-storage RK3 / Crank-Nicolson
substep (Sec. 2.1 third paragraph, Sec. 2.2 first and last paragraphs).

Sec. 2.1: a provisional velocity is advanced with the old pressure; the
"delta" form then solves a Poisson equation for a correction phi, and the
velocity and pressure are updated with it so that the velocity is
discretely solenoidal. Time advancement is a three-substep low-storage RK3
with Crank-Nicolson for the implicit terms; Sec. 2.2 keeps only the
wall-normal viscous terms implicit (the horizontal ones are explicit).

Readings where the paper defers to its references:
* RK3 coefficients gamma = (8/15, 5/12, 3/4), rho = (0, -17/60, -5/12),
  alpha = gamma + rho (the standard low-storage set of the cited scheme);
* substep l:  R_q = dt [gamma_l H_q + rho_l H_q^prev - alpha_l G_q p
                      + alpha_l nu dzz q],
  (I - beta_l dzz) dq = R_q with beta_l = alpha_l dt nu / 2, q* = q + dq;
  H_q = -A_q + nu (dxx + dyy) q (+ T on w) is the explicit part;
* pressure correction with s = alpha_l dt: L phi = D(u*)/s,
  u = u* - s G phi, p <- p + phi - beta_l dzz phi (the last term keeps the
  delta form consistent with a wall-normal-only implicit operator);
* the temperature is advanced in the same substep from the state at the
  substep start (buoyancy also uses T at the substep start);
* Nu = 1 + sqrt(Ra Pr) <w T>_V, the volume form of the Nusselt number.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import torch

from .grid import Grid
from . import operators as op
from . import poisson

GAMMA = (8.0 / 15.0, 5.0 / 12.0, 3.0 / 4.0)
RHO = (0.0, -17.0 / 60.0, -5.0 / 12.0)
ALPHA = tuple(g + r for g, r in zip(GAMMA, RHO))


@dataclass
class Phys:
    nu: float = 0.0
    kappa: float = 0.0
    buoyancy: float = 0.0
    u_bot: float = 0.0
    u_top: float = 0.0
    T_bot: float = 0.0
    T_top: float = 0.0


# generic low-storage RK3 + CN increment (used by the field substep and by the
# order tests on scalar problems) ----------------------------------------------
def rk3_rhs(l: int, dt: float, H, Hprev, lin):
    """R = dt [gamma_l H + rho_l Hprev + alpha_l lin]; Hprev is unused at l = 0."""
    r = GAMMA[l] * H + ALPHA[l] * lin
    if RHO[l] != 0.0:
        r = r + RHO[l] * Hprev
    return dt * r


def cn_beta(l: int, dt: float, diff: float) -> float:
    return ALPHA[l] * dt * diff / 2.0


# Crank-Nicolson wall-normal solves (homogeneous Dirichlet increments) ----------
def cn_solve_cell(g: Grid, beta: float, R):
    """(I - beta dzz) dq = R for a cell field with Dirichlet walls half a cell away."""
    nz = g.nz
    a = 1.0 / (g.dzc * g.dzf[:-1])      # couples k-1 (the wall for k = 0)
    c = 1.0 / (g.dzc * g.dzf[1:])       # couples k+1 (the wall for k = nz-1)
    diag = (1.0 + beta * (a + c))[:, None, None].expand(nz, g.ny, g.nx)
    return poisson.thomas(-beta * a, diag, -beta * c, R)


def cn_solve_face(g: Grid, beta: float, R):
    """(I - beta dzz) dq = R on interior faces 1..nz-1; walls stay zero."""
    n = g.nz - 1
    dzf = g.dzf[1:-1]
    a = 1.0 / (dzf * g.dzc[:-1])
    c = 1.0 / (dzf * g.dzc[1:])
    diag = (1.0 + beta * (a + c))[:, None, None].expand(n, g.ny, g.nx)
    inner = poisson.thomas(-beta * a, diag, -beta * c, R[1:-1])
    zero = torch.zeros_like(R[:1])
    return torch.cat([zero, inner, zero], dim=0)


# pressure correction (Sec. 2.2) ------------------------------------------------
def project(g: Grid, u, v, w, p, phi, s: float, beta: float):
    gu, gv, gw = op.gradient(g, phi)
    return (u - s * gu, v - s * gv, w - s * gw,
            p + phi - beta * op.dzz_cell_neumann(g, phi))


def pressure_correction(g: Grid, u, v, w, p, s: float = 1.0, beta: float = 0.0):
    """Divergence -> Poisson solve -> projection; returns (u, v, w, p, phi)."""
    b = op.divergence(g, u, v, w) / s
    phi = poisson.solve(g, b)
    u, v, w, p = project(g, u, v, w, p, phi, s, beta)
    return u, v, w, p, phi


# explicit terms --------------------------------------------------------------------
def explicit_terms(g: Grid, ph: Phys, u, v, w, T):
    """H for u, v (cells), w and T (faces, zero on walls). T may be None."""
    Hu = -op.adv_u(g, u, v, w) + ph.nu * op.lap_h(g, u)
    Hv = -op.adv_v(g, u, v, w) + ph.nu * op.lap_h(g, v)
    Hw = -op.adv_face(g, u, v, w, w) + ph.nu * op.lap_h(g, w)
    if T is not None:
        Hw = Hw + ph.buoyancy * T
    Hw = _zero_walls(Hw)
    HT = None
    if T is not None:
        HT = _zero_walls(-op.adv_face(g, u, v, w, T) + ph.kappa * op.lap_h(g, T))
    return Hu, Hv, Hw, HT


def _zero_walls(f):
    zero = torch.zeros_like(f[:1])
    return torch.cat([zero, f[1:-1], zero], dim=0)


# one RK3 substep ----------------------------------------------------------------
def substep(g: Grid, ph: Phys, l: int, dt: float, state, Hprev, advance_scalar: bool = True,
            return_provisional: bool = False):
    """state = (u, v, w, T, p) (T may be None); Hprev = (Hu, Hv, Hw, HT) of the
    previous substep (ignored at l = 0). Returns (new_state, H), and with
    return_provisional also the provisional velocity (u*, v*, w*) that entered
    the pressure correction.

    advance_scalar=False: T only supplies the buoyancy of the w equation and is
    returned unchanged (HT is None), as when the temperature lives on its own
    refined grid and is advanced separately (multires.py)."""
    u, v, w, T, p = state
    Hu, Hv, Hw, HT = explicit_terms(g, ph, u, v, w, T)
    if not advance_scalar:
        HT = None
    if Hprev is None:
        Hprev = (None, None, None, None)
    gpu, gpv, gpw = op.gradient(g, p)
    bn = cn_beta(l, dt, ph.nu)
    Ru = rk3_rhs(l, dt, Hu, Hprev[0], -gpu + ph.nu * op.dzz_cell_dirichlet(g, u, ph.u_bot, ph.u_top))
    Rv = rk3_rhs(l, dt, Hv, Hprev[1], -gpv + ph.nu * op.dzz_cell_dirichlet(g, v, 0.0, 0.0))
    Rw = rk3_rhs(l, dt, Hw, Hprev[2], -gpw + ph.nu * op.dzz_face(g, w))
    us = u + cn_solve_cell(g, bn, Ru)
    vs = v + cn_solve_cell(g, bn, Rv)
    ws = w + cn_solve_face(g, bn, Rw)
    Tn = T if not advance_scalar else None
    if T is not None and advance_scalar:
        RT = rk3_rhs(l, dt, HT, Hprev[3], ph.kappa * op.dzz_face(g, T))
        Tn = T + cn_solve_face(g, cn_beta(l, dt, ph.kappa), RT)
    s = ALPHA[l] * dt
    un, vn, wn, pn, _ = pressure_correction(g, us, vs, ws, p, s, bn)
    if return_provisional:
        return (un, vn, wn, Tn, pn), (Hu, Hv, Hw, HT), (us, vs, ws)
    return (un, vn, wn, Tn, pn), (Hu, Hv, Hw, HT)


def step(g: Grid, ph: Phys, dt: float, state, H=None):
    """Three substeps with one dt; returns (state, H)."""
    for l in range(3):
        state, H = substep(g, ph, l, dt, state, H)
    return state, H


def nusselt(g: Grid, w, T, ra: float, pr: float):
    """Nu = 1 + sqrt(Ra Pr) sum_f W_f w T / V over interior faces."""
    return 1.0 + math.sqrt(ra * pr) * (g.w_face() * w * T).sum() / g.volume()
