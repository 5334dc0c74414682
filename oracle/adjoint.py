"""Reverse-mode derivatives of the oracle's forward maps.

Each adjoint here is the exact transpose of the oracle's own forward code,
obtained by automatic differentiation (torch.autograd) of exactly the
functions in poisson.py and timestep.py; no adjoint formula is written by
hand, so the CUDA path's hand-written adjoints are checked against an
independent derivation. The time step dt is treated as a constant (the CFL
maximum is not differentiated): a rollout records its dt sequence forward and
reuses it backward.
"""
from __future__ import annotations

import torch

from .grid import Grid
from . import poisson, timestep as ts


def _vjp(fn, inputs, cotangents):
    inputs = [x.detach().clone().requires_grad_(True) if x is not None else None for x in inputs]
    live = [x for x in inputs if x is not None]
    outs = fn(*inputs)
    pairs = [(o, c) for o, c in zip(outs, cotangents) if o is not None and c is not None]
    grads = torch.autograd.grad([o for o, _ in pairs], live, [c for _, c in pairs],
                                allow_unused=True)
    it = iter(grads)
    res = []
    for x in inputs:
        if x is None:
            res.append(None)
        else:
            gx = next(it)
            res.append(torch.zeros_like(x) if gx is None else gx.detach())
    return res


def poisson_vjp(g: Grid, gphi):
    """Transpose of the linear map b -> phi = solve(b)."""
    zero = torch.zeros(g.cell_shape(), dtype=torch.float64)
    return _vjp(lambda b: (poisson.solve(g, b),), [zero], [gphi])[0]


def project_vjp(g: Grid, s: float, beta: float, gu, gv, gw, gp):
    """Transpose of the linear pressure-correction map (u, v, w, p) -> (u', v', w', p')."""
    zc = torch.zeros(g.cell_shape(), dtype=torch.float64)
    zf = torch.zeros(g.face_shape(), dtype=torch.float64)

    def fwd(u, v, w, p):
        return ts.pressure_correction(g, u, v, w, p, s, beta)[:4]

    return _vjp(fwd, [zc, zc.clone(), zf, zc.clone()], [gu, gv, gw, gp])


def substep_vjp(g: Grid, ph: ts.Phys, l: int, dt: float, state, Hprev, cot_state, cot_H):
    """VJP of (state, Hprev) -> (state', H) at the given forward input."""
    u, v, w, T, p = state
    if Hprev is None:
        Hprev = (torch.zeros_like(u), torch.zeros_like(v), torch.zeros_like(w),
                 None if T is None else torch.zeros_like(T))

    def fwd(u, v, w, T, p, hu, hv, hw, hT):
        (un, vn, wn, Tn, pn), (Hu, Hv, Hw, HT) = ts.substep(
            g, ph, l, dt, (u, v, w, T, p), (hu, hv, hw, hT))
        return un, vn, wn, Tn, pn, Hu, Hv, Hw, HT

    return _vjp(fwd, [u, v, w, T, p, *Hprev], list(cot_state) + list(cot_H))


def rollout(g: Grid, ph: ts.Phys, state, dts):
    """Forward rollout with a fixed dt sequence; returns the final state."""
    H = None
    for dt in dts:
        state, H = ts.step(g, ph, dt, state, H)
    return state


def nusselt_grad_T0(g: Grid, ph: ts.Phys, state0, dts, ra: float, pr: float):
    """(Nu after the rollout, dNu/dT0) by reverse-mode differentiation."""
    u, v, w, T, p = state0
    T0 = T.detach().clone().requires_grad_(True)
    s = rollout(g, ph, (u, v, w, T0, p), dts)
    nu = ts.nusselt(g, s[2], s[3], ra, pr)
    (gT,) = torch.autograd.grad(nu, [T0])
    return float(nu.detach()), gT.detach()
