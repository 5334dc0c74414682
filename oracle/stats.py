"""Wall-normal statistics: horizontal (x, y) means per wall-normal plane and
the scalars built from them (Sec. 3.2: the statistics are accumulated only
along the wall-normal direction, a vector reduction; Sec. 5: the Nusselt
number of Rayleigh-Benard flow, the friction velocity and friction Reynolds
number of plane Couette flow, Table 4).

TEST INFRASTRUCTURE ONLY (see the package header).

Profiles, one row per plane (cell planes k = 0..nz-1 for the cell-centred
quantities, face planes k = 0..nz for the face quantities; rows a quantity
does not have are zero):
   0 <u>   1 <v>   2 <u^2>   3 <v^2>             (cell planes)
   4 <w>   5 <w^2> 6 <T>     7 <T^2>   8 <w T>   (face planes)

Scalars (H = 1, Delta T = T_bot - T_top, h = H/2 the half height):
  nu_volume = 1 + <w T>_V / kappa, <.>_V over interior faces weighted by
              dzf (kappa = 1/sqrt(Ra Pr) in free-fall units, so 1/kappa is the
              sqrt(Ra Pr) of Nu = 1 + sqrt(Ra Pr) <w T>_V);
  nu_bottom = -(<T>_1 - <T>_0) / dzc_0 / Delta T, nu_top = -(<T>_nz -
              <T>_{nz-1}) / dzc_{nz-1} / Delta T: the conductive flux through
              the wall cells;
  tau_bottom = nu (<u>_0 - u_bot) / (dzc_0 / 2), tau_top = nu (u_top -
              <u>_{nz-1}) / (dzc_{nz-1} / 2): the wall shear stress from the
              wall value half a cell away (the wall treatment of the viscous
              term);
  re_tau    = h u_tau / nu with u_tau = sqrt((|tau_bottom| + |tau_top|) / 2)
              (Table 4's definition u_tau = sqrt(tau_w / rho), rho = 1);
  ke        = <(u^2 + v^2 + w^2) / 2>_V, the u, v means weighted by dzc over
              the cell planes, the w mean by dzf over the interior faces.
"""
from __future__ import annotations

import math

import torch

from .grid import Grid

NQ = 9


def plane_means(g: Grid, u, v, w, T=None):
    """[nz+1][NQ] tensor of the horizontal means listed in the header."""
    nz = g.nz
    out = torch.zeros((nz + 1, NQ), dtype=torch.float64)
    hm = lambda f: f.mean(dim=(1, 2))
    out[:nz, 0] = hm(u)
    out[:nz, 1] = hm(v)
    out[:nz, 2] = hm(u * u)
    out[:nz, 3] = hm(v * v)
    out[:, 4] = hm(w)
    out[:, 5] = hm(w * w)
    if T is not None:
        out[:, 6] = hm(T)
        out[:, 7] = hm(T * T)
        out[:, 8] = hm(w * T)
    return out


def scalars(g: Grid, prof, nu: float, kappa: float, u_bot: float, u_top: float,
            T_bot: float, T_top: float) -> dict:
    """The scalars of the header from the profiles."""
    nz = g.nz
    dzc = g.dzc.double()
    dzf = g.dzf.double()
    height = float(g.zf[-1] - g.zf[0])
    dT = T_bot - T_top
    interior = dzf[1:nz]
    wT_V = float((interior * prof[1:nz, 8]).sum()) / height
    out = {
        "nu_volume": 1.0 + wT_V / kappa if kappa > 0 else 0.0,
        "nu_bottom": -float(prof[1, 6] - prof[0, 6]) / float(dzc[0]) / dT if dT != 0 else 0.0,
        "nu_top": -float(prof[nz, 6] - prof[nz - 1, 6]) / float(dzc[nz - 1]) / dT if dT != 0 else 0.0,
        "tau_bottom": nu * float(prof[0, 0] - u_bot) / (0.5 * float(dzc[0])),
        "tau_top": nu * float(u_top - prof[nz - 1, 0]) / (0.5 * float(dzc[nz - 1])),
    }
    u_tau = math.sqrt(0.5 * (abs(out["tau_bottom"]) + abs(out["tau_top"])))
    out["re_tau"] = 0.5 * height * u_tau / nu if nu > 0 else 0.0
    ke_uv = float((dzc * (prof[:nz, 2] + prof[:nz, 3])).sum())
    ke_w = float((interior * prof[1:nz, 5]).sum())
    out["ke"] = 0.5 * (ke_uv + ke_w) / height
    return out
