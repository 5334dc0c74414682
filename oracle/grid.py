"""Staggered grid with a stretched wall-normal direction (Sec. 2.1, Fig. 1).

Pressure sits at cell centres; each velocity component sits on the cell face
normal to it; temperature is collocated with the wall-normal velocity (Fig. 1).
In this package's coordinates the periodic directions are x, y (uniform
spacing) and the wall-normal direction is z (faces z_0 = 0 < ... < z_nz = 1).

Metric:
  dzc[k] = z_{k+1} - z_k                 cell widths, k = 0..nz-1
  zc[k]  = (z_k + z_{k+1}) / 2           cell centres
  dzf[k] = zc[k] - zc[k-1]               centre spacing at interior face k = 1..nz-1
  dzf[0] = dzc[0]/2, dzf[nz] = dzc[nz-1]/2   wall to first/last centre
"""
from __future__ import annotations

import torch

f64 = torch.float64


class Grid:
    def __init__(self, nx: int, ny: int, nz: int, lx: float, ly: float, zf):
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.lx, self.ly = float(lx), float(ly)
        self.dx = self.lx / self.nx
        self.dy = self.ly / self.ny
        zf = torch.as_tensor(zf, dtype=f64)
        assert zf.shape == (self.nz + 1,)
        self.zf = zf
        self.dzc = zf[1:] - zf[:-1]
        self.zc = 0.5 * (zf[1:] + zf[:-1])
        dzf = torch.empty(self.nz + 1, dtype=f64)
        dzf[1:-1] = self.zc[1:] - self.zc[:-1]
        dzf[0] = 0.5 * self.dzc[0]
        dzf[-1] = 0.5 * self.dzc[-1]
        self.dzf = dzf

    # quadrature weights of the cell and face control volumes
    def w_cell(self) -> torch.Tensor:
        """W_c = dx dy dzc_k, broadcastable to [nz][ny][nx]."""
        return (self.dx * self.dy * self.dzc)[:, None, None]

    def w_face(self) -> torch.Tensor:
        """W_f = dx dy dzf_k on interior faces, zero on the two walls, [nz+1][1][1]."""
        w = self.dx * self.dy * self.dzf.clone()
        w[0] = 0.0
        w[-1] = 0.0
        return w[:, None, None]

    def volume(self) -> float:
        return self.lx * self.ly * float(self.zf[-1] - self.zf[0])

    def cell_shape(self):
        return (self.nz, self.ny, self.nx)

    def face_shape(self):
        return (self.nz + 1, self.ny, self.nx)
