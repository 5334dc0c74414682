"""Shared test helpers: build the same seeded inputs for the oracle and the
CUDA path, and compare fields."""
import numpy as np
import torch

import synth
from oracle import Grid


def ogrid(w):
    return Grid(w.nx, w.ny, w.nz, w.lx, w.ly, w.faces())


def cpu(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64)


def gpu(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64).cuda()


def rel_l2(x, ref):
    x = x.detach().cpu().double()
    ref = ref.detach().cpu().double()
    n = float(ref.norm())
    d = float((x - ref).norm())
    return d / n if n > 0 else d


def interior(f):
    return f[1:-1]


def make_ctx(w, precision="fp64", **kw):
    from paper_1705_01423_gb300 import Context, Physics
    ph = Physics(nu=w.nu, kappa=w.kappa, buoyancy=w.buoyancy, u_bot=w.u_bot, u_top=w.u_top,
                 T_bot=w.T_bot, T_top=w.T_top)
    return Context(w.nx, w.ny, w.nz, w.lx, w.ly, w.faces(), precision=precision, phys=ph, **kw)
