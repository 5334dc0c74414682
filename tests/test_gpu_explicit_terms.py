"""The explicit terms H of the RK3 substep (Sec. 2.1: central, second-order,
conservative differences on the staggered grid) computed by afid_rk3_substep
for single Fourier modes, against their closed forms -- not against the
oracle, so that a misreading shared by the oracle and the kernels would fail
here too.

* u = cos(2 pi b y/ly):  Hu = -nu 4 sin^2(pi b/ny)/dy^2 u
* v = cos(2 pi a x/lx):  Hv = -nu 4 sin^2(pi a/nx)/dx^2 v
* T = h(z) cos cos:      HT = -kappa (lambda_x + lambda_y) T, Hw = buoyancy T
* v = eps sin(2 pi a x/lx) under a uniform u = U:
                         Hv = -U eps cos(2 pi a x/lx) sin(2 pi a/nx)/dx
* u = eps sin(2 pi b y/ly) under a uniform v = V:
                         Hu = -V eps cos(2 pi b y/ly) sin(2 pi b/ny)/dy
* T = eps h(z) sin(theta) under a uniform (U, V):
                         HT = -eps h cos(theta) (U sin(2 pi a/nx)/dx + V sin(2 pi b/ny)/dy)

H is compared within 1e-12 of the closed form's scale; the terms that vanish
exactly for these fields are checked to be zero at that scale.
"""
import math

import numpy as np
import pytest
import torch

import synth
from tests.helpers import gpu, make_ctx

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


NX, NY, NZ, LX, LY = 32, 24, 9, 2.3, 1.1


def setup(nu=0.0, kappa=0.0, buoyancy=0.0):
    w = synth.workload("rb512", nx=NX, ny=NY, nz=NZ, lx=LX, ly=LY, stretch=1.7)
    w.nu, w.kappa, w.buoyancy, w.T_bot, w.T_top = nu, kappa, buoyancy, 0.0, 0.0
    return w, make_ctx(w)


def coords():
    dx, dy = LX / NX, LY / NY
    xc = ((np.arange(NX) + 0.5) * dx)[None, None, :]
    yc = ((np.arange(NY) + 0.5) * dy)[None, :, None]
    return dx, dy, xc, yc


def run_substep(ctx, u, v, w, T):
    """H of substep 0 for the state (u, v, w, T) with p = 0 (dt small; H depends
    only on the state at the substep start)."""
    S = [gpu(np.broadcast_to(a, s).copy()) for a, s in
         ((u, (NZ, NY, NX)), (v, (NZ, NY, NX)), (w, (NZ + 1, NY, NX)), (T, (NZ + 1, NY, NX)))]
    p = torch.zeros((NZ, NY, NX), dtype=torch.float64, device="cuda")
    H = [torch.full_like(S[0], np.nan), torch.full_like(S[1], np.nan),
         torch.full_like(S[2], np.nan), torch.full_like(S[3], np.nan)]
    ctx.rk3_substep(0, 1e-4, S[0], S[1], S[2], S[3], p, *H)
    torch.cuda.synchronize()
    return [h.cpu().numpy() for h in H]


def close(a, ref, scale):
    return float(np.abs(a - np.broadcast_to(ref, a.shape)).max()) <= TOL * scale


def test_gpu_horizontal_diffusion_closed_form():
    nu, kappa, bu = 0.013, 0.021, 0.7
    w, ctx = setup(nu, kappa, bu)
    dx, dy, xc, yc = coords()
    a, b = 3, 2
    lamx = 4 * math.sin(math.pi * a / NX) ** 2 / dx ** 2
    lamy = 4 * math.sin(math.pi * b / NY) ** 2 / dy ** 2
    zc0 = np.zeros((NZ, NY, NX))
    zf0 = np.zeros((NZ + 1, NY, NX))
    u = np.cos(2 * np.pi * b * yc / LY) + zc0
    Hu, Hv, Hw, HT = run_substep(ctx, u, zc0, zf0, zf0)
    assert close(Hu, -nu * lamy * u, nu * lamy)
    assert close(Hv, 0.0, nu * lamy) and close(Hw, 0.0, nu * lamy)
    v = np.cos(2 * np.pi * a * xc / LX) + zc0
    Hu, Hv, Hw, HT = run_substep(ctx, zc0, v, zf0, zf0)
    assert close(Hv, -nu * lamx * v, nu * lamx)
    assert close(Hu, 0.0, nu * lamx) and close(Hw, 0.0, nu * lamx)
    zf = synth.tanh_faces(NZ, 1.7)
    T = np.sin(np.pi * zf)[:, None, None] * np.cos(2 * np.pi * a * xc / LX) * np.cos(2 * np.pi * b * yc / LY)
    T[0] = 0.0
    T[-1] = 0.0
    Hu, Hv, Hw, HT = run_substep(ctx, zc0, zc0, zf0, T)
    lam = lamx + lamy
    assert close(HT[1:-1], -kappa * lam * T[1:-1], kappa * lam)
    assert close(HT[[0, -1]], 0.0, kappa * lam)
    assert close(Hw[1:-1], bu * T[1:-1], bu)
    assert close(Hu, 0.0, bu) and close(Hv, 0.0, bu)


def test_gpu_advection_by_uniform_flow_closed_form():
    w, ctx = setup()
    dx, dy, xc, yc = coords()
    zc0 = np.zeros((NZ, NY, NX))
    zf0 = np.zeros((NZ + 1, NY, NX))
    a, b, U, V, eps = 3, 2, 0.8, -0.6, 0.05
    # v carried by u = U
    v = eps * np.sin(2 * np.pi * a * xc / LX) + zc0
    Hu, Hv, Hw, _ = run_substep(ctx, U + zc0, v, zf0, zf0)
    scale = U * eps / dx
    assert close(Hv, -U * eps * np.cos(2 * np.pi * a * xc / LX) * math.sin(2 * np.pi * a / NX) / dx, scale)
    assert close(Hu, 0.0, scale) and close(Hw, 0.0, scale)
    # u carried by v = V
    u = eps * np.sin(2 * np.pi * b * yc / LY) + zc0
    Hu, Hv, Hw, _ = run_substep(ctx, u, V + zc0, zf0, zf0)
    scale = abs(V) * eps / dy
    assert close(Hu, -V * eps * np.cos(2 * np.pi * b * yc / LY) * math.sin(2 * np.pi * b / NY) / dy, scale)
    assert close(Hv, 0.0, scale) and close(Hw, 0.0, scale)
    # a face scalar carried by (U, V)
    zf = synth.tanh_faces(NZ, 1.7)
    hz = (1.0 + zf)[:, None, None]
    a2, b2 = 2, 3
    th = 2 * np.pi * (a2 * xc / LX + b2 * yc / LY)
    T = eps * hz * np.sin(th) + zf0
    T[0] = 0.0
    T[-1] = 0.0
    Hu, Hv, Hw, HT = run_substep(ctx, U + zc0, V + zc0, zf0, T)
    ref = -eps * hz * np.cos(th) * (U * math.sin(2 * np.pi * a2 / NX) / dx + V * math.sin(2 * np.pi * b2 / NY) / dy)
    scale = eps * (abs(U) / dx + abs(V) / dy) * 2
    assert close(HT[1:-1], ref[1:-1], scale)
    assert close(HT[[0, -1]], 0.0, scale)
