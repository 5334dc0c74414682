"""Pins of the oracle's reverse-mode derivatives: the transpose structure that
the mathematics fixes for the Poisson solve (L = W_c^-1 K with K symmetric, so
solve^T = W_c solve W_c^-1 on gauge-free data), and central finite differences
for the nonlinear substep and the Nusselt-number rollout gradient."""
import math

import numpy as np
import torch

import synth
from oracle import Grid, adjoint, poisson, timestep as ts


def t(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64)


def test_poisson_transpose_structure():
    g = Grid(8, 6, 7, 1.0, 2.0, synth.tanh_faces(7, 1.5))
    y = t(synth.noise(g.cell_shape(), seed=21))
    got = adjoint.poisson_vjp(g, y)
    dzc = g.dzc[:, None, None]
    ref = dzc * poisson.solve(g, y / dzc)
    assert float((got - ref).norm() / ref.norm()) < 1e-12


def small_rb(seed=0, nx=8, ny=8, nz=8):
    wl = synth.workload("rb512", nx=nx, ny=ny, nz=nz)
    g = Grid(wl.nx, wl.ny, wl.nz, wl.lx, wl.ly, wl.faces())
    ph = ts.Phys(nu=3e-2, kappa=3e-2, buoyancy=1.0, T_bot=1.0, T_top=0.0)
    u, v, w, T, p = (t(a) for a in synth.rb_initial(wl, seed, amp=0.3))
    vel = [t(a) * 0.3 for a in synth.velocity_noise(wl, seed + 1)]
    u, v, w = vel
    u, v, w, p, _ = ts.pressure_correction(g, u, v, w, p)
    return g, ph, (u, v, w, T, p)


def test_substep_vjp_finite_difference():
    g, ph, state = small_rb()
    Hp = tuple(t(synth.noise(x.shape, seed=30 + i)) * 0.1 for i, x in enumerate(state[:4]))
    l, dt = 1, 0.02
    cot_s = [t(synth.noise(x.shape, seed=40 + i)) for i, x in enumerate(state)]
    cot_H = [t(synth.noise(x.shape, seed=50 + i)) for i, x in enumerate(Hp)]
    for c in (cot_s[2], cot_s[3], cot_H[2], cot_H[3]):
        c[0] = 0.0
        c[-1] = 0.0
    grads = adjoint.substep_vjp(g, ph, l, dt, state, Hp, cot_s, cot_H)
    dirs = [t(synth.noise(x.shape, seed=60 + i)) for i, x in enumerate(list(state) + list(Hp))]
    for i in (2, 3, 6, 7):
        dirs[i][0] = 0.0
        dirs[i][-1] = 0.0

    def J(eps):
        xs = [x + eps * d for x, d in zip(list(state) + list(Hp), dirs)]
        s2, H2 = ts.substep(g, ph, l, dt, tuple(xs[:5]), tuple(xs[5:]))
        return sum(float((o * c).sum()) for o, c in zip(list(s2) + list(H2), cot_s + cot_H))

    eps = 1e-6
    fd = (J(eps) - J(-eps)) / (2 * eps)
    an = sum(float((gx * d).sum()) for gx, d in zip(grads, dirs))
    assert abs(fd - an) < 1e-6 * max(1.0, abs(an)), (fd, an)


def test_nusselt_gradient_finite_difference():
    g, ph, state = small_rb(seed=3)
    dts = [0.02, 0.02]
    nu, gT = adjoint.nusselt_grad_T0(g, ph, state, dts, ra=1e3, pr=1.0)
    d = t(synth.noise(state[3].shape, seed=77))
    d[0] = 0.0
    d[-1] = 0.0

    def N(eps):
        u, v, w, T, p = state
        s = adjoint.rollout(g, ph, (u, v, w, T + eps * d, p), dts)
        return float(ts.nusselt(g, s[2], s[3], 1e3, 1.0))

    eps = 1e-6
    fd = (N(eps) - N(-eps)) / (2 * eps)
    an = float((gT * d).sum())
    assert abs(fd - an) < 1e-6 * max(1.0, abs(an)), (fd, an)
    assert math.isfinite(nu)
