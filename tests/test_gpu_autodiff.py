"""Autograd wrappers and the checkpointed Nusselt-number gradient on the GPU.

* RK3StepFn / ProjectFn backward (hand-written adjoints through the C ABI)
  against the oracle's reverse-mode derivative of the same step;
* dNu/dT0 after a checkpointed rollout against the oracle's gradient on a
  32^3 copy (the FP64 reference gradient), and against central finite
  differences (eps = 1e-6) along 4 seeded directions at 32^3 and on the full
  256 x 256 x 128 adjoint workload (Ra = 1e7, 20 steps, checkpoints every 5).
"""
import math

import numpy as np
import pytest
import torch

import synth
from oracle import adjoint as oadj, operators as op, timestep as ts
from tests.helpers import cpu, gpu, make_ctx, ogrid, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def rb_workload(nx, ny, nz, ra=1e7):
    w = synth.workload("adj256", nx=nx, ny=ny, nz=nz)
    w.nu, w.kappa = synth.rb_params(ra, 1.0)
    return w


def initial(w, seed, amp=1e-3, vel=0.0):
    u, v, ww, T, p = synth.rb_initial(w, seed, amp=amp)
    if vel:
        un, vn, wn = synth.velocity_noise(w, seed + 50, sigma=vel)
        u, v, ww = u + un, v + vn, ww + wn
    return [u, v, ww, T, p]


def test_rk3stepfn_matches_oracle_vjp():
    from paper_1705_01423_gb300.autodiff import RK3StepFn
    w = rb_workload(16, 16, 11, ra=1e4)
    g = ogrid(w)
    ph = ts.Phys(nu=w.nu, kappa=w.kappa, buoyancy=1.0, T_bot=1.0, T_top=0.0)
    st = initial(w, 3, amp=0.2, vel=0.2)
    dt = 0.02
    cot = [synth.noise(a.shape, seed=60 + i) for i, a in enumerate(st)]
    for c in (cot[2], cot[3]):
        c[0] = 0.0
        c[-1] = 0.0
    # oracle: VJP of the full step by reverse-mode differentiation
    X = [cpu(a).requires_grad_(True) for a in st]
    out, _ = ts.step(g, ph, dt, tuple(X))
    J = sum((o * cpu(c)).sum() for o, c in zip(out, cot))
    ref = torch.autograd.grad(J, X)
    ctx = make_ctx(w)
    G = [gpu(a).requires_grad_(True) for a in st]
    outg = RK3StepFn.apply(ctx, dt, *G)
    Jg = sum((o * gpu(c)).sum() for o, c in zip(outg, cot))
    got = torch.autograd.grad(Jg, G)
    names = ["u", "v", "w", "T", "p"]
    for n, a, b in zip(names, got, ref):
        if n in ("w", "T"):
            a, b = a[1:-1], b[1:-1]
        assert rel_l2(a, b) < 1e-11, n


def test_projectfn_matches_oracle_vjp():
    from paper_1705_01423_gb300.autodiff import ProjectFn
    w = synth.workload("pc64", nx=32, ny=16, nz=12)
    g = ogrid(w)
    u, v, ww = synth.velocity_noise(w, seed=8)
    p = synth.noise(g.cell_shape(), seed=9)
    cot = [synth.noise(a.shape, seed=20 + i) for i, a in enumerate((u, v, ww, p))]
    cot[2][0] = 0.0
    cot[2][-1] = 0.0
    ref = oadj.project_vjp(g, 0.4, 1e-3, *[cpu(c) for c in cot])
    ctx = make_ctx(w)
    X = [gpu(a).requires_grad_(True) for a in (u, v, ww, p)]
    out = ProjectFn.apply(ctx, *X, 0.4, 1e-3)
    J = sum((o * gpu(c)).sum() for o, c in zip(out, cot))
    got = torch.autograd.grad(J, X)
    for i, (a, b) in enumerate(zip(got, ref)):
        if i == 2:
            a, b = a[1:-1], b[1:-1]
        assert rel_l2(a, b) < 1e-12


def rollout_dts(ctx, w, st, n):
    """dt sequence of the forward rollout (CFL of Listing 1, frozen afterwards)."""
    from paper_1705_01423_gb300.autodiff import _run_step
    S = [a.clone() for a in st]
    dts = []
    for _ in range(n):
        cflm = float(ctx.cfl(S[0], S[1], S[2], w.cfl, w.dt_max))
        dt = min(w.cfl / cflm, w.dt_max)
        dts.append(dt)
        _run_step(ctx, dt, S)
    return dts


def nu_forward(ctx, st, dts, ra):
    from paper_1705_01423_gb300.autodiff import _run_step
    S = [a.clone() for a in st]
    for dt in dts:
        _run_step(ctx, dt, S)
    return ctx.nusselt(S[2], S[3], math.sqrt(ra)), S


def face_weights(ctx, device):
    """dx dy dzf_k on the interior faces, zero on the walls (test-side weights)."""
    zf = torch.as_tensor(ctx._zf, dtype=torch.float64)
    zc = 0.5 * (zf[1:] + zf[:-1])
    dzf = torch.zeros(ctx.nz + 1, dtype=torch.float64)
    dzf[1:-1] = zc[1:] - zc[:-1]
    return (ctx.lx / ctx.nx * ctx.ly / ctx.ny * dzf).to(device)


def test_nusselt_gradient_vs_oracle_32cubed():
    from paper_1705_01423_gb300.autodiff import nusselt_gradient
    ra = 1e5
    w = rb_workload(32, 32, 32, ra=ra)
    g = ogrid(w)
    ph = ts.Phys(nu=w.nu, kappa=w.kappa, buoyancy=1.0, T_bot=1.0, T_top=0.0)
    st = initial(w, 1, amp=0.05, vel=0.02)
    ctx = make_ctx(w)
    S = [gpu(a) for a in st]
    dts = rollout_dts(ctx, w, S, 6)
    nu, gT = nusselt_gradient(ctx, S, dts, ra, 1.0, checkpoint_every=2)
    nu_ref, gT_ref = oadj.nusselt_grad_T0(g, ph, tuple(cpu(a) for a in st), dts, ra, 1.0)
    assert abs(nu - nu_ref) < 1e-12 * abs(nu_ref)
    assert rel_l2(gT[1:-1], gT_ref[1:-1]) < 1e-10


def fd_check(ctx, w, st, dts, ra, gT, ndir=4, eps=1e-6, seed=900):
    """Central differences (Nu(T0 + eps d) - Nu(T0 - eps d)) / (2 eps), with the
    difference of the two Nusselt numbers summed face by face,
    sqrt(Ra Pr)/V sum_f W_f (w+ T+ - w- T-), so that the constant 1 and the
    large common part of <w T> do not cancel in floating point."""
    wf = face_weights(ctx, st[0].device)[:, None, None]
    coef = math.sqrt(ra) / (ctx.lx * ctx.ly)
    errs = []
    for d in range(ndir):
        dirn = gpu(synth.noise(st[3].shape, seed=seed + d))
        dirn[0] = 0.0
        dirn[-1] = 0.0
        sp = [a.clone() for a in st]
        sm = [a.clone() for a in st]
        sp[3] += eps * dirn
        sm[3] -= eps * dirn
        _, Sp = nu_forward(ctx, sp, dts, ra)
        _, Sm = nu_forward(ctx, sm, dts, ra)
        fd = coef * float((wf * (Sp[2] * Sp[3] - Sm[2] * Sm[3])).sum()) / (2 * eps)
        an = float((gT * dirn).sum())
        errs.append(abs(fd - an) / max(abs(an), 1e-30))
    return errs


def test_nusselt_gradient_fd_32cubed():
    from paper_1705_01423_gb300.autodiff import nusselt_gradient
    ra = 1e5
    w = rb_workload(32, 32, 32, ra=ra)
    st = [gpu(a) for a in initial(w, 2, amp=0.05, vel=0.02)]
    ctx = make_ctx(w)
    dts = rollout_dts(ctx, w, st, 5)
    _, gT = nusselt_gradient(ctx, st, dts, ra, 1.0, checkpoint_every=2)
    errs = fd_check(ctx, w, st, dts, ra, gT)
    assert max(errs) < 1e-6, errs


def test_nusselt_gradient_fd_adjoint_workload():
    """Config of the adjoint workload: Ra = 1e7, Pr = 1, 256 x 256 x 128,
    20 steps, checkpoints every 5, central differences at eps = 1e-6."""
    from paper_1705_01423_gb300.autodiff import nusselt_gradient
    w = synth.workload("adj256")
    ra = w.extra["Ra"]
    st = [gpu(a) for a in initial(w, 0, amp=1e-3)]
    ctx = make_ctx(w)
    dts = rollout_dts(ctx, w, st, w.steps)
    nu, gT = nusselt_gradient(ctx, st, dts, ra, 1.0, checkpoint_every=w.extra["checkpoint_every"])
    assert math.isfinite(nu) and float(gT.abs().max()) > 0
    errs = fd_check(ctx, w, st, dts, ra, gT)
    assert max(errs) < 1e-6, errs


def test_afid_nusselt_and_seeds_vs_oracle():
    """afid_nusselt against oracle.timestep.nusselt (1e-12) and its seed
    cotangents against the oracle's reverse-mode derivative of Nu with respect
    to w and T (1e-12 relative L2), on a stretched 48 x 40 x 21 grid."""
    ra = 1e6
    w = rb_workload(48, 40, 21, ra=ra)
    g = ogrid(w)
    st = initial(w, 3, amp=0.05, vel=0.1)
    ctx = make_ctx(w)
    W, T = gpu(st[2]), gpu(st[3])
    nu, gw, gT = ctx.nusselt(W, T, math.sqrt(ra), seeds=True)
    wr = cpu(st[2]).requires_grad_(True)
    Tr = cpu(st[3]).requires_grad_(True)
    nu_ref = ts.nusselt(g, wr, Tr, ra, 1.0)
    nu_ref.backward()
    assert abs(nu - float(nu_ref)) < 1e-12 * abs(float(nu_ref))
    assert rel_l2(gw, wr.grad) < 1e-12 and rel_l2(gT, Tr.grad) < 1e-12
    assert float(gw[0].abs().max()) == 0.0 and float(gT[-1].abs().max()) == 0.0
    assert ctx.nusselt(W, T, math.sqrt(ra)) == nu       # deterministic, no seeds
