"""GPU hand-written adjoints through the C ABI against the oracle's
reverse-mode derivatives (automatic differentiation of the oracle's forward
code), plus dot-product identities of the linear maps on the device.

Wall planes of w and T are boundary data, not unknowns: their cotangents are
zero on the CUDA side and are excluded from the comparison."""
import numpy as np
import pytest
import torch

import synth
from oracle import adjoint, timestep as ts
from tests.helpers import cpu, gpu, make_ctx, ogrid, rel_l2

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_poisson_adjoint():
    w = synth.workload("pc64", nx=32, ny=16, nz=13, lx=1.5)
    g = ogrid(w)
    y = synth.noise(g.cell_shape(), seed=31)
    ref = adjoint.poisson_vjp(g, cpu(y))
    ctx = make_ctx(w, poisson_only=True)
    got = ctx.poisson_solve_adjoint(gpu(y))
    assert rel_l2(got, ref) < TOL
    # <solve(b), y> == <b, solve^T(y)> on the device
    b = gpu(synth.noise(g.cell_shape(), seed=32))
    lhs = float((ctx.poisson_solve(b) * gpu(y)).sum())
    rhs = float((b * got).sum())
    assert abs(lhs - rhs) < 1e-12 * max(abs(lhs), 1.0)


@pytest.mark.parametrize("s,beta", [(1.0, 0.0), (0.02, 3e-4)])
def test_project_adjoint(s, beta):
    w = synth.workload("pc64", nx=32, ny=32, nz=15, ly=2.0)
    g = ogrid(w)
    cu_, cv, cw = synth.velocity_noise(w, seed=41)
    cp = synth.noise(g.cell_shape(), seed=42)
    ref = adjoint.project_vjp(g, s, beta, cpu(cu_), cpu(cv), cpu(cw), cpu(cp))
    ctx = make_ctx(w)
    G = [gpu(a) for a in (cu_, cv, cw, cp)]
    ctx.project_adjoint(*G, s, beta)
    assert rel_l2(G[0], ref[0]) < TOL
    assert rel_l2(G[1], ref[1]) < TOL
    assert rel_l2(G[2][1:-1], ref[2][1:-1]) < TOL
    assert rel_l2(G[3], ref[3]) < TOL
    assert float(G[2][0].abs().max()) == 0.0 and float(G[2][-1].abs().max()) == 0.0


def rb_state(w, seed):
    u, v, ww, T, p = synth.rb_initial(w, seed, amp=0.1)
    un, vn, wn = synth.velocity_noise(w, seed + 100, sigma=0.1)
    return [u + un, v + vn, ww + wn, T, synth.noise(p.shape, seed + 200, 0.1)]


@pytest.mark.parametrize("l", [0, 1, 2])
def test_substep_adjoint(l):
    w = synth.workload("rb512", nx=16, ny=16, nz=11)
    w.nu, w.kappa = 3e-2, 2e-2
    g = ogrid(w)
    ph = ts.Phys(nu=w.nu, kappa=w.kappa, buoyancy=1.0, T_bot=1.0, T_top=0.0)
    st = rb_state(w, 5)
    Hp = [synth.noise(a.shape, seed=70 + i, sigma=0.1) for i, a in enumerate(st[:4])]
    for a in Hp[2:]:
        a[0] = 0.0
        a[-1] = 0.0
    cs = [synth.noise(a.shape, seed=80 + i) for i, a in enumerate(st)]
    cH = [synth.noise(a.shape, seed=90 + i) for i, a in enumerate(Hp)]
    for a in (cs[2], cs[3], cH[2], cH[3]):
        a[0] = 0.0
        a[-1] = 0.0
    dt = 0.03
    ref = adjoint.substep_vjp(g, ph, l, dt, tuple(cpu(a) for a in st), tuple(cpu(a) for a in Hp),
                              [cpu(a) for a in cs], [cpu(a) for a in cH])
    ctx = make_ctx(w)
    S = [gpu(a) for a in st]
    G = [gpu(a) for a in cs]            # gu, gv, gw, gT, gp
    GH = [gpu(a) for a in cH]
    ctx.rk3_substep_adjoint(l, dt, S[0], S[1], S[2], S[3], *G, *GH)
    names = ["u", "v", "w", "T", "p", "Hu", "Hv", "Hw", "HT"]
    for i, (got, r) in enumerate(zip(G + GH, ref)):
        if names[i] in ("w", "T", "Hw", "HT"):
            got, r = got[1:-1], r[1:-1]
        e = rel_l2(got, r)
        assert e < 1e-11, (names[i], e)
