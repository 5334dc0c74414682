"""Refined temperature grid through the C ABI (afid_mr_*, and afid_rk3_substep
with a buoyancy-only temperature) against the oracle (oracle/multires.py) on
the same seeded inputs: fine faces, velocity prolongation at the step start
and at intermediate times, restriction, refined temperature steps and whole
coupled steps, each within 1e-12 relative; at full size (momentum 512 x 512 x
384, temperature 1024 x 1024 x 768) the properties that hold at any size: the
steady conduction state and the closed-form advection of a Fourier mode by a
uniform velocity."""
import math

import numpy as np
import pytest
import torch

import synth
from oracle import multires as omr, timestep as ts
from paper_1705_01423_gb300 import MultiRes
from tests.helpers import cpu, gpu, make_ctx, ogrid, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def oracle_phys(w):
    return ts.Phys(nu=w.nu, kappa=w.kappa, buoyancy=w.buoyancy, u_bot=w.u_bot, u_top=w.u_top,
                   T_bot=w.T_bot, T_top=w.T_top)


def setup(name, shape, r, **over):
    nx, ny, nz = shape
    w = synth.workload(name, nx=nx, ny=ny, nz=nz, **over)
    ctx = make_ctx(w)
    m = MultiRes(ctx, *r)
    g = ogrid(w)
    gf = omr.fine_grid(g, *r)
    return w, ctx, m, g, gf


def maxrel(x, ref):
    x = x.detach().cpu()
    s = float(ref.abs().max())
    return float((x - ref).abs().max()) / (s if s > 0 else 1.0)


def noisy_velocity(w, seed, sigma=1.0):
    u, v, ww = synth.velocity_noise(w, seed, sigma=sigma)
    return cpu(u), cpu(v), cpu(ww)


@pytest.mark.parametrize("r", [(2, 2, 2), (3, 1, 2), (1, 2, 3)])
def test_fine_faces(r):
    w, ctx, m, g, gf = setup("rb512", (32, 16, 12), r)
    assert (m.nx, m.ny, m.nz) == (gf.nx, gf.ny, gf.nz)
    assert np.abs(m.faces() - gf.zf.numpy()).max() <= 1e-15


@pytest.mark.parametrize("shape,r,theta", [((32, 16, 10), (1, 1, 1), 0.0),
                                           ((32, 16, 10), (2, 2, 2), 0.0),
                                           ((32, 16, 10), (2, 2, 2), 0.37),
                                           ((32, 16, 10), (3, 2, 1), 8.0 / 15.0),
                                           ((32, 16, 10), (1, 3, 4), 1.0),
                                           ((32, 8, 10), (1, 1, 1), 0.0),   # 8 coarse rows, ry = 1: 9 block rows wrap
                                           ((48, 16, 10), (1, 2, 2), 0.5)])  # 48 fine columns: per-column kernel
def test_prolong_parity(shape, r, theta):
    w, ctx, m, g, gf = setup("couette1024", shape, r)  # u wall values -1, +1
    vel0 = noisy_velocity(w, 1)
    vel1 = noisy_velocity(w, 2)
    out = m.prolong(tuple(gpu(a) for a in vel0), tuple(gpu(a) for a in vel1), theta)
    ref = omr.velocity_at(g, gf, r, oracle_phys(w), vel0, vel1, theta)
    for a, b in zip(out, ref):
        assert maxrel(a, b) <= 1e-12


@pytest.mark.parametrize("r", [(2, 2, 2), (3, 2, 1)])
def test_restrict_parity(r):
    w, ctx, m, g, gf = setup("rb512", (32, 16, 12), r)
    Tf = cpu(synth.noise((gf.nz + 1, gf.ny, gf.nx), 3))
    Tc = m.restrict(gpu(Tf))
    assert maxrel(Tc, omr.restrict(r, Tf)) <= 1e-13


@pytest.mark.parametrize("shape,r,n_sub", [((32, 16, 12), (2, 2, 2), 1),   # 64-wide shared-flux blocks
                                           ((32, 16, 12), (2, 2, 2), 2),
                                           ((32, 16, 12), (3, 1, 2), 3),   # 32-wide shared-flux blocks
                                           ((48, 16, 12), (1, 1, 2), 1)])  # plain kernel (48 columns)
def test_scalar_advance_parity(shape, r, n_sub):
    w, ctx, m, g, gf = setup("rb512", shape, r)
    vel0 = noisy_velocity(w, 4, 0.5)
    vel1 = noisy_velocity(w, 5, 0.5)
    ph = oracle_phys(w)
    Tf = cpu(synth.conduction_temperature(gf.zf.numpy(), gf.ny, gf.nx, w.T_bot, w.T_top, 6, amp=0.1))
    dt = 2e-3
    Tg = gpu(Tf)
    m.scalar_advance(dt, n_sub, tuple(gpu(a) for a in vel0), tuple(gpu(a) for a in vel1), Tg)
    ref = omr.scalar_advance(g, gf, r, ph, dt, n_sub, vel0, vel1, Tf)
    assert rel_l2(Tg.cpu()[1:-1] - Tf[1:-1], ref[1:-1] - Tf[1:-1]) <= 1e-11  # the change itself
    assert rel_l2(Tg, ref) <= 1e-12
    assert torch.equal(Tg[0].cpu(), Tf[0]) and torch.equal(Tg[-1].cpu(), Tf[-1])


@pytest.mark.parametrize("name,shape,r,n_sub", [("rb512", (32, 16, 12), (2, 2, 2), 1),
                                                ("rb512", (48, 24, 10), (2, 3, 2), 2),
                                                ("couette1024", (32, 16, 12), (2, 1, 3), 1)])
def test_step_parity(name, shape, r, n_sub):
    """Two coupled steps (momentum with the restricted buoyancy, then the
    refined temperature); the Couette case starts from its workload's state
    (laminar profile plus N(0, 0.05) noise) and carries T as a passive scalar."""
    over = {} if name == "rb512" else dict(kappa=2e-3, T_bot=1.0, T_top=-1.0)
    w, ctx, m, g, gf = setup(name, shape, r, **over)
    ph = oracle_phys(w)
    p = torch.zeros(g.cell_shape(), dtype=torch.float64)
    if name == "rb512":
        u, v, ww = noisy_velocity(w, 7, 0.2)
    else:
        u, v, ww, _ = (cpu(a) for a in synth.couette_initial(w, seed=7))
    # make the start solenoidal (as a time step leaves it)
    u, v, ww, _, _ = ts.pressure_correction(g, u, v, ww, p)
    Tf = cpu(synth.conduction_temperature(gf.zf.numpy(), gf.ny, gf.nx, w.T_bot, w.T_top, 8, amp=0.05))
    # the workload's time step (its CFL limit is above the cap dt_max): the
    # pressure takes rounding of order eps |u| / dt from each projection, so a
    # much smaller dt than the run's makes its relative error grow as 1/dt
    dt = 2e-3 if name == "rb512" else w.dt_max
    gs = [gpu(a) for a in (u, v, ww, p)]
    H = [torch.zeros_like(gs[0]), torch.zeros_like(gs[0]), torch.zeros_like(gs[2])]
    Tg = gpu(Tf)
    ref_state, ref_T = (u, v, ww, p), Tf
    for _ in range(2):
        m.step(dt, n_sub, *gs, *H, Tg)
        ref_state, ref_T = omr.step(g, gf, r, ph, dt, n_sub, ref_state, ref_T)
    errs = [rel_l2(a, b) for a, b in zip(gs, ref_state)]
    assert max(errs) <= 1e-12, errs
    assert rel_l2(Tg, ref_T) <= 1e-12
    assert rel_l2(Tg.cpu()[1:-1] - Tf[1:-1], ref_T[1:-1] - Tf[1:-1]) <= 1e-10


@pytest.mark.parametrize("l", [0, 1, 2])
def test_buoyancy_only_substep(l):
    """afid_rk3_substep with T and no HT: T enters the w equation only and is
    not changed (the momentum half of a coupled step)."""
    w = synth.workload("rb512", nx=32, ny=16, nz=12)
    g = ogrid(w)
    ctx = make_ctx(w)
    ph = oracle_phys(w)
    u, v, ww = noisy_velocity(w, 9, 0.3)
    T = cpu(synth.conduction_temperature(g.zf.numpy(), g.ny, g.nx, w.T_bot, w.T_top, 10, amp=0.2))
    p = cpu(synth.noise(g.cell_shape(), 11, 0.1))
    Hp = [cpu(synth.noise(s, 12 + i, 0.1)) for i, s in enumerate([g.cell_shape(), g.cell_shape(), g.face_shape()])]
    dt = 3e-3
    gs = [gpu(a) for a in (u, v, ww, T, p)]
    gH = [gpu(a) for a in Hp]
    ctx.rk3_substep(l, dt, *gs, *gH, None)
    (ur, vr, wr, Tr, pr), (Hu, Hv, Hw, HT) = ts.substep(g, ph, l, dt, (u, v, ww, T, p),
                                                        tuple(Hp) + (None,), advance_scalar=False)
    assert HT is None and torch.equal(gs[3].cpu(), T)
    for a, b in zip(gs[:3] + gs[4:], (ur, vr, wr, pr)):
        assert rel_l2(a, b) <= 1e-12
    for a, b in zip(gH, (Hu, Hv, Hw)):
        assert rel_l2(a, b) <= 1e-12


# full size (the refined Rayleigh-Benard workload of the benchmark) ------------------
def fullsize():
    w = synth.workload("rb512")
    ctx = make_ctx(w)
    m = MultiRes(ctx, 2, 2, 2)
    return w, ctx, m


def test_fullsize_conduction_steady():
    """No velocity, T linear in z on the fine grid: one coupled step leaves T
    unchanged and the velocity zero (the buoyancy, a function of z alone, is
    taken up by the pressure)."""
    w, ctx, m = fullsize()
    zf = m.faces()
    Tf = torch.as_tensor(synth.conduction_temperature(zf, m.ny, m.nx, w.T_bot, w.T_top, 0, amp=0.0),
                         device="cuda")
    T0 = Tf.clone()
    z = lambda s: torch.zeros(s, dtype=torch.float64, device="cuda")
    u, v, ww, p = z(ctx.cell), z(ctx.cell), z(ctx.face), z(ctx.cell)
    H = [z(ctx.cell), z(ctx.cell), z(ctx.face)]
    m.step(1e-3, 2, u, v, ww, p, *H, Tf)
    torch.cuda.synchronize()
    assert float((Tf - T0).abs().max()) <= 1e-14
    assert max(float(u.abs().max()), float(v.abs().max()), float(ww.abs().max())) <= 1e-13
    assert float(p.abs().max()) > 1e-6


def test_fullsize_fourier_mode_closed_form():
    """Uniform velocity (U, 0, 0) with u_bot = u_top = U, no diffusion: each
    interior fine plane of T = cos(kx x + ky y) is multiplied by the RK3
    amplification 1 + z + z^2/2 + z^3/6 per refined step, z = -i U sin(kx dx_f)
    dt_f / dx_f (the y flux vanishes with v = 0)."""
    U = 0.6
    w = synth.workload("rb512", kappa=0.0, u_bot=U, u_top=U, buoyancy=0.0)
    ctx = make_ctx(w)
    m = MultiRes(ctx, 2, 2, 2)
    lx, ly = w.lx, w.ly
    dxf, dyf = lx / m.nx, ly / m.ny
    a, b = 7, 3
    kx, ky = 2 * math.pi * a / lx, 2 * math.pi * b / ly
    X = (torch.arange(m.nx, dtype=torch.float64, device="cuda") + 0.5) * dxf
    Y = (torch.arange(m.ny, dtype=torch.float64, device="cuda") + 0.5) * dyf
    phase = kx * X[None, :] + ky * Y[:, None]
    Tf = torch.cos(phase)[None].expand(m.nz + 1, -1, -1).contiguous()
    Tf[0] = 1.0
    Tf[-1] = 0.0
    uc = torch.full(ctx.cell, U, dtype=torch.float64, device="cuda")
    vc = torch.zeros(ctx.cell, dtype=torch.float64, device="cuda")
    wc = torch.zeros(ctx.face, dtype=torch.float64, device="cuda")
    dt, n_sub = 2e-3, 2
    m.scalar_advance(dt, n_sub, (uc, vc, wc), (uc, vc, wc), Tf)
    zz = -1j * U * math.sin(kx * dxf) / dxf * dt / n_sub
    G = (1 + zz + zz * zz / 2 + zz ** 3 / 6) ** n_sub
    exact = (G.real * torch.cos(phase) - G.imag * torch.sin(phase))
    err = float((Tf[1:-1] - exact[None]).abs().max())
    assert err <= 1e-12, err
    assert float((Tf[0] - 1.0).abs().max()) == 0.0 and float(Tf[-1].abs().max()) == 0.0


def test_refined_grid_argument_checks():
    """Host-side validation with a live context: refinement factors outside
    1..8, a context without the RK3 workspace, dt <= 0 and n_sub < 1 are
    refused before anything is launched, and the context stays usable."""
    from paper_1705_01423_gb300 import AfidError
    from paper_1705_01423_gb300.afid import AFID_ERR_INVALID_ARG
    w = synth.workload("rb512", nx=32, ny=16, nz=8)
    ctx = make_ctx(w)
    for r in [(0, 1, 1), (1, 9, 1), (2, 2, -1)]:
        with pytest.raises(AfidError) as e:
            MultiRes(ctx, *r)
        assert e.value.status == AFID_ERR_INVALID_ARG
    pctx = make_ctx(w, poisson_only=True)
    with pytest.raises(AfidError):
        MultiRes(pctx, 2, 2, 2)
    m = MultiRes(ctx, 2, 2, 2)
    z = lambda s: torch.zeros(s, dtype=torch.float64, device="cuda")
    vel = (z(ctx.cell), z(ctx.cell), z(ctx.face))
    Tf = z(m.fface)
    for dt, n in [(0.0, 1), (-1e-3, 1), (1e-3, 0)]:
        with pytest.raises(AfidError):
            m.scalar_advance(dt, n, vel, vel, Tf)
    with pytest.raises(ValueError):  # wrong fine shape, caught by the binding
        m.restrict(z(ctx.face))
    m.scalar_advance(1e-3, 1, vel, vel, Tf)  # still usable
    torch.cuda.synchronize()
    assert float(Tf.abs().max()) == 0.0


def test_context_close_releases_its_refined_grids_first():
    w = synth.workload("rb512", nx=32, ny=16, nz=8)
    ctx = make_ctx(w)
    m = MultiRes(ctx, 2, 1, 2)
    assert m.workspace_bytes > 0
    ctx.close()          # closes m first: the refined grid refers to the context
    assert m._h is None and ctx._h is None
    m.close()            # no-op


def test_ten_coupled_steps_parity():
    """Ten coupled steps on a small Rayleigh-Benard copy (momentum 32 x 32 x 16,
    temperature 64 x 64 x 32, two refined steps per momentum step) against the
    oracle advanced side by side: the errors stay at round-off."""
    w, ctx, m, g, gf = setup("rb512", (32, 32, 16), (2, 2, 2), nu=2e-3, kappa=2e-3)
    ph = oracle_phys(w)
    u, v, ww = noisy_velocity(w, 21, 0.05)
    p = torch.zeros(g.cell_shape(), dtype=torch.float64)
    u, v, ww, _, _ = ts.pressure_correction(g, u, v, ww, p)
    Tf = cpu(synth.conduction_temperature(gf.zf.numpy(), gf.ny, gf.nx, w.T_bot, w.T_top, 22, amp=0.05))
    gs = [gpu(a) for a in (u, v, ww, p)]
    H = [torch.zeros_like(gs[0]), torch.zeros_like(gs[0]), torch.zeros_like(gs[2])]
    Tg = gpu(Tf)
    ref_state, ref_T = (u, v, ww, p), Tf
    errs = []
    for _ in range(10):
        m.step(5e-3, 2, *gs, *H, Tg)
        ref_state, ref_T = omr.step(g, gf, (2, 2, 2), ph, 5e-3, 2, ref_state, ref_T)
        errs.append(max([rel_l2(a, b) for a, b in zip(gs, ref_state)] + [rel_l2(Tg, ref_T)]))
    assert max(errs) <= 1e-12, errs


@pytest.mark.parametrize("name,shape,r", [("rb512", (32, 16, 12), (2, 2, 2)),
                                          ("couette1024", (32, 16, 10), (2, 1, 3))])
def test_refined_statistics_parity(name, shape, r):
    """afid_mr_statistics = the oracle's statistics (plane means and scalars)
    of the prolonged velocity and the fine temperature on the fine grid."""
    from oracle import stats as ostats
    over = {} if name == "rb512" else dict(kappa=2e-3, T_bot=1.0, T_top=-1.0)
    w, ctx, m, g, gf = setup(name, shape, r, **over)
    u, v, ww = noisy_velocity(w, 31, 0.3)
    Tf = cpu(synth.conduction_temperature(gf.zf.numpy(), gf.ny, gf.nx, w.T_bot, w.T_top, 32, amp=0.1))
    prof, sc = m.statistics(gpu(u), gpu(v), gpu(ww), gpu(Tf))
    velf = omr.prolong(g, gf, r, u, v, ww, w.u_bot, w.u_top)
    ref = ostats.plane_means(gf, *velf, Tf).numpy()
    scale = np.maximum(np.abs(ref).max(axis=0), 1e-300)
    assert np.all(np.abs(prof - ref).max(axis=0) <= 1e-12 * scale + 1e-300)
    rs = ostats.scalars(gf, torch.as_tensor(ref), w.nu, w.kappa, w.u_bot, w.u_top, w.T_bot, w.T_top)
    for k, v_ in rs.items():
        assert abs(sc[k] - v_) <= 1e-12 * max(abs(v_), 1e-30), (k, sc[k], v_)


def test_fullsize_refined_conduction_nusselt():
    """Conduction profile on the refined grid (temperature 1024 x 1024 x 768):
    Nu = 1 at both walls and in the volume from the fine temperature."""
    w, ctx, m = fullsize()
    zf = m.faces()
    Tf = torch.as_tensor(synth.conduction_temperature(zf, m.ny, m.nx, w.T_bot, w.T_top, 0, amp=0.0),
                         device="cuda")
    z = lambda s: torch.zeros(s, dtype=torch.float64, device="cuda")
    prof, sc = m.statistics(z(ctx.cell), z(ctx.cell), z(ctx.face), Tf)
    assert prof.shape == (m.nz + 1, 9)
    for k in ("nu_bottom", "nu_top", "nu_volume"):
        assert abs(sc[k] - 1.0) <= 1e-12, (k, sc[k])
