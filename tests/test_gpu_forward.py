"""GPU parity of the forward path through the C ABI against the FP64 oracle.

Tolerance: FP64 results within 1e-12 relative L2 of the oracle (the paper's
GPU and CPU codes agree to machine precision, Sec. 5; residual divergence
O(1e-13), Sec. 2.2); mixed precision within 1e-10. Grids are chosen so that
every kernel runs several blocks and ragged tails (odd nz, partial kx tiles,
nx/2+1 columns)."""
import math

import numpy as np
import pytest
import torch

import synth
from oracle import operators as op, poisson, timestep as ts
from tests.helpers import cpu, gpu, make_ctx, ogrid, rel_l2

pytestmark = pytest.mark.gpu
TOL64 = 1e-12
TOLMIX = 1e-10


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


SHAPES = [(16, 8, 3), (16, 8, 5), (32, 16, 12), (64, 32, 37), (128, 64, 24), (64, 128, 19)]


@pytest.mark.parametrize("shape", SHAPES)
def test_poisson_fp64(shape):
    nx, ny, nz = shape
    w = synth.workload("pc64", nx=nx, ny=ny, nz=nz, lx=2.0, ly=1.3)
    g = ogrid(w)
    b = synth.noise(g.cell_shape(), seed=nx + nz) + 0.25     # non-zero weighted mean
    ref, mb = poisson.solve(g, cpu(b), return_mean=True)
    ctx = make_ctx(w, poisson_only=True)
    phi, info = ctx.poisson_solve(gpu(b), info=True)
    assert rel_l2(phi, ref) < TOL64
    assert abs(info["rhs_mean"] - float(mb)) < 1e-13
    assert info["status"] == 5          # the non-zero mean is reported (and removed)
    assert abs(info["rhs_absmax"] - float(np.abs(b).max())) < 1e-15 * float(np.abs(b).max())


# Pass structures of the FP64 transforms with tangent-form twiddles (power-of-two
# lengths >= 64): x lengths nx/2 = 256 (radix 8, 8, 4) and 512 (8, 8, 8); y lengths
# 256 (8, 8, 4), 1024 (8, 8, 8, 2: a plain radix-2 last pass), 2048 (8, 8, 8, 4) and
# 4096 (four radix-8 passes, the largest ny a context takes).
TANGENT_SHAPES = [(512, 16, 6), (1024, 8, 4), (16, 256, 6), (16, 1024, 4), (16, 2048, 3), (16, 4096, 3)]


@pytest.mark.parametrize("shape", TANGENT_SHAPES)
def test_poisson_fp64_tangent_twiddle_passes(shape):
    nx, ny, nz = shape
    w = synth.workload("pc64", nx=nx, ny=ny, nz=nz, lx=2.0, ly=1.3)
    g = ogrid(w)
    b = synth.noise(g.cell_shape(), seed=nx + ny + nz)
    ref = poisson.solve(g, cpu(b))
    phi = make_ctx(w, poisson_only=True).poisson_solve(gpu(b))
    assert rel_l2(phi, ref) < TOL64


def test_poisson_aliasing_and_repeat():
    w = synth.workload("pc64", nx=32, ny=32, nz=9)
    g = ogrid(w)
    b = synth.noise(g.cell_shape(), seed=3)
    ref = poisson.solve(g, cpu(b))
    ctx = make_ctx(w, poisson_only=True)
    x = gpu(b)
    ctx.poisson_solve(x, x)              # in place
    assert rel_l2(x, ref) < TOL64
    y = ctx.poisson_solve(gpu(b))        # second call on the same context
    assert torch.equal(x, y)


def test_poisson_uniform_closed_form():
    """Exact discrete eigenfunction on a uniform z grid: phi = -b / lambda."""
    w = synth.workload("pc64", nx=32, ny=16, nz=16, stretch=0.0, lx=1.0, ly=1.0)
    g = ogrid(w)
    xc = (np.arange(w.nx) + 0.5) / w.nx
    yc = (np.arange(w.ny) + 0.5) / w.ny
    zc = g.zc.numpy()
    a, bb, m = 3, 2, 5
    f = (np.cos(np.pi * m * zc)[:, None, None] * np.cos(2 * np.pi * bb * yc)[None, :, None]
         * np.cos(2 * np.pi * a * xc)[None, None, :])
    lam = (4 * math.sin(math.pi * a / w.nx) ** 2 * w.nx**2 + 4 * math.sin(math.pi * bb / w.ny) ** 2 * w.ny**2
           + 4 * math.sin(math.pi * m / (2 * w.nz)) ** 2 * w.nz**2)
    ctx = make_ctx(w, poisson_only=True)
    phi = ctx.poisson_solve(gpu(f)).cpu().numpy()
    assert np.abs(phi + f / lam).max() < 1e-13 * np.abs(f).max() / lam * 10


def test_pressure_correction_64cubed():
    """64^3, stretch 1.5, u, v, w ~ N(0,1): max|div| after projection < 1e-12."""
    w = synth.workload("pc64")
    g = ogrid(w)
    u, v, ww = synth.velocity_noise(w, seed=0)
    p = np.zeros(g.cell_shape())
    ru, rv, rw, rp, _ = ts.pressure_correction(g, cpu(u), cpu(v), cpu(ww), cpu(p))
    ctx = make_ctx(w)
    U, V, W, Pp = gpu(u), gpu(v), gpu(ww), gpu(p)
    info = ctx.project(U, V, W, Pp, 1.0, 0.0, info=True)
    for got, ref in ((U, ru), (V, rv), (W, rw), (Pp, rp)):
        assert rel_l2(got, ref) < TOL64
    assert info["max_div"] < 1e-12
    md = float(ctx.max_divergence(U, V, W))
    assert md == info["max_div"]
    assert float(op.divergence(g, U.cpu(), V.cpu(), W.cpu()).abs().max()) < 1e-12


@pytest.mark.parametrize("s,beta", [(0.3, 0.0), (2.0e-3, 1.0e-4)])
def test_project_scaled(s, beta):
    w = synth.workload("pc64", nx=32, ny=64, nz=21, lx=3.0)
    g = ogrid(w)
    u, v, ww = synth.velocity_noise(w, seed=5)
    p = synth.noise(g.cell_shape(), seed=6)
    ref = ts.pressure_correction(g, cpu(u), cpu(v), cpu(ww), cpu(p), s, beta)
    ctx = make_ctx(w)
    X = [gpu(a) for a in (u, v, ww, p)]
    ctx.project(*X, s, beta)
    for got, r in zip(X, ref[:4]):
        assert rel_l2(got, r) < TOL64


def test_cfl_listing1():
    w = synth.workload("pc64", nx=32, ny=16, nz=11, lx=2.0, ly=0.5)
    g = ogrid(w)
    u, v, ww = synth.velocity_noise(w, seed=9)
    ref = op.cfl_number(g, cpu(u), cpu(v), cpu(ww))
    ctx = make_ctx(w)
    c = float(ctx.cfl(gpu(u), gpu(v), gpu(ww), 0.7, 1.0))
    assert abs(c - ref) < 1e-14 * ref
    z = torch.zeros(g.cell_shape(), dtype=torch.float64, device="cuda")
    zw = torch.zeros(g.face_shape(), dtype=torch.float64, device="cuda")
    assert float(ctx.cfl(z, z, zw, 0.7, 1.0)) == 1e-8          # Listing 1 floor


def rb_state(w, seed):
    u, v, ww, T, p = synth.rb_initial(w, seed, amp=0.05)
    un, vn, wn = synth.velocity_noise(w, seed + 100, sigma=0.05)
    return [u + un, v + vn, ww + wn, T, p]


def compare_state(got, ref, tol):
    names = ("u", "v", "w", "T", "p")
    for n, a, b in zip(names, got, ref):
        if b is None:
            continue
        e = rel_l2(a, b)
        assert e < tol, (n, e)


@pytest.mark.parametrize("shape", [(32, 32, 16), (64, 16, 13)])
def test_rk3_step_rb(shape):
    nx, ny, nz = shape
    w = synth.workload("rb512", nx=nx, ny=ny, nz=nz)
    w.nu, w.kappa = 2e-3, 2e-3
    g = ogrid(w)
    ph = ts.Phys(nu=w.nu, kappa=w.kappa, buoyancy=1.0, T_bot=1.0, T_top=0.0)
    st = rb_state(w, 1)
    ref_state = tuple(cpu(a) for a in st)
    ctx = make_ctx(w)
    S = [gpu(a) for a in st]
    H = [torch.zeros_like(S[0]), torch.zeros_like(S[1]), torch.zeros_like(S[2]), torch.zeros_like(S[3])]
    Href = None
    dt = 1e-2
    for step in range(2):
        for l in range(3):
            ref_state, Href = ts.substep(g, ph, l, dt, ref_state, Href)
            ctx.rk3_substep(l, dt, *S, *H)
            compare_state(S, ref_state, TOL64)
            for a, b in zip(H, Href):
                assert rel_l2(a, b) < TOL64


def test_rk3_couette_no_scalar_and_device_dt():
    w = synth.workload("couette1024", nx=32, ny=16, nz=12)
    g = ogrid(w)
    ph = ts.Phys(nu=w.nu, u_bot=-1.0, u_top=1.0)
    u, v, ww, p = synth.couette_initial(w, seed=2)
    ref = (cpu(u), cpu(v), cpu(ww), None, cpu(p))
    dt_ref = op.cfl_dt(g, ref[0], ref[1], ref[2], w.cfl, w.dt_max)
    ctx = make_ctx(w)
    S = [gpu(u), gpu(v), gpu(ww), None, gpu(p)]
    H = [torch.zeros_like(S[0]), torch.zeros_like(S[1]), torch.zeros_like(S[2]), None]
    ctx.cfl(S[0], S[1], S[2], w.cfl, w.dt_max)       # dt stays on the device
    Href = None
    for l in range(3):
        ref, Href = ts.substep(g, ph, l, dt_ref, ref, Href)
        ctx.rk3_substep(l, -1.0, *S, *H)
    compare_state(S, ref, TOL64)


def test_rb_conduction_steady_gpu():
    w = synth.workload("rb512", nx=32, ny=32, nz=24)
    u, v, ww, T, p = synth.rb_initial(w, 0, amp=0.0)
    ctx = make_ctx(w)
    S = [gpu(a) for a in (u, v, ww, T, p)]
    T0 = S[3].clone()
    H = [torch.zeros_like(S[0]), torch.zeros_like(S[1]), torch.zeros_like(S[2]), torch.zeros_like(S[3])]
    for _ in range(3):
        for l in range(3):
            ctx.rk3_substep(l, 5e-3, *S, *H)
    assert max(float(S[i].abs().max()) for i in range(3)) < 1e-13
    assert float((S[3] - T0).abs().max()) < 1e-13


@pytest.mark.parametrize("fuse", [True, False, None])
@pytest.mark.parametrize("shape", [(64, 64, 33), (128, 32, 48)])
def test_mixed_poisson(shape, fuse):
    """fuse: the small-nz kernel that runs the y transforms and the wall-normal
    solves of one kx column in shared memory (these grids qualify), the
    separate passes, or the context's own choice."""
    nx, ny, nz = shape
    w = synth.workload("pc64", nx=nx, ny=ny, nz=nz)
    g = ogrid(w)
    b = synth.noise(g.cell_shape(), seed=11)
    ref = poisson.solve(g, cpu(b))
    ctx = make_ctx(w, precision="mixed", refine_tol=1e-12, refine_max_iter=8, poisson_only=True, fuse=fuse)
    phi, info = ctx.poisson_solve(gpu(b), info=True)
    assert info["status"] in (0, 5)
    err = rel_l2(phi, ref)
    assert err < TOLMIX, (err, info)
    assert 2 <= info["iters"] <= 8
    assert info["err_estimate"] <= 1e-12


@pytest.mark.parametrize("fuse", [True, False])
@pytest.mark.parametrize("shape", [(64, 64, 33), (128, 32, 48), (64, 32, 37)])
def test_mixed_poisson_at_1e10(shape, fuse):
    """refine_tol = 1e-10, the accuracy the mixed solve is held to: three FP32
    solves at most on these grids, and the error against the oracle below the
    tolerance and consistent with the estimate."""
    nx, ny, nz = shape
    w = synth.workload("pc64", nx=nx, ny=ny, nz=nz)
    g = ogrid(w)
    b = synth.noise(g.cell_shape(), seed=13)
    ref = poisson.solve(g, cpu(b))
    ctx = make_ctx(w, precision="mixed", refine_tol=1e-10, refine_max_iter=8, poisson_only=True, fuse=fuse)
    phi, info = ctx.poisson_solve(gpu(b), info=True)
    assert info["status"] in (0, 5)
    err = rel_l2(phi, ref)
    assert err < TOLMIX, (err, info)
    assert info["iters"] <= 3, info
    assert info["err_estimate"] <= 1e-10
    assert err <= max(10 * info["err_estimate"], 1e-13), (err, info)


def test_mixed_pressure_correction():
    w = synth.workload("pc64", nx=64, ny=64, nz=40)
    g = ogrid(w)
    u, v, ww = synth.velocity_noise(w, seed=4)
    p = np.zeros(g.cell_shape())
    ref = ts.pressure_correction(g, cpu(u), cpu(v), cpu(ww), cpu(p))
    ctx = make_ctx(w, precision="mixed", refine_tol=1e-12, refine_max_iter=8)
    X = [gpu(a) for a in (u, v, ww, p)]
    info = ctx.project(*X, 1.0, 0.0, info=True)
    for got, r in zip(X, ref[:4]):
        assert rel_l2(got, r) < TOLMIX
    assert info["max_div"] < 1e-10


def test_mixed_reports_not_converged():
    """One refinement iteration cannot reach 1e-12: the call reports it and
    returns the best phi (no spin, no trap)."""
    w = synth.workload("pc64", nx=32, ny=32, nz=24)
    g = ogrid(w)
    b = synth.noise(g.cell_shape(), seed=12)
    ctx = make_ctx(w, precision="mixed", refine_tol=1e-12, refine_max_iter=1, poisson_only=True)
    phi, info = ctx.poisson_solve(gpu(b), info=True)
    assert info["status"] == 4 and info["iters"] == 1
    ref = poisson.solve(g, cpu(b))
    assert rel_l2(phi, ref) < 1e-3


@pytest.mark.parametrize("shape", [(16, 8, 3), (32, 16, 100), (16, 16, 384), (32, 8, 1000)])
def test_poisson_fp64_warp_partitioned_tridiag(shape):
    """Every (kx, ky) system through the warp-partitioned solver (chunked Thomas
    per lane + parallel cyclic reduction over the warp), long columns."""
    nx, ny, nz = shape
    w = synth.workload("pc64", nx=nx, ny=ny, nz=nz)
    g = ogrid(w)
    b = synth.noise(g.cell_shape(), seed=nz)
    ref = poisson.solve(g, cpu(b))
    ctx = make_ctx(w, poisson_only=True, warp_tridiag=True)
    phi = ctx.poisson_solve(gpu(b))
    assert rel_l2(phi, ref) < TOL64


@pytest.mark.parametrize("shape", [(32, 16, 1024), (64, 32, 300)])
def test_poisson_fp64_tridiag_choice_long_columns(shape):
    """Long columns and few systems: the context picks the warp-partitioned
    solver by itself; it, the forced per-thread solver and the oracle agree."""
    nx, ny, nz = shape
    w = synth.workload("pc64", nx=nx, ny=ny, nz=nz)
    g = ogrid(w)
    b = synth.noise(g.cell_shape(), seed=nz + 1)
    ref = poisson.solve(g, cpu(b))
    auto = make_ctx(w, poisson_only=True).poisson_solve(gpu(b))
    per_thread = make_ctx(w, poisson_only=True, warp_tridiag=False).poisson_solve(gpu(b))
    assert rel_l2(auto, ref) < TOL64 and rel_l2(per_thread, ref) < TOL64
    assert rel_l2(auto, per_thread) < TOL64


@pytest.mark.parametrize("shape", [(32, 16, 12), (64, 32, 37), (128, 64, 24), (64, 128, 19),
                                   (64, 64, 33), (128, 32, 48), (64, 256, 9), (32, 512, 5),
                                   (64, 1024, 4), (48, 2048, 3), (16, 2048, 4)])
def test_tma_y_transform_matches_plain_kernel(shape):
    """Mixed precision: the TMA-staged FP32 y transform runs the same Stockham
    passes with the same twiddles on every line as the plain kernel, so both
    refined solves agree to round-off; both match the oracle. Shapes span one to several column tiles,
    the zero-filled ragged last tile (M + 1 not a multiple of the tile width),
    ny below and at one TMA box, and the narrower tiles past ny = 512 (8
    columns at ny = 1024, 4 at 2048: several boxes of 256 rows per tile)."""
    nx, ny, nz = shape
    w = synth.workload("pc64", nx=nx, ny=ny, nz=nz)
    g = ogrid(w)
    b = synth.noise(g.cell_shape(), seed=nx + ny)
    kw = dict(precision="mixed", refine_tol=1e-12, refine_max_iter=8, poisson_only=True, fuse=False)
    a = make_ctx(w, **kw).poisson_solve(gpu(b))
    p = make_ctx(w, tma=False, **kw).poisson_solve(gpu(b))
    torch.cuda.synchronize()
    assert rel_l2(a, p) < 1e-11
    ref = poisson.solve(g, cpu(b))
    assert rel_l2(a, ref) < TOLMIX


@pytest.mark.parametrize("shape", [(64, 64, 8), (128, 64, 13), (32, 128, 5), (96, 48, 9), (48, 120, 11),
                                   (64, 32, 37), (256, 256, 32), (16, 8, 3)])
def test_mixed_fused_small_nz_matches_separate_passes(shape):
    """The fused small-nz kernel (y transforms, FP32 Thomas, FP64 low modes,
    exact (0,0) mode, one kernel per kx column) against the separate passes:
    the same solve to round-off (the low modes take the table-based FP64
    sweep instead of the warp-partitioned one), both within 1e-10 of the
    oracle. Shapes: powers of two, radix-3/5 lines (96, 48, 120), odd and
    short nz, several column counts."""
    nx, ny, nz = shape
    w = synth.workload("pc64", nx=nx, ny=ny, nz=nz, lx=1.6, ly=0.7)
    g = ogrid(w)
    b = synth.noise(g.cell_shape(), seed=nx + 3 * nz) + 0.05
    ref = poisson.solve(g, cpu(b))
    kw = dict(precision="mixed", refine_tol=1e-12, refine_max_iter=8, poisson_only=True)
    fused = make_ctx(w, fuse=True, **kw)
    fused.profile(True)
    fused.profile_read()
    a, ia = fused.poisson_solve(gpu(b), info=True)
    fams = fused.profile_read()
    assert fams["yfft_thomas"][1] >= 1 and fams["thomas"][1] == 0     # the fused kernel ran
    p, ip = make_ctx(w, fuse=False, **kw).poisson_solve(gpu(b), info=True)
    torch.cuda.synchronize()
    assert ia["status"] in (0, 5) and ip["status"] in (0, 5)
    assert rel_l2(a, p) < 1e-11
    assert rel_l2(a, ref) < TOLMIX and rel_l2(p, ref) < TOLMIX


RADIX35 = [(96, 48, 9), (160, 40, 7), (48, 120, 11), (384, 24, 5), (240, 24, 6)]


@pytest.mark.parametrize("shape", RADIX35)
def test_poisson_fp64_radix_3_and_5(shape):
    """Sizes with factors 3 and 5 (radix-3 and radix-5 Stockham passes after the
    radix-8/4/2 ones; nx/2 and ny both mixed-radix): FP64 solve against the
    oracle within 1e-12."""
    nx, ny, nz = shape
    w = synth.workload("pc64", nx=nx, ny=ny, nz=nz, lx=1.7, ly=0.9)
    g = ogrid(w)
    b = synth.noise(g.cell_shape(), seed=nx + 3 * ny)
    ref = poisson.solve(g, cpu(b))
    phi = make_ctx(w, poisson_only=True).poisson_solve(gpu(b))
    assert rel_l2(phi, ref) < TOL64


@pytest.mark.parametrize("shape", [(96, 48, 9), (160, 40, 7)])
def test_mixed_poisson_radix_3_and_5(shape):
    nx, ny, nz = shape
    w = synth.workload("pc64", nx=nx, ny=ny, nz=nz)
    g = ogrid(w)
    b = synth.noise(g.cell_shape(), seed=nx + ny + 1)
    ref = poisson.solve(g, cpu(b))
    phi, info = make_ctx(w, precision="mixed", refine_tol=1e-10, refine_max_iter=8,
                         poisson_only=True).poisson_solve(gpu(b), info=True)
    assert rel_l2(phi, ref) < TOLMIX, info


@pytest.mark.parametrize("shape", [(96, 40, 12), (80, 24, 7)])
def test_rk3_step_rb_radix_3_and_5(shape):
    """Two full RK3 steps (explicit terms with periodic wraps at nx, ny not
    powers of two, 32- and 16-wide blocks) against the oracle."""
    nx, ny, nz = shape
    w = synth.workload("rb512", nx=nx, ny=ny, nz=nz)
    w.nu, w.kappa = 2e-3, 2e-3
    g = ogrid(w)
    ph = ts.Phys(nu=w.nu, kappa=w.kappa, buoyancy=1.0, T_bot=1.0, T_top=0.0)
    st = rb_state(w, 2)
    ref_state = tuple(cpu(a) for a in st)
    ctx = make_ctx(w)
    S = [gpu(a) for a in st]
    H = [torch.zeros_like(S[0]), torch.zeros_like(S[1]), torch.zeros_like(S[2]), torch.zeros_like(S[3])]
    Href = None
    for step in range(2):
        for l in range(3):
            ref_state, Href = ts.substep(g, ph, l, 1e-2, ref_state, Href)
            ctx.rk3_substep(l, 1e-2, *S, *H)
    compare_state(S, ref_state, TOL64)
