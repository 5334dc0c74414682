"""Wall-normal statistics through the C ABI (afid_statistics) against the
oracle (oracle/stats.py) on the same seeded states: every profile entry and
every scalar within 1e-12 (relative to the quantity's scale), on a turbulent-
like Rayleigh-Benard state, on plane Couette without a scalar, at a radix-3
grid, and the exact values of the conduction and laminar Couette states at
full size."""
import math

import numpy as np
import pytest
import torch

import synth
from oracle import stats as ostats, timestep as ts
from tests.helpers import cpu, gpu, make_ctx, ogrid

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def check(w, state, has_T=True):
    g = ogrid(w)
    u, v, ww, T = state
    ctx = make_ctx(w)
    prof, sc = ctx.statistics(gpu(u), gpu(v), gpu(ww), gpu(T) if has_T else None)
    ref = ostats.plane_means(g, cpu(u), cpu(v), cpu(ww), cpu(T) if has_T else None).numpy()
    scale = np.maximum(np.abs(ref).max(axis=0), 1e-300)
    assert np.abs(prof - ref).max(axis=0).max() <= 1e-12 * scale.max()
    assert np.all(np.abs(prof - ref).max(axis=0) <= 1e-12 * scale + 1e-300)
    rs = ostats.scalars(g, torch.as_tensor(ref), w.nu, w.kappa, w.u_bot, w.u_top, w.T_bot, w.T_top)
    for k, v_ in rs.items():
        assert abs(sc[k] - v_) <= 1e-12 * max(abs(v_), 1e-30), (k, sc[k], v_)
    return prof, sc


@pytest.mark.parametrize("shape", [(64, 32, 21), (96, 40, 12)])
def test_stats_rb_noisy_state(shape):
    nx, ny, nz = shape
    w = synth.workload("rb512", nx=nx, ny=ny, nz=nz)
    u, v, ww, T, p = synth.rb_initial(w, 3, amp=0.05)
    un, vn, wn = synth.velocity_noise(w, 4, sigma=0.1)
    check(w, (u + un, v + vn, ww + wn, T))


def test_stats_couette_no_scalar():
    w = synth.workload("couette1024", nx=64, ny=32, nz=17)
    u, v, ww, p = synth.couette_initial(w, seed=5)
    check(w, (u, v, ww, np.zeros((w.nz + 1, w.ny, w.nx))), has_T=False)


def test_stats_exact_states_fullsize():
    """512 x 512 x 384: the conduction profile gives Nu = 1 at both walls and in
    the volume; the laminar Couette profile on 1024 x 512 x 256 gives a wall
    shear stress of exactly 2 nu at both walls."""
    w = synth.workload("rb512")
    u, v, ww, T, p = synth.rb_initial(w, 0, amp=0.0)
    ctx = make_ctx(w)
    _, sc = ctx.statistics(gpu(u), gpu(v), gpu(ww), gpu(T))
    for k in ("nu_volume", "nu_bottom", "nu_top"):
        assert abs(sc[k] - 1.0) < 1e-12, (k, sc[k])
    del ctx
    wc = synth.workload("couette1024")
    g = ogrid(wc)
    zc = g.zc.numpy()
    uc = np.broadcast_to((2.0 * zc - 1.0)[:, None, None], (wc.nz, wc.ny, wc.nx)).copy()
    z0 = np.zeros((wc.nz, wc.ny, wc.nx))
    ctx = make_ctx(wc)
    _, sc = ctx.statistics(gpu(uc), gpu(z0), gpu(np.zeros((wc.nz + 1, wc.ny, wc.nx))))
    assert abs(sc["tau_bottom"] - 2 * wc.nu) < 1e-12 * wc.nu
    assert abs(sc["tau_top"] - 2 * wc.nu) < 1e-12 * wc.nu
