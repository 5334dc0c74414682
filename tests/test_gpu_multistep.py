"""Multi-step parity of whole RK3 steps (CFL dt kept on the device, three
substeps) against the FP64 oracle.

* Small copies at the workloads' full step counts: Rayleigh-Benard (Ra = 1e8,
  Pr = 1) on 64 x 64 x 48 cells for 100 steps, plane Couette (Re_w = 4000,
  4pi x 2pi x 1) on 64 x 32 x 32 cells for 50 steps; within 1e-12 relative L2
  after steps 1, 10 and the last, field by field.
* The full sizes (512 x 512 x 384 and 1024 x 512 x 256) over 10 steps, within
  1e-12 after every step, each error measured against the scale of the
  quantities the step formed it from (the normwise forward error of the
  step): the velocity error relative to the largest provisional velocity
  (u*, v*, w*) that entered a pressure correction during the step, the
  pressure error relative to the largest pressure the step held after a
  substep, T relative to itself. Field by field the first step is dominated
  by cancellation: in Rayleigh-Benard from rest the velocity after the first
  substep is the remainder of projecting a provisional velocity about a thousand
  times larger (the hydrostatic response to the buoyancy), and in plane
  Couette the first substep's pressure (the potential that makes the
  non-solenoidal initial perturbation solenoidal) is removed again by the
  next substep; the oracle itself, run on the same inputs shifted
  periodically or with x and y exchanged (exact symmetries of the discrete
  equations), changes these fields by up to 2.3e-12 (RB u, v) and 1e-12
  (Couette p). The field-by-field errors are printed and bounded by 1e-10.

The dt of every step comes from the CFL formula of Listing 1 on each side and
is compared too, within 1e-12 (the maximum is order-independent; it inherits
the round-off difference of the velocities at the maximising cell).
"""
import math

import pytest
import torch

import synth
from oracle import operators as op, timestep as ts
from tests.helpers import cpu, gpu, make_ctx, ogrid, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def phys_of(w):
    return ts.Phys(nu=w.nu, kappa=w.kappa, buoyancy=w.buoyancy, u_bot=w.u_bot, u_top=w.u_top,
                   T_bot=w.T_bot, T_top=w.T_top)


def initial(w, seed):
    if w.has_T:
        return list(synth.rb_initial(w, seed))
    u, v, ww, p = synth.couette_initial(w, seed)
    return [u, v, ww, None, p]


def state_errors(S, ref):
    return {n: rel_l2(a, b) for n, a, b in zip("uvwTp", S, ref) if b is not None}


def run_pair(w, steps, check_at, seed=0):
    """Advances the GPU and the oracle side by side; returns {step: errors}:
    each field's relative L2 error, and the step's normwise errors "vel*"
    (velocity against the largest provisional velocity of its substeps) and
    "p*" (pressure against the largest pressure after one of its substeps)."""
    g = ogrid(w)
    ph = phys_of(w)
    host = initial(w, seed)
    ref = tuple(cpu(a) if a is not None else None for a in host)
    ctx = make_ctx(w)
    S = [gpu(a) if a is not None else None for a in host]
    del host
    H = [torch.zeros_like(S[0]), torch.zeros_like(S[1]), torch.zeros_like(S[2]),
         torch.zeros_like(S[3]) if S[3] is not None else None]
    Href = None
    out = {}
    for n in range(1, steps + 1):
        cfl_gpu = float(ctx.cfl(S[0], S[1], S[2], w.cfl, w.dt_max))
        cfl_ref = float(op.cfl_number(g, ref[0], ref[1], ref[2]))
        assert abs(cfl_gpu - cfl_ref) <= 1e-12 * cfl_ref, (n, cfl_gpu, cfl_ref)
        dt = op.cfl_dt(g, ref[0], ref[1], ref[2], w.cfl, w.dt_max)
        vel_scale = p_scale = 0.0
        for l in range(3):
            ctx.rk3_substep(l, -1.0, *S, *H)
            ref, Href, prov = ts.substep(g, ph, l, dt, ref, Href, return_provisional=True)
            vel_scale = max(vel_scale, math.sqrt(sum(float(x.norm()) ** 2 for x in prov)))
            p_scale = max(p_scale, float(ref[4].norm()))
        if n in check_at:
            torch.cuda.synchronize()
            e = state_errors(S, ref)
            dv = math.sqrt(sum(float((S[i].cpu() - ref[i]).norm()) ** 2 for i in range(3)))
            e["vel*"] = dv / vel_scale
            e["p*"] = float((S[4].cpu() - ref[4]).norm()) / p_scale
            out[n] = e
    return out


def assert_all(errs, tol):
    for n, e in errs.items():
        for name, v in e.items():
            assert v < tol, (n, name, v)


def test_rb_small_copy_100_steps():
    w = synth.workload("rb512", nx=64, ny=64, nz=48)
    errs = run_pair(w, 100, (1, 10, 100))
    print("rb 64x64x48:", errs)
    assert_all(errs, 1e-12)


def test_couette_small_copy_50_steps():
    w = synth.workload("couette1024", nx=64, ny=32, nz=32)
    errs = run_pair(w, 50, (1, 10, 50))
    print("couette 64x32x32:", errs)
    assert_all(errs, 1e-12)


@pytest.mark.parametrize("name", ["rb512", "couette1024"])
def test_fullsize_ten_steps_error_growth(name):
    w = synth.workload(name)
    errs = run_pair(w, 10, tuple(range(1, 11)))
    for n in sorted(errs):
        print("%s step %2d: %s" % (name, n, " ".join("%s %.2e" % kv for kv in errs[n].items())))
    for n, e in errs.items():
        assert e["vel*"] < 1e-12 and e["p*"] < 1e-12, (n, e)
        if "T" in e:
            assert e["T"] < 1e-12, (n, e)
    assert_all({n: {k: v for k, v in e.items() if k not in ("vel*", "p*")} for n, e in errs.items()}, 1e-10)
