"""Failure paths that run without faulting or hanging the GPU, through the C ABI.

* A bounded device-side wait that runs out: afid_test_tma_timeout makes the
  next TMA y-transform launch arm one block's first tile stage for the tile's
  bytes without issuing the copy, under a 1 ms limit. The block gives up,
  flags the fault and returns; the solve reports AFID_ERR_TIMEOUT through
  afid_info, and the next solve on the same context is correct again.
* Misaligned device pointers (8 bytes off a 16-byte boundary) are refused with
  AFID_ERR_ALIGNMENT before anything is launched, and the context stays usable.
"""
import ctypes as C

import pytest
import torch

import synth
from oracle import poisson
from tests.helpers import cpu, gpu, make_ctx, ogrid, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_tma_wait_timeout_is_reported_and_the_context_recovers():
    from paper_1705_01423_gb300 import afid
    w = synth.workload("pc64", nx=64, ny=64, nz=21, lx=1.3, ly=1.0)
    g = ogrid(w)
    b = synth.noise(g.cell_shape(), seed=31)
    ref = poisson.solve(g, cpu(b))
    # the separate passes (the fused small-nz kernel would take the y transforms)
    ctx = make_ctx(w, precision="mixed", refine_tol=1e-12, refine_max_iter=6, poisson_only=True,
                   fuse=False)
    B = gpu(b)
    assert afid.lib().afid_test_tma_timeout(ctx._h) == afid.AFID_OK
    with pytest.raises(afid.AfidError) as e:
        ctx.poisson_solve(B, info=True)
    assert e.value.status == afid.AFID_ERR_TIMEOUT
    phi, info = ctx.poisson_solve(B, info=True)        # the next solve is clean
    assert info["status"] in (0, 5)
    assert rel_l2(phi, ref) < 1e-10
    # contexts without a TMA transform refuse the hook
    ctx64 = make_ctx(w, poisson_only=True)
    assert afid.lib().afid_test_tma_timeout(ctx64._h) == afid.AFID_ERR_INVALID_ARG


def test_misaligned_pointers_are_refused():
    from paper_1705_01423_gb300 import afid
    L = afid.lib()
    w = synth.workload("pc64", nx=32, ny=16, nz=9)
    g = ogrid(w)
    ctx = make_ctx(w)
    nf = w.nx * w.ny * (w.nz + 1)
    buf = torch.zeros(2 * nf + 8, dtype=torch.float64, device="cuda")
    ok = buf.data_ptr()
    assert ok % 16 == 0
    off = ok + 8                                        # 8-byte aligned, not 16
    P = C.c_void_p
    A = afid.AFID_ERR_ALIGNMENT
    assert L.afid_poisson_solve(ctx._h, P(off), P(ok), None) == A
    assert L.afid_poisson_solve(ctx._h, P(ok), P(off), None) == A
    assert L.afid_project(ctx._h, P(off), P(ok), P(ok), P(ok), 1.0, 0.0, None) == A
    assert L.afid_max_divergence(ctx._h, P(ok), P(off), P(ok), P(ok)) == A
    assert L.afid_statistics(ctx._h, P(ok), P(ok), P(off), None, None, None) == A
    assert L.afid_nusselt(ctx._h, P(ok), P(off), 1.0, None, None, None) == A
    assert L.afid_poisson_solve_adjoint(ctx._h, P(off), P(ok)) == A
    assert L.afid_rk3_substep(ctx._h, 0, 1e-3, P(ok), P(ok), P(off), None, P(ok), P(ok), P(ok), P(ok),
                              None, None) == A
    zf = w.faces()
    assert L.afid_poisson_solve_noalloc(w.nx, w.ny, w.nz, w.lx, w.ly, zf.ctypes.data_as(P), P(off),
                                        P(ok), None) == A
    # nothing was launched by the refused calls; the context still solves correctly
    b = synth.noise(g.cell_shape(), seed=5)
    assert rel_l2(ctx.poisson_solve(gpu(b)), poisson.solve(g, cpu(b))) < 1e-12
