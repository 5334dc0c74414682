"""The allocation-free Poisson solve (afid_poisson_solve_noalloc) against the
regular context-based afid_poisson_solve, through the C ABI.

The entry point serves callers that cannot call cudaMalloc (code under a
device memory pool it does not own, loops that must never allocate, plugins
without a context object): all its workspace sits in a fixed 16 MiB device
array inside the library. This file is collected last on purpose, so that a
run stopping at the first failure has already run every other test; it also
passes on its own in a fresh process."""
import ctypes as C

import numpy as np
import pytest
import torch

import synth
from oracle import poisson
from tests.helpers import cpu, gpu, make_ctx, ogrid, rel_l2

pytestmark = pytest.mark.gpu
TOL64 = 1e-12


@pytest.fixture(autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def noalloc(w, rhs, phi):
    from paper_1705_01423_gb300 import afid
    zf = np.ascontiguousarray(w.faces())
    st = afid.lib().afid_poisson_solve_noalloc(
        w.nx, w.ny, w.nz, w.lx, w.ly, zf.ctypes.data_as(C.c_void_p), C.c_void_p(rhs.data_ptr()),
        C.c_void_p(phi.data_ptr()), C.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st


@pytest.mark.parametrize("shape", [(64, 64, 64), (32, 16, 13), (128, 128, 80)])
def test_noalloc_matches_context_solve_twice(shape):
    nx, ny, nz = shape
    w = synth.workload("pc64", nx=nx, ny=ny, nz=nz, lx=1.7, ly=0.9)
    ctx = make_ctx(w, poisson_only=True)
    for seed in (101, 102):                       # two calls in a row, different data
        b = gpu(synth.noise((nz, ny, nx), seed=seed) + 0.1)
        ref = ctx.poisson_solve(b)
        out = torch.full_like(b, float("nan"))
        assert noalloc(w, b, out) == 0
        torch.cuda.synchronize()
        assert rel_l2(out, ref) < TOL64


def test_noalloc_in_place_and_against_the_oracle():
    """rhs and phi may be the same buffer; the result is the FP64 solve of the
    oracle within 1e-12 relative L2 (printed), on two calls in a row."""
    nx, ny, nz = 32, 16, 13
    w = synth.workload("pc64", nx=nx, ny=ny, nz=nz, lx=1.7, ly=0.9)
    g = ogrid(w)
    for seed in (201, 202):
        b = synth.noise((nz, ny, nx), seed=seed) + 0.1
        ref = poisson.solve(g, cpu(b))
        x = gpu(b)
        assert noalloc(w, x, x) == 0
        torch.cuda.synchronize()
        err = rel_l2(x, ref)
        print("noalloc in place, seed %d: rel L2 vs oracle %.2e" % (seed, err))
        assert err < TOL64


def test_noalloc_rejects_oversized_grid():
    from paper_1705_01423_gb300 import afid
    w = synth.workload("pc64", nx=256, ny=256, nz=256)   # needs far more than 16 MiB
    b = torch.zeros(8, dtype=torch.float64, device="cuda")
    assert noalloc(w, b, b) == afid.AFID_ERR_UNSUPPORTED_SIZE
