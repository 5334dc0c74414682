"""The C-ABI library builds, loads and exports every entry point that
include/afid.h declares; host-side validation rejects bad arguments before
anything is launched (no GPU needed)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_1705_01423_gb300 import build
    build.build()
    from paper_1705_01423_gb300 import afid
    return afid.lib()


def declared():
    src = open(os.path.join(ROOT, "include", "afid.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(afid_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(L):
    names = declared()
    assert len(names) >= 14
    for n in names:
        assert hasattr(L, n), n
    from paper_1705_01423_gb300 import afid
    assert sorted(afid.exported_symbols()) == names


def test_status_strings(L):
    for s in range(8):
        assert L.afid_status_string(s)
    assert b"unknown" in L.afid_status_string(99)


def desc(nx=32, ny=16, nz=8, zf=None, prec=0):
    from paper_1705_01423_gb300 import afid
    import synth
    z = np.ascontiguousarray(synth.tanh_faces(nz, 1.5) if zf is None else zf)
    d = afid.GridDesc(nx, ny, nz, 1.0, 1.0, z.ctypes.data_as(C.POINTER(C.c_double)), prec, 1e-12, 4, 0)
    return d, z


@pytest.mark.parametrize("nx,ny,nz,code", [(24, 16, 8, 2), (32, 12, 8, 2), (8, 16, 8, 2), (32, 16, 2, 2),
                                            (8192, 16, 8, 2), (32, 4, 8, 2), (112, 16, 8, 2),
                                            (96, 56, 8, 2), (16 * 11, 48, 8, 2), (4800, 48, 8, 2)])
def test_create_rejects_unsupported_sizes(L, nx, ny, nz, code):
    from paper_1705_01423_gb300 import afid
    d, z = desc(nx, ny, nz, zf=np.linspace(0, 1, nz + 1))
    h = C.c_void_p()
    assert L.afid_create(C.byref(d), None, None, C.byref(h)) == code
    assert not h.value
    assert L.afid_workspace_bytes(C.byref(d)) == 0


@pytest.mark.parametrize("nx,ny", [(96, 48), (160, 40), (384, 24), (1280, 1024), (768, 768), (48, 120)])
def test_sizes_with_factors_3_and_5_accepted(L, nx, ny):
    """nx, ny of the form 2^a 3^b 5^c (nx a multiple of 16, ny of 8) -- the
    paper's Table 3/4 grids among them -- pass validation (host only)."""
    d, z = desc(nx, ny, 8)
    assert L.afid_workspace_bytes(C.byref(d)) > 0


def test_create_rejects_bad_faces_and_precision(L):
    from paper_1705_01423_gb300 import afid
    z = np.linspace(0, 1, 9)
    z[4] = z[3]                         # not strictly increasing
    d, _ = desc(zf=z)
    h = C.c_void_p()
    assert L.afid_create(C.byref(d), None, None, C.byref(h)) == afid.AFID_ERR_INVALID_ARG
    d, z2 = desc(prec=7)
    assert L.afid_create(C.byref(d), None, None, C.byref(h)) == afid.AFID_ERR_INVALID_ARG
    assert L.afid_create(None, None, None, C.byref(h)) == afid.AFID_ERR_INVALID_ARG
    d, z3 = desc()
    assert L.afid_create(C.byref(d), None, None, None) == afid.AFID_ERR_INVALID_ARG


def test_null_context_is_rejected(L):
    from paper_1705_01423_gb300 import afid
    assert L.afid_poisson_solve(None, None, None, None) == afid.AFID_ERR_INVALID_ARG
    assert L.afid_project(None, None, None, None, None, 1.0, 0.0, None) == afid.AFID_ERR_INVALID_ARG
    assert L.afid_destroy(None) == afid.AFID_ERR_INVALID_ARG
    assert L.afid_kernel_launches(None) == -1


def test_workspace_bytes(L):
    d, z = desc(64, 32, 16)
    b64 = L.afid_workspace_bytes(C.byref(d))
    n = 64 * 32 * 16
    assert b64 > 8 * n * 5
    d2, z2 = desc(64, 32, 16, prec=1)
    assert L.afid_workspace_bytes(C.byref(d2)) > 0


def test_refined_grid_calls_reject_null_handles(L):
    """The afid_mr_* entry points validate on the host: a NULL context or
    handle is refused before any CUDA call."""
    from paper_1705_01423_gb300 import afid
    bad = afid.AFID_ERR_INVALID_ARG
    h = C.c_void_p(123)
    assert L.afid_mr_create(None, 2, 2, 2, C.byref(h)) == bad
    assert not h.value  # the out handle is cleared first
    assert L.afid_mr_create(None, 2, 2, 2, None) == bad
    assert L.afid_mr_destroy(None) == bad
    a, b, c = C.c_int(), C.c_int(), C.c_int()
    assert L.afid_mr_dims(None, C.byref(a), C.byref(b), C.byref(c)) == bad
    assert L.afid_mr_workspace_bytes(None) == 0
    assert L.afid_mr_faces(None, None) == bad
    assert L.afid_mr_restrict(None, None, None) == bad
    assert L.afid_mr_prolong(None, None, None, None, None, None, None, 0.0, None, None, None) == bad
    assert L.afid_mr_scalar_advance(None, 1e-3, 1, None, None, None, None, None, None, None) == bad
    assert L.afid_mr_step(None, 1e-3, 1, None, None, None, None, None, None, None, None, None) == bad
    assert L.afid_mr_statistics(None, None, None, None, None, None, None) == bad


def test_mixed_refinement_needs_at_least_one_iteration(L):
    """refine_max_iter = 0 (and a negative or NaN tolerance) in AFID_MIXED is
    refused on the host before any CUDA call; FP64 ignores both fields."""
    from paper_1705_01423_gb300 import afid
    z = np.ascontiguousarray(np.linspace(0.0, 1.0, 9))
    h = C.c_void_p()
    for it, tol in ((0, 1e-10), (-1, 1e-10), (4, -1.0), (4, float("nan"))):
        d = afid.GridDesc(32, 16, 8, 1.0, 1.0, z.ctypes.data_as(C.POINTER(C.c_double)), afid.AFID_MIXED,
                          tol, it, 0)
        assert L.afid_create(C.byref(d), None, None, C.byref(h)) == afid.AFID_ERR_INVALID_ARG
        assert not h.value
        assert L.afid_workspace_bytes(C.byref(d)) == 0
    d = afid.GridDesc(32, 16, 8, 1.0, 1.0, z.ctypes.data_as(C.POINTER(C.c_double)), afid.AFID_FP64, 1e-10, 0, 0)
    assert L.afid_workspace_bytes(C.byref(d)) > 0


def test_new_calls_reject_null_context(L):
    from paper_1705_01423_gb300 import afid
    bad = afid.AFID_ERR_INVALID_ARG
    r = C.c_double()
    assert L.afid_nusselt(None, None, None, 1.0, None, None, None) == bad
    assert L.afid_probe_fp64_rate(None, 100, C.byref(r), None) == bad
    assert L.afid_test_tma_timeout(None) == bad
