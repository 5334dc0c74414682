"""Thin ctypes binding of libafid (include/afid.h): argument marshalling only.

Every computation runs in the CUDA kernels of libafid.so; this module checks
tensor shapes, dtypes, devices and contiguity, passes raw device pointers and
the current CUDA stream, and turns status codes into exceptions. There is no
fallback: if the library is missing or no GPU is present, calls raise.

Field layout (C order, x fastest, torch.float64, CUDA, contiguous):
  u, v, p, phi, rhs   [nz][ny][nx]
  w, T                [nz+1][ny][nx]   (planes 0 and nz are the walls)
"""
from __future__ import annotations

import ctypes as C
import os
import weakref
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libafid.so")

AFID_OK = 0
AFID_ERR_INVALID_ARG = 1
AFID_ERR_UNSUPPORTED_SIZE = 2
AFID_ERR_ALIGNMENT = 3
AFID_ERR_NOT_CONVERGED = 4
AFID_ERR_INCONSISTENT_RHS = 5
AFID_ERR_CUDA = 6
AFID_ERR_OOM = 7
AFID_ERR_TIMEOUT = 8
AFID_FP64 = 0
AFID_MIXED = 1
AFID_POISSON_ONLY = 1
AFID_WARP_TRIDIAG = 2
AFID_NO_TMA = 4
AFID_FUSE_SMALL_NZ = 8
AFID_NO_FUSE = 32
AFID_THREAD_TRIDIAG = 16


class GridDesc(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("lx", C.c_double),
                ("ly", C.c_double), ("zf", C.POINTER(C.c_double)), ("precision", C.c_int),
                ("refine_tol", C.c_double), ("refine_max_iter", C.c_int), ("flags", C.c_int)]


class PhysDesc(C.Structure):
    _fields_ = [("nu", C.c_double), ("kappa", C.c_double), ("buoyancy", C.c_double),
                ("u_bot", C.c_double), ("u_top", C.c_double), ("T_bot", C.c_double),
                ("T_top", C.c_double)]


class Info(C.Structure):
    _fields_ = [("iters", C.c_int), ("rel_residual", C.c_double), ("rhs_mean", C.c_double),
                ("rhs_absmax", C.c_double), ("max_div", C.c_double), ("err_estimate", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class AfidError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__("%s: %s (status %d)" % (where, status_string(status), status))


_lib = None
P = C.c_void_p
D = C.c_double
I = C.c_int

_SIGS = {
    "afid_create": (I, [C.POINTER(GridDesc), C.POINTER(PhysDesc), P, C.POINTER(P)]),
    "afid_destroy": (I, [P]),
    "afid_set_stream": (I, [P, P]),
    "afid_workspace_bytes": (C.c_size_t, [C.POINTER(GridDesc)]),
    "afid_poisson_solve": (I, [P, P, P, C.POINTER(Info)]),
    "afid_project": (I, [P, P, P, P, P, D, D, C.POINTER(Info)]),
    "afid_cfl": (I, [P, P, P, P, D, D, P]),
    "afid_rk3_substep": (I, [P, I, D, P, P, P, P, P, P, P, P, P, C.POINTER(Info)]),
    "afid_max_divergence": (I, [P, P, P, P, P]),
    "afid_statistics": (I, [P, P, P, P, P, P, P]),
    "afid_nusselt": (I, [P, P, P, D, C.POINTER(C.c_double), P, P]),
    "afid_probe_fp64_rate": (I, [P, I, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "afid_test_tma_timeout": (I, [P]),
    "afid_poisson_solve_adjoint": (I, [P, P, P]),
    "afid_project_adjoint": (I, [P, P, P, P, P, D, D]),
    "afid_rk3_substep_adjoint": (I, [P, I, D, P, P, P, P, P, P, P, P, P, P, P, P, P]),
    "afid_status_string": (C.c_char_p, [I]),
    "afid_kernel_launches": (C.c_longlong, [P]),
    "afid_profile_enable": (I, [P, I]),
    "afid_profile_read": (I, [P, C.POINTER(C.c_double), C.POINTER(C.c_longlong), I]),
    "afid_kernel_family_name": (C.c_char_p, [I]),
    "afid_poisson_solve_noalloc": (I, [I, I, I, D, D, P, P, P, P]),
    "afid_mr_create": (I, [P, I, I, I, C.POINTER(P)]),
    "afid_mr_destroy": (I, [P]),
    "afid_mr_dims": (I, [P, C.POINTER(I), C.POINTER(I), C.POINTER(I)]),
    "afid_mr_workspace_bytes": (C.c_size_t, [P]),
    "afid_mr_faces": (I, [P, P]),
    "afid_mr_prolong": (I, [P, P, P, P, P, P, P, D, P, P, P]),
    "afid_mr_restrict": (I, [P, P, P]),
    "afid_mr_scalar_advance": (I, [P, D, I, P, P, P, P, P, P, P]),
    "afid_mr_step": (I, [P, D, I, P, P, P, P, P, P, P, P, C.POINTER(Info)]),
    "afid_mr_statistics": (I, [P, P, P, P, P, P, P]),
}
KERNEL_FAMILIES = 16


def lib():
    """Load libafid.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libafid.so not found at %s: run paper_1705_01423_gb300/build.py "
                               "(there is no CPU fallback)" % LIB_PATH)
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def exported_symbols():
    return sorted(_SIGS)


def status_string(s: int) -> str:
    try:
        return lib().afid_status_string(s).decode()
    except Exception:
        return "status %d" % s


def _ptr(t, shape, name):
    import torch
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError("%s must be a torch.Tensor" % name)
    if t.dtype != torch.float64 or not t.is_cuda or not t.is_contiguous():
        raise ValueError("%s must be a contiguous float64 CUDA tensor" % name)
    if tuple(t.shape) != tuple(shape):
        raise ValueError("%s has shape %s, expected %s" % (name, tuple(t.shape), tuple(shape)))
    return C.c_void_p(t.data_ptr())


def _check(st: int, where: str, allow=()):
    if st != AFID_OK and st not in allow:
        raise AfidError(st, where)
    return st


@dataclass
class Physics:
    nu: float = 0.0
    kappa: float = 0.0
    buoyancy: float = 0.0
    u_bot: float = 0.0
    u_top: float = 0.0
    T_bot: float = 0.0
    T_top: float = 0.0


STAT_NQ = 9


class Stats(C.Structure):
    _fields_ = [("nu_volume", C.c_double), ("nu_bottom", C.c_double), ("nu_top", C.c_double),
                ("tau_bottom", C.c_double), ("tau_top", C.c_double), ("re_tau", C.c_double),
                ("ke", C.c_double)]


class Context:
    """One grid on the current CUDA device (afid_create / afid_destroy)."""

    def __init__(self, nx, ny, nz, lx, ly, zf, precision="fp64", refine_tol=1e-12,
                 refine_max_iter=10, phys: Physics | None = None, poisson_only=False,
                 warp_tridiag=None, tma=True, fuse=None, stream=None):
        import torch
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.lx, self.ly = float(lx), float(ly)
        self._zf = np.ascontiguousarray(np.asarray(zf, dtype=np.float64))
        if self._zf.shape != (self.nz + 1,):
            raise ValueError("zf must hold nz+1 face coordinates")
        self.precision = precision
        self.phys = phys or Physics()
        desc = GridDesc(self.nx, self.ny, self.nz, self.lx, self.ly,
                        self._zf.ctypes.data_as(C.POINTER(C.c_double)),
                        AFID_MIXED if precision == "mixed" else AFID_FP64, float(refine_tol),
                        int(refine_max_iter),
                        (AFID_POISSON_ONLY if poisson_only else 0)
                        | (0 if warp_tridiag is None else (AFID_WARP_TRIDIAG if warp_tridiag else AFID_THREAD_TRIDIAG))
                        | (0 if tma else AFID_NO_TMA) | (0 if fuse is None else (AFID_FUSE_SMALL_NZ if fuse else AFID_NO_FUSE)))
        self._desc = desc
        ph = PhysDesc(self.phys.nu, self.phys.kappa, self.phys.buoyancy, self.phys.u_bot,
                      self.phys.u_top, self.phys.T_bot, self.phys.T_top)
        if stream is None:
            stream = torch.cuda.current_stream()
        self._stream = stream
        h = C.c_void_p()
        _check(lib().afid_create(C.byref(desc), C.byref(ph), C.c_void_p(stream.cuda_stream),
                                 C.byref(h)), "afid_create")
        self._h = h
        self._children = weakref.WeakSet()
        self.workspace_bytes = int(lib().afid_workspace_bytes(C.byref(desc)))

    # shapes
    @property
    def cell(self):
        return (self.nz, self.ny, self.nx)

    @property
    def face(self):
        return (self.nz + 1, self.ny, self.nx)

    def close(self):
        # refined grids built on this context go first (they refer to it)
        for child in list(getattr(self, "_children", ())):
            child.close()
        if getattr(self, "_h", None):
            lib().afid_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream):
        self._stream = stream
        _check(lib().afid_set_stream(self._h, C.c_void_p(stream.cuda_stream)), "afid_set_stream")

    def kernel_launches(self) -> int:
        return int(lib().afid_kernel_launches(self._h))

    def probe_fp64_rate(self, iters=20000):
        """(FP64 operations per second, ms) of the FMA-chain probe
        (afid_probe_fp64_rate); an FMA counts as one operation."""
        r, ms = C.c_double(), C.c_double()
        _check(lib().afid_probe_fp64_rate(self._h, int(iters), C.byref(r), C.byref(ms)),
               "afid_probe_fp64_rate")
        return r.value, ms.value

    def profile(self, on=True):
        _check(lib().afid_profile_enable(self._h, 1 if on else 0), "afid_profile_enable")

    def profile_read(self):
        """{family: (ms, launch groups)} since the last read (synchronises)."""
        n = KERNEL_FAMILIES
        ms = (C.c_double * n)()
        cnt = (C.c_longlong * n)()
        _check(lib().afid_profile_read(self._h, ms, cnt, n), "afid_profile_read")
        return {lib().afid_kernel_family_name(i).decode(): (ms[i], int(cnt[i])) for i in range(n)}

    # ---- forward calls
    def poisson_solve(self, rhs, phi=None, info=False):
        import torch
        if phi is None:
            phi = torch.empty_like(rhs)
        inf = Info() if info else None
        st = lib().afid_poisson_solve(self._h, _ptr(rhs, self.cell, "rhs"), _ptr(phi, self.cell, "phi"),
                                      C.byref(inf) if inf else None)
        _check(st, "afid_poisson_solve", allow=(AFID_ERR_NOT_CONVERGED, AFID_ERR_INCONSISTENT_RHS))
        if info:
            d = inf.as_dict()
            d["status"] = st
            return phi, d
        return phi

    def project(self, u, v, w, p, s=1.0, beta=0.0, info=False):
        inf = Info() if info else None
        st = lib().afid_project(self._h, _ptr(u, self.cell, "u"), _ptr(v, self.cell, "v"),
                                _ptr(w, self.face, "w"), _ptr(p, self.cell, "p"), float(s),
                                float(beta), C.byref(inf) if inf else None)
        _check(st, "afid_project", allow=(AFID_ERR_NOT_CONVERGED, AFID_ERR_INCONSISTENT_RHS))
        if info:
            d = inf.as_dict()
            d["status"] = st
            return d
        return None

    def cfl(self, u, v, w, cfl=0.7, dt_max=1e-2):
        """Returns the CFL number as a 1-element device tensor and sets the
        context's device-resident dt = min(cfl/cflm, dt_max)."""
        import torch
        out = torch.empty(1, dtype=torch.float64, device=u.device)
        _check(lib().afid_cfl(self._h, _ptr(u, self.cell, "u"), _ptr(v, self.cell, "v"),
                              _ptr(w, self.face, "w"), float(cfl), float(dt_max),
                              C.c_void_p(out.data_ptr())), "afid_cfl")
        return out

    def max_divergence(self, u, v, w):
        import torch
        out = torch.empty(1, dtype=torch.float64, device=u.device)
        _check(lib().afid_max_divergence(self._h, _ptr(u, self.cell, "u"), _ptr(v, self.cell, "v"),
                                         _ptr(w, self.face, "w"), C.c_void_p(out.data_ptr())),
               "afid_max_divergence")
        return out

    def statistics(self, u, v, w, T=None):
        """Wall-normal statistics (afid_statistics): returns (profiles, scalars),
        profiles a [nz+1][9] numpy array of horizontal means (<u>, <v>, <u^2>,
        <v^2> on cell planes; <w>, <w^2>, <T>, <T^2>, <w T> on face planes) and
        scalars a dict (nu_volume, nu_bottom, nu_top, tau_bottom, tau_top,
        re_tau, ke)."""
        prof = np.zeros((self.nz + 1, STAT_NQ), dtype=np.float64)
        st = Stats()
        _check(lib().afid_statistics(self._h, _ptr(u, self.cell, "u"), _ptr(v, self.cell, "v"),
                                     _ptr(w, self.face, "w"),
                                     _ptr(T, self.face, "T") if T is not None else None,
                                     prof.ctypes.data_as(C.c_void_p), C.byref(st)), "afid_statistics")
        return prof, {name: getattr(st, name) for name, _ in Stats._fields_}

    def nusselt(self, w, T, coef, seeds=False):
        """Volume Nusselt number 1 + coef <w T>_V (afid_nusselt; coef = sqrt(Ra Pr)).
        With seeds=True also returns (dNu/dw, dNu/dT) as new device tensors."""
        import torch
        nu = C.c_double()
        gw = torch.empty_like(w) if seeds else None
        gT = torch.empty_like(T) if seeds else None
        _check(lib().afid_nusselt(self._h, _ptr(w, self.face, "w"), _ptr(T, self.face, "T"),
                                  float(coef), C.byref(nu), _ptr(gw, self.face, "gw"),
                                  _ptr(gT, self.face, "gT")), "afid_nusselt")
        return (nu.value, gw, gT) if seeds else nu.value

    def rk3_substep(self, l, dt, u, v, w, T, p, Hu, Hv, Hw, HT, info=False):
        """dt <= 0 uses the dt set by the last cfl() call (device resident)."""
        inf = Info() if info else None
        st = lib().afid_rk3_substep(self._h, int(l), float(dt), _ptr(u, self.cell, "u"),
                                    _ptr(v, self.cell, "v"), _ptr(w, self.face, "w"),
                                    _ptr(T, self.face, "T"), _ptr(p, self.cell, "p"),
                                    _ptr(Hu, self.cell, "Hu"), _ptr(Hv, self.cell, "Hv"),
                                    _ptr(Hw, self.face, "Hw"), _ptr(HT, self.face, "HT"),
                                    C.byref(inf) if inf else None)
        _check(st, "afid_rk3_substep", allow=(AFID_ERR_NOT_CONVERGED, AFID_ERR_INCONSISTENT_RHS))
        if info:
            d = inf.as_dict()
            d["status"] = st
            return d
        return None

    def rk3_step(self, state, H, dt):
        """Three substeps in place; state = (u, v, w, T, p), H = (Hu, Hv, Hw, HT)."""
        u, v, w, T, p = state
        for l in range(3):
            self.rk3_substep(l, dt, u, v, w, T, p, *H)

    # ---- adjoints
    def poisson_solve_adjoint(self, gphi, grhs=None):
        import torch
        if grhs is None:
            grhs = torch.empty_like(gphi)
        _check(lib().afid_poisson_solve_adjoint(self._h, _ptr(gphi, self.cell, "gphi"),
                                                _ptr(grhs, self.cell, "grhs")),
               "afid_poisson_solve_adjoint")
        return grhs

    def project_adjoint(self, gu, gv, gw, gp, s=1.0, beta=0.0):
        _check(lib().afid_project_adjoint(self._h, _ptr(gu, self.cell, "gu"), _ptr(gv, self.cell, "gv"),
                                          _ptr(gw, self.face, "gw"), _ptr(gp, self.cell, "gp"),
                                          float(s), float(beta)), "afid_project_adjoint")

    def rk3_substep_adjoint(self, l, dt, u, v, w, T, gu, gv, gw, gT, gp, gHu, gHv, gHw, gHT):
        _check(lib().afid_rk3_substep_adjoint(
            self._h, int(l), float(dt), _ptr(u, self.cell, "u"), _ptr(v, self.cell, "v"),
            _ptr(w, self.face, "w"), _ptr(T, self.face, "T"), _ptr(gu, self.cell, "gu"),
            _ptr(gv, self.cell, "gv"), _ptr(gw, self.face, "gw"), _ptr(gT, self.face, "gT"),
            _ptr(gp, self.cell, "gp"), _ptr(gHu, self.cell, "gHu"), _ptr(gHv, self.cell, "gHv"),
            _ptr(gHw, self.face, "gHw"), _ptr(gHT, self.face, "gHT")), "afid_rk3_substep_adjoint")


class MultiRes:
    """Refined temperature grid over a Context (afid_mr_*): the grid refined
    rx x ry x rz times, the velocity prolongation, the restriction of the
    temperature and the refined temperature steps. Fine fields: velocity
    cells `fcell` = (nzf, nyf, nxf), faces and temperature `fface` =
    (nzf + 1, nyf, nxf)."""

    def __init__(self, ctx: Context, rx: int, ry: int, rz: int):
        self.ctx = ctx
        self.r = (int(rx), int(ry), int(rz))
        h = C.c_void_p()
        _check(lib().afid_mr_create(ctx._h, self.r[0], self.r[1], self.r[2], C.byref(h)), "afid_mr_create")
        self._h = h
        ctx._children.add(self)
        a, b, c = I(), I(), I()
        _check(lib().afid_mr_dims(h, C.byref(a), C.byref(b), C.byref(c)), "afid_mr_dims")
        self.nx, self.ny, self.nz = a.value, b.value, c.value
        self.workspace_bytes = int(lib().afid_mr_workspace_bytes(h))

    def faces(self):
        """The nzf + 1 fine face coordinates (numpy)."""
        zf = np.zeros(self.nz + 1, dtype=np.float64)
        _check(lib().afid_mr_faces(self._h, zf.ctypes.data_as(C.c_void_p)), "afid_mr_faces")
        return zf

    @property
    def fcell(self):
        return (self.nz, self.ny, self.nx)

    @property
    def fface(self):
        return (self.nz + 1, self.ny, self.nx)

    def close(self):
        if getattr(self, "_h", None):
            lib().afid_mr_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def prolong(self, vel0, vel1=None, theta=0.0, out=None):
        """Fine (uf, vf, wf) at t + theta dt from the coarse states vel0 at t
        and vel1 at t + dt."""
        import torch
        cc, cf = self.ctx.cell, self.ctx.face
        u0, v0, w0 = vel0
        if out is None:
            out = (torch.empty(self.fcell, dtype=torch.float64, device=u0.device),
                   torch.empty(self.fcell, dtype=torch.float64, device=u0.device),
                   torch.empty(self.fface, dtype=torch.float64, device=u0.device))
        u1, v1, w1 = vel1 if vel1 is not None else (None, None, None)
        _check(lib().afid_mr_prolong(
            self._h, _ptr(u0, cc, "u0"), _ptr(v0, cc, "v0"), _ptr(w0, cf, "w0"), _ptr(u1, cc, "u1"),
            _ptr(v1, cc, "v1"), _ptr(w1, cf, "w1"), float(theta), _ptr(out[0], self.fcell, "uf"),
            _ptr(out[1], self.fcell, "vf"), _ptr(out[2], self.fface, "wf")), "afid_mr_prolong")
        return out

    def restrict(self, Tf, Tc=None):
        import torch
        if Tc is None:
            Tc = torch.empty(self.ctx.face, dtype=torch.float64, device=Tf.device)
        _check(lib().afid_mr_restrict(self._h, _ptr(Tf, self.fface, "Tf"), _ptr(Tc, self.ctx.face, "Tc")),
               "afid_mr_restrict")
        return Tc

    def scalar_advance(self, dt, n_sub, vel0, vel1, Tf):
        cc, cf = self.ctx.cell, self.ctx.face
        (u0, v0, w0), (u1, v1, w1) = vel0, vel1
        _check(lib().afid_mr_scalar_advance(
            self._h, float(dt), int(n_sub), _ptr(u0, cc, "u0"), _ptr(v0, cc, "v0"), _ptr(w0, cf, "w0"),
            _ptr(u1, cc, "u1"), _ptr(v1, cc, "v1"), _ptr(w1, cf, "w1"), _ptr(Tf, self.fface, "Tf")),
            "afid_mr_scalar_advance")

    def statistics(self, u, v, w, Tf):
        """Wall-normal statistics on the refined grid (afid_mr_statistics):
        (profiles [nzf+1][9] numpy, scalars dict), as Context.statistics."""
        cc, cf = self.ctx.cell, self.ctx.face
        prof = np.zeros((self.nz + 1, STAT_NQ), dtype=np.float64)
        st = Stats()
        _check(lib().afid_mr_statistics(self._h, _ptr(u, cc, "u"), _ptr(v, cc, "v"), _ptr(w, cf, "w"),
                                        _ptr(Tf, self.fface, "Tf"), prof.ctypes.data_as(C.c_void_p),
                                        C.byref(st)), "afid_mr_statistics")
        return prof, {name: getattr(st, name) for name, _ in Stats._fields_}

    def step(self, dt, n_sub, u, v, w, p, Hu, Hv, Hw, Tf, info=False):
        """One coupled step in place (momentum on the context's grid, Tf on
        the fine grid)."""
        cc, cf = self.ctx.cell, self.ctx.face
        inf = Info() if info else None
        st = lib().afid_mr_step(self._h, float(dt), int(n_sub), _ptr(u, cc, "u"), _ptr(v, cc, "v"),
                                _ptr(w, cf, "w"), _ptr(p, cc, "p"), _ptr(Hu, cc, "Hu"), _ptr(Hv, cc, "Hv"),
                                _ptr(Hw, cf, "Hw"), _ptr(Tf, self.fface, "Tf"), C.byref(inf) if inf else None)
        _check(st, "afid_mr_step", allow=(AFID_ERR_NOT_CONVERGED, AFID_ERR_INCONSISTENT_RHS))
        if info:
            d = inf.as_dict()
            d["status"] = st
            return d
        return None
