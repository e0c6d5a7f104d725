"""Python access to the FP64 CPU oracle (oracle/sfx_oracle.c).

TEST INFRASTRUCTURE: the tests, the smoke check and the benchmark's CPU
baseline leg use this module to check and time the CUDA library.  The
library itself never imports it.

All arrays are float64 numpy arrays laid out as described in the workloads
module: cells (nz, ny, nx), faces ux (nz, ny, nx+1), uy (nz, ny+1, nx),
uz (nz+1, ny, nx).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sfx_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SO_OMP = os.path.join(_BUILD, "liboracle_omp.so")


def _compile(out, extra):
    tmp = out + ".%d.tmp" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c99",
                           *extra, "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, out)


def build(force: bool = False, openmp: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no FMA contraction).  With
    openmp=True the same source with -fopenmp: its order-independent loops
    (operator applications, residual maxima, coefficients, advection,
    normals) run on all host cores; the Gauss-Seidel sweeps stay serial, so
    every result is bitwise the serial one."""
    os.makedirs(_BUILD, exist_ok=True)
    so = _SO_OMP if openmp else _SO
    stale = (not os.path.exists(so)) or os.path.getmtime(so) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "sfx_oracle.h")))
    if force or stale:
        _compile(so, ["-fopenmp"] if openmp else [])
    return so


_use_openmp = False


def use_openmp(on: bool) -> None:
    """Route the calls below to the OpenMP build (threads: OMP_NUM_THREADS,
    else every host core) or back to the serial one."""
    global _use_openmp
    _use_openmp = bool(on)


class Grid(C.Structure):
    _fields_ = [("geom", C.c_int), ("nx", C.c_int), ("ny", C.c_int),
                ("nz", C.c_int), ("h", C.c_double)]


class Params(C.Structure):
    _fields_ = [("ka", C.c_double), ("kd", C.c_double), ("gamma_inf", C.c_double),
                ("Df", C.c_double), ("DF", C.c_double), ("eps", C.c_double),
                ("eta", C.c_double), ("sigma0", C.c_double), ("E", C.c_double),
                ("eos", C.c_int), ("literal_upwind", C.c_int),
                ("bc_F", C.c_double), ("bc_f", C.c_double)]


class Opts(C.Structure):
    _fields_ = [("tol", C.c_double), ("max_picard", C.c_int), ("max_sweeps", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("picard", C.c_int), ("sweeps", C.c_int), ("res_f", C.c_double),
                ("res_F", C.c_double), ("mass_f", C.c_double),
                ("mass_F", C.c_double), ("converged", C.c_int)]


_libs = {}
_P = C.POINTER(C.c_double)


def lib():
    key = bool(_use_openmp)
    if key not in _libs:
        L = C.CDLL(build(openmp=key))
        G, Pp = C.POINTER(Grid), C.POINTER(Params)
        L.orc_threads.restype = C.c_int
        L.orc_threads.argtypes = []
        L.orc_cell_volume.restype = C.c_double
        L.orc_cell_volume.argtypes = [G, C.c_int, C.c_int, C.c_int]
        L.orc_redistance.argtypes = [G, _P, C.c_int, C.c_double, _P]
        L.orc_phase_field.argtypes = [G, _P, C.c_double, _P, _P]
        L.orc_phase_field_build.argtypes = [G, _P, C.c_int, C.c_double, C.c_double, _P, _P, _P]
        L.orc_normals.argtypes = [G, _P, C.c_double, _P]
        L.orc_face_drift.argtypes = [G, Pp, _P, C.c_int, _P, _P, _P]
        L.orc_apply_operator.argtypes = [G, C.c_double, _P, _P, _P, C.c_int, _P, _P, _P]
        L.orc_elliptic_solve.restype = C.c_int
        L.orc_elliptic_solve.argtypes = [G, C.c_double, _P, _P, _P, C.c_int, _P, _P, _P,
                                         C.c_double, C.c_int, _P]
        L.orc_advect_bcg.argtypes = [G, _P, _P, _P, C.c_double, _P, C.c_double, _P]
        L.orc_vof_advect.argtypes = [G, _P, _P, _P, C.c_double, C.c_int, _P]
        L.orc_coupled_implicit.argtypes = [G, Pp, _P, _P, _P, C.c_double, C.POINTER(Opts),
                                           _P, _P, C.POINTER(Stats)]
        L.orc_surfactant_step.argtypes = [G, Pp, _P, _P, _P, _P, C.c_double,
                                          C.POINTER(Opts), _P, _P, C.POINTER(Stats)]
        L.orc_coupled_residual.argtypes = [G, Pp, _P, _P, _P, C.c_double, _P, _P, _P, _P,
                                           _P, _P]
        L.orc_total.restype = C.c_double
        L.orc_total.argtypes = [G, _P]
        L.orc_eos.argtypes = [G, Pp, _P, _P, _P, _P]
        L.orc_marangoni.argtypes = [G, Pp, _P, _P, _P, C.c_int, _P, _P]
        L.orc_capillary.argtypes = [G, _P, _P, _P, C.c_double, _P, _P]
        L.orc_acdi_step.argtypes = [G, _P, _P, _P, C.c_double, C.c_double, C.c_double, C.c_int,
                                    _P, _P]
        L.orc_plic_volume.restype = C.c_double
        L.orc_plic_volume.argtypes = [C.c_int, _P, C.c_double]
        L.orc_plic_area.restype = C.c_double
        L.orc_plic_area.argtypes = [C.c_int, _P, C.c_double]
        L.orc_cfl_dt.restype = C.c_double
        L.orc_cfl_dt.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, C.c_double,
                                 C.c_double]
        _libs[key] = L
    return _libs[key]


# ------------------------------------------------------------ helpers
def _ptr(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_P)


def _arr(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def cgrid(g) -> Grid:
    return Grid(int(g.geom), int(g.nx), int(g.ny), int(g.nz), float(g.h))


def cparams(p) -> Params:
    return Params(p.ka, p.kd, p.gamma_inf, p.Df, p.DF, p.eps, p.eta, p.sigma0, p.E,
                  int(p.eos), int(p.literal_upwind), p.bc_F, p.bc_f)


def _face_shapes(g):
    nz, ny, nx = g.nz, g.ny, g.nx
    return [(nz, ny, nx + 1), (nz, ny + 1, nx), (nz + 1, ny, nx)]


# ------------------------------------------------------------ API
def threads():
    """Threads of the build in use (1 for the serial oracle)."""
    return int(lib().orc_threads())


def cell_volumes(g):
    L, G = lib(), cgrid(g)
    V = np.empty((g.nz, g.ny, g.nx))
    for k in range(g.nz):
        for j in range(g.ny):
            for i in range(g.nx):
                V[k, j, i] = L.orc_cell_volume(C.byref(G), i, j, k)
    return V


def redistance(g, Cf, iters, dtau):
    chi = np.empty((g.nz, g.ny, g.nx))
    lib().orc_redistance(C.byref(cgrid(g)), _ptr(_arr(Cf)), int(iters), float(dtau), _ptr(chi))
    return chi


def phase_field(g, chi, eps):
    phi = np.empty((g.nz, g.ny, g.nx))
    delta = np.empty_like(phi)
    lib().orc_phase_field(C.byref(cgrid(g)), _ptr(_arr(chi)), float(eps), _ptr(phi), _ptr(delta))
    return phi, delta


def phase_field_build(g, Cf, iters, dtau, eps):
    shp = (g.nz, g.ny, g.nx)
    chi, phi, delta = np.empty(shp), np.empty(shp), np.empty(shp)
    lib().orc_phase_field_build(C.byref(cgrid(g)), _ptr(_arr(Cf)), int(iters), float(dtau),
                                float(eps), _ptr(chi), _ptr(phi), _ptr(delta))
    return chi, phi, delta


def normals(g, phi, eps):
    n = np.empty((g.ndim, g.nz, g.ny, g.nx))
    lib().orc_normals(C.byref(cgrid(g)), _ptr(_arr(phi)), float(eps), _ptr(n))
    return n


def face_drift(g, p, phi, which):
    sh = _face_shapes(g)
    Bx, By = np.empty(sh[0]), np.empty(sh[1])
    Bz = np.empty(sh[2]) if g.ndim == 3 else np.zeros(1)
    lib().orc_face_drift(C.byref(cgrid(g)), C.byref(cparams(p)), _ptr(_arr(phi)), int(which),
                         _ptr(Bx), _ptr(By), _ptr(Bz))
    return Bx, By, (Bz if g.ndim == 3 else None)


def _bz(g, Bz):
    return _arr(Bz) if (g.ndim == 3 and Bz is not None) else np.zeros(1)


def apply_operator(g, D, Bx, By, Bz, lam, a, literal=0):
    out = np.empty((g.nz, g.ny, g.nx))
    lib().orc_apply_operator(C.byref(cgrid(g)), float(D), _ptr(_arr(Bx)), _ptr(_arr(By)),
                             _ptr(_bz(g, Bz)), int(literal), _ptr(_arr(lam)), _ptr(_arr(a)),
                             _ptr(out))
    return out


def elliptic_solve(g, D, Bx, By, Bz, lam, b, a0=None, tol=1e-13, max_sweeps=100000,
                   literal=0):
    a = np.zeros((g.nz, g.ny, g.nx)) if a0 is None else _arr(a0).copy()
    rr = C.c_double(0)
    s = lib().orc_elliptic_solve(C.byref(cgrid(g)), float(D), _ptr(_arr(Bx)), _ptr(_arr(By)),
                                 _ptr(_bz(g, Bz)), int(literal), _ptr(_arr(lam)),
                                 _ptr(_arr(b)), _ptr(a), float(tol), int(max_sweeps),
                                 C.byref(rr))
    return a, s, rr.value


def advect_bcg(g, ux, uy, uz, dt, xi, bc_in):
    out = np.empty((g.nz, g.ny, g.nx))
    uzp = _arr(uz) if g.ndim == 3 else np.zeros(1)
    lib().orc_advect_bcg(C.byref(cgrid(g)), _ptr(_arr(ux)), _ptr(_arr(uy)), _ptr(uzp),
                         float(dt), _ptr(_arr(xi)), float(bc_in), _ptr(out))
    return out


def vof_advect(g, ux, uy, uz, dt, Cf, order=0):
    """One split PLIC step of the volume fraction (returns a new array)."""
    out = np.array(Cf, dtype=np.float64, copy=True)
    uzp = _arr(uz) if g.ndim == 3 else np.zeros(1)
    lib().orc_vof_advect(C.byref(cgrid(g)), _ptr(_arr(ux)), _ptr(_arr(uy)), _ptr(uzp),
                         float(dt), int(order), _ptr(out))
    return out


def coupled_implicit(g, p, phi, fstar, Fstar, dt, tol, max_picard=200, max_sweeps=100000):
    f = np.empty((g.nz, g.ny, g.nx))
    F = np.empty_like(f)
    st = Stats()
    o = Opts(float(tol), int(max_picard), int(max_sweeps))
    lib().orc_coupled_implicit(C.byref(cgrid(g)), C.byref(cparams(p)), _ptr(_arr(phi)),
                               _ptr(_arr(fstar)), _ptr(_arr(Fstar)), float(dt), C.byref(o),
                               _ptr(f), _ptr(F), C.byref(st))
    return f, F, st


def surfactant_step(g, p, phi, f, F, dt, tol, ux=None, uy=None, uz=None, max_picard=200,
                    max_sweeps=100000):
    """One coupled step; returns new (f, F, stats).  Inputs are not modified."""
    f = _arr(f).copy()
    F = _arr(F).copy()
    st = Stats()
    o = Opts(float(tol), int(max_picard), int(max_sweeps))
    uzp = _arr(uz) if (ux is not None and g.ndim == 3) else (np.zeros(1) if ux is not None else None)
    lib().orc_surfactant_step(C.byref(cgrid(g)), C.byref(cparams(p)), _ptr(_arr(phi)),
                              _ptr(_arr(ux)), _ptr(_arr(uy)), _ptr(uzp), float(dt),
                              C.byref(o), _ptr(f), _ptr(F), C.byref(st))
    return f, F, st


def coupled_residual(g, p, phi, fstar, Fstar, dt, f, F):
    rf = np.empty((g.nz, g.ny, g.nx))
    rF = np.empty_like(rf)
    a, b = C.c_double(0), C.c_double(0)
    lib().orc_coupled_residual(C.byref(cgrid(g)), C.byref(cparams(p)), _ptr(_arr(phi)),
                               _ptr(_arr(fstar)), _ptr(_arr(Fstar)), float(dt), _ptr(_arr(f)),
                               _ptr(_arr(F)), _ptr(rf), _ptr(rF), C.byref(a), C.byref(b))
    return rf, rF, a.value, b.value


def total(g, x):
    return lib().orc_total(C.byref(cgrid(g)), _ptr(_arr(x)))


def eos(g, p, f, phi):
    gam = np.empty((g.nz, g.ny, g.nx))
    sig = np.empty_like(gam)
    lib().orc_eos(C.byref(cgrid(g)), C.byref(cparams(p)), _ptr(_arr(f)), _ptr(_arr(phi)),
                  _ptr(gam), _ptr(sig))
    return gam, sig


def marangoni(g, p, f, phi, Cf, dm_mode=1):
    sig = np.empty((g.nz, g.ny, g.nx))
    force = np.empty((g.ndim, g.nz, g.ny, g.nx))
    lib().orc_marangoni(C.byref(cgrid(g)), C.byref(cparams(p)), _ptr(_arr(f)), _ptr(_arr(phi)),
                        _ptr(_arr(Cf)), int(dm_mode), _ptr(sig), _ptr(force))
    return sig, force


def acdi_step(g, phi, dt, zeta, eps, ux=None, uy=None, uz=None, clip=False):
    """One ACDI step of phi (advection when ux is given; result clipped to
    [0, 1] with clip); returns a new array."""
    out = np.empty((g.nz, g.ny, g.nx))
    cl = 1 if clip else 0
    if ux is None:
        lib().orc_acdi_step(C.byref(cgrid(g)), None, None, None, float(dt), float(zeta), float(eps),
                            cl, _ptr(_arr(phi)), _ptr(out))
    else:
        uzp = _arr(uz) if g.ndim == 3 else np.zeros(1)
        lib().orc_acdi_step(C.byref(cgrid(g)), _ptr(_arr(ux)), _ptr(_arr(uy)), _ptr(uzp), float(dt),
                            float(zeta), float(eps), cl, _ptr(_arr(phi)), _ptr(out))
    return out


def capillary(g, phi, Cf, sigma, eps):
    """(kappa, force): curvature -div n and F_cap = sigma kappa |grad C| n."""
    kap = np.empty((g.nz, g.ny, g.nx))
    force = np.empty((g.ndim, g.nz, g.ny, g.nx))
    lib().orc_capillary(C.byref(cgrid(g)), _ptr(_arr(phi)), _ptr(_arr(Cf)), _ptr(_arr(sigma)),
                        float(eps), _ptr(kap), _ptr(force))
    return kap, force


def plic_volume(dim, m, alpha):
    m = np.ascontiguousarray(m, dtype=np.float64)
    return lib().orc_plic_volume(int(dim), _ptr(m), float(alpha))


def plic_area(dim, m, Cv):
    m = np.ascontiguousarray(m, dtype=np.float64)
    return lib().orc_plic_area(int(dim), _ptr(m), float(Cv))


def cfl_dt(ndim, h, umax, D, eps, safety=1.0):
    return lib().orc_cfl_dt(int(ndim), float(h), float(umax), float(D), float(eps),
                            float(safety))
