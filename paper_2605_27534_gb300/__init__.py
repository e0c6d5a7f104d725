"""GB300 (sm_103a) library for the coupled soluble-surfactant step of the hybrid
VoF / phase-field method (arxiv 2605.27534).

This module is a thin binding: it marshals torch CUDA tensors (device
pointers) and the current torch stream into the C-ABI of libsfx
(include/sfx.h).  Every step of the method runs in the library's CUDA
kernels; nothing here computes on the CPU, and nothing falls back when the
library is missing.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
from typing import Optional, Sequence

from . import _lib
from ._lib import (SFX_AXISYM, SFX_CART3D, SFX_F32, SFX_F64, SFX_OK, SFX_ERR_NOT_CONVERGED,
                   SFX_PLANAR2D, Grid, Params, SolveOpts, StepStats)

__all__ = ["SfxError", "Context", "Batch", "SurfactantRollout", "RolloutSetup", "lib", "default_opts", "SFX_PLANAR2D", "SFX_AXISYM",
           "SFX_CART3D", "SFX_F64", "SFX_F32"]


class SfxError(RuntimeError):
    def __init__(self, status: int, where: str):
        L = lib()
        msg = L.sfx_status_string(status).decode()
        if status == _lib.SFX_ERR_CUDA:
            msg += " (%s)" % L.sfx_last_cuda_error().decode()
        super().__init__("%s: %s" % (where, msg))
        self.status = status


def lib():
    return _lib.load()


def _check(st: int, where: str, allow=()):
    if st != SFX_OK and st not in allow:
        raise SfxError(st, where)
    return st


def default_opts(**kw) -> SolveOpts:
    o = SolveOpts()
    lib().sfx_default_opts(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("libsfx takes CUDA tensors (device pointers)")
    if not t.is_contiguous():
        raise ValueError("libsfx takes contiguous tensors")
    return t.data_ptr()


def _stream():
    import torch
    return torch.cuda.current_stream().cuda_stream


def params_struct(p) -> Params:
    """Params from any object with the fields of sfx_params."""
    return Params(p.ka, p.kd, p.gamma_inf, p.Df, p.DF, p.eps, p.eta, p.sigma0, p.E, int(p.eos),
                  int(p.literal_upwind), p.bc_F, p.bc_f)


class Context:
    """One grid shape and precision (owns the multigrid pyramid and scratch)."""

    def __init__(self, geom: int, nx: int, ny: int, nz: int, h: float, precision: int = SFX_F64):
        self.grid = Grid(int(geom), int(nx), int(ny), int(nz), float(h))
        self.precision = int(precision)
        h_ = C.c_void_p()
        _check(lib().sfx_ctx_create(C.byref(self.grid), self.precision, C.byref(h_)),
               "sfx_ctx_create")
        self._h = h_

    @classmethod
    def for_grid(cls, g, precision=SFX_F64):
        return cls(g.geom, g.nx, g.ny, g.nz, g.h, precision)

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            lib().sfx_ctx_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------ calls
    def sfx_phase_field_build(self, Cf, chi, phi, delta=None, iters=24, dtau=None, eps=None):
        dtau = dtau if dtau is not None else 0.5 * self.grid.h
        _check(lib().sfx_phase_field_build(self._h, _ptr(Cf), _ptr(chi), _ptr(phi), _ptr(delta),
                                           int(iters), float(dtau), float(eps), _stream()),
               "sfx_phase_field_build")

    def sfx_phase_field_from_chi(self, chi, phi, delta=None, eps=None):
        _check(lib().sfx_phase_field_from_chi(self._h, _ptr(chi), _ptr(phi), _ptr(delta),
                                              float(eps), _stream()), "sfx_phase_field_from_chi")

    def sfx_advect(self, ux, uy, uz, dt, xi, bc_in, xi_out):
        _check(lib().sfx_advect(self._h, _ptr(ux), _ptr(uy), _ptr(uz), float(dt), _ptr(xi),
                                float(bc_in), _ptr(xi_out), _stream()), "sfx_advect")

    def sfx_vof_advect(self, ux, uy, uz, dt, Cf, order=0):
        """One split PLIC step of the volume fraction Cf (double, in place)."""
        _check(lib().sfx_vof_advect(self._h, _ptr(ux), _ptr(uy), _ptr(uz), float(dt), int(order),
                                    _ptr(Cf), _stream()), "sfx_vof_advect")

    def sfx_mg_solve(self, D, Bx, By, Bz, lam, b, a, opts=None, literal_upwind=0):
        o = opts if opts is not None else default_opts()
        cyc, res = C.c_int(0), C.c_double(0)
        st = lib().sfx_mg_solve(self._h, float(D), _ptr(Bx), _ptr(By), _ptr(Bz),
                                int(literal_upwind), _ptr(lam), _ptr(b), _ptr(a), C.byref(o),
                                C.byref(cyc), C.byref(res), _stream())
        _check(st, "sfx_mg_solve", allow=(SFX_ERR_NOT_CONVERGED,))
        return cyc.value, res.value, st == SFX_OK

    def sfx_surfactant_step(self, params, phi, f, F, dt, ux=None, uy=None, uz=None, opts=None,
                            stats=True, allow_not_converged=False):
        o = opts if opts is not None else default_opts()
        st_ = StepStats()
        ps = params if isinstance(params, Params) else params_struct(params)
        st = lib().sfx_surfactant_step(self._h, C.byref(ps), _ptr(phi), _ptr(ux), _ptr(uy),
                                       _ptr(uz), _ptr(f), _ptr(F), float(dt), C.byref(o),
                                       C.byref(st_) if stats else None, _stream())
        _check(st, "sfx_surfactant_step",
               allow=(SFX_ERR_NOT_CONVERGED,) if allow_not_converged else ())
        return st_

    def sfx_totals(self, fields: Sequence):
        n = len(fields)
        arr = (C.c_void_p * n)(*[_ptr(t) for t in fields])
        out = (C.c_double * n)()
        _check(lib().sfx_totals(self._h, arr, n, out, _stream()), "sfx_totals")
        return [out[i] for i in range(n)]

    def sfx_marangoni_force(self, params, f, phi, Cf, sigma, force, dm_mode=1):
        ps = params if isinstance(params, Params) else params_struct(params)
        _check(lib().sfx_marangoni_force(self._h, C.byref(ps), _ptr(f), _ptr(phi), _ptr(Cf),
                                         int(dm_mode), _ptr(sigma), _ptr(force), _stream()),
               "sfx_marangoni_force")

    def sfx_acdi_step(self, phi, dt, zeta, eps, ux=None, uy=None, uz=None, clip=False):
        """One ACDI step of the double phase field `phi`, in place (result
        clipped to [0, 1] with clip)."""
        _check(lib().sfx_acdi_step(self._h, _ptr(ux), _ptr(uy), _ptr(uz), float(dt), float(zeta),
                                   float(eps), 1 if clip else 0, _ptr(phi), _stream()),
               "sfx_acdi_step")

    def sfx_capillary_force(self, params, phi, Cf, sigma, force, kappa=None):
        """F_cap = sigma kappa |grad C| n into `force` (ndim x N), the
        curvature into `kappa` when given."""
        ps = params if isinstance(params, Params) else params_struct(params)
        _check(lib().sfx_capillary_force(self._h, C.byref(ps), _ptr(phi), _ptr(Cf), _ptr(sigma),
                                         _ptr(kappa), _ptr(force), _stream()),
               "sfx_capillary_force")

    def sfx_df_pack(self, x, out=None):
        return sfx_df_pack(x, out)

    def sfx_df_unpack(self, p, out=None):
        return sfx_df_unpack(p, out)

    def sfx_set_tuning(self, key: int, value: int):
        _check(lib().sfx_set_tuning(self._h, int(key), int(value)), "sfx_set_tuning")

    def sfx_profile(self, on: bool):
        _check(lib().sfx_profile(self._h, 1 if on else 0), "sfx_profile")

    def sfx_profile_read(self):
        """{kind: (launches, total_ms, timed_launches)} since sfx_profile(True)."""
        out = {}
        for k, name in enumerate(_lib.KERNEL_KINDS):
            n, ms, nt = C.c_longlong(0), C.c_double(0), C.c_longlong(0)
            _check(lib().sfx_profile_read(self._h, k, C.byref(n), C.byref(ms), C.byref(nt)),
                   "sfx_profile_read")
            out[name] = (n.value, ms.value, nt.value)
        return out

    def sfx_profile_work(self):
        """{kind: launches that did work} for the kinds the library counts
        (the FP32 Newton solve's residual passes)."""
        out = {}
        for k, name in enumerate(_lib.KERNEL_KINDS):
            w = C.c_longlong(0)
            _check(lib().sfx_profile_work(self._h, k, C.byref(w)), "sfx_profile_work")
            if w.value >= 0:
                out[name] = w.value
        return out

    # ------------------------------------------------------------ adjoint
    def sfx_f_from_gamma(self, gamma, phi, eps, out=None):
        """f = Gamma delta_phi (double tensors); also maps dL/df to dL/dGamma."""
        import torch
        if out is None:
            out = torch.empty_like(gamma)
        _check(lib().sfx_f_from_gamma(self._h, _ptr(gamma), _ptr(phi), float(eps), _ptr(out),
                                      _stream()), "sfx_f_from_gamma")
        return out

    def sfx_marangoni_loss(self, params, f, phi, Cf, dm_mode=1, grad=True):
        """(L = sum V |F_Ma|^2, dL/df or None); all double tensors."""
        import torch
        ps = params if isinstance(params, Params) else params_struct(params)
        g = torch.empty_like(f) if grad else None
        L = C.c_double(0)
        _check(lib().sfx_marangoni_loss(self._h, C.byref(ps), _ptr(f), _ptr(phi), _ptr(Cf),
                                        int(dm_mode), C.byref(L), _ptr(g), _stream()),
               "sfx_marangoni_loss")
        return L.value, g

    def sfx_adjoint_apply(self, params, phi, f, F, dt, vf, vF, transpose=False):
        """((-J) v) or ((-J)^T v) at the state (f, F) after a step."""
        import torch
        ps = params if isinstance(params, Params) else params_struct(params)
        of, oF = torch.empty_like(vf), torch.empty_like(vF)
        _check(lib().sfx_adjoint_apply(self._h, C.byref(ps), _ptr(phi), _ptr(f), _ptr(F),
                                       float(dt), 1 if transpose else 0, _ptr(vf), _ptr(vF),
                                       _ptr(of), _ptr(oF), _stream()), "sfx_adjoint_apply")
        return of, oF

    def sfx_adjoint_step(self, params, phi, f, F, dt, lam_f, lam_F, dparams=None, opts=None):
        """lam (in place) from dL/dx after the step to dL/dx before it; adds
        the step's dL/d(k_a, k_d, D_f, D_F) to dparams (4 floats, a list)."""
        ps = params if isinstance(params, Params) else params_struct(params)
        o = opts if opts is not None else default_opts(tol=1e-13, max_cycles=500, nu1=10, nu2=10)
        dp = (C.c_double * 4)(*(dparams if dparams is not None else [0.0] * 4))
        st_ = StepStats()
        _check(lib().sfx_adjoint_step(self._h, C.byref(ps), _ptr(phi), _ptr(f), _ptr(F),
                                      float(dt), _ptr(lam_f), _ptr(lam_F), dp, C.byref(o),
                                      C.byref(st_), _stream()), "sfx_adjoint_step")
        if dparams is not None:
            for k in range(4):
                dparams[k] = dp[k]
        return st_

    def sfx_cfl_dt(self, ux, uy, uz, D, eps, safety=1.0):
        out = C.c_double(0)
        _check(lib().sfx_cfl_dt(self._h, _ptr(ux), _ptr(uy), _ptr(uz), float(D), float(eps),
                                float(safety), C.byref(out), _stream()), "sfx_cfl_dt")
        return out.value


class Batch:
    """Many independent instances stepped together (sfx_batch_*).

    `instances` is a sequence of (nr, nz, h, dt, params); fields are packed
    back to back, instance i at the offsets of `layout()`.  geom is
    SFX_AXISYM (rings) or SFX_PLANAR2D (planar cells of unit depth).
    """

    def __init__(self, instances, geom=None):
        n = len(instances)
        arr = (_lib.BatchInstance * n)()
        for i, (nr, nz, h, dt, p) in enumerate(instances):
            ps = p if isinstance(p, Params) else params_struct(p)
            arr[i] = _lib.BatchInstance(int(nr), int(nz), float(h), float(dt), ps)
        self.n = n
        h_ = C.c_void_p()
        if geom is None:
            _check(lib().sfx_batch_create(arr, n, C.byref(h_)), "sfx_batch_create")
        else:
            _check(lib().sfx_batch_create_geom(arr, n, int(geom), C.byref(h_)),
                   "sfx_batch_create_geom")
        self._h = h_

    def close(self):
        if self._h:
            lib().sfx_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sfx_batch_layout(self):
        """(n_cells, n_rfaces, n_zfaces, cell_off, rface_off, zface_off)."""
        n = self.n
        nc, nr, nz = C.c_size_t(0), C.c_size_t(0), C.c_size_t(0)
        co, ro, zo = (C.c_size_t * n)(), (C.c_size_t * n)(), (C.c_size_t * n)()
        _check(lib().sfx_batch_layout(self._h, C.byref(nc), C.byref(nr), C.byref(nz), co, ro, zo),
               "sfx_batch_layout")
        return nc.value, nr.value, nz.value, list(co), list(ro), list(zo)

    def sfx_batch_set_schedule(self, block=256, sweeps=3, max_iters=8):
        _check(lib().sfx_batch_set_schedule(self._h, int(block), int(sweeps), int(max_iters)),
               "sfx_batch_set_schedule")

    def sfx_batch_set_tuning(self, key, value):
        """Batch solver tuning (SFX_TUNE_F32_FAST_RESID only)."""
        _check(lib().sfx_batch_set_tuning(self._h, int(key), int(value)), "sfx_batch_set_tuning")

    def sfx_batch_reuse_phi(self, on=True):
        """Static phi: fold and drift faces outside the step graph."""
        _check(lib().sfx_batch_reuse_phi(self._h, 1 if on else 0), "sfx_batch_reuse_phi")

    def sfx_batch_step(self, phi, f, F, tol, ur=None, uz=None):
        _check(lib().sfx_batch_step(self._h, _ptr(phi), _ptr(ur), _ptr(uz), _ptr(f), _ptr(F),
                                    float(tol), _stream()), "sfx_batch_step")

    def sfx_batch_stats(self):
        """dict of per-instance lists: iters, res_f, res_F, mass_f, mass_F, converged."""
        n = self.n
        it, cv = (C.c_int * n)(), (C.c_int * n)()
        rf, rF = (C.c_float * n)(), (C.c_float * n)()
        mf, mF = (C.c_double * n)(), (C.c_double * n)()
        _check(lib().sfx_batch_stats(self._h, it, rf, rF, mf, mF, cv, _stream()),
               "sfx_batch_stats")
        return {"iters": list(it), "res_f": list(rf), "res_F": list(rF), "mass_f": list(mf),
                "mass_F": list(mF), "converged": [bool(x) for x in cv]}

    def sfx_batch_work(self, reset=False):
        """(residual passes, sweep groups) per instance since creation or reset."""
        n = self.n
        r, w = (C.c_longlong * n)(), (C.c_longlong * n)()
        _check(lib().sfx_batch_work(self._h, r, w, 1 if reset else 0, _stream()), "sfx_batch_work")
        return list(r), list(w)

    def sfx_batch_autotune(self, phi, f, F, tol, ur=None, uz=None):
        """Pick block size, sweeps and iteration budget; returns them."""
        ch = (C.c_int * 3)()
        _check(lib().sfx_batch_autotune(self._h, _ptr(phi), _ptr(ur), _ptr(uz), _ptr(f), _ptr(F),
                                        float(tol), _stream(), ch), "sfx_batch_autotune")
        return tuple(ch)


def sfx_df_pack(x, out=None):
    """double tensor -> double-float pairs (float32 tensor, last dim 2)."""
    import torch
    if out is None:
        out = torch.empty(tuple(x.shape) + (2,), dtype=torch.float32, device=x.device)
    _check(lib().sfx_df_pack(_ptr(x), _ptr(out), x.numel(), _stream()), "sfx_df_pack")
    return out


def sfx_df_unpack(p, out=None):
    """double-float pairs (float32, last dim 2) -> double tensor."""
    import torch
    if out is None:
        out = torch.empty(tuple(p.shape[:-1]), dtype=torch.float64, device=p.device)
    _check(lib().sfx_df_unpack(_ptr(p), _ptr(out), out.numel(), _stream()), "sfx_df_unpack")
    return out


from .adjoint import RolloutSetup, SurfactantRollout  # noqa: E402
