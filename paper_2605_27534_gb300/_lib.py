"""ctypes declarations of the libsfx C-ABI (include/sfx.h).

Loading fails loudly when the library has not been built: there is no CPU
or Python fallback for any call.
"""
from __future__ import annotations

import ctypes as C
import os

PKG = os.path.dirname(os.path.abspath(__file__))
SO_PATH = os.path.join(PKG, "libsfx.so")

SFX_OK, SFX_ERR_ARG, SFX_ERR_NOT_CONVERGED, SFX_ERR_NONFINITE, SFX_ERR_TIMEOUT, \
    SFX_ERR_CUDA, SFX_ERR_WORKSPACE = range(7)
SFX_PLANAR2D, SFX_AXISYM, SFX_CART3D = 0, 1, 2
SFX_F64, SFX_F32 = 0, 1

#: every entry point declared in include/sfx.h
EXPORTS = [
    "sfx_version", "sfx_status_string", "sfx_last_cuda_error", "sfx_ctx_create",
    "sfx_ctx_destroy", "sfx_default_opts", "sfx_phase_field_build", "sfx_advect",
    "sfx_mg_solve", "sfx_surfactant_step", "sfx_totals", "sfx_marangoni_force", "sfx_cfl_dt",
    "sfx_profile", "sfx_profile_read", "sfx_totals_noalloc", "sfx_df_pack", "sfx_df_unpack",
    "sfx_set_tuning", "sfx_batch_create", "sfx_batch_create_geom", "sfx_batch_destroy",
    "sfx_batch_layout", "sfx_batch_set_schedule", "sfx_batch_set_tuning", "sfx_batch_step",
    "sfx_batch_stats",
    "sfx_batch_autotune", "sfx_batch_work", "sfx_f_from_gamma", "sfx_marangoni_loss",
    "sfx_adjoint_apply", "sfx_adjoint_step", "sfx_vof_advect", "sfx_capillary_force", "sfx_acdi_step", "sfx_batch_reuse_phi",
    "sfx_phase_field_from_chi", "sfx_profile_work",
]
SFX_TUNE_FUSED_SWEEP = 0
SFX_TUNE_F32_SOLVER = 1
SFX_TUNE_REUSE_DRIFT = 2
SFX_TUNE_PREDICT = 3
SFX_TUNE_F32_REDIST = 4
SFX_TUNE_SWEEP_PLANES = 5
SFX_TUNE_TILED_SWEEP = 6
SFX_TUNE_TILED_ZCHUNK = 7
SFX_TUNE_F32_FAST_RESID = 8
SFX_TUNE_ADVECT_STAGED = 9
SFX_TUNE_F32_INCR_RESID = 10
SFX_TUNE_F32_SOR = 11
KERNEL_KINDS = ["smooth_fine", "smooth_coarse", "restrict", "prolong", "setup", "residual",
                "advect", "totals", "forces", "phase", "other", "smooth_tiled",
                "residual_fp32", "residual_incr"]


class Grid(C.Structure):
    _fields_ = [("geom", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("h", C.c_double)]


class Params(C.Structure):
    _fields_ = [("ka", C.c_double), ("kd", C.c_double), ("gamma_inf", C.c_double),
                ("Df", C.c_double), ("DF", C.c_double), ("eps", C.c_double),
                ("eta", C.c_double), ("sigma0", C.c_double), ("E", C.c_double),
                ("eos", C.c_int), ("literal_upwind", C.c_int), ("bc_F", C.c_double),
                ("bc_f", C.c_double)]


class SolveOpts(C.Structure):
    _fields_ = [("tol", C.c_double), ("max_cycles", C.c_int), ("nu1", C.c_int),
                ("nu2", C.c_int), ("mg_levels", C.c_int), ("vcycles", C.c_int),
                ("check_every", C.c_int), ("coarse_sweeps", C.c_int)]


class StepStats(C.Structure):
    _fields_ = [("picard", C.c_int), ("vcycles", C.c_int), ("res_f", C.c_double),
                ("res_F", C.c_double), ("mass_f", C.c_double), ("mass_F", C.c_double),
                ("converged", C.c_int)]


class BatchInstance(C.Structure):
    _fields_ = [("nr", C.c_int), ("nz", C.c_int), ("h", C.c_double), ("dt", C.c_double),
                ("params", Params)]


_lib = None
vp, dp = C.c_void_p, C.c_double


def load(path: str = SO_PATH):
    """Load libsfx.so (raises OSError if it is missing or unloadable)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError("libsfx.so not built (%s): run __graft_entry__.build() or "
                      "python paper_2605_27534_gb300/build.py" % path)
    L = C.CDLL(path)
    L.sfx_version.restype = C.c_char_p
    L.sfx_version.argtypes = []
    L.sfx_status_string.restype = C.c_char_p
    L.sfx_status_string.argtypes = [C.c_int]
    L.sfx_last_cuda_error.restype = C.c_char_p
    L.sfx_last_cuda_error.argtypes = []
    L.sfx_ctx_create.restype = C.c_int
    L.sfx_ctx_create.argtypes = [C.POINTER(Grid), C.c_int, C.POINTER(vp)]
    L.sfx_ctx_destroy.restype = None
    L.sfx_ctx_destroy.argtypes = [vp]
    L.sfx_default_opts.restype = None
    L.sfx_default_opts.argtypes = [C.POINTER(SolveOpts)]
    L.sfx_phase_field_build.restype = C.c_int
    L.sfx_phase_field_build.argtypes = [vp, vp, vp, vp, vp, C.c_int, dp, dp, vp]
    L.sfx_phase_field_from_chi.restype = C.c_int
    L.sfx_phase_field_from_chi.argtypes = [vp, vp, vp, vp, dp, vp]
    L.sfx_advect.restype = C.c_int
    L.sfx_advect.argtypes = [vp, vp, vp, vp, dp, vp, dp, vp, vp]
    L.sfx_mg_solve.restype = C.c_int
    L.sfx_mg_solve.argtypes = [vp, dp, vp, vp, vp, C.c_int, vp, vp, vp, C.POINTER(SolveOpts),
                               C.POINTER(C.c_int), C.POINTER(C.c_double), vp]
    L.sfx_surfactant_step.restype = C.c_int
    L.sfx_surfactant_step.argtypes = [vp, C.POINTER(Params), vp, vp, vp, vp, vp, vp, dp,
                                      C.POINTER(SolveOpts), C.POINTER(StepStats), vp]
    L.sfx_totals.restype = C.c_int
    L.sfx_totals.argtypes = [vp, C.POINTER(C.c_void_p), C.c_int, C.POINTER(C.c_double), vp]
    L.sfx_marangoni_force.restype = C.c_int
    L.sfx_marangoni_force.argtypes = [vp, C.POINTER(Params), vp, vp, vp, C.c_int, vp, vp, vp]
    L.sfx_cfl_dt.restype = C.c_int
    L.sfx_cfl_dt.argtypes = [vp, vp, vp, vp, dp, dp, dp, C.POINTER(C.c_double), vp]
    L.sfx_profile.restype = C.c_int
    L.sfx_profile.argtypes = [vp, C.c_int]
    L.sfx_profile_read.restype = C.c_int
    L.sfx_profile_read.argtypes = [vp, C.c_int, C.POINTER(C.c_longlong), C.POINTER(C.c_double),
                                   C.POINTER(C.c_longlong)]
    L.sfx_profile_work.restype = C.c_int
    L.sfx_profile_work.argtypes = [vp, C.c_int, C.POINTER(C.c_longlong)]
    L.sfx_df_pack.restype = C.c_int
    L.sfx_df_pack.argtypes = [vp, vp, C.c_size_t, vp]
    L.sfx_df_unpack.restype = C.c_int
    L.sfx_df_unpack.argtypes = [vp, vp, C.c_size_t, vp]
    L.sfx_set_tuning.restype = C.c_int
    L.sfx_set_tuning.argtypes = [vp, C.c_int, C.c_int]
    L.sfx_totals_noalloc.restype = C.c_int
    L.sfx_totals_noalloc.argtypes = [C.POINTER(Grid), C.POINTER(C.c_void_p), C.c_int,
                                     C.POINTER(C.c_double), vp]
    szp = C.POINTER(C.c_size_t)
    ip, fp, dpp = C.POINTER(C.c_int), C.POINTER(C.c_float), C.POINTER(C.c_double)
    L.sfx_batch_create.restype = C.c_int
    L.sfx_batch_create.argtypes = [C.POINTER(BatchInstance), C.c_int, C.POINTER(vp)]
    L.sfx_batch_create_geom.restype = C.c_int
    L.sfx_batch_create_geom.argtypes = [C.POINTER(BatchInstance), C.c_int, C.c_int, C.POINTER(vp)]
    L.sfx_batch_destroy.restype = None
    L.sfx_batch_destroy.argtypes = [vp]
    L.sfx_batch_layout.restype = C.c_int
    L.sfx_batch_layout.argtypes = [vp, szp, szp, szp, szp, szp, szp]
    L.sfx_batch_set_schedule.restype = C.c_int
    L.sfx_batch_set_schedule.argtypes = [vp, C.c_int, C.c_int, C.c_int]
    L.sfx_batch_set_tuning.restype = C.c_int
    L.sfx_batch_set_tuning.argtypes = [vp, C.c_int, C.c_int]
    L.sfx_batch_step.restype = C.c_int
    L.sfx_batch_step.argtypes = [vp, vp, vp, vp, vp, vp, dp, vp]
    L.sfx_batch_stats.restype = C.c_int
    L.sfx_batch_stats.argtypes = [vp, ip, fp, fp, dpp, dpp, ip, vp]
    L.sfx_batch_autotune.restype = C.c_int
    L.sfx_batch_autotune.argtypes = [vp, vp, vp, vp, vp, vp, dp, vp, ip]
    L.sfx_batch_work.restype = C.c_int
    L.sfx_batch_work.argtypes = [vp, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong), C.c_int,
                                 vp]
    L.sfx_f_from_gamma.restype = C.c_int
    L.sfx_f_from_gamma.argtypes = [vp, vp, vp, dp, vp, vp]
    L.sfx_marangoni_loss.restype = C.c_int
    L.sfx_marangoni_loss.argtypes = [vp, C.POINTER(Params), vp, vp, vp, C.c_int,
                                     C.POINTER(C.c_double), vp, vp]
    L.sfx_adjoint_apply.restype = C.c_int
    L.sfx_adjoint_apply.argtypes = [vp, C.POINTER(Params), vp, vp, vp, dp, C.c_int, vp, vp, vp,
                                    vp, vp]
    L.sfx_adjoint_step.restype = C.c_int
    L.sfx_adjoint_step.argtypes = [vp, C.POINTER(Params), vp, vp, vp, dp, vp, vp,
                                   C.POINTER(C.c_double), C.POINTER(SolveOpts),
                                   C.POINTER(StepStats), vp]
    L.sfx_acdi_step.restype = C.c_int
    L.sfx_acdi_step.argtypes = [vp, vp, vp, vp, dp, dp, dp, C.c_int, vp, vp]
    L.sfx_capillary_force.restype = C.c_int
    L.sfx_capillary_force.argtypes = [vp, C.POINTER(Params), vp, vp, vp, vp, vp, vp]
    L.sfx_vof_advect.restype = C.c_int
    L.sfx_vof_advect.argtypes = [vp, vp, vp, vp, dp, C.c_int, vp, vp]
    L.sfx_batch_reuse_phi.restype = C.c_int
    L.sfx_batch_reuse_phi.argtypes = [vp, C.c_int]
    _lib = L
    return L
