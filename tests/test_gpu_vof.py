"""GPU geometric VoF advection (sfx_vof_advect) against the oracle's split
PLIC scheme, conservation on the device, and the moving-interface
pipeline of the single-vortex workload (VoF step, phase-field rebuild,
coupled surfactant step) against the same pipeline in the oracle."""
import numpy as np
import pytest

import oracle
import workloads as W
from gpu_util import dev, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sfx():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2605_27534_gb300 as m
    m.lib()
    return m


def _rotation_3d(n, h, omega=2.0):
    ux, uy = W.solid_rotation_faces(n, h, (0.5, 0.5), omega)
    ux3 = np.repeat(ux, n, axis=0)
    uy3 = np.repeat(uy, n, axis=0)
    for u in (ux3,):
        u[..., 0] = u[..., -1] = 0.0
    uy3[:, 0, :] = uy3[:, -1, :] = 0.0
    return ux3, uy3, np.zeros((n + 1, n, n))


@pytest.mark.parametrize("precision", [0, 1])
def test_vof_matches_oracle_in_the_single_vortex(sfx, precision):
    import torch
    n = 64
    h = 1.0 / n
    g = W.Grid(W.PLANAR, n, n, 1, h)
    Cf = W.circle_vof(n, n, h, 0.5, 0.75, 0.15)
    T, steps = 2.0, 40
    dt = 0.4 * h
    ctx = sfx.Context.for_grid(g, precision)
    vt = torch.float32 if precision else torch.float64
    Cd = dev(Cf)
    Co = Cf.copy()
    for s in range(steps):
        ux, uy = W.single_vortex_faces(n, h, (s + 0.5) * dt, T)
        uxd, uyd = dev(ux, vt), dev(uy, vt)
        ctx.sfx_vof_advect(uxd, uyd, None, dt, Cd, s % 2)
        Co = oracle.vof_advect(g, host(uxd), host(uyd), None, dt, Co, s % 2)
    # SFX_F32 contexts evaluate the PLIC geometry in float: each flux carries
    # a few float roundings (~1e-7 of the Courant number), four fluxes per
    # cell and step over 40 steps stay below 1e-5; the update itself is
    # double and conservative
    tol = 1e-5 if precision else 1e-12
    assert np.abs(host(Cd) - Co).max() <= tol
    # sum C is kept up to the discrete divergence of the face velocities,
    # which rounding them to float (6e-8) makes non-zero
    assert abs(host(Cd).sum() - Cf.sum()) <= (1e-10 if precision else 1e-12) * Cf.sum()


def test_vof_matches_oracle_in_3d_and_conserves(sfx):
    n = 20
    h = 1.0 / n
    g = W.Grid(W.CART3D, n, n, n, h)
    Cf = W.sphere_vof(n, h, (0.5, 0.7, 0.5), 0.2)
    ux, uy, uz = _rotation_3d(n, h)
    dt = 0.2 * h
    ctx = sfx.Context.for_grid(g, 0)
    Cd = dev(Cf)
    Co = Cf.copy()
    u = [dev(ux), dev(uy), dev(uz)]
    for s in range(12):
        ctx.sfx_vof_advect(*u, dt, Cd, s % 2)
        Co = oracle.vof_advect(g, ux, uy, uz, dt, Co, s % 2)
    got = host(Cd)
    assert np.abs(got - Co).max() <= 1e-12
    assert abs(got.sum() - Cf.sum()) <= 1e-13 * Cf.sum()


def test_vof_rejects_axisymmetric_grids(sfx):
    g = W.Grid(W.AXI, 8, 8, 1, 0.1)
    ctx = sfx.Context.for_grid(g, 0)
    import torch
    C = torch.zeros(g.shape, dtype=torch.float64, device="cuda")
    ur = torch.zeros((1, 8, 9), dtype=torch.float64, device="cuda")
    uz = torch.zeros((1, 9, 8), dtype=torch.float64, device="cuda")
    with pytest.raises(sfx.SfxError):
        ctx.sfx_vof_advect(ur, uz, None, 1e-3, C)


@pytest.mark.parametrize("rebuild_every", [1, 3])
def test_moving_interface_pipeline_matches_oracle(sfx, rebuild_every):
    """Single vortex with a soluble surfactant at 48^2: each step advects C,
    rebuilds phi from it (or, between rebuilds every rebuild_every steps,
    carries phi by one ACDI step with zeta = 1.1 max|u|) and takes the
    coupled step with the same velocity, in the oracle and in an FP64
    context."""
    import torch
    n = 48
    c = W.case_vortex_2d(n=n, soluble=True)
    g, p = c.grid, c.params
    T = c.extra["T"]
    dt = c.dt
    _, phi0, delta0 = oracle.phase_field_build(g, c.C, c.redist_iters, c.dtau, p.eps)
    f0 = 0.5 * delta0
    Co, fo, Fo = c.C.copy(), f0.copy(), c.F0.copy()
    ctx = sfx.Context.for_grid(g, 0)
    Cd, fd, Fd = dev(c.C), dev(f0), dev(c.F0)
    chi = torch.empty_like(Cd)
    phid = torch.empty_like(Cd)
    opts = sfx.default_opts(tol=1e-13, max_cycles=200)
    for s in range(6):
        ux, uy = W.single_vortex_faces(n, g.h, (s + 0.5) * dt, T)
        Co = oracle.vof_advect(g, ux, uy, None, dt, Co, s % 2)
        rebuild = s % rebuild_every == 0
        zeta = 1.1 * max(np.abs(ux).max(), np.abs(uy).max())
        if rebuild:
            _, phio, _ = oracle.phase_field_build(g, Co, c.redist_iters, c.dtau, p.eps)
        else:
            phio = oracle.acdi_step(g, phio, dt, zeta, p.eps, ux, uy, None, clip=True)
        fo, Fo, st = oracle.surfactant_step(g, p, phio, fo, Fo, dt, 1e-14, ux, uy, None)
        assert st.converged
        uxd, uyd = dev(ux), dev(uy)
        ctx.sfx_vof_advect(uxd, uyd, None, dt, Cd, s % 2)
        if rebuild:
            ctx.sfx_phase_field_build(Cd, chi, phid, None, iters=c.redist_iters, dtau=c.dtau,
                                      eps=p.eps)
        else:
            ctx.sfx_acdi_step(phid, dt, zeta, p.eps, uxd, uyd, clip=True)
        stt = ctx.sfx_surfactant_step(p, phid, fd, Fd, dt, uxd, uyd, None, opts=opts)
        assert stt.converged
    assert np.abs(host(Cd) - Co).max() <= 1e-12
    scale = max(np.abs(Fo).max(), np.abs(fo).max())
    assert np.abs(host(Fd) - Fo).max() <= 1e-12 * scale
    assert np.abs(host(fd) - fo).max() <= 1e-12 * scale


def test_fp32_moving_interface_pipeline_matches_oracle(sfx):
    """The FP32 form of the single-vortex pipeline at 128^2: VoF fluxes with
    FP32 PLIC geometry, the fused FP32 redistancing (eight Jacobi steps per
    launch) and the FP32 Newton step, four steps, against the FP64 oracle's
    pipeline (1e-5)."""
    import torch
    n = 128
    c = W.case_vortex_2d(n=n, soluble=True)
    g, p = c.grid, c.params
    T, dt = c.extra["T"], c.dt
    _, phi0, delta0 = oracle.phase_field_build(g, c.C, c.redist_iters, c.dtau, p.eps)
    f0 = 0.5 * delta0
    Co, fo, Fo = c.C.copy(), f0.copy(), c.F0.copy()
    ctx = sfx.Context.for_grid(g, 1)
    ctx.sfx_set_tuning(sfx._lib.SFX_TUNE_F32_REDIST, 1)
    Cd = dev(c.C)
    fd, Fd = ctx.sfx_df_pack(dev(f0)), ctx.sfx_df_pack(dev(c.F0))
    chi, phid = torch.empty_like(Cd), torch.empty_like(Cd)
    opts = sfx.default_opts(tol=1e-10, max_cycles=400)
    for s in range(4):
        ux, uy = W.single_vortex_faces(n, g.h, (s + 0.5) * dt, T)
        uxd, uyd = dev(ux, torch.float32), dev(uy, torch.float32)
        ux, uy = host(uxd), host(uyd)        # the oracle takes the same rounded velocities
        Co = oracle.vof_advect(g, ux, uy, None, dt, Co, s % 2)
        _, phio, _ = oracle.phase_field_build(g, Co, c.redist_iters, c.dtau, p.eps)
        fo, Fo, st = oracle.surfactant_step(g, p, phio, fo, Fo, dt, 1e-13, ux, uy, None)
        assert st.converged
        ctx.sfx_vof_advect(uxd, uyd, None, dt, Cd, s % 2)
        ctx.sfx_phase_field_build(Cd, chi, phid, None, iters=c.redist_iters, dtau=c.dtau,
                                  eps=p.eps)
        assert ctx.sfx_surfactant_step(p, phid, fd, Fd, dt, uxd, uyd, None, opts=opts).converged
    assert np.abs(host(Cd) - Co).max() <= 1e-6
    scale = max(np.abs(Fo).max(), np.abs(fo).max())
    assert np.abs(host(ctx.sfx_df_unpack(Fd)) - Fo).max() <= 1e-5 * scale
    assert np.abs(host(ctx.sfx_df_unpack(fd)) - fo).max() <= 1e-5 * scale
