"""GPU (libsfx, C-ABI) against the FP64 CPU oracle on the same seeded
inputs.  FP64 contexts must agree to 1e-12 normwise relative
(||x_gpu - x_oracle||_inf / ||x_oracle||_inf) when both sides converge to
tol = 1e-13; FP32 contexts to 1e-5 with totals conserved to 1e-10."""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from gpu_util import dev, host, rel_err

pytestmark = pytest.mark.gpu

PARITY = 1e-12
TOL = 1e-13


@pytest.fixture(scope="module")
def sfx():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2605_27534_gb300 as m
    m.lib()
    return m


def _ctx(sfx, g, prec=0):
    return sfx.Context.for_grid(g, prec)


def _planar_circle(nx, ny, R=0.25):
    h = 1.0 / max(nx, ny)
    g = W.Grid(W.PLANAR, nx, ny, 1, h)
    return g, W.circle_vof(nx, ny, h, 0.5 * nx * h, 0.5 * ny * h, R * min(nx, ny) * h)


def _axi_sphere(nr, nz, R=0.2):
    h = 1.0 / nr
    g = W.Grid(W.AXI, nr, nz, 1, h)
    return g, W.ring_vof(nr, nz, h, 0.5 * nz * h, R)


def _sphere(nx, ny, nz, R=0.3):
    h = 1.0 / max(nx, ny, nz)
    g = W.Grid(W.CART3D, nx, ny, nz, h)
    assert nx == ny == nz or True
    Cf = np.zeros((nz, ny, nx))
    n = max(nx, ny, nz)
    full = W.sphere_vof(n, h, (0.5, 0.5, 0.5), R)
    Cf[:] = full[:nz, :ny, :nx]
    return g, Cf


GEOMS = {
    "planar": lambda: _planar_circle(70, 52),
    "axi": lambda: _axi_sphere(40, 80),
    "3d": lambda: _sphere(24, 20, 28, 0.3),
}


@pytest.mark.parametrize("geom", list(GEOMS))
def test_phase_field_build_parity(sfx, geom):
    import torch
    g, Cf = GEOMS[geom]()
    eps, dtau = 0.75 * g.h, (g.h / 3 if g.geom == W.CART3D else 0.5 * g.h)
    chi_o, phi_o, del_o = oracle.phase_field_build(g, Cf, 24, dtau, eps)
    ctx = _ctx(sfx, g)
    Cd = dev(Cf)
    chi = torch.empty_like(Cd)
    phi = torch.empty_like(Cd)
    dl = torch.empty_like(Cd)
    ctx.sfx_phase_field_build(Cd, chi, phi, dl, iters=24, dtau=dtau, eps=eps)
    assert rel_err(host(chi), chi_o) < PARITY
    assert rel_err(host(phi), phi_o) < PARITY
    assert rel_err(host(dl), del_o) < PARITY
    # SFX_F32 contexts redistance in FP64 by default (the same bits) ...
    ctx32 = _ctx(sfx, g, 1)
    phi32, chi32 = torch.empty_like(Cd), torch.empty_like(Cd)
    ctx32.sfx_phase_field_build(Cd, chi32, phi32, None, iters=24, dtau=dtau, eps=eps)
    assert np.array_equal(host(chi32), host(chi)) and np.array_equal(host(phi32), host(phi))
    # ... and in FP32 with SFX_TUNE_F32_REDIST
    ctx32.sfx_set_tuning(sfx._lib.SFX_TUNE_F32_REDIST, 1)
    ctx32.sfx_phase_field_build(Cd, chi32, phi32, None, iters=24, dtau=dtau, eps=eps)
    assert rel_err(host(chi32), chi_o) < 1e-6      # float iterate
    assert np.abs(host(phi32) - phi_o).max() < 5e-6


@pytest.mark.parametrize("geom", ["planar", "axi"])
@pytest.mark.parametrize("iters", [1, 8, 13, 17])
def test_fp32_redistancing_step_counts(sfx, geom, iters):
    """2D SFX_F32 contexts take up to eight redistancing steps per launch in
    shared memory; step counts below, at and between multiples of eight
    against the FP64 oracle."""
    import torch
    g, Cf = GEOMS[geom]()
    eps, dtau = 0.75 * g.h, 0.5 * g.h
    chi_o, phi_o, _ = oracle.phase_field_build(g, Cf, iters, dtau, eps)
    ctx32 = _ctx(sfx, g, 1)
    ctx32.sfx_set_tuning(sfx._lib.SFX_TUNE_F32_REDIST, 1)
    Cd = dev(Cf)
    phi32, chi32 = torch.empty_like(Cd), torch.empty_like(Cd)
    ctx32.sfx_phase_field_build(Cd, chi32, phi32, None, iters=iters, dtau=dtau, eps=eps)
    assert rel_err(host(chi32), chi_o) < 1e-6
    assert np.abs(host(phi32) - phi_o).max() < 5e-6


def _random_problem(g, seed, scale=2.0):
    rng = np.random.default_rng(seed)
    nz, ny, nx = g.shape
    Bx = np.zeros((nz, ny, nx + 1))
    By = np.zeros((nz, ny + 1, nx))
    Bz = np.zeros((nz + 1, ny, nx)) if g.ndim == 3 else None
    Bx[..., 1:-1] = rng.uniform(-scale, scale, Bx[..., 1:-1].shape)
    By[:, 1:-1, :] = rng.uniform(-scale, scale, By[:, 1:-1, :].shape)
    if Bz is not None:
        Bz[1:-1] = rng.uniform(-scale, scale, Bz[1:-1].shape)
    lam = rng.uniform(50.0, 100.0, g.shape)
    b = rng.uniform(-1.0, 1.0, g.shape)
    return Bx, By, Bz, lam, b


@pytest.mark.parametrize("shape,geom", [((1, 48, 64), W.PLANAR), ((1, 64, 32), W.AXI),
                                        ((24, 16, 16), W.CART3D), ((1, 29, 37), W.PLANAR),
                                        ((1, 1, 1), W.PLANAR), ((2, 2, 2), W.CART3D)])
def test_mg_solve_parity(sfx, shape, geom):
    import torch
    nz, ny, nx = shape
    g = W.Grid(geom, nx, ny, nz, 1.0 / max(shape))
    D = 0.05
    Bx, By, Bz, lam, b = _random_problem(g, 3)
    a_o, s, _ = oracle.elliptic_solve(g, D, Bx, By, Bz, lam, b, tol=1e-15)
    assert s > 0
    ctx = _ctx(sfx, g)
    a = torch.zeros(shape, dtype=torch.float64, device="cuda")
    opts = sfx.default_opts(tol=TOL, max_cycles=100)
    cyc, res, ok = ctx.sfx_mg_solve(D, dev(Bx), dev(By), None if Bz is None else dev(Bz),
                                    dev(lam), dev(b), a, opts)
    assert ok and res <= TOL
    assert rel_err(host(a), a_o) < PARITY


@pytest.mark.parametrize("case", ["vortex", "hr3d", "hraxi", "uniform3d"])
def test_advection_parity(sfx, case):
    import torch
    rng = np.random.default_rng(1)
    if case == "vortex":
        n = 48
        g = W.Grid(W.PLANAR, n, n, 1, 1.0 / n)
        ux, uy = W.single_vortex_faces(n, g.h, 0.3, 4.0)
        uz, dt = None, 0.4 * g.h
        xi = W.circle_vof(n, n, g.h, 0.5, 0.75, 0.15)
    elif case == "hr3d":
        n = 20
        g = W.Grid(W.CART3D, n, n, n, 1.0 / n)
        ux, uy, uz = W.hr_faces_3d(n, g.h, (0.5, 0.5, 0.5), 0.2)
        dt = 0.3 * g.h
        xi = rng.uniform(0, 1, g.shape)
    elif case == "hraxi":
        g = W.Grid(W.AXI, 24, 48, 1, 1.0 / 24)
        ux, uy = W.hr_faces_axi(24, 48, g.h, 1.0, 0.2)
        uz, dt = None, 0.3 * g.h
        xi = rng.uniform(0, 1, g.shape)
    else:
        g = W.Grid(W.CART3D, 12, 10, 14, 0.1)
        ux, uy, uz = W.uniform_faces(g, (0.3, -0.2, 0.45))
        dt = 0.1
        xi = rng.uniform(0, 1, g.shape)
    ref = oracle.advect_bcg(g, ux, uy, uz, dt, xi, 0.4)
    ctx = _ctx(sfx, g)
    out = torch.empty(g.shape, dtype=torch.float64, device="cuda")
    ctx.sfx_advect(dev(ux), dev(uy), None if uz is None else dev(uz), dt, dev(xi), 0.4, out)
    assert rel_err(host(out), ref) < 1e-14


def _step_case(name):
    if name == "adsorption2d":
        c = W.case_adsorption_2d(n=48, steps=5, tol=TOL)
        return c, None, None, None
    if name == "vortex2d":
        c = W.case_vortex_2d(n=48, soluble=True)
        c.steps = 3
        return c, c.ux, c.uy, None
    if name == "hr3d":
        c = W.case_hr_3d(n=24, steps=2)
        return c, c.ux, c.uy, c.uz
    if name == "axi":
        c = W.case_axi(32, 64, Bi=1.0, Da=10.0, steps=3)
        return c, c.ux, c.uy, None
    raise KeyError(name)


@pytest.mark.parametrize("name", ["adsorption2d", "vortex2d", "hr3d", "axi"])
def test_surfactant_step_parity_fp64(sfx, name):
    import torch
    c, ux, uy, uz = _step_case(name)
    g, p = c.grid, c.params
    _, phi, delta = oracle.phase_field_build(g, c.C, c.redist_iters, c.dtau, p.eps)
    f0 = c.gamma0 * delta if c.gamma0 is not None else np.zeros(g.shape)
    f_o, F_o = f0.copy(), c.F0.copy()
    for _ in range(c.steps):
        f_o, F_o, st = oracle.surfactant_step(g, p, phi, f_o, F_o, c.dt, TOL / 10, ux, uy, uz)
        assert st.converged
    ctx = _ctx(sfx, g)
    f, F = dev(f0), dev(c.F0)
    phid = dev(phi)
    u = [None if v is None else dev(v) for v in (ux, uy, uz)]
    opts = sfx.default_opts(tol=TOL, max_cycles=200)
    M0 = sum(ctx.sfx_totals([f, F]))
    for _ in range(c.steps):
        stt = ctx.sfx_surfactant_step(p, phid, f, F, c.dt, *u, opts=opts)
        assert stt.converged and stt.res_f <= TOL and stt.res_F <= TOL
    scale = max(np.abs(F_o).max(), np.abs(f_o).max())
    assert np.abs(host(F) - F_o).max() / scale < PARITY
    assert np.abs(host(f) - f_o).max() / scale < PARITY
    if ux is None:   # closed box: total surfactant is invariant
        M1 = stt.mass_f + stt.mass_F
        assert abs(M1 - M0) < 1e-12 * abs(M0)


F32_TOL = 1e-5       # FP32 contexts against the FP64 oracle (normwise)
MASS_DRIFT = 1e-10   # relative drift of sum V (f + F) in a closed box


def _pairs(ctx, arr):
    return ctx.sfx_df_pack(dev(arr))


@pytest.mark.parametrize("name", ["adsorption2d", "vortex2d", "hr3d", "axi"])
def test_surfactant_step_parity_fp32(sfx, name):
    """SFX_F32 context: float carrier and velocities, double-float state,
    FP32 arithmetic; within 1e-5 of the FP64 oracle."""
    import torch
    c, ux, uy, uz = _step_case(name)
    g, p = c.grid, c.params
    _, phi, delta = oracle.phase_field_build(g, c.C, c.redist_iters, c.dtau, p.eps)
    f0 = c.gamma0 * delta if c.gamma0 is not None else np.zeros(g.shape)
    f_o, F_o = f0.copy(), c.F0.copy()
    for _ in range(c.steps):
        f_o, F_o, st = oracle.surfactant_step(g, p, phi, f_o, F_o, c.dt, 1e-13, ux, uy, uz)
    ctx = _ctx(sfx, g, 1)
    f, F = _pairs(ctx, f0), _pairs(ctx, c.F0)
    phid = dev(phi)
    u = [None if v is None else dev(v, torch.float32) for v in (ux, uy, uz)]
    opts = sfx.default_opts(tol=1e-10, max_cycles=400)
    M0 = sum(ctx.sfx_totals([f, F]))
    for _ in range(c.steps):
        stt = ctx.sfx_surfactant_step(p, phid, f, F, c.dt, *u, opts=opts)
        assert stt.converged
    scale = max(np.abs(F_o).max(), np.abs(f_o).max())
    fh, Fh = host(ctx.sfx_df_unpack(f)), host(ctx.sfx_df_unpack(F))
    assert np.abs(Fh - F_o).max() / scale < F32_TOL
    assert np.abs(fh - f_o).max() / scale < F32_TOL
    if ux is None or name == "vortex2d":   # no flow through the walls
        assert abs(stt.mass_f + stt.mass_F - M0) < MASS_DRIFT * abs(M0)


@pytest.mark.parametrize("Bi", [0.1, 1.0, 10.0])
@pytest.mark.parametrize("Da", [0.1, 1.0, 10.0])
def test_hr3d_kinetics_grid_fp32(sfx, Bi, Da):
    """The 3D HR configuration over (Bi, Da) in {0.1, 1, 10}^2 (the bench
    times (1, 1)): two SFX_F32 steps at 24^3 against the FP64 oracle."""
    import torch
    c = W.case_hr_3d(n=24, Bi=Bi, Da=Da, steps=2)
    g, p = c.grid, c.params
    _, phi, _ = oracle.phase_field_build(g, c.C, c.redist_iters, c.dtau, p.eps)
    f_o, F_o = np.zeros(g.shape), c.F0.copy()
    for _ in range(2):
        f_o, F_o, st = oracle.surfactant_step(g, p, phi, f_o, F_o, c.dt, 1e-13, c.ux, c.uy, c.uz)
        assert st.converged
    ctx = _ctx(sfx, g, 1)
    f, F = _pairs(ctx, np.zeros(g.shape)), _pairs(ctx, c.F0)
    u = [dev(v, torch.float32) for v in (c.ux, c.uy, c.uz)]
    opts = sfx.default_opts(tol=1e-10, max_cycles=400)
    for _ in range(2):
        assert ctx.sfx_surfactant_step(p, dev(phi), f, F, c.dt, *u, opts=opts).converged
    scale = max(np.abs(F_o).max(), np.abs(f_o).max())
    assert np.abs(host(ctx.sfx_df_unpack(F)) - F_o).max() / scale < F32_TOL
    assert np.abs(host(ctx.sfx_df_unpack(f)) - f_o).max() / scale < F32_TOL


@pytest.mark.parametrize("name", ["adsorption2d", "hr3d", "axi"])
def test_fused_sweep_equals_colour_launches_bitwise(sfx, name):
    import torch
    c, ux, uy, uz = _step_case(name)
    g, p = c.grid, c.params
    _, phi, delta = oracle.phase_field_build(g, c.C, c.redist_iters, c.dtau, p.eps)
    outs = []
    for fused in (1, 0):
        ctx = _ctx(sfx, g, 1)
        ctx.sfx_set_tuning(sfx._lib.SFX_TUNE_F32_SOLVER, 0)
        ctx.sfx_set_tuning(sfx._lib.SFX_TUNE_FUSED_SWEEP, fused)
        f, F = _pairs(ctx, 0.2 * delta), _pairs(ctx, c.F0)
        u = [None if v is None else dev(v, torch.float32) for v in (ux, uy, uz)]
        o = sfx.default_opts(tol=1e-10, nu1=1, nu2=0)
        for _ in range(2):
            ctx.sfx_surfactant_step(p, dev(phi), f, F, c.dt, *u, opts=o)
        torch.cuda.synchronize()
        outs.append((f.cpu().numpy().copy(), F.cpu().numpy().copy()))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])


@pytest.mark.parametrize("name", ["adsorption2d", "hr3d", "axi"])
def test_fp32_solvers_agree(sfx, name):
    """Defect correction and nonlinear pair sweeps reach the same fixed point."""
    import torch
    c, ux, uy, uz = _step_case(name)
    g, p = c.grid, c.params
    _, phi, delta = oracle.phase_field_build(g, c.C, c.redist_iters, c.dtau, p.eps)
    outs = []
    for solver in (0, 1):
        ctx = _ctx(sfx, g, 1)
        ctx.sfx_set_tuning(sfx._lib.SFX_TUNE_F32_SOLVER, solver)
        f, F = _pairs(ctx, 0.2 * delta), _pairs(ctx, c.F0)
        u = [None if v is None else dev(v, torch.float32) for v in (ux, uy, uz)]
        o = sfx.default_opts(tol=1e-12, nu1=1, nu2=0, max_cycles=400)
        for _ in range(2):
            st = ctx.sfx_surfactant_step(p, dev(phi), f, F, c.dt, *u, opts=o)
            assert st.converged
        outs.append((host(ctx.sfx_df_unpack(f)), host(ctx.sfx_df_unpack(F))))
    scale = max(np.abs(outs[0][0]).max(), np.abs(outs[0][1]).max())
    assert np.abs(outs[0][0] - outs[1][0]).max() < 1e-10 * scale
    assert np.abs(outs[0][1] - outs[1][1]).max() < 1e-10 * scale


def test_fp32_predictor_keeps_the_fixed_point_and_saves_iterations(sfx):
    """Starting each Newton iteration from x* plus the last step's increment
    reaches the same solution (within the tolerance) in fewer iterations."""
    import torch
    c = W.case_axi(32, 64, Bi=1.0, Da=10.0)
    ux, uy, uz = c.ux, c.uy, None
    g, p = c.grid, c.params
    _, phi, _ = oracle.phase_field_build(g, c.C, c.redist_iters, c.dtau, p.eps)
    out, its = [], []
    for predict in (0, 1):
        ctx = _ctx(sfx, g, 1)
        ctx.sfx_set_tuning(sfx._lib.SFX_TUNE_PREDICT, predict)
        f, F = _pairs(ctx, np.zeros(g.shape)), _pairs(ctx, c.F0)
        u = [None if v is None else dev(v, torch.float32) for v in (ux, uy, uz)]
        phid = dev(phi)
        o = sfx.default_opts(tol=1e-11, max_cycles=400, nu1=3, nu2=0)
        n_it = 0
        for _ in range(12):
            st = ctx.sfx_surfactant_step(p, phid, f, F, c.dt, *u, opts=o)
            assert st.converged and st.res_f <= 1e-11 and st.res_F <= 1e-11
            n_it += st.picard
        its.append(n_it)
        out.append((host(ctx.sfx_df_unpack(f)), host(ctx.sfx_df_unpack(F))))
    scale = np.abs(out[0][1]).max()
    assert np.abs(out[0][0] - out[1][0]).max() < 1e-8 * scale
    assert np.abs(out[0][1] - out[1][1]).max() < 1e-8 * scale
    assert its[1] < its[0], its


def test_fp32_mass_drift_over_many_steps(sfx):
    """Closed box, 100 steps of the 2D adsorption physics at tol 1e-10:
    the double-float state keeps sum V (f + F) to 1e-10."""
    import torch
    c = W.case_adsorption_2d(n=64, steps=100)
    g, p = c.grid, c.params
    ctx = _ctx(sfx, g, 1)
    Cd = dev(c.C)
    chi = torch.empty_like(Cd)
    phi = torch.empty_like(Cd)
    ctx.sfx_phase_field_build(Cd, chi, phi, None, iters=c.redist_iters, dtau=c.dtau, eps=p.eps)
    f, F = _pairs(ctx, np.zeros(g.shape)), _pairs(ctx, c.F0)
    M0 = sum(ctx.sfx_totals([f, F]))
    opts = sfx.default_opts(tol=1e-10, max_cycles=400)
    for _ in range(c.steps):
        st = ctx.sfx_surfactant_step(p, phi, f, F, c.dt, opts=opts)
        assert st.converged
    M = st.mass_f + st.mass_F
    assert abs(M - M0) < MASS_DRIFT * M0
    assert st.mass_f > 0.01 * M0   # surfactant did adsorb


def test_fp32_advection_and_totals(sfx):
    import torch
    n = 40
    g = W.Grid(W.PLANAR, n, n, 1, 1.0 / n)
    ux, uy = W.single_vortex_faces(n, g.h, 0.3, 4.0)
    xi = W.circle_vof(n, n, g.h, 0.5, 0.75, 0.15) + 0.25
    ref = oracle.advect_bcg(g, ux, uy, None, 0.4 * g.h, xi, 0.25)
    ctx = _ctx(sfx, g, 1)
    x = _pairs(ctx, xi)
    out = torch.empty_like(x)
    ctx.sfx_advect(dev(ux, torch.float32), dev(uy, torch.float32), None, 0.4 * g.h, x, 0.25, out)
    assert rel_err(host(ctx.sfx_df_unpack(out)), ref) < 1e-6
    # totals of pairs against the exact sum (walls carry no flux: conserved)
    V = oracle.cell_volumes(g)
    got = ctx.sfx_totals([out])[0]
    assert abs(got - math.fsum((V * xi).ravel())) < 1e-13 * (V * xi).sum()
    # axisymmetric flow with walls: advection alone conserves the totals
    ga = W.Grid(W.AXI, 24, 48, 1, 1.0 / 24)
    ur, uz_ = W.hr_faces_axi(24, 48, ga.h, 1.0, 0.2)
    ur[..., -1] = 0.0
    uz_[:, 0, :] = 0.0
    uz_[:, -1, :] = 0.0
    xa = np.random.default_rng(2).uniform(0.5, 1.0, ga.shape)
    cta = _ctx(sfx, ga, 1)
    xp = _pairs(cta, xa)
    oa = torch.empty_like(xp)
    cta.sfx_advect(dev(ur, torch.float32), dev(uz_, torch.float32), None, 0.2 * ga.h, xp, 0.0, oa)
    Va = oracle.cell_volumes(ga)
    assert abs(cta.sfx_totals([oa])[0] - math.fsum((Va * xa).ravel())) < 1e-13 * (Va * xa).sum()


@pytest.mark.parametrize("geom", list(GEOMS))
def test_marangoni_fp32(sfx, geom):
    import torch
    g, Cf = GEOMS[geom]()
    p = W.Params(eps=0.75 * g.h, sigma0=1.0, E=0.3, gamma_inf=1.0)
    _, phi, delta = oracle.phase_field_build(g, Cf, 24, 0.5 * g.h, p.eps)
    rng = np.random.default_rng(4)
    f = rng.uniform(0.1, 0.9, g.shape) * delta
    ctx = _ctx(sfx, g, 1)
    for eos in (W.EOS_LANGMUIR, W.EOS_LINEAR, W.EOS_TANH):
        p.eos = eos
        sig_o, force_o = oracle.marangoni(g, p, f, phi, Cf, 1)
        sig = torch.empty(g.shape, dtype=torch.float32, device="cuda")
        force = torch.empty((g.ndim,) + g.shape, dtype=torch.float32, device="cuda")
        ctx.sfx_marangoni_force(p, _pairs(ctx, f), dev(phi),
                                dev(Cf, torch.float32), sig, force, 1)
        assert rel_err(host(sig), sig_o) < 1e-6
        assert rel_err(host(force), force_o) < 1e-5


def test_totals_match_exact_sum(sfx):
    rng = np.random.default_rng(8)
    g = W.Grid(W.AXI, 333, 77, 1, 0.003)
    x = rng.standard_normal(g.shape) * 10.0 ** rng.uniform(-6, 6, g.shape)
    y = rng.uniform(0, 1, g.shape)
    ctx = _ctx(sfx, g)
    got = ctx.sfx_totals([dev(x), dev(y)])
    V = oracle.cell_volumes(g)
    for val, arr in zip(got, (x, y)):
        exact = math.fsum((V * arr).ravel())
        assert abs(val - exact) <= 4e-16 * np.abs(V * arr).sum()
    # deterministic: same bits on a second call
    assert ctx.sfx_totals([dev(x), dev(y)]) == got


@pytest.mark.parametrize("geom", list(GEOMS))
@pytest.mark.parametrize("dm_mode", [0, 1])
def test_marangoni_parity(sfx, geom, dm_mode):
    import torch
    g, Cf = GEOMS[geom]()
    p = W.Params(eps=0.75 * g.h, sigma0=1.0, E=0.3, gamma_inf=1.0)
    _, phi, delta = oracle.phase_field_build(g, Cf, 24, 0.5 * g.h, p.eps)
    rng = np.random.default_rng(4)
    Gam = rng.uniform(0.1, 0.9, g.shape)
    f = Gam * delta
    ctx = _ctx(sfx, g)
    for eos in (W.EOS_LANGMUIR, W.EOS_LINEAR, W.EOS_TANH):
        p.eos = eos
        sig_o, force_o = oracle.marangoni(g, p, f, phi, Cf, dm_mode)
        sig = torch.empty(g.shape, dtype=torch.float64, device="cuda")
        force = torch.empty((g.ndim,) + g.shape, dtype=torch.float64, device="cuda")
        ctx.sfx_marangoni_force(p, dev(f), dev(phi), dev(Cf), sig, force, dm_mode)
        assert rel_err(host(sig), sig_o) < PARITY
        assert rel_err(host(force), force_o) < 1e-11


def test_cfl_dt_matches_oracle(sfx):
    c = W.case_hr_3d(n=16, steps=1)
    ctx = _ctx(sfx, c.grid)
    dt = ctx.sfx_cfl_dt(dev(c.ux), dev(c.uy), dev(c.uz), 0.025, c.params.eps, 0.5)
    umax = max(np.abs(c.ux).max(), np.abs(c.uy).max(), np.abs(c.uz).max())
    assert dt == pytest.approx(oracle.cfl_dt(3, c.grid.h, umax, 0.025, c.params.eps, 0.5),
                               rel=1e-15)


# ----------------------------------------------------------------- edges
def test_flat_interface_axisymmetric_and_3d_steps_reduce_to_the_planar_column(sfx):
    """A flat interface normal to y, its phase field built and stepped by
    the FP64 GPU path on planar, axisymmetric and 3D blocks: every ring and
    every 3D column reproduce the oracle's planar column (whose own
    axisymmetric and 3D runs reduce to it to round-off)."""
    import torch
    ny, half, dt, steps = 48, 1.0, 2e-3, 6
    h = 2 * half / ny
    y = -half + (np.arange(ny) + 0.5) * h
    p = W.Params(ka=2.0, kd=0.5, gamma_inf=1.0, Df=0.3, DF=1.0, eps=2 * h)
    ref = None
    for geom, nx, nz in ((W.PLANAR, 2, 1), (W.AXI, 4, 1), (W.CART3D, 2, 2)):
        g = W.Grid(geom, nx, ny, nz, h)
        Cf = np.zeros(g.shape)
        Cf[:, y < 0, :] = 1.0
        dtau = h / 3 if geom == W.CART3D else 0.5 * h
        if ref is None:
            _, phi_o, del_o = oracle.phase_field_build(g, Cf, 200, dtau, p.eps)
            f_o, F_o = 0.2 * del_o, phi_o.copy()
            for _ in range(steps):
                f_o, F_o, st = oracle.surfactant_step(g, p, phi_o, f_o, F_o, dt, TOL / 10)
                assert st.converged
            ref = [a[0, :, 0] for a in (phi_o, f_o, F_o)]
        ctx = _ctx(sfx, g)
        Cd = dev(Cf)
        chi, phi, dl = torch.empty_like(Cd), torch.empty_like(Cd), torch.empty_like(Cd)
        ctx.sfx_phase_field_build(Cd, chi, phi, dl, iters=200, dtau=dtau, eps=p.eps)
        f, F = 0.2 * dl, phi.clone()
        opts = sfx.default_opts(tol=TOL, max_cycles=200)
        for _ in range(steps):
            assert ctx.sfx_surfactant_step(p, phi, f, F, dt, opts=opts).converged
        for a, r in zip((host(phi), host(f), host(F)), ref):
            err = np.abs(a - r[None, :, None]).max() / np.abs(r).max()
            assert err < PARITY, (geom, err)


def test_degenerate_single_cell_reduces_to_kinetics(sfx):
    """One cell: no faces, so App. C reduces to the pointwise kinetic system."""
    g = W.Grid(W.PLANAR, 1, 1, 1, 0.1)
    p = W.Params(ka=2.0, kd=0.5, gamma_inf=1.0, Df=0.1, DF=0.1, eps=0.075)
    phi = np.full(g.shape, 0.4)
    f0, F0 = np.full(g.shape, 0.3), np.full(g.shape, 0.8)
    f_o, F_o, _ = oracle.surfactant_step(g, p, phi, f0, F0, 0.01, 1e-15)
    ctx = _ctx(sfx, g)
    f, F = dev(f0), dev(F0)
    ctx.sfx_surfactant_step(p, dev(phi), f, F, 0.01, opts=sfx.default_opts(tol=1e-14))
    assert rel_err(host(f), f_o) < 1e-13 and rel_err(host(F), F_o) < 1e-13


def test_nonfinite_input_is_reported(sfx):
    c, *_ = _step_case("adsorption2d")
    g, p = c.grid, c.params
    _, phi, _ = oracle.phase_field_build(g, c.C, 12, c.dtau, p.eps)
    F0 = c.F0.copy()
    F0[0, 10, 10] = np.nan
    ctx = _ctx(sfx, g)
    with pytest.raises(sfx.SfxError, match="non-finite"):
        ctx.sfx_surfactant_step(p, dev(phi), dev(np.zeros(g.shape)), dev(F0), c.dt)


def test_not_converged_is_reported_with_stats(sfx):
    c, *_ = _step_case("adsorption2d")
    g, p = c.grid, c.params
    _, phi, _ = oracle.phase_field_build(g, c.C, 12, c.dtau, p.eps)
    ctx = _ctx(sfx, g)
    st = ctx.sfx_surfactant_step(p, dev(phi), dev(np.zeros(g.shape)), dev(c.F0), c.dt,
                                 opts=sfx.default_opts(tol=1e-15, max_cycles=1),
                                 allow_not_converged=True)
    assert st.converged == 0 and st.picard == 1 and st.res_f > 1e-15


def test_invalid_arguments_rejected(sfx):
    import torch
    g = W.Grid(W.PLANAR, 8, 8, 1, 0.1)
    ctx = _ctx(sfx, g)
    f = torch.zeros(g.shape, dtype=torch.float64, device="cuda")
    p = W.Params(eps=0.075)
    with pytest.raises(sfx.SfxError, match="invalid argument"):
        ctx.sfx_surfactant_step(p, f, f, f, 0.1)          # f aliases F
    with pytest.raises(sfx.SfxError, match="invalid argument"):
        ctx.sfx_surfactant_step(p, f, f.clone(), f.clone(), -1.0)
    bad = W.Params(eps=0.0)
    with pytest.raises(sfx.SfxError, match="invalid argument"):
        ctx.sfx_surfactant_step(bad, f, f.clone(), f.clone(), 0.1)
    with pytest.raises(sfx.SfxError, match="invalid argument"):
        sfx.Context(W.PLANAR, 8, 8, 2, 0.1)               # nz > 1 in 2D


def _wide_case(name):
    """Grids whose colour rows fill one 128-thread block of the FP32 Newton
    kernels and spill into more with a ragged tail: planar 520 x 40 (260
    cells per colour row: 128 + 128 + 4) and 3D 258 x 20 x 16 (129: 128 + 1),
    a circle (an extruded cylinder in 3D) in solid-body rotation (plus a
    uniform axial velocity in 3D), soluble surfactant."""
    nx, ny, nz = (520, 40, 1) if name == "planar520" else (258, 20, 16)
    h = 1.0 / 64
    xc, yc, R = 0.5 * nx * h, 0.5 * ny * h, 0.2
    C2 = W.circle_vof(nx, ny, h, xc, yc, R)
    ux, uy = W.solid_rotation_faces((nx, ny), h, (xc, yc), 2.0)
    if nz == 1:
        g = W.Grid(W.PLANAR, nx, ny, 1, h)
        Cf, uz = C2, None
    else:
        g = W.Grid(W.CART3D, nx, ny, nz, h)
        Cf = np.repeat(C2, nz, axis=0)
        ux, uy = np.repeat(ux, nz, axis=0), np.repeat(uy, nz, axis=0)
        uz = np.full((nz + 1, ny, nx), 0.3)
    p = W.Params(ka=2.0, kd=0.5, gamma_inf=1.0, Df=2e-3, DF=5e-3, eps=0.75 * h, bc_F=1.0,
                 bc_f=0.0)
    return g, Cf, p, ux, uy, uz, 0.25 * h


@pytest.mark.parametrize("name", ["planar520", "cyl258"])
def test_fp32_step_on_rows_wider_than_one_block(sfx, name):
    """SFX_F32 steps on full and multi-block colour rows with a ragged tail
    against the FP64 oracle (three steps, 1e-5)."""
    import torch
    g, Cf, p, ux, uy, uz, dt = _wide_case(name)
    redist = W.redist_dtau(g)
    _, phi, delta = oracle.phase_field_build(g, Cf, 24, redist, p.eps)
    f0, F0 = 0.3 * delta, 1.0 - Cf
    f_o, F_o = f0.copy(), F0.copy()
    for _ in range(3):
        f_o, F_o, st = oracle.surfactant_step(g, p, phi, f_o, F_o, dt, 1e-13, ux, uy, uz)
        assert st.converged
    ctx = _ctx(sfx, g, 1)
    f, F = _pairs(ctx, f0), _pairs(ctx, F0)
    u = [None if v is None else dev(v, torch.float32) for v in (ux, uy, uz)]
    opts = sfx.default_opts(tol=1e-10, max_cycles=400)
    for _ in range(3):
        assert ctx.sfx_surfactant_step(p, dev(phi), f, F, dt, *u, opts=opts).converged
    scale = max(np.abs(F_o).max(), np.abs(f_o).max())
    assert np.abs(host(ctx.sfx_df_unpack(F)) - F_o).max() / scale < F32_TOL
    assert np.abs(host(ctx.sfx_df_unpack(f)) - f_o).max() / scale < F32_TOL


@pytest.mark.parametrize("redist32", [0, 1])
def test_fp32_phase_field_build_and_step_against_oracle(sfx, redist32):
    """The FP32 form end to end on the 3D HR workload at 40^3: the phase
    field from the SFX_F32 context's own build (FP64 redistancing, or FP32
    with SFX_TUNE_F32_REDIST), then two FP32 steps, against the oracle's
    FP64 build and steps."""
    import torch
    c = W.case_hr_3d(n=40, steps=2)
    g, p = c.grid, c.params
    _, phi_o, _ = oracle.phase_field_build(g, c.C, c.redist_iters, c.dtau, p.eps)
    f_o, F_o = np.zeros(g.shape), c.F0.copy()
    for _ in range(2):
        f_o, F_o, st = oracle.surfactant_step(g, p, phi_o, f_o, F_o, c.dt, 1e-13, c.ux, c.uy,
                                              c.uz)
        assert st.converged
    ctx = _ctx(sfx, g, 1)
    ctx.sfx_set_tuning(sfx._lib.SFX_TUNE_F32_REDIST, redist32)
    Cd = dev(c.C)
    chi, phi = torch.empty_like(Cd), torch.empty_like(Cd)
    ctx.sfx_phase_field_build(Cd, chi, phi, None, iters=c.redist_iters, dtau=c.dtau, eps=p.eps)
    f, F = _pairs(ctx, np.zeros(g.shape)), _pairs(ctx, c.F0)
    u = [dev(v, torch.float32) for v in (c.ux, c.uy, c.uz)]
    opts = sfx.default_opts(tol=1e-10, max_cycles=400)
    for _ in range(2):
        assert ctx.sfx_surfactant_step(p, phi, f, F, c.dt, *u, opts=opts).converged
    scale = max(np.abs(F_o).max(), np.abs(f_o).max())
    assert np.abs(host(ctx.sfx_df_unpack(F)) - F_o).max() / scale < F32_TOL
    assert np.abs(host(ctx.sfx_df_unpack(f)) - f_o).max() / scale < F32_TOL


def test_fp32_build_and_step_at_256_cubed_match_the_fp64_path(sfx):
    """The timed 256^3 workload: the SFX_F32 context's own phase-field build
    (FP64 redistancing, the default) and two FP32 steps against the FP64
    path, which the tests above hold to the oracle at 1e-12; the FP32 form
    within 1e-5.  (With SFX_TUNE_F32_REDIST the float redistancing moves
    the step by 5e-5 here: F = 1 fills the sphere, and at the front of the
    redistanced band the drift's direction follows chi's float rounding.)"""
    import torch
    c = W.case_hr_3d(n=256, steps=2)
    g, p = c.grid, c.params
    Cd = dev(c.C)
    out = []
    for prec in (0, 1):
        ctx = _ctx(sfx, g, prec)
        chi, phi = torch.empty_like(Cd), torch.empty_like(Cd)
        ctx.sfx_phase_field_build(Cd, chi, phi, None, iters=c.redist_iters, dtau=c.dtau,
                                  eps=p.eps)
        del chi
        vt = torch.float64 if prec == 0 else torch.float32
        u = [dev(v, vt) for v in (c.ux, c.uy, c.uz)]
        F0 = dev(c.F0)
        f, F = (torch.zeros_like(F0), F0) if prec == 0 else \
            (ctx.sfx_df_pack(torch.zeros_like(F0)), ctx.sfx_df_pack(F0))
        opts = sfx.default_opts(tol=1e-12 if prec == 0 else 1e-10, max_cycles=400)
        for _ in range(2):
            assert ctx.sfx_surfactant_step(p, phi, f, F, c.dt, *u, opts=opts).converged
        if prec == 1:
            f, F = ctx.sfx_df_unpack(f), ctx.sfx_df_unpack(F)
        out.append((host(f), host(F)))
        del ctx, u, phi
        torch.cuda.empty_cache()
    scale = max(np.abs(out[0][0]).max(), np.abs(out[0][1]).max())
    assert np.abs(out[1][0] - out[0][0]).max() / scale < F32_TOL
    assert np.abs(out[1][1] - out[0][1]).max() / scale < F32_TOL


def test_fp32_langmuir_sigma_near_saturation(sfx):
    """Gamma/Gamma_inf in [1 - 1e-6, 1 - 1e-9]: float spacing of the ratio
    (6e-8) would be a large relative error of 1 - Gamma/Gamma_inf, so the
    SFX_F32 EOS forms the Langmuir term in FP64 from the double phi and the
    whole pair of f; sigma against the oracle's."""
    import torch
    g, Cf = GEOMS["planar"]()
    p = W.Params(eps=0.75 * g.h, sigma0=1.0, E=0.2, gamma_inf=1.3, eos=W.EOS_LANGMUIR)
    _, phi, delta = oracle.phase_field_build(g, Cf, 24, 0.5 * g.h, p.eps)
    rng = np.random.default_rng(11)
    x = 1.0 - 10.0 ** rng.uniform(-9.0, -6.0, g.shape)
    f = x * p.gamma_inf * delta
    sig_o, _ = oracle.marangoni(g, p, f, phi, Cf, 1)
    band = delta >= 1e-3 / p.eps
    assert band.sum() > 100
    ctx = _ctx(sfx, g, 1)
    sig = torch.empty(g.shape, dtype=torch.float32, device="cuda")
    force = torch.empty((g.ndim,) + g.shape, dtype=torch.float32, device="cuda")
    ctx.sfx_marangoni_force(p, _pairs(ctx, f), dev(phi), dev(Cf, torch.float32), sig, force, 1)
    got = host(sig)
    assert np.abs(got[band] - sig_o[band]).max() < 1e-6 * np.abs(sig_o[band]).max()


@pytest.mark.parametrize("shape,geom", [((1, 64, 64), W.PLANAR), ((1, 96, 48), W.AXI),
                                        ((16, 16, 32), W.CART3D)])
def test_mg_solve_parity_when_diffusion_dominates(sfx, shape, geom):
    """The multigrid regime: D/(lambda h^2) of 25-50 (smooth error that
    relaxation alone barely damps; the oracle's Gauss-Seidel still reaches
    its round-off floor)."""
    import torch
    nz, ny, nx = shape
    g = W.Grid(geom, nx, ny, nz, 1.0 / max(shape))
    D = 0.05
    Bx, By, Bz, lam, b = _random_problem(g, 7, scale=0.5)
    lam = D / (g.h ** 2) * np.random.default_rng(8).uniform(0.02, 0.04, g.shape)
    assert D / (lam.max() * g.h ** 2) >= 25
    a_o, s, _ = oracle.elliptic_solve(g, D, Bx, By, Bz, lam, b, tol=1e-14, max_sweeps=400000)
    assert s > 0
    ctx = _ctx(sfx, g)
    a = torch.zeros(shape, dtype=torch.float64, device="cuda")
    opts = sfx.default_opts(tol=1e-14, max_cycles=200)
    cyc, res, ok = ctx.sfx_mg_solve(D, dev(Bx), dev(By), None if Bz is None else dev(Bz),
                                    dev(lam), dev(b), a, opts)
    assert ok and res <= 1e-14 and cyc <= 40, (cyc, res)
    assert rel_err(host(a), a_o) < PARITY


def _diffusive_case(geom):
    """A soluble-surfactant step whose implicit problem is diffusion
    dominated: D dt/h^2 = 20 (an interface of radius 0.3 in flow)."""
    if geom == W.PLANAR:
        g, Cf = _planar_circle(64, 64, R=0.3)
        ux, uy = W.solid_rotation_faces(64, g.h, (0.5, 0.5), 1.0)
        uz = None
    elif geom == W.AXI:
        g, Cf = _axi_sphere(48, 96, R=0.3)
        ux, uy = W.hr_faces_axi(48, 96, g.h, 0.5 * 96 * g.h, 0.3)
        uz = None
    else:
        g, Cf = _sphere(20, 20, 20, 0.3)
        ux, uy, uz = W.hr_faces_3d(20, g.h, (0.5, 0.5, 0.5), 0.3)
    dt = 2e-3
    D = 20.0 * g.h ** 2 / dt
    p = W.Params(ka=5.0, kd=1.0, gamma_inf=1.0, Df=D, DF=D, eps=0.75 * g.h)
    return g, Cf, p, ux, uy, uz, dt


@pytest.mark.parametrize("geom", [W.PLANAR, W.AXI, W.CART3D])
def test_fp32_multigrid_correction_when_diffusion_dominates(sfx, geom):
    """D dt/h^2 = 20: the FP32 Newton correction relaxed by red-black sweeps
    alone needs many iterations; with the FP32 V-cycle (chosen by default
    above D dt/h^2 = 1) the step converges in a bounded number and matches
    the FP64 oracle to 1e-5."""
    import torch
    g, Cf, p, ux, uy, uz, dt = _diffusive_case(geom)
    _, phi, delta = oracle.phase_field_build(g, Cf, 24, W.redist_dtau(g), p.eps)
    f0, F0 = 0.2 * delta, 1.0 - Cf
    f_o, F_o = f0.copy(), F0.copy()
    for _ in range(2):
        f_o, F_o, st = oracle.surfactant_step(g, p, phi, f_o, F_o, dt, 1e-13, ux, uy, uz)
        assert st.converged
    u = [None if v is None else dev(v, torch.float32) for v in (ux, uy, uz)]
    iters = {}
    for mg in (0, 1):
        ctx = _ctx(sfx, g, 1)
        ctx.sfx_set_tuning(sfx._lib.SFX_TUNE_PREDICT, 0)
        f, F = _pairs(ctx, f0), _pairs(ctx, F0)
        opts = sfx.default_opts(tol=1e-10, max_cycles=60, mg_levels=mg)
        its = []
        for _ in range(2):
            try:
                st = ctx.sfx_surfactant_step(p, dev(phi), f, F, dt, *u, opts=opts,
                                             allow_not_converged=(mg == 1))
                its.append(st.picard if st.converged else 10 ** 6)
            except sfx.SfxError:
                if mg == 0:
                    raise
                its.append(10 ** 6)     # relaxation alone diverged
                break
        iters[mg] = max(its)
        if mg == 0:
            scale = max(np.abs(F_o).max(), np.abs(f_o).max())
            assert np.abs(host(ctx.sfx_df_unpack(F)) - F_o).max() / scale < F32_TOL
            assert np.abs(host(ctx.sfx_df_unpack(f)) - f_o).max() / scale < F32_TOL
    assert iters[0] <= 20 and iters[0] * 2 < iters[1], iters


@pytest.mark.parametrize("shape", [(24, 24, 24), (23, 20, 26), (25, 21, 22)])
def test_sweep_planes_per_thread_bitwise(sfx, shape):
    """Two planes per thread in the 3D correction sweep (both cells' loads
    in flight before their arithmetic) give the same bits as one, on even
    and odd rows and an odd plane count."""
    import torch
    nz, ny, nx = shape
    g, Cf = _sphere(nx, ny, nz, 0.3)
    ux, uy, uz = W.uniform_faces(g, (0.3, -0.2, 0.25))
    p = W.Params(ka=2.0, kd=0.5, Df=2e-3, DF=5e-3, eps=0.75 * g.h)
    _, phi, delta = oracle.phase_field_build(g, Cf, 24, W.redist_dtau(g), p.eps)
    outs = []
    for planes in (1, 2):
        ctx = _ctx(sfx, g, 1)
        ctx.sfx_set_tuning(sfx._lib.SFX_TUNE_SWEEP_PLANES, planes)
        f, F = _pairs(ctx, 0.3 * delta), _pairs(ctx, 1.0 - Cf)
        u = [dev(v, torch.float32) for v in (ux, uy, uz)]
        for _ in range(2):
            assert ctx.sfx_surfactant_step(p, dev(phi), f, F, 0.2 * g.h, *u,
                                           opts=sfx.default_opts(tol=1e-10)).converged
        torch.cuda.synchronize()
        outs.append((f.cpu().numpy().copy(), F.cpu().numpy().copy()))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])


@pytest.mark.parametrize("shape,zchunk", [((37, 19, 136), 32), ((37, 19, 136), 4),
                                          ((9, 8, 64), 32), ((24, 24, 24), 5)])
def test_tiled_sweep_bitwise(sfx, shape, zchunk):
    """The tiled sweep (one launch per red-black sweep, z-planes staged in
    shared memory by tensor copies) gives the colour launches' bits: x tiles
    with a ragged last tile (136 = 2 x 64 + 8), rows and planes that do not
    fill the last tile or z-chunk, chunks of 4 and 5 planes (many chunk
    seams); it runs 4 instead of 7 sweep launches per Newton iteration.  The
    red updates are over-relaxed (the default) in both."""
    import torch
    nz, ny, nx = shape
    g, Cf = _sphere(nx, ny, nz, 0.3)
    ux, uy, uz = W.uniform_faces(g, (0.3, -0.2, 0.25))
    p = W.Params(ka=2.0, kd=0.5, Df=2e-3, DF=5e-3, eps=0.75 * g.h)
    _, phi, delta = oracle.phase_field_build(g, Cf, 24, W.redist_dtau(g), p.eps)
    outs, launches = [], []
    for tiled in (0, 1):
        ctx = _ctx(sfx, g, 1)
        ctx.sfx_set_tuning(sfx._lib.SFX_TUNE_TILED_SWEEP, tiled)
        ctx.sfx_set_tuning(sfx._lib.SFX_TUNE_TILED_ZCHUNK, zchunk)
        # (the colour-launch path evaluates no incremental residuals)
        ctx.sfx_set_tuning(sfx._lib.SFX_TUNE_F32_INCR_RESID, 0)
        f, F = _pairs(ctx, 0.3 * delta), _pairs(ctx, 1.0 - Cf)
        u = [dev(v, torch.float32) for v in (ux, uy, uz)]
        ctx.sfx_profile(True)
        for _ in range(3):
            assert ctx.sfx_surfactant_step(p, dev(phi), f, F, 0.2 * g.h, *u,
                                           opts=sfx.default_opts(tol=1e-10)).converged
        torch.cuda.synchronize()
        pr = ctx.sfx_profile_read()
        launches.append((pr["smooth_fine"][0], pr["smooth_tiled"][0]))
        ctx.sfx_profile(False)
        outs.append((f.cpu().numpy().copy(), F.cpu().numpy().copy()))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    (colour, none), (last_black, tiled) = launches
    assert none == 0 and tiled == 3 * last_black and (tiled + last_black) * 7 == colour * 4, \
        launches


@pytest.mark.parametrize("fast", [1, 2, 4])
def test_fp32_residual_iterations_reach_the_same_fixed_point(sfx, fast):
    """Newton iterations with FP32 residuals early in each solve (at most
    `fast` of them, until the relative residual falls below 1e-3) end on the
    pair residual's fixed point: the state matches the pair-only solve to
    far below the FP32 tolerance, each solve converges on a pair residual,
    and no solve needs more than one extra iteration."""
    import torch
    nz, ny, nx = 24, 20, 32
    g, Cf = _sphere(nx, ny, nz, 0.3)
    ux, uy, uz = W.uniform_faces(g, (0.3, -0.2, 0.25))
    p = W.Params(ka=2.0, kd=0.5, Df=2e-3, DF=5e-3, eps=0.75 * g.h)
    _, phi, delta = oracle.phase_field_build(g, Cf, 24, W.redist_dtau(g), p.eps)
    outs, its = [], []
    for mode in (0, fast):
        ctx = _ctx(sfx, g, 1)
        ctx.sfx_set_tuning(sfx._lib.SFX_TUNE_F32_FAST_RESID, mode)
        f, F = _pairs(ctx, 0.3 * delta), _pairs(ctx, 1.0 - Cf)
        u = [dev(v, torch.float32) for v in (ux, uy, uz)]
        n = []
        for _ in range(3):
            st = ctx.sfx_surfactant_step(p, dev(phi), f, F, 0.2 * g.h, *u,
                                         opts=sfx.default_opts(tol=1e-10))
            assert st.converged
            n.append(st.picard)
        its.append(n)
        outs.append((host(ctx.sfx_df_unpack(f)), host(ctx.sfx_df_unpack(F))))
    for a, b in zip(outs[0], outs[1]):
        assert np.abs(a - b).max() / np.abs(a).max() < 1e-8
    assert all(m <= k + 1 for k, m in zip(its[0], its[1])), its


@pytest.mark.parametrize("tiled", [0, 1])
def test_over_relaxed_sweeps_reach_the_same_fixed_point(sfx, tiled):
    """Red updates over-relaxed (omega from the Jacobi-radius bound, and a
    fixed omega_F = 1.15) end on the Gauss-Seidel solve's fixed point: the
    state matches to far below the FP32 tolerance and each solve converges,
    with no more iterations than Gauss-Seidel at one sweep fewer per
    iteration; colour launches (tiled = 0) and tiled sweeps alike."""
    import torch
    nz, ny, nx = 24, 20, 32
    g, Cf = _sphere(nx, ny, nz, 0.3)
    ux, uy, uz = W.uniform_faces(g, (0.3, -0.2, 0.25))
    p = W.Params(ka=2.0, kd=0.5, Df=2e-3, DF=5e-2, eps=0.75 * g.h)
    _, phi, delta = oracle.phase_field_build(g, Cf, 24, W.redist_dtau(g), p.eps)
    outs, its = [], []
    for sor, sweeps in ((0, 4), (1, 3), (1150, 3)):
        ctx = _ctx(sfx, g, 1)
        ctx.sfx_set_tuning(sfx._lib.SFX_TUNE_TILED_SWEEP, tiled)
        ctx.sfx_set_tuning(sfx._lib.SFX_TUNE_F32_SOR, sor)
        f, F = _pairs(ctx, 0.3 * delta), _pairs(ctx, 1.0 - Cf)
        u = [dev(v, torch.float32) for v in (ux, uy, uz)]
        o = sfx.default_opts(tol=1e-10, nu1=sweeps, nu2=0)
        n = []
        for _ in range(3):
            st = ctx.sfx_surfactant_step(p, dev(phi), f, F, 0.2 * g.h, *u, opts=o)
            assert st.converged
            n.append(st.picard)
        its.append(n)
        outs.append((host(ctx.sfx_df_unpack(f)), host(ctx.sfx_df_unpack(F))))
    for k in (1, 2):
        for a, b in zip(outs[0], outs[k]):
            assert np.abs(a - b).max() / np.abs(a).max() < 1e-8
        assert all(m <= q + 1 for q, m in zip(its[0], its[k])), its


@pytest.mark.parametrize("geom", ["planar", "axi"])
def test_over_relaxed_sweeps_reach_the_same_fixed_point_2d(sfx, geom):
    """The over-relaxed red updates on planar and axisymmetric grids (omega
    from the Jacobi-radius bound, D dt/h^2 ~ 0.5 for F): the same fixed
    point as Gauss-Seidel to far below the FP32 tolerance, every solve
    converged, and no more Newton iterations over three steps."""
    import torch
    if geom == "planar":
        g, Cf = _planar_circle(96, 80)
    else:
        g, Cf = _axi_sphere(48, 96)
    ux, uy = W.uniform_faces(g, (0.3, -0.2))[:2] if geom == "planar" else (None, None)
    p = W.Params(ka=2.0, kd=0.5, Df=2e-3, DF=5e-2, eps=0.75 * g.h)
    _, phi, delta = oracle.phase_field_build(g, Cf, 24, W.redist_dtau(g), p.eps)
    dt = 0.5 * g.h * g.h / p.DF
    outs, its = [], []
    for sor in (0, 1):
        ctx = _ctx(sfx, g, 1)
        ctx.sfx_set_tuning(sfx._lib.SFX_TUNE_F32_SOR, sor)
        f, F = _pairs(ctx, 0.3 * delta), _pairs(ctx, 1.0 - Cf)
        u = [dev(v, torch.float32) if v is not None else None for v in (ux, uy)] + [None]
        n = 0
        for _ in range(3):
            st = ctx.sfx_surfactant_step(p, dev(phi), f, F, dt, *u,
                                         opts=sfx.default_opts(tol=1e-10, mg_levels=1))
            assert st.converged
            n += st.picard
        its.append(n)
        outs.append((host(ctx.sfx_df_unpack(f)), host(ctx.sfx_df_unpack(F))))
    for a, b in zip(outs[0], outs[1]):
        assert np.abs(a - b).max() / np.abs(a).max() < 1e-8
    assert its[1] <= its[0], its


@pytest.mark.parametrize("shape", [(24, 24, 24), (19, 17, 70), (5, 9, 33)])
def test_staged_advection_bitwise(sfx, shape):
    """The 3D BCG step from shared-memory planes (values rounded once,
    neighbours past a wall clamped in the staging) gives the bits of the
    tiles that gather from global memory: ragged x tiles (70 = 2 x 31 + 8,
    33 = 31 + 2), rows and planes that do not fill a tile or z-chunk, and
    inflow values on the walls."""
    import torch
    nz, ny, nx = shape
    g, Cf = _sphere(nx, ny, nz, 0.3)
    ux, uy, uz = W.uniform_faces(g, (0.3, -0.2, 0.25))
    p = W.Params(ka=2.0, kd=0.5, Df=2e-3, DF=5e-3, eps=0.75 * g.h, bc_f=0.1, bc_F=1.0)
    _, phi, delta = oracle.phase_field_build(g, Cf, 24, W.redist_dtau(g), p.eps)
    outs = []
    for staged in (0, 1):
        ctx = _ctx(sfx, g, 1)
        ctx.sfx_set_tuning(sfx._lib.SFX_TUNE_ADVECT_STAGED, staged)
        f, F = _pairs(ctx, 0.3 * delta), _pairs(ctx, 1.0 - Cf)
        u = [dev(v, torch.float32) for v in (ux, uy, uz)]
        for _ in range(2):
            assert ctx.sfx_surfactant_step(p, dev(phi), f, F, 0.2 * g.h, *u,
                                           opts=sfx.default_opts(tol=1e-10)).converged
        torch.cuda.synchronize()
        outs.append((f.cpu().numpy().copy(), F.cpu().numpy().copy()))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])


@pytest.mark.parametrize("shape", [(24, 24, 32), (20, 16, 64)])
def test_incremental_residuals_reach_the_same_fixed_point(sfx, shape):
    """After the pair residual pass, residuals formed in FP32 from the
    previous residual and the correction just added (the tiled path) end on
    the pair-only fixed point: the state matches the pair-only solve far
    below the FP32 tolerance, each solve converges, no solve needs more than
    one extra iteration, and the passes were counted as incremental."""
    import torch
    nz, ny, nx = shape
    g, Cf = _sphere(nx, ny, nz, 0.3)
    ux, uy, uz = W.uniform_faces(g, (0.3, -0.2, 0.25))
    p = W.Params(ka=2.0, kd=0.5, Df=2e-3, DF=5e-3, eps=0.75 * g.h)
    _, phi, delta = oracle.phase_field_build(g, Cf, 24, W.redist_dtau(g), p.eps)
    outs, its, work = [], [], []
    for incr in (0, 1):
        ctx = _ctx(sfx, g, 1)
        ctx.sfx_set_tuning(sfx._lib.SFX_TUNE_F32_INCR_RESID, incr)
        f, F = _pairs(ctx, 0.3 * delta), _pairs(ctx, 1.0 - Cf)
        u = [dev(v, torch.float32) for v in (ux, uy, uz)]
        ctx.sfx_profile(True)
        n = []
        for _ in range(3):
            st = ctx.sfx_surfactant_step(p, dev(phi), f, F, 0.2 * g.h, *u,
                                         opts=sfx.default_opts(tol=1e-10))
            assert st.converged and st.res_f <= 1e-10 and st.res_F <= 1e-10
            n.append(st.picard)
        torch.cuda.synchronize()
        work.append(ctx.sfx_profile_work())
        ctx.sfx_profile(False)
        its.append(n)
        outs.append((host(ctx.sfx_df_unpack(f)), host(ctx.sfx_df_unpack(F))))
    for a, b in zip(outs[0], outs[1]):
        assert np.abs(a - b).max() / np.abs(a).max() < 1e-8
    assert all(m <= k + 1 for k, m in zip(its[0], its[1])), its
    assert work[0]["residual_incr"] == 0 and work[1]["residual_incr"] > 0, work
