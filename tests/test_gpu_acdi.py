"""GPU ACDI step of the phase field (sfx_acdi_step, Sec. 2.5) against the
FP64 oracle: planar, axisymmetric and 3D grids in closed divergence-free
flows and at rest, over several steps; FP32 contexts (float face
velocities, FP64 arithmetic on phi) against the oracle fed the same
rounded velocities; conservation of sum V phi; argument checks."""
import numpy as np
import pytest

import oracle
import workloads as W
from gpu_util import dev, host, rel_err

pytestmark = pytest.mark.gpu

PARITY = 1e-12      # normwise, against the FP64 oracle


@pytest.fixture(scope="module")
def sfx():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2605_27534_gb300 as m
    m.lib()
    return m


def _profile(r, R, eps):
    return 0.5 * (1.0 + np.tanh((r - R) / (2.0 * eps)))


def _case(geom):
    """(grid, phi0, (ux, uy, uz)) with a closed divergence-free flow."""
    if geom == "planar":
        nx, ny = 70, 66
        h = 1.0 / 70
        g = W.Grid(W.PLANAR, nx, ny, 1, h)
        # single-vortex stream function of the nx x ny box: zero on its walls
        x = np.arange(nx + 1) * h
        y = np.arange(ny + 1) * h
        psi = (np.sin(np.pi * x / x[-1]) ** 2)[None, :] * (np.sin(np.pi * y / y[-1]) ** 2)[:, None]
        ux = ((psi[1:, :] - psi[:-1, :]) / h)[None]
        uy = (-(psi[:, 1:] - psi[:, :-1]) / h)[None]
        xc = (np.arange(nx) + 0.5) * h
        yc = (np.arange(ny) + 0.5) * h
        r = np.hypot(xc[None, :] - 0.5, yc[:, None] - 0.6)[None]
        return g, _profile(r, 0.2, 0.75 * h), (ux, uy, None)
    if geom == "axi":
        g = W.Grid(W.AXI, 40, 80, 1, 1.0 / 40)
        ur, uz = W.ring_vortex_faces_axi(40, 80, g.h)
        r = (np.arange(40) + 0.5) * g.h
        z = (np.arange(80) + 0.5) * g.h
        rho = np.hypot(r[None, :], z[:, None] - 1.1)[None]
        return g, _profile(rho, 0.35, 0.75 * g.h), (ur, uz, None)
    n = 36
    g = W.Grid(W.CART3D, n, n, n, 1.0 / n)
    vx, vy = W.single_vortex_faces(n, g.h, 0.0, 4.0)
    u = (np.repeat(vx, n, axis=0), np.repeat(vy, n, axis=0), np.zeros((n + 1, n, n)))
    c = (np.arange(n) + 0.5) * g.h
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    rho = np.sqrt((X - 0.55) ** 2 + (Y - 0.5) ** 2 + (Z - 0.45) ** 2)
    return g, _profile(rho, 0.25, 0.75 * g.h), u


GEOMS = ["planar", "axi", "3d"]


def _run_oracle(g, phi, u, dt, zeta, eps, steps, flow=True):
    for _ in range(steps):
        phi = oracle.acdi_step(g, phi, dt, zeta, eps, *(u if flow else (None, None, None)))
    return phi


@pytest.mark.parametrize("geom", GEOMS)
@pytest.mark.parametrize("flow", [True, False])
def test_acdi_fp64_matches_the_oracle(sfx, geom, flow):
    import torch
    g, phi0, u = _case(geom)
    umax = max(np.abs(a).max() for a in u if a is not None)
    dt, zeta, eps = 0.3 * g.h / umax, 1.1 * umax, 0.75 * g.h
    want = _run_oracle(g, phi0, u, dt, zeta, eps, 6, flow)
    ctx = sfx.Context.for_grid(g, sfx.SFX_F64)
    phi = dev(phi0)
    ud = [dev(a) if a is not None else None for a in u] if flow else [None, None, None]
    for _ in range(6):
        ctx.sfx_acdi_step(phi, dt, zeta, eps, *ud)
    assert rel_err(host(phi), want) < PARITY
    assert rel_err(host(phi) - phi0, want - phi0) < 1e-9   # the change itself
    # conservation in the closed box
    V = oracle.cell_volumes(g)
    assert abs((V * host(phi)).sum() - (V * phi0).sum()) <= 1e-13 * (V * phi0).sum()
    torch.cuda.synchronize()


@pytest.mark.parametrize("geom", GEOMS)
def test_acdi_in_fp32_contexts_matches_the_oracle(sfx, geom):
    """Float face velocities: the oracle takes the same rounded values; phi
    and the arithmetic stay FP64."""
    import torch
    g, phi0, u = _case(geom)
    u32 = [a.astype(np.float32) if a is not None else None for a in u]
    u64 = [a.astype(np.float64) if a is not None else None for a in u32]
    umax = max(np.abs(a).max() for a in u64 if a is not None)
    dt, zeta, eps = 0.3 * g.h / umax, 1.1 * umax, 0.75 * g.h
    want = _run_oracle(g, phi0, u64, dt, zeta, eps, 4)
    ctx = sfx.Context.for_grid(g, sfx.SFX_F32)
    phi = dev(phi0)
    ud = [dev(a) if a is not None else None for a in u32]
    for _ in range(4):
        ctx.sfx_acdi_step(phi, dt, zeta, eps, *ud)
    assert rel_err(host(phi), want) < PARITY
    assert ud[0].dtype == torch.float32


@pytest.mark.parametrize("clip", [False, True])
def test_acdi_overshoots_and_clipping_match_the_oracle(sfx, clip):
    """phi beyond 1 + veps and below -veps (no psi there without the clamp),
    with and without clipping of the result, in the closed planar flow."""
    g, phi0, u = _case("planar")
    phi0 = phi0.copy()
    phi0[phi0 > 1.0 - 1e-6] = 1.0 + 3e-6
    phi0[phi0 < 1e-6] = -3e-6
    umax = max(np.abs(a).max() for a in u if a is not None)
    dt, zeta, eps = 0.3 * g.h / umax, 1.1 * umax, 0.75 * g.h
    want = phi0
    for _ in range(3):
        want = oracle.acdi_step(g, want, dt, zeta, eps, *u, clip=clip)
    ctx = sfx.Context.for_grid(g, sfx.SFX_F64)
    phi = dev(phi0)
    ud = [dev(a) if a is not None else None for a in u]
    for _ in range(3):
        ctx.sfx_acdi_step(phi, dt, zeta, eps, *ud, clip=clip)
    got = host(phi)
    assert np.all(np.isfinite(got))
    assert rel_err(got, want) < PARITY
    if clip:
        assert got.min() >= 0.0 and got.max() <= 1.0


def test_acdi_rejects_bad_arguments(sfx):
    g, phi0, u = _case("planar")
    ctx = sfx.Context.for_grid(g, sfx.SFX_F64)
    phi = dev(phi0)
    with pytest.raises(sfx.SfxError):
        ctx.sfx_acdi_step(phi, -1e-3, 1.0, 0.75 * g.h)
    with pytest.raises(sfx.SfxError):
        ctx.sfx_acdi_step(phi, 1e-3, 1.0, 0.0)
    with pytest.raises(sfx.SfxError):
        ctx.sfx_acdi_step(phi, 1e-3, -1.0, 0.75 * g.h)
    with pytest.raises(sfx.SfxError):
        ctx.sfx_acdi_step(phi, 1e-3, 1.0, 0.75 * g.h, dev(u[0]), None)
    with pytest.raises(sfx.SfxError):
        ctx.sfx_acdi_step(None, 1e-3, 1.0, 0.75 * g.h)
