"""GPU capillary force (sfx_capillary_force) against the FP64 oracle:
F_cap = sigma kappa |grad C| n with kappa = -div n (Sec. 2.2, 2.4), on
planar, axisymmetric and 3D grids whose extents leave ragged tiles (32 x 8
cells per block, 32 planes per z chunk), with a non-uniform sigma."""
import numpy as np
import pytest

import oracle
import workloads as W
from gpu_util import dev, host, rel_err

pytestmark = pytest.mark.gpu

PARITY = 1e-12      # FP64 context against the FP64 oracle (normwise)
# SFX_F32: the normals are rounded to float (2^-24 relative) and kappa is
# their difference over h, so its rounding error is ~2^-23/h against the
# force scale sigma |kappa| |grad C| ~ 1/(R h); on grids of <= 100 cells
# across with R >= 0.2 that is < 1e-5 of the largest force.
F32_TOL = 1e-5


@pytest.fixture(scope="module")
def sfx():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2605_27534_gb300 as m
    m.lib()
    return m


def _case(geom):
    if geom == "planar":
        nx, ny = 77, 53
        h = 1.0 / 77
        g = W.Grid(W.PLANAR, nx, ny, 1, h)
        Cf = W.circle_vof(nx, ny, h, 0.47, 0.5 * ny * h, 0.2)
    elif geom == "axi":
        g = W.Grid(W.AXI, 45, 90, 1, 1.0 / 45)
        Cf = W.ring_vof(45, 90, g.h, 1.0, 0.3)
    else:
        n = 70      # three z chunks, the last one ragged
        g = W.Grid(W.CART3D, 37, 41, n, 1.0 / n)
        Cf = W.sphere_vof(n, g.h, (0.26, 0.29, 0.5), 0.2)[:, :41, :37].copy()
    p = W.Params(eps=0.75 * g.h, sigma0=1.0, E=0.3, gamma_inf=1.0)
    dtau = 0.5 * g.h if g.ndim == 2 else g.h / 3
    _, phi, _ = oracle.phase_field_build(g, Cf, 24, dtau, p.eps)
    Z, Y, X = np.meshgrid(*[(np.arange(m) + 0.5) * g.h for m in (g.nz, g.ny, g.nx)],
                          indexing="ij")
    sigma = 1.0 - 0.2 * np.sin(5 * X + 1) * np.cos(3 * Y) * np.cos(2 * Z)
    return g, p, Cf, phi, sigma


GEOMS = ["planar", "axi", "3d"]


@pytest.mark.parametrize("geom", GEOMS)
def test_capillary_force_fp64_matches_the_oracle(sfx, geom):
    import torch
    g, p, Cf, phi, sigma = _case(geom)
    kap_o, force_o = oracle.capillary(g, phi, Cf, sigma, p.eps)
    assert np.abs(force_o).max() > 0
    ctx = sfx.Context.for_grid(g, sfx.SFX_F64)
    kap = torch.full(g.shape, np.nan, dtype=torch.float64, device="cuda")
    force = torch.full((g.ndim,) + g.shape, np.nan, dtype=torch.float64, device="cuda")
    ctx.sfx_capillary_force(p, dev(phi), dev(Cf), dev(sigma), force, kappa=kap)
    assert rel_err(host(kap), kap_o) < PARITY
    assert rel_err(host(force), force_o) < PARITY
    # without the curvature output: the same force, bit for bit
    force2 = torch.empty_like(force)
    ctx.sfx_capillary_force(p, dev(phi), dev(Cf), dev(sigma), force2)
    assert torch.equal(force, force2)


@pytest.mark.parametrize("geom", GEOMS)
def test_capillary_force_fp32_matches_the_oracle(sfx, geom):
    import torch
    g, p, Cf, phi, sigma = _case(geom)
    kap_o, force_o = oracle.capillary(g, phi, Cf, sigma, p.eps)
    ctx = sfx.Context.for_grid(g, sfx.SFX_F32)
    kap = torch.full(g.shape, np.nan, dtype=torch.float32, device="cuda")
    force = torch.full((g.ndim,) + g.shape, np.nan, dtype=torch.float32, device="cuda")
    ctx.sfx_capillary_force(p, dev(phi), dev(Cf, torch.float32), dev(sigma, torch.float32), force,
                            kappa=kap)
    assert rel_err(host(force), force_o) < F32_TOL
    # the curvature where the force lives (elsewhere n may switch off at a
    # slightly different cell where phi turns flat)
    live = np.abs(force_o).sum(axis=0) > 0
    k32 = host(kap)
    assert np.abs(k32[live] - kap_o[live]).max() < F32_TOL * np.abs(kap_o[live]).max()


def test_capillary_force_degenerate_grids(sfx):
    """One cell and a single row: no interface can be resolved, the force is
    zero; a uniform C has no force either."""
    import torch
    for nx, ny in ((1, 1), (33, 1)):
        g = W.Grid(W.PLANAR, nx, ny, 1, 1.0 / 33)
        rng = np.random.default_rng(1)
        phi = rng.uniform(0, 1, g.shape)
        Cf = np.ones(g.shape)
        sig = np.ones(g.shape)
        p = W.Params(eps=0.75 * g.h)
        kap_o, force_o = oracle.capillary(g, phi, Cf, sig, p.eps)
        ctx = sfx.Context.for_grid(g, sfx.SFX_F64)
        kap = torch.empty(g.shape, dtype=torch.float64, device="cuda")
        force = torch.empty((2,) + g.shape, dtype=torch.float64, device="cuda")
        ctx.sfx_capillary_force(p, dev(phi), dev(Cf), dev(sig), force, kappa=kap)
        assert np.all(host(force) == 0.0) and np.all(force_o == 0.0)
        assert rel_err(host(kap), kap_o) < PARITY


def test_capillary_force_rejects_null_arguments(sfx):
    import torch
    g, p, Cf, phi, sigma = _case("planar")
    ctx = sfx.Context.for_grid(g, sfx.SFX_F64)
    force = torch.empty((2,) + g.shape, dtype=torch.float64, device="cuda")
    with pytest.raises(sfx.SfxError):
        ctx.sfx_capillary_force(p, dev(phi), dev(Cf), None, force)
    with pytest.raises(sfx.SfxError):
        ctx.sfx_capillary_force(p, dev(phi), None, dev(sigma), force)
