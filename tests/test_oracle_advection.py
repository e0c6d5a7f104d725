"""Pins of the oracle's explicit BCG advection step (Sec. 3.1)."""
import math

import numpy as np
import pytest

import oracle
import workloads as W


@pytest.mark.parametrize("geom,axis", [(W.PLANAR, 0), (W.PLANAR, 1), (W.AXI, 1), (W.CART3D, 2)])
def test_courant_one_translation_is_an_exact_shift(geom, axis):
    """At Courant number 1 the time-centred face value is the upwind cell
    value, so one step shifts the field by one cell (Gamma unchanged under
    uniform translation); the inflow value enters at the wall."""
    shape = (8, 7, 6) if geom == W.CART3D else (1, 12, 10)
    g = W.Grid(geom, shape[2], shape[1], shape[0], 0.1)
    dt = 0.05
    vel = [0.0, 0.0, 0.0]
    vel[axis] = g.h / dt
    ux, uy, uz = W.uniform_faces(g, vel)
    rng = np.random.default_rng(5)
    xi = rng.uniform(0, 1, shape)
    cur = xi.copy()
    ax = 2 - axis  # numpy axis of the grid direction
    for s in range(3):
        cur = oracle.advect_bcg(g, ux, uy, uz, dt, cur, 0.25)
    expect = np.roll(xi, 3, axis=ax)
    sl = [slice(None)] * 3
    sl[ax] = slice(0, 3)
    expect[tuple(sl)] = 0.25
    np.testing.assert_allclose(cur, expect, rtol=0, atol=1e-14)


@pytest.mark.parametrize("which", ["vortex", "hr3d", "hraxi"])
def test_uniform_field_is_preserved_by_divergence_free_flow(which):
    if which == "vortex":
        n = 32
        g = W.Grid(W.PLANAR, n, n, 1, 1.0 / n)
        ux, uy = W.single_vortex_faces(n, g.h, 0.7, 4.0)
        uz, dt = None, 0.5 * g.h
    elif which == "hr3d":
        n = 16
        g = W.Grid(W.CART3D, n, n, n, 1.0 / n)
        ux, uy, uz = W.hr_faces_3d(n, g.h, (0.5, 0.5, 0.5), 0.2)
        dt = 0.3 * g.h
    else:
        nr, nz = 16, 32
        g = W.Grid(W.AXI, nr, nz, 1, 1.0 / nr)
        ux, uy = W.hr_faces_axi(nr, nz, g.h, 1.0, 0.2)
        uz, dt = None, 0.3 * g.h
    xi = np.full(g.shape, 0.7)
    out = oracle.advect_bcg(g, ux, uy, uz, dt, xi, 0.7)
    np.testing.assert_allclose(out, 0.7, rtol=0, atol=1e-14)


def test_closed_domain_conserves_and_stays_bounded():
    n = 48
    g = W.Grid(W.PLANAR, n, n, 1, 1.0 / n)
    Cf = W.circle_vof(n, n, g.h, 0.5, 0.75, 0.15)
    xi = Cf.copy()
    V = oracle.cell_volumes(g)
    M0 = (V * xi).sum()
    dt = 0.4 * g.h
    for s in range(40):
        ux, uy = W.single_vortex_faces(n, g.h, s * dt, 4.0)
        xi = oracle.advect_bcg(g, ux, uy, None, dt, xi, 0.0)
    assert abs((V * xi).sum() - M0) < 1e-14
    assert xi.min() > -0.02 and xi.max() < 1.02


def _rotation_error(n):
    """Smooth bump rotated a quarter turn by solid-body rotation."""
    g = W.Grid(W.PLANAR, n, n, 1, 1.0 / n)
    omega = 2 * math.pi
    ux, uy = W.solid_rotation_faces(n, g.h, (0.5, 0.5), omega)
    x = (np.arange(n) + 0.5) * g.h

    def bump(cx, cy):
        r2 = (x[None, :] - cx) ** 2 + (x[:, None] - cy) ** 2
        return np.exp(-r2 / (2 * 0.08 ** 2))[None]

    T = 0.25
    steps = int(round(T / (0.25 * g.h / (omega * 0.5))))
    dt = T / steps
    xi = bump(0.75, 0.5)
    for _ in range(steps):
        xi = oracle.advect_bcg(g, ux, uy, None, dt, xi, 0.0)
    exact = bump(0.5, 0.75)  # counter-clockwise quarter turn
    # L1 norm: the limiter clips the peak, which lowers the max-norm order
    return np.abs(xi - exact).sum() * g.h ** 2


def test_rotation_converges_at_second_order():
    e1, e2 = _rotation_error(48), _rotation_error(96)
    order = math.log2(e1 / e2)
    assert order > 1.7, (e1, e2, order)
