"""Pins of the oracle's geometric VoF advection (split conservative PLIC,
the reading of Sec. 2's geometric VoF): an exact one-cell shift at Courant
number 1, exact conservation and boundedness in divergence-free flows with
closed walls, and the return of the single-vortex shape, converging under
refinement."""
import math

import numpy as np
import pytest

import oracle
import workloads as W


def _closed(ux, uy):
    ux = ux.copy()
    uy = uy.copy()
    ux[..., 0] = ux[..., -1] = 0.0
    uy[:, 0, :] = uy[:, -1, :] = 0.0
    return ux, uy


@pytest.mark.parametrize("order", [0, 1])
def test_courant_one_shifts_by_exactly_one_cell(order):
    n = 24
    h = 1.0 / n
    g = W.Grid(W.PLANAR, n, n, 1, h)
    Cf = W.circle_vof(n, n, h, 0.45, 0.5, 0.2)
    dt = 1e-2
    ux, uy, _ = W.uniform_faces(g, (h / dt, 0.0, 0.0))
    ux, uy = _closed(ux, uy)
    out = oracle.vof_advect(g, ux, uy, None, dt, Cf, order)
    np.testing.assert_allclose(out[..., 1:-1], Cf[..., :-2], rtol=0, atol=1e-14)


def test_courant_one_shift_in_3d():
    n = 12
    h = 1.0 / n
    g = W.Grid(W.CART3D, n, n, n, h)
    Cf = W.sphere_vof(n, h, (0.5, 0.5, 0.4), 0.25)
    dt = 1e-2
    ux, uy, uz = W.uniform_faces(g, (0.0, 0.0, h / dt))
    uz[0] = uz[-1] = 0.0
    out = oracle.vof_advect(g, ux, uy, uz, dt, Cf, 0)
    np.testing.assert_allclose(out[1:-1], Cf[:-2], rtol=0, atol=1e-14)


def test_single_vortex_conserves_and_stays_bounded():
    n = 48
    h = 1.0 / n
    g = W.Grid(W.PLANAR, n, n, 1, h)
    Cf = W.circle_vof(n, n, h, 0.5, 0.75, 0.15)
    T, steps = 2.0, 400
    dt = T / steps
    M0 = Cf.sum()
    C = Cf
    for s in range(steps // 2):
        ux, uy = W.single_vortex_faces(n, h, (s + 0.5) * dt, T)
        C = oracle.vof_advect(g, ux, uy, None, dt, C, s % 2)
    assert abs(C.sum() - M0) < 1e-13 * M0
    assert C.min() > -1e-12 and C.max() < 1.0 + 1e-12
    assert np.abs(C - Cf).sum() > 0.1 * M0   # the shape did move


def _vortex_error(n, T=2.0, courant=0.4):
    h = 1.0 / n
    g = W.Grid(W.PLANAR, n, n, 1, h)
    Cf = W.circle_vof(n, n, h, 0.5, 0.75, 0.15)
    steps = int(math.ceil(T / (courant * h)))
    dt = T / steps
    C = Cf
    for s in range(steps):
        ux, uy = W.single_vortex_faces(n, h, (s + 0.5) * dt, T)
        C = oracle.vof_advect(g, ux, uy, None, dt, C, s % 2)
    return np.abs(C - Cf).sum() * h * h


def test_single_vortex_returns_and_converges():
    e32, e64 = _vortex_error(32), _vortex_error(64)
    area = math.pi * 0.15 ** 2
    assert e64 < 0.05 * area
    assert e64 < e32 / 1.6, (e32, e64)
