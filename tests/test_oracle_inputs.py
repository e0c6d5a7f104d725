"""Checks of the seeded input generators against exact geometry and the
divergence-free property of the prescribed flows."""
import math

import numpy as np
import pytest

import oracle
import workloads as W


def test_circle_vof_total_area_exact():
    n, R = 64, 0.25
    Cf = W.circle_vof(n, n, 1.0 / n, 0.5, 0.5, R)
    assert abs(Cf.sum() / n ** 2 - math.pi * R * R) < 1e-13
    # off-centre circle
    Cf = W.circle_vof(n, n, 1.0 / n, 0.431, 0.577, 0.2)
    assert abs(Cf.sum() / n ** 2 - math.pi * 0.04) < 1e-13
    assert Cf.min() >= 0 and Cf.max() <= 1


def test_circle_rect_area_brute_force():
    rng = np.random.default_rng(1)
    for _ in range(20):
        x0, y0 = rng.uniform(-0.3, 0.2, 2)
        w, hgt = rng.uniform(0.01, 0.2, 2)
        R = 0.25
        exact = float(W.circle_rect_area(x0, x0 + w, y0, y0 + hgt, R))
        m = 800
        xs = x0 + (np.arange(m) + 0.5) * w / m
        ys = y0 + (np.arange(m) + 0.5) * hgt / m
        inside = (xs[None, :] ** 2 + ys[:, None] ** 2) <= R * R
        approx = inside.mean() * w * hgt
        assert abs(exact - approx) < 3e-3 * w * hgt + 1e-9


def test_ring_vof_sphere_volume_exact():
    nr, nz, R = 32, 64, 0.4
    h = 1.0 / nr
    Cf = W.ring_vof(nr, nz, h, 1.0, R)
    g = W.Grid(W.AXI, nr, nz, 1, h)
    V = oracle.cell_volumes(g)
    assert abs((Cf * V).sum() - 4.0 / 3.0 * math.pi * R ** 3) < 1e-13


def test_sphere_vof_volume():
    n, R = 32, 0.3
    Cf = W.sphere_vof(n, 1.0 / n, (0.5, 0.5, 0.5), R)
    vol = Cf.sum() / n ** 3
    assert abs(vol - 4.0 / 3.0 * math.pi * R ** 3) < 1e-9


def _div_3d(ux, uy, uz, h):
    return ((ux[:, :, 1:] - ux[:, :, :-1]) + (uy[:, 1:, :] - uy[:, :-1, :]) +
            (uz[1:, :, :] - uz[:-1, :, :])) * h * h


def test_hr_3d_divergence_free_and_tangent():
    n = 32
    h = 1.0 / n
    ux, uy, uz = W.hr_faces_3d(n, h, (0.5, 0.5, 0.5), 0.25)
    div = _div_3d(ux, uy, uz, h)
    assert np.abs(div).max() < 1e-15
    # on the axis below the drop, Stokes flow gives u_z = U(1 - A R/r + B R^3/r^3)
    lam, R = 0.01, 0.25
    A, B = (2 + 3 * lam) / (2 * (1 + lam)), lam / (2 * (1 + lam))
    # the z-face on the axis averages the field over one face: compare loosely
    r = 0.5
    assert abs(uz[0, n // 2, n // 2] - (1 - A * R / r + B * R ** 3 / r ** 3)) < 0.02
    # no flow through the drop surface: z-faces on the axis at the poles
    zf = np.arange(n + 1) * h - 0.5
    k = int(np.argmin(np.abs(np.abs(zf) - 0.25)))
    assert abs(uz[k, n // 2, n // 2]) < 0.1


def test_hr_axi_divergence_free():
    nr, nz = 32, 64
    h = 1.0 / nr
    ur, uz = W.hr_faces_axi(nr, nz, h, 1.0, 0.2)
    r = np.arange(nr + 1) * h
    Ar = 2 * np.pi * r * h
    Az = np.pi * (r[1:] ** 2 - r[:-1] ** 2)
    net = (ur[0][:, 1:] * Ar[1:] - ur[0][:, :-1] * Ar[:-1]) + \
          (uz[0][1:, :] * Az - uz[0][:-1, :] * Az)
    assert np.abs(net).max() < 1e-14
    assert np.all(ur[0][:, 0] == 0.0)


def test_single_vortex_divergence_free_and_walls():
    n = 64
    ux, uy = W.single_vortex_faces(n, 1.0 / n, 0.3, 4.0)
    div = (ux[0][:, 1:] - ux[0][:, :-1]) + (uy[0][1:, :] - uy[0][:-1, :])
    assert np.abs(div).max() < 1e-15
    assert np.abs(ux[0][:, 0]).max() < 1e-15 and np.abs(uy[0][0, :]).max() < 1e-15


def test_workload_time_steps_within_cfl():
    """The fixed dt of each synthetic workload respects the Sec. 3.3 bound."""
    c = W.case_hr_3d(n=32, steps=1)
    p = c.params
    bound = oracle.cfl_dt(3, c.grid.h, c.extra["umax"], max(p.DF, p.Df), p.eps, 1.0)
    assert c.dt <= bound
    bound256 = oracle.cfl_dt(3, 1 / 256, 1.0, 0.025, 0.75 / 256, 1.0)
    assert W.HR3D_DT[256] <= bound256
    for nr in (16, 64, 128, 256):
        c = W.case_axi(nr, 2 * nr, 1.0, 1.0, steps=1) if nr <= 64 else None
        h = 1.0 / nr
        D = 0.4 / 100.0
        dt = W.AXI_DT.get(nr, 0.1 * h)
        assert dt <= oracle.cfl_dt(2, h, 1.2, D, 0.75 * h, 1.0)
    n = 128
    cv = W.case_vortex_2d(n=n)
    assert cv.dt <= oracle.cfl_dt(2, 1.0 / n, 1.0, 1e-4, 0.75 / n, 1.0)


def test_cfl_reduces_to_cell_peclet_when_eps_is_dx():
    """Sec. 3.3: with eps = dx the combined bound is dx <= D/|u|; at equality
    the advective and diffusive limits of the rule meet (2D: dx^2/(4D) vs
    dx/(u + D/dx) = dx^2/(2D))."""
    D, u = 0.01, 2.0
    h = D / u
    dt = oracle.cfl_dt(2, h, u, D, h, 1.0)
    assert math.isclose(dt, min(h / (u + D / h), h * h / (4 * D)), rel_tol=1e-15)
    assert math.isclose(h / (u + D / h), h * h / (2 * D), rel_tol=1e-14)
