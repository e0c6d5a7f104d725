"""Pins of the oracle's phase-field build (redistancing, tanh carrier and
regularised delta, Sec. 2.5-2.6)."""
import math

import numpy as np

import oracle
import workloads as W
from paper_values import PAPER


def _circle(n, R=0.25, c=(0.5, 0.5)):
    h = 1.0 / n
    g = W.Grid(W.PLANAR, n, n, 1, h)
    Cf = W.circle_vof(n, n, h, c[0], c[1], R)
    x = (np.arange(n) + 0.5) * h
    r = np.sqrt((x[None, :] - c[0]) ** 2 + (x[:, None] - c[1]) ** 2)[None]
    return g, Cf, R - r  # exact signed distance, positive inside fluid 1


def test_redistance_matches_exact_distance_in_band():
    errs = []
    for n in (32, 64, 128):
        g, Cf, chi_ex = _circle(n)
        chi = oracle.redistance(g, Cf, 3 * n // 4, 0.5 * g.h)
        band = np.abs(chi_ex) < 6 * g.h
        errs.append(np.abs(chi - chi_ex)[band].max() / g.h)
    # within a fraction of a cell everywhere in the band, at every resolution
    assert max(errs) < 0.35, errs


def test_redistance_far_field_gradient_is_unit():
    n = 64
    g, Cf, chi_ex = _circle(n)
    chi = oracle.redistance(g, Cf, 3 * n // 4, 0.5 * g.h)[0]
    gy, gx = np.gradient(chi, g.h)
    mask = (np.abs(chi_ex[0]) > 3 * g.h) & (np.abs(chi_ex[0]) < 10 * g.h)
    assert np.abs(np.hypot(gx, gy)[mask] - 1).max() < 0.15


def test_phase_field_closed_form_and_delta_identity():
    n = 64
    g, Cf, chi_ex = _circle(n)
    eps = PAPER["eps_over_dx"] * g.h
    phi, delta = oracle.phase_field(g, chi_ex, eps)
    # phi = 1/(1 + exp(chi/eps)) is the same logistic written without tanh
    # (absolute tolerance: 1 - tanh loses relative precision where phi ~ 0)
    np.testing.assert_allclose(phi, 1.0 / (1.0 + np.exp(chi_ex / eps)), rtol=1e-12, atol=1e-15)
    # delta = phi(1-phi)/eps = sech^2(chi/2eps)/(4 eps) = |d phi / d chi|
    np.testing.assert_allclose(delta, 1.0 / (4 * eps * np.cosh(chi_ex / (2 * eps)) ** 2),
                               rtol=1e-12, atol=1e-15 / eps)
    # fluid 1 (C = 1) carries phi ~ 0; the bulk side phi ~ 1 (Sec. 2.7)
    assert phi[chi_ex > 4 * g.h].max() < 0.01 and phi[chi_ex < -4 * g.h].min() > 0.99


def test_delta_integrates_to_interface_measure():
    """int delta_phi dV -> interface measure: perimeter (2D), sphere area
    (axisymmetric and 3D)."""
    R = 0.25
    errs = []
    for n in (32, 64, 128):
        g, Cf, _ = _circle(n, R)
        eps = 0.75 * g.h
        _, phi, delta = oracle.phase_field_build(g, Cf, 3 * n // 4, 0.5 * g.h, eps)
        errs.append(abs(oracle.total(g, delta) - 2 * math.pi * R) / (2 * math.pi * R))
    # the grid sampling of a width-0.75h profile leaves a small O(1)-in-h
    # error (below 0.5 %); a wrong width or normalisation would be O(1)
    assert max(errs) < 5e-3, errs
    # axisymmetric sphere: surface area 4 pi R^2
    nr, nz, R = 64, 128, 0.5
    h = 2.0 / nr
    ga = W.Grid(W.AXI, nr, nz, 1, h)
    Ca = W.ring_vof(nr, nz, h, nz * h / 2, R)
    _, _, da = oracle.phase_field_build(ga, Ca, 48, 0.5 * h, 0.75 * h)
    assert abs(oracle.total(ga, da) - 4 * math.pi * R * R) / (4 * math.pi * R * R) < 1e-2
    # 3D sphere
    n, R = 32, 0.3
    h = 1.0 / n
    g3 = W.Grid(W.CART3D, n, n, n, h)
    C3 = W.sphere_vof(n, h, (0.5, 0.5, 0.5), R)
    _, _, d3 = oracle.phase_field_build(g3, C3, 24, h / 3, 0.75 * h)
    assert abs(oracle.total(g3, d3) - 4 * math.pi * R * R) / (4 * math.pi * R * R) < 2e-2


def test_normals_of_circle_are_radial():
    n = 64
    g, Cf, chi_ex = _circle(n)
    phi, _ = oracle.phase_field(g, chi_ex, 0.75 * g.h)
    nrm = oracle.normals(g, phi, 0.75 * g.h)
    x = (np.arange(n) + 0.5) * g.h - 0.5
    r = np.hypot(x[None, :], x[:, None])
    band = (np.abs(chi_ex[0]) < 3 * g.h)
    # grad phi points out of fluid 1: along +e_r
    dot = (nrm[0, 0] * x[None, :] + nrm[1, 0] * x[:, None]) / r
    assert dot[band].min() > 0.99
