"""Pins of the oracle's unit normal n = grad phi/|grad phi| (Sec. 2.6) and
of its reading where phi is flat: with q = |grad phi| / (phi (1 - phi)/eps),
the ratio to the slope of the equilibrium profile, n = 0 for q <= 1e-3, the
unit vector for q >= 2e-3 and a linear fade between."""
import numpy as np

import oracle
import workloads as W


def _grid(n, geom=W.PLANAR):
    return W.Grid(geom, n, n, 1 if geom != W.CART3D else n, 1.0 / n)


def test_plane_profiles_give_the_plane_normal_everywhere():
    """phi of a plane chi = x.m - c along an axis and along the diagonal
    (where the centred differences of both components are equal by
    symmetry): every cell sees the plane's normal to round-off; the flatness
    guard removes none of them out to |chi| = 10 eps (phi ~ 1e-6)."""
    n = 48
    g = _grid(n)
    eps = 0.75 * g.h
    x = (np.arange(n) + 0.5) * g.h
    for th in (0.0, np.pi / 4):
        m = np.array([np.cos(th), np.sin(th)])
        chi = (x[None, :] * m[0] + x[:, None] * m[1] - 0.7)[None]
        phi, _ = oracle.phase_field(g, chi, eps)
        nrm = oracle.normals(g, phi, eps)
        inner = (slice(None), slice(1, -1), slice(1, -1))
        sel = np.abs(chi[inner]) < 10 * eps
        assert sel.sum() > 200
        # grad phi points against grad chi (phi decreases with chi)
        for d in range(2):
            assert np.abs(nrm[d][inner][sel] + m[d]).max() < 1e-9


def test_flat_phi_with_round_off_variations_has_no_normal():
    """A bulk plateau phi = 6e-6 perturbed at the 1e-12 relative level: the
    perturbation has no resolvable direction and n = 0; a constant field
    gives n = 0 as well."""
    n = 16
    g = _grid(n)
    eps = 0.75 * g.h
    rng = np.random.default_rng(1)
    phi = 6e-6 * (1.0 + 1e-12 * rng.standard_normal(g.shape))
    assert np.all(oracle.normals(g, phi, eps) == 0.0)
    assert np.all(oracle.normals(g, np.full(g.shape, 0.3), eps) == 0.0)


def test_guard_threshold_is_relative_to_the_profile_slope():
    """phi = a + s x with |grad phi| = s: at or above 2e-3 a (1 - a)/eps the
    normal is e_x, at or below 1e-3 a (1 - a)/eps it is 0, and between the
    two it fades linearly (cells away from the walls, where phi's cell
    value is a + s (x - 1/2), so q varies by a few per cent along x)."""
    n = 16
    g = _grid(n)
    eps = 0.75 * g.h
    a = 0.2
    slope_eq = a * (1 - a) / eps
    x = (np.arange(n) + 0.5) * g.h
    inner = (slice(None), slice(None), slice(3, -3))
    for fac, want in ((3e-3, 1.0), (3e-4, 0.0)):
        s = fac * slope_eq
        phi = np.broadcast_to(a + s * (x - 0.5)[None, None, :], g.shape).copy()
        nrm = oracle.normals(g, phi, eps)
        np.testing.assert_allclose(nrm[0][inner], want, rtol=0, atol=1e-12)
        assert np.all(nrm[1][inner] == 0.0)
    # the fade: n_x = q/1e-3 - 1 with q = s/(phi (1 - phi)/eps) per cell
    s = 1.5e-3 * slope_eq
    phi = np.broadcast_to(a + s * (x - 0.5)[None, None, :], g.shape).copy()
    nrm = oracle.normals(g, phi, eps)
    q = s / (phi * (1 - phi) / eps)
    np.testing.assert_allclose(nrm[0][inner], (q / 1e-3 - 1.0)[inner], rtol=0, atol=1e-9)
    assert 0.3 < nrm[0][inner].min() and nrm[0][inner].max() < 0.7


def test_normal_depends_continuously_on_phi_where_it_fades():
    """Across the fade a relative change of 1e-9 in grad phi moves n by at
    most ~1e-9 / 1e-3 of the ramp's slope, never by a jump."""
    n = 16
    g = _grid(n)
    eps = 0.75 * g.h
    a = 0.2
    x = (np.arange(n) + 0.5) * g.h
    inner = (slice(None), slice(None), slice(3, -3))
    for fac in np.linspace(0.9e-3, 2.1e-3, 13):
        s = fac * a * (1 - a) / eps
        out = []
        for ds in (0.0, 1e-9):
            phi = np.broadcast_to(a + s * (1 + ds) * (x - 0.5)[None, None, :], g.shape).copy()
            out.append(oracle.normals(g, phi, eps)[0][inner])
        assert np.abs(out[1] - out[0]).max() < 1e-5


def test_sphere_normals_are_radial_in_3d():
    n = 24
    g = _grid(n, W.CART3D)
    eps = 0.75 * g.h
    x = (np.arange(n) + 0.5) * g.h - 0.5
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    r = np.sqrt(X * X + Y * Y + Z * Z)
    chi = r - 0.3
    phi, _ = oracle.phase_field(g, chi, eps)
    nrm = oracle.normals(g, phi, eps)
    band = np.abs(chi) < 3 * g.h
    dot = -(nrm[0] * X + nrm[1] * Y + nrm[2] * Z) / r
    assert dot[band].min() > 0.99
