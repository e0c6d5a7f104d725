"""Pins of the oracle's capillary force F_cap = sigma kappa delta_s n with
kappa = -div n and delta_s = |grad C| (Sec. 2.2, 2.4): the curvature of
circles, spheres, cylinders and axisymmetric spheres against its closed
form, second-order convergence, a plane (no force), the pointwise role of
sigma, mirror symmetry and the Young-Laplace force on half a circle."""
import numpy as np

import oracle
import workloads as W


def _phi_of(g, chi, eps):
    phi, _ = oracle.phase_field(g, chi, eps)
    return phi


def _centres(g):
    x = (np.arange(g.nx) + 0.5) * g.h
    y = (np.arange(g.ny) + 0.5) * g.h
    z = (np.arange(g.nz) + 0.5) * g.h
    return np.meshgrid(z, y, x, indexing="ij")   # (Z, Y, X) with shape (nz, ny, nx)


def _circle_kappa_error(n, eps=1.0 / 16, R=0.25):
    g = W.Grid(W.PLANAR, n, n, 1, 1.0 / n)
    _, Y, X = _centres(g)
    r = np.hypot(X - 0.5, Y - 0.5)
    phi = _phi_of(g, R - r, eps)
    kap, _ = oracle.capillary(g, phi, np.zeros(g.shape), np.ones(g.shape), eps)
    band = (r > 0.5 * R) & (r < 1.5 * R)
    return np.abs(kap[band] * r[band] + 1.0).max()


def test_circle_curvature_is_minus_one_over_r_to_second_order():
    """n = grad phi/|grad phi| of a circle's profile is the outward radial
    direction, so kappa = -div n = -1/r at every cell of the band, not only
    on the interface.  With the profile width eps held fixed the error falls
    by ~4 per halving of h (the centred gradient of the tanh profile turns n
    by O((h/eps)^2), so at a fixed eps/h the error would not fall)."""
    e = [_circle_kappa_error(n) for n in (32, 64, 128)]
    assert e[2] < 3e-3, e
    assert e[0] / e[1] > 3.2 and e[1] / e[2] > 3.2, e


def test_sphere_and_cylinder_curvatures_in_3d():
    n = 48
    g = W.Grid(W.CART3D, n, n, n, 1.0 / n)
    Z, Y, X = _centres(g)
    eps = 1.0 / 12
    R = 0.25
    rho = np.sqrt((X - 0.5) ** 2 + (Y - 0.5) ** 2 + (Z - 0.5) ** 2)
    kap, _ = oracle.capillary(g, _phi_of(g, R - rho, eps), np.zeros(g.shape), np.ones(g.shape),
                              eps)
    band = (rho > 0.6 * R) & (rho < 1.4 * R)
    assert np.abs(kap[band] * rho[band] + 2.0).max() < 2e-2
    # a cylinder along z: one principal curvature
    s = np.hypot(X - 0.5, Y - 0.5)
    kap, _ = oracle.capillary(g, _phi_of(g, R - s, eps), np.zeros(g.shape), np.ones(g.shape), eps)
    band = (s > 0.6 * R) & (s < 1.4 * R)
    assert np.abs(kap[band] * s[band] + 1.0).max() < 1.5e-2


def test_axisymmetric_sphere_has_twice_the_planar_curvature():
    """A sphere on the axis of an (r, z) grid: kappa = -2/rho, the hoop term
    n_r/r coming from the face areas; cells on the axis included."""
    errs = []
    for nr in (32, 64, 128):
        g = W.Grid(W.AXI, nr, 2 * nr, 1, 1.0 / nr)
        _, Z, Rr = _centres(g)
        rho = np.hypot(Rr, Z - 1.0)
        eps = 1.0 / 16
        kap, _ = oracle.capillary(g, _phi_of(g, 0.4 - rho, eps), np.zeros(g.shape),
                                  np.ones(g.shape), eps)
        band = (rho > 0.25) & (rho < 0.55)
        assert band[..., 0].any()
        errs.append(np.abs(kap[band] * rho[band] + 2.0).max())
    assert errs[2] < 5e-3 and errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5, errs


def test_plane_interface_has_no_capillary_force():
    """A straight interface (C from exact areas, phi its profile): kappa is
    zero wherever delta_s is non-zero, and so is the force."""
    n = 48
    g = W.Grid(W.PLANAR, n, n, 1, 1.0 / n)
    _, Y, X = _centres(g)
    Cf = np.clip((0.4 - (X - 0.5 * g.h)) / g.h, 0.0, 1.0)       # x = 0.4 plane
    phi = _phi_of(g, 0.4 - X, 0.75 * g.h)
    kap, force = oracle.capillary(g, phi, Cf, np.full(g.shape, 0.7), 0.75 * g.h)
    assert np.count_nonzero(Cf * (1 - Cf)) + np.count_nonzero(np.diff(Cf, axis=2)) > 0
    assert np.all(force == 0.0)
    ds = np.abs(np.gradient(Cf, axis=2))
    assert np.all(kap[ds > 0] == 0.0)


def _circle_case(n, R=0.25, xc=0.5, yc=0.5):
    g = W.Grid(W.PLANAR, n, n, 1, 1.0 / n)
    Cf = W.circle_vof(n, n, g.h, xc, yc, R)
    _, Y, X = _centres(g)
    eps = 0.75 * g.h
    phi = _phi_of(g, R - np.hypot(X - xc, Y - yc), eps)
    return g, Cf, phi, eps, X, Y


def test_sigma_enters_pointwise():
    """F_cap(s sigma) = s F_cap(sigma) cell by cell for any positive field s:
    sigma multiplies the force and is not differentiated."""
    g, Cf, phi, eps, X, Y = _circle_case(48, xc=0.47, yc=0.52)
    s = 1.0 + 0.5 * np.sin(7 * X) * np.cos(5 * Y)
    _, f1 = oracle.capillary(g, phi, Cf, np.ones(g.shape), eps)
    _, f2 = oracle.capillary(g, phi, Cf, s, eps)
    np.testing.assert_allclose(f2, s[None] * f1, rtol=1e-15, atol=0)


def test_centred_circle_is_mirror_symmetric_and_force_free():
    """A circle centred in the box: F_x is odd in x and even in y, F_y the
    other way round, F_y is F_x transposed (up to the rounding of the
    exact-area C, 5e-14), and the total force vanishes."""
    g, Cf, phi, eps, X, Y = _circle_case(64)
    _, force = oracle.capillary(g, phi, Cf, np.ones(g.shape), eps)
    fx, fy = force[0, 0], force[1, 0]
    tol = 1e-13 * np.abs(fx).max()
    assert np.abs(fx + fx[:, ::-1]).max() <= tol and np.abs(fx - fx[::-1, :]).max() <= tol
    assert np.abs(fy + fy[::-1, :]).max() <= tol and np.abs(fy - fy[:, ::-1]).max() <= tol
    assert np.abs(fx - fy.T).max() <= 1e3 * tol
    scale = np.abs(fx).sum()
    assert abs(fx.sum()) <= 1e-14 * scale and abs(fy.sum()) <= 1e-14 * scale


def test_young_laplace_force_on_half_a_circle():
    """Sum of V F_cap over the half x > xc of a circle of radius R with
    uniform sigma: sigma kappa times the projected length of the half arc,
    sigma (-1/R)(2R) = -2 sigma along x, 0 along y; first-order in h."""
    sig = 0.8
    errs = []
    for n in (64, 128, 256):
        g, Cf, phi, eps, X, Y = _circle_case(n)
        _, force = oracle.capillary(g, phi, Cf, np.full(g.shape, sig), eps)
        half = X > 0.5
        V = g.h * g.h
        Fx = (force[0][half]).sum() * V
        Fy = (force[1][half]).sum() * V
        assert abs(Fy) < 1e-12
        errs.append(abs(Fx / (-2 * sig) - 1.0))
    assert errs[-1] < 0.02 and errs[0] > errs[1] > errs[2], errs
