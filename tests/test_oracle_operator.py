"""Pins of the oracle's generalised elliptic operator
L(a) = div(alpha grad a + beta a) + lambda a  (Sec. 3.1-3.2, App. A, App. B)
and of its Gauss-Seidel solver."""
import math

import numpy as np
import pytest

import oracle
import workloads as W


def _zero_faces(g):
    nz, ny, nx = g.shape
    Bx = np.zeros((nz, ny, nx + 1))
    By = np.zeros((nz, ny + 1, nx))
    Bz = np.zeros((nz + 1, ny, nx)) if g.ndim == 3 else None
    return Bx, By, Bz


def _random_faces(g, rng, scale):
    Bx, By, Bz = _zero_faces(g)
    Bx[..., 1:-1] = rng.uniform(-scale, scale, Bx[..., 1:-1].shape)
    By[:, 1:-1, :] = rng.uniform(-scale, scale, By[:, 1:-1, :].shape)
    if Bz is not None:
        Bz[1:-1] = rng.uniform(-scale, scale, Bz[1:-1].shape)
    return Bx, By, Bz


@pytest.mark.parametrize("geom,shape", [(W.PLANAR, (1, 12, 16)), (W.CART3D, (6, 8, 10))])
def test_cosine_modes_are_discrete_eigenvectors(geom, shape):
    """With B = 0 and no-flux walls, cos(k pi (i+1/2)/n) is an exact
    eigenvector of the 3-point diffusion stencil with eigenvalue
    (2D/h^2)(1 - cos(k pi / n))."""
    nz, ny, nx = shape
    h, D, lam = 0.1, 0.37, 5.0
    g = W.Grid(geom, nx, ny, nz, h)
    Bx, By, Bz = _zero_faces(g)
    kx, ky, kz = 3, 2, (1 if geom == W.CART3D else 0)
    cx = np.cos(kx * np.pi * (np.arange(nx) + 0.5) / nx)
    cy = np.cos(ky * np.pi * (np.arange(ny) + 0.5) / ny)
    cz = np.cos(kz * np.pi * (np.arange(nz) + 0.5) / nz)
    a = cz[:, None, None] * cy[None, :, None] * cx[None, None, :]
    ev = lam + sum(2 * D / h ** 2 * (1 - math.cos(k * math.pi / n))
                   for k, n in ((kx, nx), (ky, ny), (kz, nz)))
    La = oracle.apply_operator(g, D, Bx, By, Bz, np.full(shape, lam), a)
    np.testing.assert_allclose(La, ev * a, atol=1e-12 * ev)


def test_axisymmetric_axial_cosine_mode():
    nr, nz, h, D, lam = 8, 16, 0.05, 0.2, 1.0
    g = W.Grid(W.AXI, nr, nz, 1, h)
    Bx, By, _ = _zero_faces(g)
    a = np.cos(3 * np.pi * (np.arange(nz) + 0.5) / nz)[None, :, None] * np.ones((1, nz, nr))
    ev = lam + 2 * D / h ** 2 * (1 - math.cos(3 * math.pi / nz))
    La = oracle.apply_operator(g, D, Bx, By, None, np.full(a.shape, lam), a)
    np.testing.assert_allclose(La, ev * a, atol=1e-12 * ev)


def test_laplacian_of_quadratics_is_exact():
    """Centred fluxes are exact for quadratics: div grad (r^2) = 4 in the
    axisymmetric metric (including the axis cell), |x|^2 -> 2 N_d."""
    D = 1.0
    # axisymmetric r^2 (App. B volumes and face areas)
    nr, nz, h = 10, 6, 0.1
    g = W.Grid(W.AXI, nr, nz, 1, h)
    r = (np.arange(nr) + 0.5) * h
    a = np.broadcast_to(r[None, None, :] ** 2, (1, nz, nr)).copy()
    Bx, By, _ = _zero_faces(g)
    La = oracle.apply_operator(g, D, Bx, By, None, np.zeros_like(a), a)
    np.testing.assert_allclose(La[0, :, :-1], -4.0, rtol=1e-12)
    # 3D |x|^2
    n = 6
    g3 = W.Grid(W.CART3D, n, n, n, h)
    x = (np.arange(n) + 0.5) * h
    a3 = x[:, None, None] ** 2 + x[None, :, None] ** 2 + x[None, None, :] ** 2
    Bx, By, Bz = _zero_faces(g3)
    L3 = oracle.apply_operator(g3, D, Bx, By, Bz, np.zeros_like(a3), a3)
    np.testing.assert_allclose(L3[1:-1, 1:-1, 1:-1], -6.0, rtol=1e-12)
    # planar
    g2 = W.Grid(W.PLANAR, n, n, 1, h)
    a2 = (x[None, :, None] ** 2 + x[None, None, :] ** 2)
    Bx, By, _ = _zero_faces(g2)
    L2 = oracle.apply_operator(g2, D, Bx, By, None, np.zeros_like(a2), a2)
    np.testing.assert_allclose(L2[:, 1:-1, 1:-1], -4.0, rtol=1e-12)


@pytest.mark.parametrize("geom", [W.PLANAR, W.AXI, W.CART3D])
def test_flux_form_conserves(geom):
    """Every face flux leaves one cell and enters its neighbour with the same
    area, and walls carry none: sum V (lambda a - L(a)) = 0 for any a, B."""
    rng = np.random.default_rng(7)
    shape = (5, 6, 7) if geom == W.CART3D else (1, 9, 8)
    g = W.Grid(geom, shape[2], shape[1], shape[0], 0.07)
    Bx, By, Bz = _random_faces(g, rng, 3.0)
    a = rng.uniform(0.1, 2.0, shape)
    lam = rng.uniform(1.0, 2.0, shape)
    La = oracle.apply_operator(g, 0.3, Bx, By, Bz, lam, a)
    V = oracle.cell_volumes(g)
    s = (V * (lam * a - La)).sum()
    assert abs(s) < 1e-13 * (V * np.abs(lam * a)).sum()


def test_upwind_reading_keeps_maximum_principle():
    """Implicit steps of an upwinded drift keep a positive field positive
    (M-matrix); the face value printed in Sec. 3.2 (left value when B > 0)
    does not once the cell Peclet number |B| h / D exceeds 2."""
    n = 24
    h = 1.0 / n
    g = W.Grid(W.PLANAR, n, n, 1, h)
    Cf = W.circle_vof(n, n, h, 0.5, 0.5, 0.25)
    p = W.Params(Df=1e-5, DF=1e-5, eps=0.75 * h)
    _, phi, _ = oracle.phase_field_build(g, Cf, 18, 0.5 * h, p.eps)
    Bx, By, _ = oracle.face_drift(g, p, phi, 0)
    Bx *= 1e3
    By *= 1e3
    rng = np.random.default_rng(3)
    b = rng.uniform(0.0, 1.0, g.shape)
    lam = np.full(g.shape, 1.0 / 1e-3)
    a, s, rr = oracle.elliptic_solve(g, 1e-5, Bx, By, None, lam, b, tol=1e-13, literal=0)
    assert s > 0 and a.min() >= 0.0
    a_lit, s_lit, _ = oracle.elliptic_solve(g, 1e-5, Bx, By, None, lam, b, tol=1e-13,
                                            max_sweeps=400, literal=1)
    assert s_lit < 0 or a_lit.min() < 0.0


@pytest.mark.parametrize("geom", [W.PLANAR, W.AXI, W.CART3D])
def test_gauss_seidel_matches_dense_solve(geom):
    rng = np.random.default_rng(11)
    shape = (3, 4, 5) if geom == W.CART3D else (1, 6, 5)
    g = W.Grid(geom, shape[2], shape[1], shape[0], 0.2)
    Bx, By, Bz = _random_faces(g, rng, 0.5)
    lam = rng.uniform(5.0, 10.0, shape)
    b = rng.uniform(-1, 1, shape)
    D = 0.05
    N = g.ncell
    M = np.zeros((N, N))
    for c in range(N):
        e = np.zeros(N)
        e[c] = 1.0
        M[:, c] = oracle.apply_operator(g, D, Bx, By, Bz, lam, e.reshape(shape)).ravel()
    a_ref = np.linalg.solve(M, b.ravel()).reshape(shape)
    a, s, rr = oracle.elliptic_solve(g, D, Bx, By, Bz, lam, b, tol=1e-14)
    assert s > 0
    np.testing.assert_allclose(a, a_ref, rtol=0, atol=1e-13 * np.abs(a_ref).max())


def test_face_drift_is_mean_of_cell_values_and_zero_on_walls():
    n = 16
    h = 1.0 / n
    g = W.Grid(W.PLANAR, n, n, 1, h)
    Cf = W.circle_vof(n, n, h, 0.5, 0.5, 0.3)
    p = W.Params(Df=0.02, DF=0.03, eps=0.75 * h)
    _, phi, _ = oracle.phase_field_build(g, Cf, 12, 0.5 * h, p.eps)
    nrm = oracle.normals(g, phi, p.eps)
    for which, s in ((0, -p.Df * 2 * (0.5 - phi) / p.eps), (1, -p.DF * (1 - phi) / p.eps)):
        Bx, By, _ = oracle.face_drift(g, p, phi, which)
        Bc = s * nrm[0]
        np.testing.assert_allclose(Bx[..., 1:-1], 0.5 * (Bc[..., :-1] + Bc[..., 1:]), rtol=1e-14,
                                   atol=1e-300)
        assert np.all(Bx[..., 0] == 0) and np.all(Bx[..., -1] == 0)
        assert np.all(By[:, 0, :] == 0) and np.all(By[:, -1, :] == 0)
