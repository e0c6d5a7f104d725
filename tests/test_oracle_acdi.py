"""Pins of the oracle's ACDI step of the phase field (Sec. 2.5, central face
fluxes of the regularisation after a BCG advection): the equilibrium tanh
profile of width eps and its O((h/eps)^2) discrete residual, relaxation of
a wider profile to the thickness integral eps, exact conservation in closed
divergence-free flows (planar, axisymmetric, 3D), commutation with an exact
Courant-1 shift, mirror symmetry, and the reading of the normal where psi
is flat (no normal there, so that the step is well conditioned)."""
import numpy as np

import oracle
import workloads as W


def _slab(n, L=1.0):
    """A planar strip n x 4 of width L along x."""
    h = L / n
    g = W.Grid(W.PLANAR, n, 4, 1, h)
    x = (np.arange(n) + 0.5) * h
    return g, np.broadcast_to(x[None, None, :], g.shape).copy()


def _tanh_profile(x, x0, w):
    # phi = 1/2 (1 + tanh((x - x0)/(2 w))): phi -> 1 (fluid 2) for x > x0
    return 0.5 * (1.0 + np.tanh((x - x0) / (2.0 * w)))


def test_equilibrium_profile_residual_is_second_order():
    """The continuous tanh profile of width eps is a steady state of the
    regularisation; the discrete rate |phi1 - phi0|/(dt zeta) of its
    sampled profile falls by ~4 per halving of h (eps fixed)."""
    eps, zeta, dt = 0.05, 1.0, 1e-5
    rates = []
    for n in (64, 128, 256):
        g, X = _slab(n)
        phi0 = _tanh_profile(X, 0.5, eps)
        phi1 = oracle.acdi_step(g, phi0, dt, zeta, eps)
        rates.append(np.abs(phi1 - phi0).max() / (dt * zeta))
    assert rates[2] < 2e-3, rates
    assert rates[0] / rates[1] > 3.5 and rates[1] / rates[2] > 3.5, rates


def test_wide_profile_relaxes_to_the_equilibrium_width():
    """A profile of width 2 eps relaxes (u = 0) to the tanh of width eps: the
    thickness integral sum phi (1 - phi) h matches that of the equilibrium
    tanh over the box (eps up to the tails) to 1e-4, and the profile matches
    the tanh whose position keeps the mass, the error falling as (h/eps)^2."""
    eps, zeta = 0.05, 1.0
    errs = []
    for n in (64, 128):
        g, X = _slab(n)
        h = g.h
        dt = 0.2 * h * h / (zeta * eps)
        phi = _tanh_profile(X, 0.5, 2 * eps)
        mass0 = phi.sum()
        for _ in range(int(3.0 / dt)):     # ~15 decay times of the width
            phi = oracle.acdi_step(g, phi, dt, zeta, eps)
        assert abs(phi.sum() - mass0) <= 1e-12 * mass0
        thick = (phi * (1 - phi))[0, 0].sum() * h
        x = X[0, 0]
        # position of the equilibrium tanh with the same mass: 1 - x0 = mass
        x0 = 1.0 - phi[0, 0].sum() * h
        # its thickness integral over the box [0, 1] (eps up to the tails)
        want = 0.5 * eps * (np.tanh((1.0 - x0) / (2 * eps)) + np.tanh(x0 / (2 * eps)))
        errs.append((abs(thick / want - 1.0),
                     np.abs(phi[0, 0] - _tanh_profile(x, x0, eps)).max()))
    assert errs[0][0] < 1e-4 and errs[1][0] < 1e-4, errs
    assert errs[1][1] < 1e-4 and errs[0][1] / errs[1][1] > 3.5, errs


def _circle_phi(g, xc, yc, R, eps):
    x = (np.arange(g.nx) + 0.5) * g.h
    y = (np.arange(g.ny) + 0.5) * g.h
    r = np.hypot(x[None, :] - xc, y[:, None] - yc)[None]
    return _tanh_profile(r, R, eps)


def test_conserved_in_closed_divergence_free_flow():
    """Single-vortex flow (no normal velocity on the walls) on the planar
    grid and in every plane of the 3D grid, a closed ring vortex on the
    axisymmetric grid: sum V phi is kept to round-off over 20 steps."""
    n = 48
    g = W.Grid(W.PLANAR, n, n, 1, 1.0 / n)
    ux, uy = W.single_vortex_faces(n, g.h, 0.0, 4.0)
    cases = [(g, _circle_phi(g, 0.5, 0.75, 0.15, 0.75 * g.h), (ux, uy, None))]
    ga = W.Grid(W.AXI, 24, 48, 1, 1.0 / 24)
    ur, uz = W.ring_vortex_faces_axi(24, 48, ga.h)
    r = (np.arange(24) + 0.5) * ga.h
    z = (np.arange(48) + 0.5) * ga.h
    rho = np.hypot(r[None, :], z[:, None] - 1.0)[None]
    cases.append((ga, _tanh_profile(rho, 0.3, 0.75 * ga.h), (ur, uz, None)))
    n3 = 16
    g3 = W.Grid(W.CART3D, n3, n3, n3, 1.0 / n3)
    vx, vy = W.single_vortex_faces(n3, g3.h, 0.0, 4.0)
    u3 = (np.repeat(vx, n3, axis=0), np.repeat(vy, n3, axis=0), np.zeros((n3 + 1, n3, n3)))
    c3 = (np.arange(n3) + 0.5) * g3.h
    Z, Y, X = np.meshgrid(c3, c3, c3, indexing="ij")
    rho3 = np.sqrt((X - 0.6) ** 2 + (Y - 0.5) ** 2 + (Z - 0.5) ** 2)
    cases.append((g3, _tanh_profile(rho3, 0.25, 0.75 * g3.h), u3))
    for gg, phi, u in cases:
        V = oracle.cell_volumes(gg)
        umax = max(np.abs(a).max() for a in u if a is not None)
        dt = 0.25 * gg.h / umax
        m0 = (V * phi).sum()
        for _ in range(20):
            phi = oracle.acdi_step(gg, phi, dt, 1.1 * umax, 0.75 * gg.h, *u)
        assert abs((V * phi).sum() - m0) <= 1e-13 * m0, gg.geom
        assert phi.min() > -1e-3 and phi.max() < 1 + 1e-3, gg.geom


def test_commutes_with_an_exact_courant_one_shift():
    """u = h/dt along x: the BCG step is an exact shift by one cell and the
    regularisation is translation invariant, so away from the walls the step
    equals the shifted step of the same profile at rest."""
    n = 40
    g = W.Grid(W.PLANAR, n, n, 1, 1.0 / n)
    dt = 1e-3
    u = g.h / dt
    ux = np.full((1, n, n + 1), u)
    uy = np.zeros((1, n + 1, n))
    eps = 0.75 * g.h
    phi0 = _circle_phi(g, 0.45, 0.5, 0.2, eps)
    moved = oracle.acdi_step(g, phi0, dt, 1.1 * u, eps, ux, uy, None)
    rest = oracle.acdi_step(g, np.roll(phi0, 1, axis=2), dt, 1.1 * u, eps)
    inner = (slice(None), slice(3, -3), slice(4, -3))
    assert np.abs(moved[inner] - rest[inner]).max() < 1e-13


def test_centred_circle_stays_mirror_symmetric():
    n = 40
    g = W.Grid(W.PLANAR, n, n, 1, 1.0 / n)
    eps = 0.75 * g.h
    phi = _circle_phi(g, 0.5, 0.5, 0.2, eps)
    for _ in range(5):
        phi = oracle.acdi_step(g, phi, 2e-3, 1.0, eps)
    p = phi[0]
    assert np.abs(p - p[:, ::-1]).max() < 1e-14
    assert np.abs(p - p[::-1, :]).max() < 1e-14
    assert np.abs(p - p.T).max() < 1e-14


def test_step_is_well_conditioned_where_phi_saturates():
    """Where phi saturates psi is flat to round-off and its gradient has no
    direction; with n = 0 there (|grad psi| < 0.1) perturbing phi by 1e-15
    relative moves six steps by < 1e-13.  With the round-off direction kept
    one step moves by ~1e-6 (1 - tanh^2 is ~4e-6 there, not 0)."""
    n = 64
    g = W.Grid(W.PLANAR, n, n, 1, 1.0 / n)
    eps = 0.75 * g.h
    phi0 = _circle_phi(g, 0.5, 0.55, 0.2, eps)
    rng = np.random.default_rng(3)
    phi1 = phi0 * (1.0 + 1e-15 * rng.standard_normal(phi0.shape))
    for u in ((None, None, None), W.single_vortex_faces(n, g.h, 0.0, 4.0) + (None,)):
        a, b = phi0, phi1
        for _ in range(6):
            a = oracle.acdi_step(g, a, 0.3 * g.h, 1.1, eps, *u)
            b = oracle.acdi_step(g, b, 0.3 * g.h, 1.1, eps, *u)
        assert np.abs(a - b).max() < 1e-13


def test_flat_plateau_only_diffuses():
    """A saturated plateau phi = 1e-12 (1 + noise) far below veps: psi is
    flat, n = 0 everywhere, and the step is the pure discrete diffusion
    zeta eps lap(phi) of the noise (no-flux walls)."""
    n = 16
    g = W.Grid(W.PLANAR, n, n, 1, 1.0 / n)
    rng = np.random.default_rng(5)
    phi = 1e-12 * (1.0 + rng.uniform(0, 1, g.shape))
    eps, zeta, dt = 0.75 * g.h, 1.0, 1e-4
    out = oracle.acdi_step(g, phi, dt, zeta, eps)
    p = np.pad(phi[0], 1, mode="edge")
    lap = (p[1:-1, 2:] + p[1:-1, :-2] + p[2:, 1:-1] + p[:-2, 1:-1] - 4 * p[1:-1, 1:-1]) / g.h ** 2
    want = dt * zeta * eps * lap
    np.testing.assert_allclose(out[0] - phi[0], want, rtol=0, atol=1e-9 * np.abs(want).max())


def test_overshoots_past_one_plus_veps_stay_finite_and_clip_bounds():
    """phi* beyond 1 + veps (or below -veps) has no psi; psi is formed from
    phi* clipped to [0, 1], so the step stays finite.  With clip the result
    lies in [0, 1] and differs from the unclipped step only where that one
    leaves [0, 1]; the unclipped step conserves sum V phi."""
    n = 32
    g = W.Grid(W.PLANAR, n, n, 1, 1.0 / n)
    eps = 0.75 * g.h
    phi = _circle_phi(g, 0.5, 0.5, 0.25, eps)
    phi[phi > 1.0 - 1e-6] = 1.0 + 3e-6
    phi[phi < 1e-6] = -3e-6
    raw = oracle.acdi_step(g, phi, 2e-3, 1.0, eps)
    cl = oracle.acdi_step(g, phi, 2e-3, 1.0, eps, clip=True)
    assert np.all(np.isfinite(raw))
    assert abs(raw.sum() - phi.sum()) <= 1e-13 * phi.sum()
    assert cl.min() >= 0.0 and cl.max() <= 1.0
    inside = (raw >= 0.0) & (raw <= 1.0)
    assert np.array_equal(cl[inside], raw[inside])
    assert np.array_equal(cl[raw > 1.0], np.ones(int((raw > 1.0).sum())))
    assert np.all(cl[raw < 0.0] == 0.0)
