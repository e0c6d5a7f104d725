"""Pins of the oracle's coupled implicit source step (App. C) against the
flat-interface kinetics of Sec. 4.3 and against conservation.

The closed forms are sharp-interface limits.  The diffuse band converges to
them as eps -> 0 with eps/h fixed and large enough for the first-order
upwind drift to resolve the tanh profile; at the paper's eps = 0.75 h the
band-averaged F/phi keeps an O(1)-in-h bias of about 15 %, so these pins run
with eps = 4 h."""
import math

import numpy as np
import pytest
from scipy.integrate import quad
from scipy.special import erfc

import oracle
import workloads as W
from paper_values import PAPER

L = PAPER["e3a_domain_half"]


def _flat(ny, nx=2):
    """Flat interface y = 0 in [-L, L]: fluid 1 (no bulk surfactant) below."""
    h = 2 * L / ny
    g = W.Grid(W.PLANAR, nx, ny, 1, h)
    y = -L + (np.arange(ny) + 0.5) * h
    Cf = np.zeros((1, ny, nx))
    Cf[0, y < 0, :] = 1.0
    return g, Cf, y


def _gamma_constant_adsorption(Da, t):
    """Sec. 4.3.1 closed form for the interfacial concentration."""
    return (math.exp(Da * Da * t) * erfc(Da * math.sqrt(t)) - 1.0
            + 2.0 * Da * math.sqrt(t) / math.sqrt(math.pi)) / Da


def _run_e3a(ny, t_end=0.5, dt=1e-3):
    Da = PAPER["e3a_Da"]
    g, Cf, y = _flat(ny)
    big = 1e8   # J = r_a F_s Gamma_inf: the Langmuir law with Gamma << Gamma_inf
    p = W.Params(ka=Da / big, kd=0.0, gamma_inf=big, Df=1.0, DF=1.0, eps=4 * g.h)
    _, phi, delta = oracle.phase_field_build(g, Cf, 200, 0.5 * g.h, p.eps)
    f, F = np.zeros(g.shape), phi.copy()
    n = int(round(t_end / dt))
    for _ in range(n):
        f, F, st = oracle.surfactant_step(g, p, phi, f, F, dt, 1e-12)
        assert st.converged
    G = oracle.total(g, f) / oracle.total(g, delta)
    return G, _gamma_constant_adsorption(Da, n * dt)


def test_constant_adsorption_converges_to_closed_form():
    """E3a (Sec. 4.3.1): Gamma(t) -> the erfc closed form as eps -> 0."""
    e1 = [abs(a - b) / b for a, b in [_run_e3a(128)]][0]
    e2 = [abs(a - b) / b for a, b in [_run_e3a(256)]][0]
    assert e2 < 0.1 and e2 < 0.6 * e1, (e1, e2)


def test_pure_desorption_exact_discrete_decay_and_bulk_profile():
    """E3b (Sec. 4.3.2).  With r_a = 0 the f problem is linear and its flux
    form telescopes, so implicit Euler gives sum V f = M0 (1 + r_d dt)^-n
    exactly; Gamma = exp(-Bi t) is its dt -> 0 limit, and the released
    surfactant enters the bulk side with the closed-form profile."""
    Bi = PAPER["e3b_Bi"]
    ny, dt, n = 256, 1e-3, 500
    g, Cf, y = _flat(ny)
    p = W.Params(ka=0.0, kd=Bi, gamma_inf=1.0, Df=1.0, DF=1.0, eps=4 * g.h)
    _, phi, delta = oracle.phase_field_build(g, Cf, 200, 0.5 * g.h, p.eps)
    f, F = delta.copy(), np.zeros(g.shape)
    M0 = oracle.total(g, f)
    for _ in range(n):
        f, F, st = oracle.surfactant_step(g, p, phi, f, F, dt, 1e-13)
    Mf = oracle.total(g, f)
    assert abs(Mf / M0 - (1 + Bi * dt) ** -n) < 1e-10
    assert abs(Mf / M0 - math.exp(-Bi * n * dt)) < 1e-3
    # total conserved: what left the interface is in the bulk
    assert abs(oracle.total(g, F) + Mf - M0) < 1e-11 * M0   # 500 steps at tol 1e-13
    t = n * dt

    def F_exact(yy):
        v, _ = quad(lambda tau: math.exp(Bi * tau - yy * yy / (4 * tau)) / math.sqrt(tau), 0, t)
        return Bi * math.exp(-Bi * t) * v / math.sqrt(math.pi)

    for yy in (1.0, 1.5):
        j = int(np.argmin(np.abs(y - yy)))
        assert abs(F[0, j, 0] - F_exact(y[j])) < 0.1 * F_exact(y[j])
        jm = int(np.argmin(np.abs(y + yy)))
        assert F[0, jm, 0] < 0.01 * F[0, j, 0]   # nothing goes into fluid 1


def test_langmuir_equilibrium():
    """E3c (Sec. 4.3.3): with a reservoir that barely depletes, Gamma relaxes
    to Gamma_inf r_a F / (r_a F + r_d) = Da/(Da + Bi)."""
    ny = 64
    g, Cf, y = _flat(ny)
    ka, kd = 2.0, 1.0
    p = W.Params(ka=ka, kd=kd, gamma_inf=0.01, Df=1.0, DF=1.0, eps=4 * g.h)
    _, phi, delta = oracle.phase_field_build(g, Cf, 200, 0.5 * g.h, p.eps)
    f, F = np.zeros(g.shape), phi.copy()
    for _ in range(400):
        f, F, st = oracle.surfactant_step(g, p, phi, f, F, 1e-2, 1e-13)
    G = oracle.total(g, f) / oracle.total(g, delta) / p.gamma_inf
    assert abs(G - ka / (ka + kd)) < 0.02


def _c0_small(n=32):
    c = W.case_adsorption_2d(n=n, steps=10)
    g, p = c.grid, c.params
    _, phi, delta = oracle.phase_field_build(g, c.C, 24, c.dtau, p.eps)
    return c, g, p, phi, delta


def test_total_surfactant_conserved_to_round_off():
    """No-flux walls: sum V (f + F) is invariant (Sec. 3.2 flux form; the
    source enters the two equations with opposite signs, App. C)."""
    c, g, p, phi, delta = _c0_small(32)
    f, F = np.zeros(g.shape), c.F0.copy()
    M0 = oracle.total(g, f) + oracle.total(g, F)
    for _ in range(10):
        f, F, st = oracle.surfactant_step(g, p, phi, f, F, c.dt, 1e-13)
        assert st.converged
    M = oracle.total(g, f) + oracle.total(g, F)
    assert abs(M - M0) < 1e-12 * M0
    assert f.sum() > 0 and F.min() > -1e-12


def test_converged_step_solves_appendix_c_system():
    """The returned state makes both App. C residuals vanish."""
    c, g, p, phi, delta = _c0_small(24)
    f0, F0 = 0.3 * delta, c.F0.copy()
    f, F, st = oracle.surfactant_step(g, p, phi, f0, F0, c.dt, 1e-13)
    _, _, rf, rF = oracle.coupled_residual(g, p, phi, f0, F0, c.dt, f, F)
    assert rf < 1e-13 and rF < 1e-13
    assert st.picard >= 2


def test_equilibrium_interface_profile_is_nearly_steady():
    """Without flow or kinetics, f = Gamma0 delta_phi is the zero-flux profile
    of the f equation (its drift balances diffusion, Sec. 2.6); the discrete
    profile (first-order upwind drift at eps = 0.75 h) relaxes to a nearby
    discrete equilibrium, moving the peak by about 11 % in 50 steps."""
    c, g, p, phi, delta = _c0_small(48)
    p.ka = p.kd = 0.0
    f, F = 0.5 * delta, np.zeros(g.shape)
    for _ in range(50):
        f, F, st = oracle.surfactant_step(g, p, phi, f, F, 1e-3, 1e-13)
    rel = np.abs(f - 0.5 * delta).max() / (0.5 * delta).max()
    assert rel < 0.15
    # with the drift switched off the same profile spreads much further
    p2 = W.Params(**{**p.__dict__})
    p2.eps = 1e6   # B = -D 2(0.5 - phi)/eps n -> 0
    f2, F2 = 0.5 * delta, np.zeros(g.shape)
    for _ in range(50):
        f2, F2, st = oracle.surfactant_step(g, p2, phi, f2, F2, 1e-3, 1e-13)
    rel2 = np.abs(f2 - 0.5 * delta).max() / (0.5 * delta).max()
    assert rel2 > 3 * rel


def _flat_in(geom, ny):
    """The flat interface y = 0 of `_flat` on a planar, axisymmetric (r
    along x, z along y) or 3D block of a few columns."""
    h = 2 * L / ny
    nx, nz = (4, 1) if geom == W.AXI else ((2, 1) if geom == W.PLANAR else (2, 3))
    g = W.Grid(geom, nx, ny, nz, h)
    y = -L + (np.arange(ny) + 0.5) * h
    Cf = np.zeros(g.shape)
    Cf[:, y < 0, :] = 1.0
    return g, Cf


def test_axisymmetric_and_3d_steps_reduce_to_the_planar_column():
    """A flat interface normal to y makes every field independent of the
    other coordinates: the axisymmetric block (the interface normal to the
    axis, so every ring carries the column's fields, the area weights of
    the axial faces cancelling the ring volumes) and the 3D block reproduce
    the planar column, to round-off, through redistancing, drifts, the
    App. C source and the implicit solve."""
    ny, dt, steps = 48, 2e-3, 6
    cols = {}
    for geom in (W.PLANAR, W.AXI, W.CART3D):
        g, Cf = _flat_in(geom, ny)
        p = W.Params(ka=2.0, kd=0.5, gamma_inf=1.0, Df=0.3, DF=1.0, eps=2 * g.h)
        dtau = g.h / 3 if geom == W.CART3D else 0.5 * g.h
        _, phi, delta = oracle.phase_field_build(g, Cf, 200, dtau, p.eps)
        f, F = 0.2 * delta, phi.copy()
        for _ in range(steps):
            f, F, st = oracle.surfactant_step(g, p, phi, f, F, dt, 1e-13)
            assert st.converged
        cols[geom] = (phi, f, F)
    ref = [a[0, :, 0] for a in cols[W.PLANAR]]
    assert ref[1].max() > 1e-3   # the interface took up surfactant
    for geom in (W.AXI, W.CART3D):
        for a, r in zip(cols[geom], ref):
            scale = np.abs(r).max()
            dev = np.abs(a - r[None, :, None]).max()
            assert dev <= 1e-12 * scale, (geom, dev / scale)
