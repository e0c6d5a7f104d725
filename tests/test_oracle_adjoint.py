"""Pins of the oracle's discrete adjoint (oracle/adjoint.py): the gradient
of the coupled step of App. C, composed over a rollout, against central
finite differences of the oracle forward itself, and one step on a single
cell against the closed form of its quadratic (implicit differentiation of
the root)."""
import dataclasses
import math

import numpy as np
import pytest

import oracle
from oracle import adjoint as A
import workloads as W

DT = 1e-3
TOL = 1e-14


@pytest.fixture(scope="module")
def case():
    return A.small_case(n=8)


def test_rollout_gradient_matches_finite_differences(case):
    g, p, Cf, phi, gamma0, F0 = case
    nsteps = 4
    L, dG, dth = A.rollout_gradient(g, p, phi, Cf, gamma0, F0, DT, nsteps, TOL)
    assert L > 0
    for k, name in enumerate(A.THETA):
        v = getattr(p, name)
        hs = 1e-4 * v
        Lp = A.rollout_loss(g, dataclasses.replace(p, **{name: v + hs}), phi, Cf, gamma0, F0,
                            DT, nsteps, TOL)
        Lm = A.rollout_loss(g, dataclasses.replace(p, **{name: v - hs}), phi, Cf, gamma0, F0,
                            DT, nsteps, TOL)
        fd = (Lp - Lm) / (2 * hs)
        assert abs(dth[k] - fd) <= 1e-6 * abs(fd) + 1e-12 * L, (name, dth[k], fd)
    # Gamma0 along two seeded directions
    rng = np.random.default_rng(7)
    for _ in range(2):
        v = rng.standard_normal(g.shape)
        hs = 1e-4 * np.abs(gamma0).max() / np.abs(v).max()
        Lp = A.rollout_loss(g, p, phi, Cf, gamma0 + hs * v, F0, DT, nsteps, TOL)
        Lm = A.rollout_loss(g, p, phi, Cf, gamma0 - hs * v, F0, DT, nsteps, TOL)
        fd = (Lp - Lm) / (2 * hs)
        got = float((dG * v).sum())
        assert abs(got - fd) <= 1e-6 * abs(fd), (got, fd)


def test_single_cell_step_adjoint_matches_closed_form():
    """One cell has no transport: the step conserves S = f + F and solves
    P(f) = c1 f^2 - B f + c1 S f_inf + f0/dt = 0 with B = c1 (S + f_inf) +
    k_d + 1/dt, c1 = k_a/(phi + eta).  Implicit differentiation of the
    physical (smaller) root gives df/dk_a, df/dk_d, df/df0, df/dF0."""
    g = W.Grid(W.PLANAR, 1, 1, 1, 0.1)
    p = W.Params(ka=3.0, kd=0.7, gamma_inf=1.0, Df=1e-2, DF=2e-2, eps=0.075)
    phi = np.full(g.shape, 0.3)
    f0, F0 = np.full(g.shape, 0.4), np.full(g.shape, 0.8)
    dt = 0.05
    f1, F1, st = oracle.surfactant_step(g, p, phi, f0, F0, dt, 1e-15)
    assert st.converged
    c1 = p.ka / (0.3 + p.eta)
    finf = p.gamma_inf * 0.3 * 0.7 / p.eps
    S = 0.4 + 0.8
    B = c1 * (S + finf) + p.kd + 1 / dt
    C0 = c1 * S * finf + 0.4 / dt
    f = (B - math.sqrt(B * B - 4 * c1 * C0)) / (2 * c1)
    assert abs(f1.item() - f) < 1e-12 * f
    dPdf = 2 * c1 * f - B
    want = {
        "ka": -((S - f) * (finf - f) / (0.3 + p.eta)) / dPdf,
        "kd": f / dPdf,
        "f0": -(1 / dt + c1 * (finf - f)) / dPdf,
        "F0": -(c1 * (finf - f)) / dPdf,
    }
    # L = f1: dL/df1 = 1, dL/dF1 = 0
    gf0, gF0, dth = A.adjoint_step(g, p, phi, f1, F1, dt, np.ones(g.shape), np.zeros(g.shape))
    assert abs(dth[0] - want["ka"]) < 1e-10 * abs(want["ka"])
    assert abs(dth[1] - want["kd"]) < 1e-10 * abs(want["kd"])
    assert dth[2] == 0.0 and dth[3] == 0.0      # no interior faces
    assert abs(gf0.item() - want["f0"]) < 1e-10 * abs(want["f0"])
    assert abs(gF0.item() - want["F0"]) < 1e-10 * abs(want["F0"])
    # L = F1 = S - f1: the same derivatives with the opposite sign, plus 1
    # for the initial values
    gf0, gF0, dth = A.adjoint_step(g, p, phi, f1, F1, dt, np.zeros(g.shape), np.ones(g.shape))
    assert abs(dth[0] + want["ka"]) < 1e-10 * abs(want["ka"])
    assert abs(gf0.item() - (1 - want["f0"])) < 1e-10
    assert abs(gF0.item() - (1 - want["F0"])) < 1e-10


def test_loss_gradient_of_the_marangoni_force(case):
    """dL/df by differences against the exact change of L along a
    direction (second-order consistent)."""
    g, p, Cf, phi, gamma0, F0 = case
    f = gamma0 * phi * (1 - phi) / p.eps
    gf = A.loss_grad(g, p, f, phi, Cf)
    rng = np.random.default_rng(3)
    v = rng.standard_normal(g.shape) * f
    for hs in (1e-4, 5e-5):
        d = (A.loss(g, p, f + hs * v, phi, Cf) - A.loss(g, p, f - hs * v, phi, Cf)) / (2 * hs)
        assert abs(d - (gf * v).sum()) <= 1e-7 * abs(d)
