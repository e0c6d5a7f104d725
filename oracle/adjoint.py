"""FP64 oracle of the discrete adjoint of the coupled surfactant step.

TEST INFRASTRUCTURE, like the rest of this package: only the tests, the
smoke check and the benchmark's CPU leg use it.

The paper has no adjoint; the gradient it stands for is fixed by the
forward scheme alone.  One step without flow solves R(x1; x0, theta) = 0 for
x1 = (f, F), where R = b - L(a) is the App. C residual of both equations
(the oracle's own coupled_residual) and x0 enters through f* = f^n,
F* = F^n.  By the implicit function theorem a loss gradient g1 = dL/dx1
pulls back as

    J^T mu = g1,   J = dR/dx1,   g0 = -(dR/dx0)^T mu,   dL/dtheta = -(dR/dtheta)^T mu,

theta = (k_a, k_d, D_f, D_F).  Every derivative of R is taken here by
differences of the oracle residual: central ones in x1 and x0, forward ones
in theta.  R is quadratic in x1 (the exchange term is bilinear in f and F)
and linear in x0 and in each of the four parameters while they keep their
sign (D_f scales both the diffusion and the drift B_f of Sec. 2.3, and the
upwind side depends only on the sign of B), so these differences are exact
up to round-off.  The matrices are dense, which limits this oracle to grids
of a few hundred cells.

The loss is the paper's Marangoni force measured in the mean-square sense,
L = sum_c V_c |F_Ma,c|^2 (Sec. 2.3, with sigma(Gamma) of the chosen EOS),
and its gradient in f is taken by central differences of the oracle force.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import cell_volumes, coupled_residual, marangoni, phase_field_build, surfactant_step

THETA = ("ka", "kd", "Df", "DF")


def _R(g, p, phi, fstar, Fstar, dt, f, F):
    rf, rF, _, _ = coupled_residual(g, p, phi, fstar, Fstar, dt, f, F)
    return np.concatenate([rf.ravel(), rF.ravel()])


def step_jacobians(g, p, phi, f1, F1, dt):
    """(J, R0, Rtheta): dR/dx1 (2N x 2N), dR/dx0 (2N x 2N) and dR/dtheta
    (2N x 4) at the state after the step."""
    N = f1.size
    x = np.concatenate([f1.ravel(), F1.ravel()])
    shp = f1.shape

    def split(v):
        return v[:N].reshape(shp), v[N:].reshape(shp)

    J = np.empty((2 * N, 2 * N))
    R0 = np.empty((2 * N, 2 * N))
    # x0 only enters as f*, F*; any value gives the same derivative
    x0 = x.copy()
    for j in range(2 * N):
        e = np.zeros(2 * N)
        e[j] = 1.0
        fp, Fp = split(x + e)
        fm, Fm = split(x - e)
        f0, F0 = split(x0)
        J[:, j] = 0.5 * (_R(g, p, phi, f0, F0, dt, fp, Fp) - _R(g, p, phi, f0, F0, dt, fm, Fm))
        sp, Sp = split(x0 + e)
        sm, Sm = split(x0 - e)
        f1_, F1_ = split(x)
        R0[:, j] = 0.5 * (_R(g, p, phi, sp, Sp, dt, f1_, F1_) - _R(g, p, phi, sm, Sm, dt, f1_, F1_))
    # R is linear in each parameter while it keeps its sign (a diffusivity
    # of the other sign would turn the drift and its upwind side round), so
    # a forward difference on [v, v + s] with v >= 0 is exact
    Rt = np.empty((2 * N, len(THETA)))
    f0, F0 = split(x0)
    R1 = _R(g, p, phi, f0, F0, dt, f1, F1)
    for k, name in enumerate(THETA):
        v = getattr(p, name)
        if v < 0:
            raise ValueError("parameters of the step are non-negative")
        step = max(v, 1e-3)
        pp = dataclasses.replace(p, **{name: v + step})
        Rt[:, k] = (_R(g, pp, phi, f0, F0, dt, f1, F1) - R1) / step
    return J, R0, Rt


def adjoint_step(g, p, phi, f1, F1, dt, gf1, gF1):
    """Pull (dL/df1, dL/dF1) back through one step: returns
    (dL/df0, dL/dF0, dL/dtheta contribution of this step)."""
    J, R0, Rt = step_jacobians(g, p, phi, f1, F1, dt)
    g1 = np.concatenate([gf1.ravel(), gF1.ravel()])
    mu = np.linalg.solve(J.T, g1)
    g0 = -R0.T @ mu
    N = f1.size
    return g0[:N].reshape(f1.shape), g0[N:].reshape(f1.shape), -Rt.T @ mu


def loss(g, p, f, phi, Cf, dm_mode=1):
    """L = sum_c V_c |F_Ma,c|^2."""
    _, force = marangoni(g, p, f, phi, Cf, dm_mode)
    V = cell_volumes(g)
    return float((V[None] * force * force).sum())


def loss_grad(g, p, f, phi, Cf, dm_mode=1, rel=1e-6):
    """dL/df by central differences, cell by cell (step rel * max|f|)."""
    h = rel * max(np.abs(f).max(), 1e-12)
    out = np.empty_like(f)
    it = np.nditer(f, flags=["multi_index"])
    for _ in it:
        i = it.multi_index
        fp = f.copy()
        fm = f.copy()
        fp[i] += h
        fm[i] -= h
        out[i] = (loss(g, p, fp, phi, Cf, dm_mode) - loss(g, p, fm, phi, Cf, dm_mode)) / (2 * h)
    return out


def rollout(g, p, phi, gamma0, F0, dt, nsteps, tol):
    """Forward states x^0 .. x^nsteps of the no-flow rollout from
    f0 = Gamma0 delta_phi (Sec. 2.3)."""
    delta = phi * (1.0 - phi) / p.eps
    f, F = gamma0 * delta, F0.copy()
    xs = [(f.copy(), F.copy())]
    for _ in range(nsteps):
        f, F, st = surfactant_step(g, p, phi, f, F, dt, tol)
        if not st.converged:
            raise RuntimeError("oracle step did not converge")
        xs.append((f.copy(), F.copy()))
    return xs


def rollout_loss(g, p, phi, Cf, gamma0, F0, dt, nsteps, tol, dm_mode=1):
    f, _ = rollout(g, p, phi, gamma0, F0, dt, nsteps, tol)[-1]
    return loss(g, p, f, phi, Cf, dm_mode)


def rollout_gradient(g, p, phi, Cf, gamma0, F0, dt, nsteps, tol, dm_mode=1):
    """(L, dL/dGamma0, dL/dtheta) by the step adjoints above."""
    xs = rollout(g, p, phi, gamma0, F0, dt, nsteps, tol)
    fN = xs[-1][0]
    L = loss(g, p, fN, phi, Cf, dm_mode)
    gf = loss_grad(g, p, fN, phi, Cf, dm_mode)
    gF = np.zeros_like(gf)
    dtheta = np.zeros(len(THETA))
    for n in range(nsteps - 1, -1, -1):
        f1, F1 = xs[n + 1]
        gf, gF, dt_ = adjoint_step(g, p, phi, f1, F1, dt, gf, gF)
        dtheta += dt_
    delta = phi * (1.0 - phi) / p.eps
    return L, gf * delta, dtheta


def small_case(n=8, seed=4, eps_cells=0.75):
    """A small no-flow adsorption case (circle R = 0.3 n h in a unit box)
    for the dense adjoint: (grid, params, C, phi, Gamma0, F0)."""
    import workloads as W
    h = 1.0 / n
    g = W.Grid(W.PLANAR, n, n, 1, h)
    Cf = W.circle_vof(n, n, h, 0.5, 0.5, 0.3)
    p = W.Params(ka=1.0, kd=0.1, gamma_inf=1.0, Df=1e-2, DF=1e-2, eps=eps_cells * h,
                 sigma0=1.0, E=0.2)
    _, phi, _ = phase_field_build(g, Cf, 24, 0.5 * h, p.eps)
    rng = np.random.default_rng(seed)
    gamma0 = 0.05 * (1.0 + rng.uniform(-1, 1, g.shape))
    F0 = 1.0 - Cf
    return g, p, Cf, phi, gamma0, F0
