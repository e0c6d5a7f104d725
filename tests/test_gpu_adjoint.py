"""GPU adjoint (sfx_adjoint_apply, sfx_adjoint_step, sfx_marangoni_loss,
sfx_f_from_gamma) and the differentiable rollout, against the dense FP64
oracle adjoint, dot-product identities and central finite differences."""

import numpy as np
import pytest

import oracle
from oracle import adjoint as OA
import workloads as W
from gpu_util import dev, host, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sfx():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2605_27534_gb300 as m
    m.lib()
    return m


def _state_case(geom, seed=0):
    """A grid with an interface, a non-trivial state (f, F) and parameters."""
    rng = np.random.default_rng(seed)
    if geom == W.PLANAR:
        n = 10
        g = W.Grid(W.PLANAR, n, n, 1, 1.0 / n)
        Cf = W.circle_vof(n, n, g.h, 0.5, 0.5, 0.3)
    elif geom == W.AXI:
        g = W.Grid(W.AXI, 7, 12, 1, 1.0 / 7)
        Cf = W.ring_vof(7, 12, g.h, 6 * g.h, 0.5)
    else:
        n = 6
        g = W.Grid(W.CART3D, n, n, n, 1.0 / n)
        Cf = W.sphere_vof(n, g.h, (0.5, 0.5, 0.5), 0.3)
    p = W.Params(ka=2.0, kd=0.3, gamma_inf=1.0, Df=0.02, DF=0.05, eps=0.75 * g.h,
                 sigma0=1.0, E=0.2)
    _, phi, delta = oracle.phase_field_build(g, Cf, 24, 0.5 * g.h if g.ndim == 2 else g.h / 3,
                                             p.eps)
    f = rng.uniform(0.1, 0.5, g.shape) * delta
    F = rng.uniform(0.5, 1.0, g.shape)
    return g, p, Cf, phi, f, F


GEOMS = [W.PLANAR, W.AXI, W.CART3D]


@pytest.mark.parametrize("geom", GEOMS)
def test_adjoint_apply_is_the_transpose_and_matches_the_oracle_jacobian(sfx, geom):
    g, p, Cf, phi, f, F = _state_case(geom)
    dt = 2e-3
    ctx = sfx.Context.for_grid(g, sfx.SFX_F64)
    rng = np.random.default_rng(5)
    v = [rng.standard_normal(g.shape) for _ in range(2)]
    w = [rng.standard_normal(g.shape) for _ in range(2)]
    d = [dev(a) for a in (phi, f, F)]
    Jv = ctx.sfx_adjoint_apply(p, *d, dt, dev(v[0]), dev(v[1]))
    JTw = ctx.sfx_adjoint_apply(p, *d, dt, dev(w[0]), dev(w[1]), transpose=True)
    Jv = [host(t) for t in Jv]
    JTw = [host(t) for t in JTw]
    lhs = (Jv[0] * w[0]).sum() + (Jv[1] * w[1]).sum()
    rhs = (v[0] * JTw[0]).sum() + (v[1] * JTw[1]).sum()
    scale = sum(np.abs(Jv[k] * w[k]).sum() for k in range(2))
    assert abs(lhs - rhs) <= 1e-13 * scale
    # against -J of the oracle, formed from its own residual
    J, _, _ = OA.step_jacobians(g, p, phi, f, F, dt)
    want = -J @ np.concatenate([v[0].ravel(), v[1].ravel()])
    got = np.concatenate([Jv[0].ravel(), Jv[1].ravel()])
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()


@pytest.mark.parametrize("geom", GEOMS)
def test_adjoint_step_matches_the_oracle(sfx, geom):
    g, p, Cf, phi, f, F = _state_case(geom, seed=1)
    dt = 2e-3
    rng = np.random.default_rng(6)
    lf, lF = rng.standard_normal(g.shape), rng.standard_normal(g.shape)
    gf0, gF0, dth = OA.adjoint_step(g, p, phi, f, F, dt, lf, lF)
    ctx = sfx.Context.for_grid(g, sfx.SFX_F64)
    lfd, lFd = dev(lf), dev(lF)
    dp = [0.0] * 4
    st = ctx.sfx_adjoint_step(p, dev(phi), dev(f), dev(F), dt, lfd, lFd, dp,
                              sfx.default_opts(tol=1e-14, max_cycles=2000, nu1=4, nu2=4))
    assert st.converged
    assert rel_err(host(lfd), gf0) < 1e-11
    assert rel_err(host(lFd), gF0) < 1e-11
    for k in range(4):
        assert abs(dp[k] - dth[k]) <= 1e-10 * max(abs(dth[k]), 1e-3 * np.abs(dth).max()), k


def test_adjoint_relaxation_graph_follows_the_sweep_count(sfx):
    """The relaxation of a check is a graph captured per context and sweep
    count: a context that changes nu1 + nu2 between steps (recapturing)
    gives bitwise the results of fresh contexts, and the same sweep count
    again gives the same bits as the first call."""
    g, p, Cf, phi, f, F = _state_case(W.AXI, seed=2)
    dt = 2e-3
    rng = np.random.default_rng(7)
    lf, lF = rng.standard_normal(g.shape), rng.standard_normal(g.shape)
    d = [dev(a) for a in (phi, f, F)]

    def run(ctx, nu):
        a, b = dev(lf), dev(lF)
        dp = [0.0] * 4
        st = ctx.sfx_adjoint_step(p, *d, dt, a, b, dp,
                                  sfx.default_opts(tol=1e-13, max_cycles=2000, nu1=nu, nu2=nu))
        assert st.converged and st.vcycles % (2 * nu) == 0
        return host(a), host(b), dp

    shared = sfx.Context.for_grid(g, sfx.SFX_F64)
    got = [run(shared, nu) for nu in (3, 7, 3)]
    for nu, r in zip((3, 7, 3), got):
        ref = run(sfx.Context.for_grid(g, sfx.SFX_F64), nu)
        assert np.array_equal(r[0], ref[0]) and np.array_equal(r[1], ref[1]), nu
        assert r[2] == ref[2], nu
    assert np.array_equal(got[0][0], got[2][0]) and got[0][2] == got[2][2]
    # different sweep counts reach the same adjoint within the tolerance
    assert rel_err(got[1][0], got[0][0]) < 1e-10


def test_adjoint_step_reports_the_checks_it_ran(sfx):
    """With too few checks the step stops after max_cycles of them
    (SFX_ERR_NOT_CONVERGED, relaxations between them only), and with enough
    it stops at the first check that passes: running it again with that
    check as the limit gives the same bits."""
    import ctypes as C
    g, p, Cf, phi, f, F = _state_case(W.PLANAR, seed=3)
    dt = 2e-3
    rng = np.random.default_rng(8)
    lf, lF = rng.standard_normal(g.shape), rng.standard_normal(g.shape)
    d = [dev(a) for a in (phi, f, F)]
    ctx = sfx.Context.for_grid(g, sfx.SFX_F64)
    ps = sfx.params_struct(p)

    def raw(max_cycles, nu=3):
        a, b = dev(lf), dev(lF)
        o = sfx.default_opts(tol=1e-13, max_cycles=max_cycles, nu1=nu, nu2=nu)
        st = sfx.StepStats()
        dp = (C.c_double * 4)()
        code = sfx.lib().sfx_adjoint_step(ctx.handle, C.byref(ps), sfx._ptr(d[0]),
                                          sfx._ptr(d[1]), sfx._ptr(d[2]), float(dt), sfx._ptr(a),
                                          sfx._ptr(b), dp, C.byref(o), C.byref(st),
                                          sfx._stream())
        return code, st, host(a), host(b), list(dp)

    code, st, *_ = raw(2)
    assert code == sfx.SFX_ERR_NOT_CONVERGED
    assert (st.picard, st.vcycles, st.converged) == (2, 6, 0) and st.res_f > 1e-13
    code, st, a1, b1, dp1 = raw(1000)
    assert code == sfx.SFX_OK and st.converged and st.res_f <= 1e-13
    assert st.vcycles == (st.picard - 1) * 6
    code, st2, a2, b2, dp2 = raw(st.picard)
    assert code == sfx.SFX_OK and st2.picard == st.picard and st2.vcycles == st.vcycles
    assert np.array_equal(a1, a2) and np.array_equal(b1, b2) and dp1 == dp2


@pytest.mark.parametrize("geom", [W.PLANAR, W.AXI])
def test_marangoni_loss_and_gradient_match_the_oracle(sfx, geom):
    g, p, Cf, phi, f, F = _state_case(geom, seed=2)
    L_o = OA.loss(g, p, f, phi, Cf)
    gf_o = OA.loss_grad(g, p, f, phi, Cf)
    ctx = sfx.Context.for_grid(g, sfx.SFX_F64)
    L, gf = ctx.sfx_marangoni_loss(p, dev(f), dev(phi), dev(Cf))
    assert abs(L - L_o) <= 1e-12 * L_o
    assert rel_err(host(gf), gf_o) < 1e-7


def test_f_from_gamma(sfx):
    g, p, Cf, phi, f, F = _state_case(W.PLANAR)
    gam = np.random.default_rng(3).uniform(0, 1, g.shape)
    ctx = sfx.Context.for_grid(g, sfx.SFX_F64)
    out = host(ctx.sfx_f_from_gamma(dev(gam), dev(phi), p.eps))
    np.testing.assert_allclose(out, gam * phi * (1 - phi) / p.eps, rtol=1e-15, atol=0)


def _setup(sfx, case, precision, nsteps, K, dt=1e-3):
    import torch
    g, p, Cf, phi, gamma0, F0 = case
    ctx = sfx.Context.for_grid(g, precision)
    setup = sfx.RolloutSetup(context=ctx, params=p, phi=dev(phi), C=dev(Cf), F0=dev(F0), dt=dt,
                             nsteps=nsteps, K=K, tol=1e-13 if precision == 0 else 1e-12)
    theta = torch.tensor([p.ka, p.kd, p.Df, p.DF], dtype=torch.float64, requires_grad=True)
    g0 = dev(gamma0).requires_grad_(True)
    return setup, theta, g0


@pytest.mark.parametrize("precision,tol", [(0, 1e-7), (1, 1e-6)])
def test_rollout_gradient_matches_the_oracle_adjoint(sfx, precision, tol):
    """8x8, 6 steps with checkpoints every 4: the autograd gradient against
    the dense oracle adjoint, whose loss gradient is itself a central
    difference (FP64 forward: 1e-7; FP32 forward: 1e-6)."""
    case = OA.small_case(n=8)
    g, p, Cf, phi, gamma0, F0 = case
    L_o, dG_o, dth_o = OA.rollout_gradient(g, p, phi, Cf, gamma0, F0, 1e-3, 6, 1e-14)
    setup, theta, g0 = _setup(sfx, case, precision, 6, 4)
    L = sfx.SurfactantRollout.apply(g0, theta, setup)
    L.backward()
    assert abs(L.item() - L_o) <= tol * L_o
    assert rel_err(host(g0.grad), dG_o) < tol
    for k in range(4):
        assert abs(theta.grad[k].item() - dth_o[k]) <= tol * abs(dth_o[k]), k


@pytest.mark.parametrize("precision,tol", [(0, 1e-6), (1, 5e-6)])
def test_rollout_gradient_at_full_size_matches_finite_differences(sfx, precision, tol):
    """The 2D adjoint workload: 256^2 no-flow adsorption with a seeded Gamma0
    perturbation, 200 steps, checkpoints every 20, loss sum V |F_Ma|^2.
    Gradients against central differences of the FP64 GPU forward (relative
    step 1e-4) for the four parameters and one Gamma0 direction: 1e-6 for
    the FP64 forward.  The FP32 forward rounds D/h and the drifts to float
    (6e-8 relative), which moves dL/dD_f of its own model by ~2e-6 from the
    FP64 model's; it is held to 5e-6."""
    import torch
    c = W.case_adjoint_2d(n=256)
    g, p = c.grid, c.params
    _, phi, _ = oracle.phase_field_build(g, c.C, c.redist_iters, c.dtau, p.eps)
    case = (g, p, c.C, phi, c.gamma0, c.F0)
    setup, theta, g0 = _setup(sfx, case, precision, 200, 20)
    L = sfx.SurfactantRollout.apply(g0, theta, setup)
    L.backward()
    fd_setup, _, _ = _setup(sfx, case, 0, 200, 200)

    def loss_at(th, gam):
        with torch.no_grad():
            return sfx.SurfactantRollout.apply(gam, th, fd_setup).item()

    base = torch.tensor([p.ka, p.kd, p.Df, p.DF], dtype=torch.float64)
    for k in range(4):
        hs = 1e-4 * base[k].item()
        tp, tm = base.clone(), base.clone()
        tp[k] += hs
        tm[k] -= hs
        fd = (loss_at(tp, g0.detach()) - loss_at(tm, g0.detach())) / (2 * hs)
        assert abs(theta.grad[k].item() - fd) <= tol * abs(fd), (k, theta.grad[k].item(), fd)
    v = torch.from_numpy(np.random.default_rng(8).standard_normal(g.shape)).cuda()
    hs = 1e-4 * g0.detach().abs().max().item() / v.abs().max().item()
    fd = (loss_at(base, g0.detach() + hs * v) - loss_at(base, g0.detach() - hs * v)) / (2 * hs)
    got = (g0.grad * v).sum().item()
    assert abs(got - fd) <= tol * abs(fd), (got, fd)
