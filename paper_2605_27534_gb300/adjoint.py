"""Differentiable no-flow rollout of the coupled surfactant step.

SurfactantRollout is a torch.autograd.Function: its forward runs `nsteps`
steps of the App. C step from f0 = Gamma0 delta_phi (Sec. 2.3) and returns
the loss L = sum_c V_c |F_Ma,c|^2 of the final Marangoni force; its backward
is the hand-written discrete adjoint of the library (sfx_adjoint_step,
sfx_marangoni_loss, sfx_f_from_gamma), giving dL/dGamma0 and dL/dtheta for
theta = (k_a, k_d, D_f, D_F).  The forward keeps a checkpoint of the state
every K steps; the backward recomputes each segment of K steps from its
checkpoint and walks it backwards.  The forward may run in an SFX_F32
context (double-float state); the adjoint always works in FP64 on the
recomputed states.  Every step of the computation runs in libsfx kernels.
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import torch

from ._lib import SFX_F32, SFX_F64, Params


@dataclasses.dataclass
class RolloutSetup:
    """Everything of the rollout that is not differentiated."""
    context: object            # Context of the grid (SFX_F64 or SFX_F32)
    params: object             # base sfx_params-like object (theta overrides 4 fields)
    phi: torch.Tensor          # double phase field
    C: torch.Tensor            # VoF fraction (double) for delta_m
    F0: torch.Tensor           # initial bulk concentration (double)
    dt: float
    nsteps: int
    K: int = 20                # checkpoint interval
    tol: float = 1e-12         # forward solve tolerance
    adj_tol: float = 1e-13     # adjoint solve tolerance
    dm_mode: int = 1
    opts: Optional[object] = None

    def params_with(self, theta):
        from . import params_struct
        ps = params_struct(self.params)
        ps.ka, ps.kd, ps.Df, ps.DF = (float(v) for v in theta)
        return ps


def _forward_steps(setup: RolloutSetup, ps: Params, f, F, n):
    """n steps from (f, F) in the context's state layout, in place."""
    from . import default_opts
    ctx = setup.context
    o = setup.opts if setup.opts is not None else default_opts(tol=setup.tol, max_cycles=400)
    for _ in range(n):
        # no stats: the step then skips its totals and their host wait (a
        # step that fails to converge still raises)
        ctx.sfx_surfactant_step(ps, setup.phi, f, F, setup.dt, opts=o, stats=False)


def _to_state(ctx, x):
    return ctx.sfx_df_pack(x) if ctx.precision == SFX_F32 else x.clone()


def _to_double(ctx, x):
    return ctx.sfx_df_unpack(x) if ctx.precision == SFX_F32 else x


class SurfactantRollout(torch.autograd.Function):
    """loss = SurfactantRollout.apply(gamma0, theta, setup)."""

    @staticmethod
    def forward(fctx, gamma0, theta, setup: RolloutSetup):
        ctx = setup.context
        ps = setup.params_with(theta.detach().cpu().tolist())
        f0 = ctx.sfx_f_from_gamma(gamma0.detach().contiguous(), setup.phi, ps.eps)
        f, F = _to_state(ctx, f0), _to_state(ctx, setup.F0)
        checkpoints = [(f.clone(), F.clone())]
        done = 0
        while done < setup.nsteps:
            n = min(setup.K, setup.nsteps - done)
            _forward_steps(setup, ps, f, F, n)
            done += n
            if done < setup.nsteps:
                checkpoints.append((f.clone(), F.clone()))
        L, _ = ctx.sfx_marangoni_loss(ps, _to_double(ctx, f), setup.phi, setup.C, setup.dm_mode,
                                      grad=False)
        fctx.setup = setup
        fctx.ps = ps
        fctx.checkpoints = checkpoints
        fctx.theta_device = theta.device
        fctx.theta_dtype = theta.dtype
        return torch.tensor(L, dtype=torch.float64)

    @staticmethod
    def backward(fctx, gL):
        from . import default_opts
        setup, ps = fctx.setup, fctx.ps
        ctx = setup.context
        o = default_opts(tol=setup.adj_tol, max_cycles=1000, nu1=10, nu2=10)
        # the final state, for dL/df
        last_f, last_F = (t.clone() for t in fctx.checkpoints[-1])
        rem = setup.nsteps - setup.K * (len(fctx.checkpoints) - 1)
        _forward_steps(setup, ps, last_f, last_F, rem)
        _, gf = ctx.sfx_marangoni_loss(ps, _to_double(ctx, last_f), setup.phi, setup.C,
                                       setup.dm_mode, grad=True)
        lam_f = gf * float(gL)
        lam_F = torch.zeros_like(lam_f)
        dtheta = [0.0, 0.0, 0.0, 0.0]
        for s in range(len(fctx.checkpoints) - 1, -1, -1):
            n = min(setup.K, setup.nsteps - s * setup.K)
            f, F = (t.clone() for t in fctx.checkpoints[s])
            states = []
            for _ in range(n):
                _forward_steps(setup, ps, f, F, 1)
                states.append((_to_double(ctx, f).clone(), _to_double(ctx, F).clone()))
            for f1, F1 in reversed(states):
                ctx.sfx_adjoint_step(ps, setup.phi, f1, F1, setup.dt, lam_f, lam_F, dtheta, o)
        dgamma = ctx.sfx_f_from_gamma(lam_f, setup.phi, ps.eps)
        dth = torch.tensor(dtheta, dtype=fctx.theta_dtype, device=fctx.theta_device)
        return dgamma, dth, None
