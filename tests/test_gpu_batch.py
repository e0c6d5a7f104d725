"""Batched SFX_F32 step (sfx_batch_*): axisymmetric instances of uneven
sizes (odd radial counts included) and per-instance Bi, Da stepped together
in one graph launch per step.  Checked per instance against the FP64 oracle
(Sec. 3.1 advection, App. C coupled system), bitwise against single-grid
SFX_F32 steps under the same fixed iteration budget, for conservation in a
closed box, and for the graph cache and the autotuner."""
import numpy as np
import pytest

import oracle
import workloads as W
from gpu_util import dev, host

pytestmark = pytest.mark.gpu

F32_TOL = 1e-5        # FP32 path against the FP64 oracle (normwise)
SPECS = [(16, 32), (32, 64), (17, 40), (24, 48), (9, 20)]


@pytest.fixture(scope="module")
def sfx():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2605_27534_gb300 as m
    m.lib()
    return m


def _instances(seed=11, steps=3):
    rng = np.random.default_rng(seed)
    out = []
    for k, (nr, nz) in enumerate(SPECS):
        Bi, Da = 10.0 ** rng.uniform(-2, 2, size=2)
        c = W.case_axi(nr, nz, Bi=Bi, Da=Da, steps=steps)
        _, phi, delta = oracle.phase_field_build(c.grid, c.C, c.redist_iters, c.dtau, c.params.eps)
        f0 = (0.3 * (k % 2)) * delta
        out.append((c, phi, f0))
    return out


def _pack(arrs):
    return np.concatenate([np.ascontiguousarray(a).ravel() for a in arrs])


class _Batch:
    """Device arrays of a batch built from _instances()."""

    def __init__(self, sfx, inst, flow=True, geom=None):
        import torch
        self.inst = inst
        self.b = sfx.Batch([(c.grid.nx, c.grid.ny, c.grid.h, c.dt, c.params) for c, _, _ in inst],
                           geom=geom)
        nc, nrf, nzf, co, ro, zo = self.b.sfx_batch_layout()
        self.co = co
        assert nc == sum(c.grid.nx * c.grid.ny for c, _, _ in inst)
        assert nrf == sum((c.grid.nx + 1) * c.grid.ny for c, _, _ in inst)
        assert nzf == sum(c.grid.nx * (c.grid.ny + 1) for c, _, _ in inst)
        self.phi = dev(_pack([p for _, p, _ in inst]))
        self.f = sfx.sfx_df_pack(dev(_pack([f0 for _, _, f0 in inst])))
        self.F = sfx.sfx_df_pack(dev(_pack([c.F0 for c, _, _ in inst])))
        if flow:
            self.ur = dev(_pack([c.ux for c, _, _ in inst]), torch.float32)
            self.uz = dev(_pack([c.uy for c, _, _ in inst]), torch.float32)
        else:
            self.ur = self.uz = None

    def step(self, tol, f=None, F=None):
        self.b.sfx_batch_step(self.phi, self.f if f is None else f, self.F if F is None else F,
                              tol, ur=self.ur, uz=self.uz)

    def fields(self, sfx, f=None, F=None):
        fh = host(sfx.sfx_df_unpack(self.f if f is None else f))
        Fh = host(sfx.sfx_df_unpack(self.F if F is None else F))
        out = []
        for (c, _, _), o in zip(self.inst, self.co):
            n = c.grid.nx * c.grid.ny
            out.append((fh[o:o + n].reshape(c.grid.shape), Fh[o:o + n].reshape(c.grid.shape)))
        return out


def test_batch_matches_oracle_per_instance(sfx):
    inst = _instances()
    B = _Batch(sfx, inst)
    B.b.sfx_batch_set_schedule(256, 3, 60)
    for _ in range(3):
        B.step(1e-10)
        st = B.b.sfx_batch_stats()
        assert all(st["converged"]), st
        assert max(st["res_f"]) <= 1e-10 and max(st["res_F"]) <= 1e-10
    got = B.fields(sfx)
    for k, ((c, phi, f0), (fg, Fg)) in enumerate(zip(inst, got)):
        f_o, F_o = f0.copy(), c.F0.copy()
        for _ in range(3):
            f_o, F_o, so = oracle.surfactant_step(c.grid, c.params, phi, f_o, F_o, c.dt, 1e-13,
                                                  c.ux, c.uy, None)
            assert so.converged
        scale = max(np.abs(F_o).max(), np.abs(f_o).max())
        assert np.abs(Fg - F_o).max() / scale < F32_TOL, k
        assert np.abs(fg - f_o).max() / scale < F32_TOL, k
        # per-instance compensated totals of the packed state
        V = oracle.cell_volumes(c.grid)
        for m, x in ((st["mass_f"][k], fg), (st["mass_F"][k], Fg)):
            assert abs(m - (V * x).sum()) <= 1e-13 * max(np.abs(V * x).sum(), 1e-300)


@pytest.mark.parametrize("fast", [0, 2])
def test_batch_bitwise_equals_single_grid_steps(sfx, fast):
    """Fixed budget (no instance meets tol = 1e-30): the batched kernels run
    the single-grid SFX_F32 arithmetic cell for cell, with the same number
    of FP32 residual passes (`fast`) before the pair residuals on both
    sides."""
    import torch
    inst = _instances(seed=5)
    B = _Batch(sfx, inst)
    B.b.sfx_batch_set_schedule(128, 2, 4)
    B.b.sfx_batch_set_tuning(sfx._lib.SFX_TUNE_F32_FAST_RESID, fast)
    for _ in range(2):
        B.step(1e-30)
    st = B.b.sfx_batch_stats()
    assert not any(st["converged"]) and set(st["iters"]) == {4}
    got = B.fields(sfx)
    fb = B.f.cpu().numpy()
    Fb = B.F.cpu().numpy()
    o = sfx.default_opts(tol=1e-30, max_cycles=4, nu1=2, nu2=0)
    for k, (c, phi, f0) in enumerate(inst):
        ctx = sfx.Context.for_grid(c.grid, sfx.SFX_F32)
        ctx.sfx_set_tuning(sfx._lib.SFX_TUNE_F32_FAST_RESID, fast)
        f, F = sfx.sfx_df_pack(dev(f0)), sfx.sfx_df_pack(dev(c.F0))
        phid = dev(phi)
        u = [dev(c.ux, torch.float32), dev(c.uy, torch.float32), None]
        for _ in range(2):
            ctx.sfx_surfactant_step(c.params, phid, f, F, c.dt, *u, opts=o,
                                    allow_not_converged=True)
        torch.cuda.synchronize()
        n = c.grid.nx * c.grid.ny
        off = B.co[k]
        assert np.array_equal(f.cpu().numpy().reshape(-1, 2), fb[off:off + n]), k
        assert np.array_equal(F.cpu().numpy().reshape(-1, 2), Fb[off:off + n]), k
    assert len(got) == len(inst)


def test_batch_early_exit_and_closed_box_mass(sfx):
    """No flow: each instance stops at its own iteration count, and the
    total sum V (f + F) of every instance is kept to 1e-10 over 5 steps."""
    inst = _instances(seed=2)
    B = _Batch(sfx, inst, flow=False)
    B.b.sfx_batch_set_schedule(256, 3, 60)
    M0 = None
    seen = set()
    its = np.zeros(len(inst), dtype=np.int64)
    B.b.sfx_batch_work(reset=True)
    for _ in range(5):
        B.step(1e-11)
        st = B.b.sfx_batch_stats()
        assert all(st["converged"])
        assert max(st["res_f"]) <= 1e-11 and max(st["res_F"]) <= 1e-11
        seen.update(st["iters"])
        its += np.array(st["iters"])
        M = np.array(st["mass_f"]) + np.array(st["mass_F"])
        if M0 is None:
            V = [oracle.cell_volumes(c.grid) for c, _, _ in inst]
            M0 = np.array([(v * (f0 + c.F0)).sum() for v, (c, _, f0) in zip(V, inst)])
        assert np.all(np.abs(M - M0) <= 1e-10 * np.abs(M0)), (M - M0) / M0
    assert len(seen) >= 2, seen   # instances converge at different counts
    # work counters: one residual pass per iteration, sweeps after all but
    # the converged one
    rp, sg = B.b.sfx_batch_work()
    assert list(rp) == list(its) and list(sg) == list(its - 5)


def test_batch_fp32_residuals_reach_the_same_fixed_point(sfx):
    """Each instance's first Newton iterations on FP32 residuals (at most
    two, per instance) end on the pair residual's fixed point: every
    instance converges on a pair residual, the states match the pair-only
    batch to far below the FP32 tolerance, and no instance needs more than
    one extra iteration per step."""
    import torch
    inst = _instances(seed=9)
    outs, its = [], []
    for fast in (0, 2):
        B = _Batch(sfx, inst)
        B.b.sfx_batch_set_schedule(256, 3, 60)
        B.b.sfx_batch_set_tuning(sfx._lib.SFX_TUNE_F32_FAST_RESID, fast)
        n = []
        for _ in range(3):
            B.step(1e-10)
            st = B.b.sfx_batch_stats()
            assert all(st["converged"])
            assert max(st["res_f"]) <= 1e-10 and max(st["res_F"]) <= 1e-10
            n.append(np.array(st["iters"]))
        torch.cuda.synchronize()
        its.append(n)
        outs.append((host(sfx.sfx_df_unpack(B.f)), host(sfx.sfx_df_unpack(B.F))))
    for a, b in zip(outs[0], outs[1]):
        assert np.abs(a - b).max() / np.abs(a).max() < 1e-8
    for k, m in zip(its[0], its[1]):
        assert np.all(m <= k + 1), (k, m)


def test_batch_over_relaxation_reaches_the_same_fixed_point(sfx):
    """Over-relaxed red updates (omega per instance from its parameters)
    end on the Gauss-Seidel batch's fixed point: every instance converges,
    the states match far below the FP32 tolerance, and the batch needs no
    more iterations in total."""
    import torch
    inst = _instances(seed=11)
    outs, its = [], []
    for sor in (0, 1):
        B = _Batch(sfx, inst)
        B.b.sfx_batch_set_schedule(256, 2, 60)
        B.b.sfx_batch_set_tuning(sfx._lib.SFX_TUNE_F32_SOR, sor)
        n = 0
        for _ in range(3):
            B.step(1e-10)
            st = B.b.sfx_batch_stats()
            assert all(st["converged"])
            n += sum(st["iters"])
        torch.cuda.synchronize()
        its.append(n)
        outs.append((host(sfx.sfx_df_unpack(B.f)), host(sfx.sfx_df_unpack(B.F))))
    for a, b in zip(outs[0], outs[1]):
        assert np.abs(a - b).max() / np.abs(a).max() < 1e-8
    assert its[1] <= its[0], its


def test_graph_cache_follows_pointers(sfx):
    """A step on other buffers recaptures the graph; results are bitwise
    those of stepping one buffer twice."""
    inst = _instances(seed=7)
    B = _Batch(sfx, inst)
    B.b.sfx_batch_set_schedule(256, 3, 40)
    f2, F2 = B.f.clone(), B.F.clone()
    B.step(1e-10)
    B.step(1e-10)
    B.step(1e-10, f2, F2)
    f3, F3 = f2.clone(), F2.clone()
    B.step(1e-10, f3, F3)
    import torch
    torch.cuda.synchronize()
    assert torch.equal(B.f, f3) and torch.equal(B.F, F3)


def test_static_phi_gives_the_same_steps(sfx):
    """With phi declared static the fold and the drifts run once outside the
    graph; the steps are bitwise those that rebuild them every step."""
    import torch
    inst = _instances(seed=3)
    outs = []
    for reuse in (False, True):
        B = _Batch(sfx, inst)
        B.b.sfx_batch_set_schedule(256, 3, 20)
        B.b.sfx_batch_reuse_phi(reuse)
        for _ in range(3):
            B.step(1e-10)
        torch.cuda.synchronize()
        outs.append((B.f.clone(), B.F.clone()))
    assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1], outs[1][1])


def test_autotune_keeps_state_and_converges(sfx):
    import torch
    inst = _instances(seed=9)
    B = _Batch(sfx, inst)
    f0, F0 = B.f.clone(), B.F.clone()
    block, sweeps, budget = B.b.sfx_batch_autotune(B.phi, B.f, B.F, 1e-10, ur=B.ur, uz=B.uz)
    torch.cuda.synchronize()
    assert torch.equal(B.f, f0) and torch.equal(B.F, F0)
    assert block in (128, 256, 512) and sweeps in (2, 3, 4) and 16 <= budget <= 200
    B.step(1e-10)
    st = B.b.sfx_batch_stats()
    assert all(st["converged"]) and max(st["iters"]) <= budget


def test_batch_rejects_bad_arguments(sfx):
    c, _, _ = _instances()[0]
    with pytest.raises(sfx.SfxError):
        sfx.Batch([(0, 8, 0.1, 1e-3, c.params)])
    with pytest.raises(sfx.SfxError):
        sfx.Batch([(8, 8, 0.1, -1.0, c.params)])
    B = _Batch(sfx, _instances()[:2])
    with pytest.raises(sfx.SfxError):
        B.b.sfx_batch_set_schedule(100, 3, 8)
    with pytest.raises(sfx.SfxError):
        B.b.sfx_batch_set_tuning(sfx._lib.SFX_TUNE_F32_FAST_RESID, 17)
    with pytest.raises(sfx.SfxError):
        B.b.sfx_batch_set_tuning(sfx._lib.SFX_TUNE_TILED_SWEEP, 1)
    with pytest.raises(sfx.SfxError):
        B.b.sfx_batch_set_tuning(sfx._lib.SFX_TUNE_F32_SOR, 2000)
    with pytest.raises(sfx.SfxError):
        B.b.sfx_batch_step(B.phi, B.f, B.F, 1e-10, ur=B.ur, uz=None)
    with pytest.raises(sfx.SfxError):
        B.b.sfx_batch_step(B.phi, B.f, B.f, 1e-10)


def _flat_instances(seed=13):
    """Flat-interface columns of Sec. 4.3 (planar) of uneven sizes, Langmuir
    kinetics with log10 Bi, log10 Da in [-2, 2]."""
    rng = np.random.default_rng(seed)
    out = []
    for nx, ny in [(4, 64), (8, 96), (5, 50), (8, 128), (3, 40)]:
        Bi, Da = 10.0 ** rng.uniform(-2, 2, size=2)
        c = W.case_flat_kinetics(ny, Bi, Da, nx=nx, steps=3)
        _, phi, _ = oracle.phase_field_build(c.grid, c.C, c.redist_iters, c.dtau, c.params.eps)
        out.append((c, phi, np.zeros(c.grid.shape)))
    return out


def test_planar_kinetics_sweep_matches_oracle_and_conserves(sfx):
    """The batched form on planar instances (sfx_batch_create_geom): each
    column against the FP64 oracle after three no-flow steps, and the total
    sum h^2 (f + F) of every column kept to 1e-10."""
    inst = _flat_instances()
    B = _Batch(sfx, inst, flow=False, geom=sfx.SFX_PLANAR2D)
    B.b.sfx_batch_set_schedule(256, 3, 60)
    for _ in range(3):
        B.step(1e-10)
        st = B.b.sfx_batch_stats()
        assert all(st["converged"]), st
    got = B.fields(sfx)
    for k, ((c, phi, f0), (fg, Fg)) in enumerate(zip(inst, got)):
        f_o, F_o = f0.copy(), c.F0.copy()
        for _ in range(3):
            f_o, F_o, so = oracle.surfactant_step(c.grid, c.params, phi, f_o, F_o, c.dt, 1e-13)
            assert so.converged
        scale = max(np.abs(F_o).max(), np.abs(f_o).max())
        assert np.abs(Fg - F_o).max() / scale < F32_TOL, k
        assert np.abs(fg - f_o).max() / scale < F32_TOL, k
        M0 = c.grid.h ** 2 * (f0 + c.F0).sum()
        M = st["mass_f"][k] + st["mass_F"][k]
        assert abs(M - M0) <= 1e-10 * M0, k
        assert abs(st["mass_f"][k] - c.grid.h ** 2 * fg.sum()) <= 1e-12 * M0, k


@pytest.mark.parametrize("fast", [0, 2])
def test_planar_batch_bitwise_equals_single_grid_steps(sfx, fast):
    """Fixed budget: planar batched kernels run the single-grid SFX_F32
    arithmetic cell for cell, as the axisymmetric ones do (the same number
    of FP32 residual passes on both sides)."""
    import torch
    inst = _flat_instances(seed=21)
    B = _Batch(sfx, inst, flow=False, geom=sfx.SFX_PLANAR2D)
    B.b.sfx_batch_set_schedule(128, 2, 4)
    B.b.sfx_batch_set_tuning(sfx._lib.SFX_TUNE_F32_FAST_RESID, fast)
    for _ in range(2):
        B.step(1e-30)
    fb, Fb = B.f.cpu().numpy(), B.F.cpu().numpy()
    o = sfx.default_opts(tol=1e-30, max_cycles=4, nu1=2, nu2=0)
    for k, (c, phi, f0) in enumerate(inst):
        ctx = sfx.Context.for_grid(c.grid, sfx.SFX_F32)
        ctx.sfx_set_tuning(sfx._lib.SFX_TUNE_F32_FAST_RESID, fast)
        f, F = sfx.sfx_df_pack(dev(f0)), sfx.sfx_df_pack(dev(c.F0))
        for _ in range(2):
            ctx.sfx_surfactant_step(c.params, dev(phi), f, F, c.dt, opts=o,
                                    allow_not_converged=True)
        torch.cuda.synchronize()
        n = c.grid.nx * c.grid.ny
        off = B.co[k]
        assert np.array_equal(f.cpu().numpy().reshape(-1, 2), fb[off:off + n]), k
        assert np.array_equal(F.cpu().numpy().reshape(-1, 2), Fb[off:off + n]), k


def test_batch_rejects_a_3d_geometry(sfx):
    c, _, _ = _flat_instances()[0]
    with pytest.raises(sfx.SfxError):
        sfx.Batch([(c.grid.nx, c.grid.ny, c.grid.h, c.dt, c.params)], geom=sfx.SFX_CART3D)
