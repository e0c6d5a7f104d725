"""sfx_totals_noalloc, the totals entry point for callers that may not
allocate device memory (their memory belongs to another allocator, or they
cannot afford cudaMalloc's device synchronisation).  Called through the
C-ABI and compared with sfx_totals on two calls in a row; the second call
must not see the first call's leftover scratch.  This file is collected
last on purpose."""
import ctypes as C
import math

import numpy as np
import pytest

import oracle
import workloads as W
from gpu_util import dev

pytestmark = pytest.mark.gpu

TOL = 4e-16   # against the exact sum, relative to sum |V x| (as the other totals tests)


@pytest.fixture(scope="module")
def sfx():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2605_27534_gb300 as m
    m.lib()
    return m


def _noalloc(sfx, g, fields):
    import torch
    grid = sfx.Grid(g.geom, g.nx, g.ny, g.nz, g.h)
    n = len(fields)
    ptrs = (C.c_void_p * n)(*[t.data_ptr() for t in fields])
    out = (C.c_double * n)()
    st = sfx.lib().sfx_totals_noalloc(C.byref(grid), ptrs, n, out,
                                      torch.cuda.current_stream().cuda_stream)
    return st, [out[i] for i in range(n)]


def test_noalloc_totals_match_context_totals_on_consecutive_calls(sfx):
    rng = np.random.default_rng(21)
    cases = [
        (W.Grid(W.AXI, 300, 91, 1, 0.004), 3),
        (W.Grid(W.CART3D, 40, 36, 30, 0.02), 1),
    ]
    for g, nf in cases:
        arrays = [rng.standard_normal(g.shape) * 10.0 ** rng.uniform(-4, 4, g.shape)
                  for _ in range(nf)]
        fields = [dev(a) for a in arrays]
        st, got = _noalloc(sfx, g, fields)
        assert st == 0, sfx.lib().sfx_status_string(st)
        ref = sfx.Context.for_grid(g).sfx_totals(fields)
        V = oracle.cell_volumes(g)
        for val, a in zip(got, arrays):
            assert abs(val - math.fsum((V * a).ravel())) <= TOL * np.abs(V * a).sum()
        # the same reduction order as sfx_totals: the same bits
        assert got == ref
        # a second call on fewer fields right after: the same bits again
        st2, got2 = _noalloc(sfx, g, fields[:1])
        assert st2 == 0 and got2[0] == ref[0]


def test_noalloc_rejects_more_fields_than_its_scratch_holds(sfx):
    import torch
    g = W.Grid(W.PLANAR, 8, 8, 1, 0.1)
    x = torch.zeros(g.shape, dtype=torch.float64, device="cuda")
    st, _ = _noalloc(sfx, g, [x] * 9)
    assert st == 6   # SFX_ERR_WORKSPACE
    assert sfx.lib().sfx_status_string(st) == b"workspace too small"
