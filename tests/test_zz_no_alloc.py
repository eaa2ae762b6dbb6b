"""inj_ybus_noalloc: Ybus-method injections for callers that cannot allocate
device memory (a host framework that owns all device memory in its own pool,
or a loop where an allocation is not acceptable).  The entry point keeps its
phasor scratch in a fixed device array inside the library, so it must give
the same result as inj_ybus on consecutive calls, whatever ran before it in
the process.  This file is collected last on purpose."""
import numpy as np
import pytest

from gridcases import random_grid, random_state, relerr

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(scope="module")
def pf():
    from paper_2302_10736_gb300 import _build
    _build.build_pfgrid()
    from paper_2302_10736_gb300 import pfgrid
    return pfgrid


def test_noalloc_matches_inj_ybus_on_two_calls(pf):
    import torch
    gr = random_grid(5000, 6800, 77, shift_max=0.2)
    grid = pf.ybus_build(gr)
    rowptr, colidx, yval = pf.ybus_get(grid)
    dev = lambda x: torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")
    for call in range(2):   # two calls in a row, different states
        vm, va = random_state(5000, 100 + call)
        vm_d, va_d = dev(vm), dev(va)
        P0 = torch.empty(grid.nb, dtype=torch.float64, device="cuda")
        Q0 = torch.empty_like(P0)
        P1 = torch.full_like(P0, np.nan)
        Q1 = torch.full_like(P0, np.nan)
        pf.inj_ybus(grid, vm_d, va_d, P0, Q0)
        pf.inj_ybus_noalloc(rowptr, colidx, yval, vm_d, va_d, P1, Q1)
        torch.cuda.synchronize()
        assert relerr(P1.cpu().numpy(), P0.cpu().numpy()) <= TOL
        assert relerr(Q1.cpu().numpy(), Q0.cpu().numpy()) <= TOL


def test_noalloc_rejects_oversized_grids(pf):
    st = pf._lib.inj_ybus_noalloc(262145, None, None, None, None, None, None, None, None)
    assert st == pf.PF_EUNSUPPORTED
    assert "262144" in pf.last_error()
