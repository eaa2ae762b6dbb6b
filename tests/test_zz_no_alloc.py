"""inj_ybus_noalloc: Ybus-method injections for callers that cannot allocate
device memory (a host framework that owns all device memory in its own pool,
or a loop where an allocation is not acceptable).  The entry point keeps its
phasor scratch in a fixed device array inside the library, so it must give
the same result as inj_ybus and as the oracle on consecutive calls, whatever
ran before it in the process - including a larger grid whose phasors are
still in the array beyond the current grid's buses.  This file is collected
last on purpose."""
import numpy as np
import pytest

import oracle
from gridcases import random_grid, random_state, relerr

pytestmark = pytest.mark.gpu
TOL = 1e-12
LIMIT = 262144   # buses the fixed scratch array holds


@pytest.fixture(scope="module")
def pf():
    from paper_2302_10736_gb300 import _build
    _build.build_pfgrid()
    from paper_2302_10736_gb300 import pfgrid
    return pfgrid


def _dev(x):
    import torch
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def _noalloc_vs_references(pf, gr, grid, Y, rowptr, colidx, yval, seed):
    """One inj_ybus_noalloc call against inj_ybus and the oracle."""
    import torch
    nb = grid.nb
    vm, va = random_state(nb, seed)
    vm_d, va_d = _dev(vm), _dev(va)
    P0 = torch.empty(nb, dtype=torch.float64, device="cuda")
    Q0 = torch.empty_like(P0)
    P1 = torch.full_like(P0, np.nan)
    Q1 = torch.full_like(P0, np.nan)
    pf.inj_ybus(grid, vm_d, va_d, P0, Q0)
    pf.inj_ybus_noalloc(rowptr, colidx, yval, vm_d, va_d, P1, Q1)
    torch.cuda.synchronize()
    Pr, Qr = oracle.inj_sparse(Y, vm, va)
    P1h, Q1h = P1.cpu().numpy(), Q1.cpu().numpy()
    assert relerr(P1h, P0.cpu().numpy()) <= TOL and relerr(Q1h, Q0.cpu().numpy()) <= TOL
    assert relerr(P1h, Pr) <= TOL and relerr(Q1h, Qr) <= TOL


def test_noalloc_matches_inj_ybus_and_oracle_on_two_calls(pf):
    # a larger grid first, so the shared scratch holds stale phasors beyond
    # the buses of the smaller grid that follows
    for nb, nl, seed, calls in ((20000, 27000, 76, 1), (5000, 6800, 77, 2)):
        gr = random_grid(nb, nl, seed, shift_max=0.2)
        grid = pf.ybus_build(gr)
        Y = oracle.ybus(gr)
        rowptr, colidx, yval = pf.ybus_get(grid)
        for call in range(calls):   # two calls in a row on the smaller grid, different states
            _noalloc_vs_references(pf, gr, grid, Y, rowptr, colidx, yval, 100 * seed + call)


def test_noalloc_at_the_size_limit(pf):
    gr = random_grid(LIMIT, int(1.32 * LIMIT), 78)
    grid = pf.ybus_build(gr)
    rowptr, colidx, yval = pf.ybus_get(grid)
    _noalloc_vs_references(pf, gr, grid, oracle.ybus(gr), rowptr, colidx, yval, 7800)


def test_noalloc_rejects_oversized_grids(pf):
    st = pf._lib.inj_ybus_noalloc(LIMIT + 1, None, None, None, None, None, None, None, None)
    assert st == pf.PF_EUNSUPPORTED
    assert str(LIMIT) in pf.last_error()


def test_noalloc_wrapper_checks_array_lengths(pf):
    import torch
    gr = random_grid(200, 270, 79)
    grid = pf.ybus_build(gr)
    rowptr, colidx, yval = pf.ybus_get(grid)
    z = torch.zeros(200, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        pf.inj_ybus_noalloc(rowptr, colidx[:-1], yval, z, z, z.clone(), z.clone())
    with pytest.raises(ValueError):
        pf.inj_ybus_noalloc(rowptr, colidx, yval[:-1], z, z, z.clone(), z.clone())
