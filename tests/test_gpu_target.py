"""Jacobian values into a caller's sparsity pattern (Alg. 2) on the GPU:
a CSC pattern that contains the Ybus-block pattern and more (random extra
positions, a TCSC-like coupled pair, rows shuffled within columns).  Both
methods write the Ybus-block positions with the values of their own
canonical evaluation placed by the oracle's Alg. 2 (bit for bit), within
1e-12 of the oracle's Jacobian, and leave every other position untouched."""
import numpy as np
import pytest

import oracle
from gridcases import hub_grid, make_grid, random_grid, random_state, relerr, superset_pattern

pytestmark = pytest.mark.gpu
TOL = 1e-12
SENTINEL = 12345.5


@pytest.fixture(scope="module")
def pf():
    from paper_2302_10736_gb300 import _build
    _build.build_pfgrid()
    from paper_2302_10736_gb300 import pfgrid
    return pfgrid


def _d(x):
    import torch
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def check_target(pf, gr, seed, extra):
    import torch
    rng = np.random.default_rng(seed)
    nb = gr["nb"]
    vm, va = random_state(nb, seed)
    Y = oracle.ybus(gr)
    colptr, rowidx = superset_pattern(Y, rng, extra)
    grid = pf.ybus_build(gr)
    pf.jac_set_target_pattern(grid, colptr, rowidx)
    Jref = oracle.jac_ybus(Y, vm, va)
    Pref, Qref = oracle.inj_sparse(Y, vm, va)
    placed_ref = oracle.jac_target(Y, Jref, colptr, rowidx, np.full(len(rowidx), np.nan))
    mapped = ~np.isnan(placed_ref)
    for method, canon in ((1, pf.jac_elementwise), (0, pf.jac_ybus)):
        Jt = torch.full((len(rowidx),), SENTINEL, dtype=torch.float64, device="cuda")
        P = torch.empty(nb, dtype=torch.float64, device="cuda")
        Q = torch.empty_like(P)
        pf.jac_target(grid, method, _d(vm), _d(va), P, Q, Jt)
        Jc = torch.empty(grid.nnzJ, dtype=torch.float64, device="cuda")
        canon(grid, _d(vm), _d(va), None, None, Jc)
        torch.cuda.synchronize()
        pf.grid_check_error(grid)
        out = Jt.cpu().numpy()
        placed = oracle.jac_target(Y, Jc.cpu().numpy(), colptr, rowidx, np.full(len(rowidx), SENTINEL))
        assert np.array_equal(out, placed), method                      # bit for bit, untouched elsewhere
        assert np.all(out[~mapped] == SENTINEL)
        assert relerr(out[mapped], placed_ref[mapped]) <= TOL, method
        assert relerr(P.cpu().numpy(), Pref) <= TOL and relerr(Q.cpu().numpy(), Qref) <= TOL
    return grid, colptr, rowidx


def _star_with_parallels():
    # a star with a triple-parallel spoke, two isolated buses, shunts everywhere
    br = [(0, 1, 1.0, -10.0, 0.02, 1.0, 0.0), (1, 0, 2.0, -8.0, 0.01, 1.03, 0.05),
          (0, 1, 0.5, -12.0, 0.0, 0.98, -0.02), (0, 2, 1.5, -9.0, 0.03, 1.0, 0.0),
          (3, 0, 0.7, -7.0, 0.04, 1.0, 0.0)]
    return make_grid(6, br, shunts={i: (0.01 * i, -0.02 * i) for i in range(6)})


@pytest.mark.parametrize("case", ["random", "hub", "parallels", "single"])
def test_target_pattern_both_methods(pf, case):
    gr = {"random": lambda: random_grid(700, 980, 31, shift_max=0.2), "hub": lambda: hub_grid(300, 33),
          "parallels": _star_with_parallels,
          "single": lambda: make_grid(1, [], shunts={0: (0.03, -0.02)})}[case]()
    check_target(pf, gr, 31, extra=500)


def test_target_pattern_rejects_a_missing_entry_and_bad_arrays(pf):
    from paper_2302_10736_gb300.pfgrid import PfError
    gr = random_grid(50, 70, 32)
    Y = oracle.ybus(gr)
    colptr, rowidx = superset_pattern(Y, np.random.default_rng(32), extra=10)
    grid = pf.ybus_build(gr)
    jrp, jci = oracle.jac_pattern(Y)
    R, C = 3, int(jci[jrp[3]])
    k = next(k for k in range(colptr[C], colptr[C + 1]) if rowidx[k] == R)
    cp2 = colptr.copy()
    cp2[C + 1:] -= 1
    with pytest.raises(PfError):
        pf.jac_set_target_pattern(grid, cp2, np.delete(rowidx, k))
    bad = rowidx.copy()
    bad[0] = 2 * gr["nb"]
    with pytest.raises(PfError):
        pf.jac_set_target_pattern(grid, colptr, bad)
    with pytest.raises(PfError):   # evaluation before any pattern was accepted
        import torch
        z = torch.zeros(gr["nb"], dtype=torch.float64, device="cuda")
        pf.jac_target(grid, 1, z, z, None, None, torch.zeros(len(rowidx), dtype=torch.float64, device="cuda"))
