"""Reduced Newton Jacobian (CSC) and mismatch vector on the GPU against the
oracle: pattern bit-exact, values within 1e-12 (max-norm relative), both
evaluation methods; Newton's method driven by the GPU's F and J_r (sparse LU
of the CSC matrix on the host) converging quadratically; the library's own
sparse LU solve against a dense solve, and its Newton loop against the
oracle's."""
import numpy as np
import pytest

import oracle
from gridcases import hub_grid, make_grid, random_grid, random_state, relerr, series, two_bus_lossless

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(scope="module")
def pf():
    from paper_2302_10736_gb300 import _build
    _build.build_pfgrid()
    from paper_2302_10736_gb300 import pfgrid
    return pfgrid


def _d(x):
    import torch
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def gpu_reduced(pf, grid, method, vm, va, Ps, Qs):
    import torch
    n, _, nnz = pf.jac_reduced_info(grid)
    F = torch.full((max(n, 1),), np.nan, dtype=torch.float64, device="cuda")
    Jr = torch.full((max(nnz, 1),), np.nan, dtype=torch.float64, device="cuda")
    pf.jac_reduced(grid, method, _d(vm), _d(va), _d(Ps), _d(Qs), F, Jr)
    torch.cuda.synchronize()
    pf.grid_check_error(grid)
    return F.cpu().numpy()[:n], Jr.cpu().numpy()[:nnz]


def check_reduced(pf, gr, bt, vm, va, Ps, Qs, grid=None):
    grid = grid or pf.ybus_build(gr)
    pf.grid_set_bus_types(grid, bt)
    Y = oracle.ybus(gr)
    P, Q, J = oracle.elementwise(gr, vm, va, Y)
    colptr, rowidx, vals = oracle.jac_reduced(Y, J, bt)
    F_ref = oracle.mismatch(P, Q, Ps, Qs, bt)
    red, npvpq, npq = oracle.reduced_index(bt)
    n, n_pvpq, nnz = pf.jac_reduced_info(grid)
    assert (n, n_pvpq, nnz) == (npvpq + npq, npvpq, len(rowidx))
    cp, ri = pf.jac_reduced_pattern(grid)
    assert np.array_equal(cp, colptr) and np.array_equal(ri, rowidx)
    for method in (0, 1):
        F, Jr = gpu_reduced(pf, grid, method, vm, va, Ps, Qs)
        assert relerr(F, F_ref) <= TOL, (method, relerr(F, F_ref))
        assert relerr(Jr, vals) <= TOL, (method, relerr(Jr, vals))
    # the element-wise kernel writes the reduced system itself: bit for bit the
    # selection of its own full evaluation (same values, same P - Pspec)
    import torch
    nb = gr["nb"]
    Pd = torch.empty(nb, dtype=torch.float64, device="cuda")
    Qd = torch.empty_like(Pd)
    Jd = torch.empty(grid.nnzJ, dtype=torch.float64, device="cuda")
    pf.jac_elementwise(grid, _d(vm), _d(va), Pd, Qd, Jd)
    _, _, vals_gpu = oracle.jac_reduced(Y, Jd.cpu().numpy(), bt)
    F_gpu = oracle.mismatch(Pd.cpu().numpy(), Qd.cpu().numpy(), Ps, Qs, bt)
    F1, Jr1 = gpu_reduced(pf, grid, 1, vm, va, Ps, Qs)
    assert np.array_equal(Jr1, vals_gpu) and np.array_equal(F1, F_gpu)
    return grid


@pytest.mark.parametrize("k", [1, 2])
def test_workload_bus_types(pf, k):
    from paper_2302_10736_gb300 import synth
    w = synth.workload(k)
    vm2, va2 = synth.voltages(w["nb"], 1, w["seed"], 1)
    Ps, Qs = oracle.inj_sparse(oracle.ybus(w), vm2[0], va2[0])
    check_reduced(pf, w, w["bustype"], w["vm"][0], w["va"][0], Ps, Qs)


def test_two_bus_and_degenerate_types(pf):
    gr = two_bus_lossless()
    vm, va = np.array([1.0, 1.0]), np.array([0.0, -0.1])
    grid = pf.ybus_build(gr)
    for bt in ([3, 1], [3, 2], [2, 3], [1, 1], [2, 2]):
        check_reduced(pf, gr, np.array(bt, np.int32), vm, va, np.array([0.5, -0.25]), np.array([0.125, 0.0625]),
                      grid=grid)
    pf.grid_set_bus_types(grid, np.array([3, 4], np.int32))   # nothing left to solve
    assert pf.jac_reduced_info(grid)[0] == 0


def test_isolated_buses_parallels_and_a_hub(pf):
    gr = hub_grid(300, 51)
    nb = gr["nb"]
    vm, va = random_state(nb, 51)
    bt = np.ones(nb, np.int32)
    bt[0], bt[3::17], bt[[5, 6]] = 3, 2, 4
    bt[(nb - 1) // 2] = 2   # the hub is a PV bus
    Ps, Qs = np.linspace(-1, 1, nb), np.linspace(0.5, -0.5, nb)
    check_reduced(pf, gr, bt, vm, va, Ps, Qs)


def test_invalid_types_and_missing_types_rejected(pf):
    import torch
    gr = random_grid(50, 70, 52)
    grid = pf.ybus_build(gr)
    e = torch.zeros(50, dtype=torch.float64, device="cuda")
    with pytest.raises(pf.PfError):
        pf.jac_reduced(grid, 1, e, e, e, e, e, e)
    bad = np.ones(50, np.int32)
    bad[7] = 5
    with pytest.raises(pf.PfError):
        pf.grid_set_bus_types(grid, bad)
    with pytest.raises(pf.PfError):
        pf.jac_reduced_info(grid)


def test_newton_with_gpu_jacobian_converges_quadratically(pf):
    """Newton's method on the 2,000-bus workload grid: F and J_r from the
    GPU (element-wise method), the step from a sparse LU of the CSC matrix on
    the host, from a start within 1e-3 of a known solution (an operating
    point with the workload's angles scaled by 0.1: the random angles
    themselves leave the reduced Jacobian near-singular, condition ~1e6)."""
    import torch
    spla = pytest.importorskip("scipy.sparse.linalg")
    sp = pytest.importorskip("scipy.sparse")
    from paper_2302_10736_gb300 import synth
    w = synth.workload(1)
    nb, bt = w["nb"], w["bustype"]
    vm_t, va_t = w["vm"][0].copy(), 0.1 * w["va"][0]
    Ps, Qs = oracle.inj_sparse(oracle.ybus(w), vm_t, va_t)
    grid = pf.ybus_build(w)
    pf.grid_set_bus_types(grid, bt)
    n, npvpq, nnz = pf.jac_reduced_info(grid)
    colptr, rowidx = pf.jac_reduced_pattern(grid)
    pvpq, pq = np.flatnonzero((bt == 1) | (bt == 2)), np.flatnonzero(bt == 1)
    rng = np.random.default_rng(53)
    vm, va = vm_t.copy(), va_t.copy()
    vm[pq] += rng.uniform(-1e-3, 1e-3, len(pq))
    va[pvpq] += rng.uniform(-1e-3, 1e-3, len(pvpq))
    norms = []
    for _ in range(6):
        F, Jr = gpu_reduced(pf, grid, 1, vm, va, Ps, Qs)
        norms.append(float(np.max(np.abs(F))))
        if norms[-1] < 1e-11:
            break
        A = sp.csc_matrix((Jr, rowidx, colptr), shape=(n, n))
        dx = spla.splu(A).solve(-F)
        va[pvpq] += dx[:npvpq]
        vm[pq] += dx[npvpq:]
    assert norms[-1] < 1e-11, norms
    for a, b in zip(norms, norms[1:]):
        if a > 1e-6:
            assert b <= 1e3 * a * a, norms
    assert torch.cuda.is_available()


@pytest.mark.parametrize("method,workload", [(0, 1), (1, 1), (1, 3)])
def test_powerflow_newton_matches_the_oracle(pf, method, workload):
    """Newton-Raphson on the GPU (reduced system, the library's sparse LU,
    update) from the same start as the oracle's Newton iteration (scipy's
    pivoting sparse LU) takes as many iterations and reaches the same solution,
    the known state that defines the specification (2k- and 10k-bus grids)."""
    import torch
    pytest.importorskip("scipy")
    from paper_2302_10736_gb300 import synth
    w = synth.workload(workload, nscen=1)
    bt = w["bustype"]
    vm_t, va_t = w["vm"][0].copy(), 0.1 * w["va"][0]
    Ps, Qs = oracle.inj_sparse(oracle.ybus(w), vm_t, va_t)
    rng = np.random.default_rng(55)
    vm0, va0 = vm_t.copy(), va_t.copy()
    pq, pvpq = bt == 1, (bt == 1) | (bt == 2)
    vm0[pq] += rng.uniform(-1e-3, 1e-3, int(pq.sum()))
    va0[pvpq] += rng.uniform(-1e-3, 1e-3, int(pvpq.sum()))
    vm_o, va_o, it_o, norms, ok_o = oracle.newton(w, bt, vm0, va0, Ps, Qs, tol=1e-11)
    assert ok_o
    grid = pf.ybus_build(w)
    pf.grid_set_bus_types(grid, bt)
    vm, va = _d(vm0), _d(va0)
    ok, it, fmax = pf.powerflow_newton(grid, method, vm, va, _d(Ps), _d(Qs), tol=1e-11, max_iter=10)
    assert ok and fmax <= 1e-11 and it == it_o, (it, it_o, fmax, norms)
    vm, va = vm.cpu().numpy(), va.cpu().numpy()
    assert np.max(np.abs(vm - vm_o)) < 1e-10 and np.max(np.abs(va - va_o)) < 1e-10
    assert np.max(np.abs(vm - vm_t)) < 1e-10 and np.max(np.abs(va - va_t)) < 1e-10
    assert np.array_equal(vm[~pq], vm0[~pq]) and va[0] == va0[0]
    torch.cuda.synchronize()


def test_powerflow_newton_reports_non_convergence(pf):
    """Zero iterations allowed from a start that is not a solution: PF_ENOCONV
    with the mismatch of the start, the state unchanged."""
    from paper_2302_10736_gb300 import synth
    w = synth.workload(1)
    grid = pf.ybus_build(w)
    pf.grid_set_bus_types(grid, w["bustype"])
    vm, va = _d(w["vm"][0]), _d(w["va"][0])
    zeros = _d(np.zeros(w["nb"]))
    ok, it, fmax = pf.powerflow_newton(grid, 1, vm, va, zeros, zeros, tol=1e-11, max_iter=0)
    P, Q = oracle.inj_sparse(oracle.ybus(w), w["vm"][0], w["va"][0])
    F = oracle.mismatch(P, Q, np.zeros(w["nb"]), np.zeros(w["nb"]), w["bustype"])
    assert not ok and it == 0 and abs(fmax - np.max(np.abs(F))) <= 1e-12 * np.max(np.abs(F))
    assert np.array_equal(vm.cpu().numpy(), w["vm"][0]) and np.array_equal(va.cpu().numpy(), w["va"][0])


def backward_error(A, x, F):
    """Normwise backward error |A x - F| / (|A| |x| + |F|) (max norms)."""
    return np.max(np.abs(A @ x - F)) / (abs(A).sum(axis=1).max() * np.max(np.abs(x)) + np.max(np.abs(F)))


def _solve_case(pf, gr, bt, seed):
    import torch
    grid = pf.ybus_build(gr)
    pf.grid_set_bus_types(grid, bt)
    vm, va = random_state(gr["nb"], seed)
    Ps, Qs = oracle.inj_sparse(oracle.ybus(gr), *random_state(gr["nb"], seed, stream=1))
    n, _, nnz = pf.jac_reduced_info(grid)
    F = torch.empty(n, dtype=torch.float64, device="cuda")
    Jr = torch.empty(nnz, dtype=torch.float64, device="cuda")
    pf.jac_reduced(grid, 1, _d(vm), _d(va), _d(Ps), _d(Qs), F, Jr)
    return grid, F, Jr, n


@pytest.mark.parametrize("case", ["workload1", "mixed_types", "hub"])
def test_lu_solve_matches_a_dense_solve(pf, case):
    """jac_reduced_solve against LAPACK's pivoting dense solve of the same
    J_r and F: solution within 1e-10 (max-norm relative), normwise backward
    error below 1e-13 (LU without pivoting; a pivoting solve reaches about
    1e-16), and two solves bitwise equal."""
    import torch
    sp = pytest.importorskip("scipy.sparse")
    from paper_2302_10736_gb300 import synth
    if case == "workload1":
        w = synth.workload(1, nscen=1)
        gr, bt = w, w["bustype"]
    elif case == "mixed_types":
        gr = random_grid(1500, 2000, 91, shift_max=0.2)
        rng = np.random.default_rng(91)
        bt = rng.choice([1, 1, 1, 2], size=1500).astype(np.int32)
        bt[0] = 3
        bt[rng.choice(1500, 20, replace=False)] = 4   # isolated buses: no rows, no columns
        bt[0] = 3
    else:
        gr = hub_grid(300, 92)
        bt = np.ones(gr["nb"], np.int32)
        bt[::5] = 2
        bt[1] = 3
    grid, F, Jr, n = _solve_case(pf, gr, bt, 93)
    dx = torch.full((n,), np.nan, dtype=torch.float64, device="cuda")
    dx2 = torch.full_like(dx, np.nan)
    pf.jac_reduced_solve(grid, Jr, F, dx)
    pf.jac_reduced_solve(grid, Jr, F, dx2)
    torch.cuda.synchronize()
    pf.grid_check_error(grid)
    colptr, rowidx = pf.jac_reduced_pattern(grid)
    A = sp.csc_matrix((Jr.cpu().numpy(), rowidx, colptr), shape=(n, n))
    Fh, xh = F.cpu().numpy(), dx.cpu().numpy()
    ref = np.linalg.solve(A.toarray(), Fh)
    assert relerr(xh, ref) <= 1e-10
    assert backward_error(A, xh, Fh) <= 1e-13
    assert torch.equal(dx, dx2)


def chain_grid(nb, seed):
    """A radial line of nb buses (bus i to bus i + 1) with random series
    admittances and charging: minimum degree eliminates its buses from one
    end, so its elimination tree is a single chain of columns."""
    rng = np.random.default_rng(seed)
    branches = []
    for i in range(nb - 1):
        g, b = series(rng.uniform(0.005, 0.02), rng.uniform(0.05, 0.2))
        branches.append((i, i + 1, g, b, rng.uniform(0.0, 0.05), 1.0, 0.0))
    return make_grid(nb, branches)


@pytest.mark.parametrize("nb", [6, 12, 200, 400])
def test_lu_solve_on_a_chain(pf, nb):
    """The solve on radial lines, whose reduced systems (n = 2 (nb - 1)) are
    all narrow levels: 6 buses (n = 10) stay below the dense tail's minimum
    of 16 columns (one launch); 12 buses (n = 22) are a tail from the first
    column on; 200 and 400 buses (n = 398, 798) have the largest tail, 384
    columns, above 14 and 414 columns of the dynamic schedule.  Solution
    within 1e-10 (max-norm relative) of LAPACK's pivoting dense solve,
    normwise backward error below 1e-13, two solves bitwise equal."""
    import torch
    import scipy.sparse as sp
    gr = chain_grid(nb, 300 + nb)
    bt = np.ones(nb, np.int32)
    bt[0] = 3
    grid, F, Jr, n = _solve_case(pf, gr, bt, 301 + nb)
    assert n == 2 * (nb - 1)
    dx = torch.full((n,), np.nan, dtype=torch.float64, device="cuda")
    dx2 = torch.full_like(dx, np.nan)
    pf.jac_reduced_solve(grid, Jr, F, dx)
    pf.jac_reduced_solve(grid, Jr, F, dx2)
    torch.cuda.synchronize()
    pf.grid_check_error(grid)
    colptr, rowidx = pf.jac_reduced_pattern(grid)
    A = sp.csc_matrix((Jr.cpu().numpy(), rowidx, colptr), shape=(n, n))
    Fh, xh = F.cpu().numpy(), dx.cpu().numpy()
    assert relerr(xh, np.linalg.solve(A.toarray(), Fh)) <= 1e-10
    assert backward_error(A, xh, Fh) <= 1e-13
    assert torch.equal(dx, dx2)


def test_lu_solve_reports_a_zero_pivot(pf):
    """A matrix without a usable pivot (all values zero) is reported through
    the grid's error word (PF_EDEVICE), not a fault; the next solve of a valid
    matrix is correct."""
    import torch
    from paper_2302_10736_gb300 import synth
    w = synth.workload(1, nscen=1)
    grid, F, Jr, n = _solve_case(pf, w, w["bustype"], 94)
    dx = torch.empty(n, dtype=torch.float64, device="cuda")
    pf.jac_reduced_solve(grid, torch.zeros_like(Jr), F, dx)
    with pytest.raises(pf.PfError) as e:
        pf.grid_check_error(grid)
    assert e.value.status == pf.PF_EDEVICE
    pf.jac_reduced_solve(grid, Jr, F, dx)
    torch.cuda.synchronize()
    pf.grid_check_error(grid)
    colptr, rowidx = pf.jac_reduced_pattern(grid)
    import scipy.sparse as sp
    A = sp.csc_matrix((Jr.cpu().numpy(), rowidx, colptr), shape=(n, n))
    assert backward_error(A, dx.cpu().numpy(), F.cpu().numpy()) <= 1e-13
