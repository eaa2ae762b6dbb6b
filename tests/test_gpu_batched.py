"""Batched N-1 evaluation and the adjoint against the oracle (GPU).

Scenario s of a batch is checked against the oracle run from scratch on the
grid without its outage branch: values within 1e-12 (max-norm relative per
vector and Jacobian block), its Jacobian pattern bit-exact.  The adjoint is
checked against J^T r of the oracle's Jacobian, complex-step branch-parameter
gradients, and (25k-bus workload) long-double central differences on 200
seeded coordinates.
"""
import os

import numpy as np
import pytest

import oracle
from gridcases import blocks, hub_grid, make_grid, random_grid, random_state, relerr

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


def _skip(nl, l):
    m = np.zeros(nl, np.uint8)
    if l >= 0:
        m[l] = 1
    return m


def _reduced(gr, l):
    """The grid without branch l (branch arrays filtered) and the index map."""
    if l < 0:
        return gr, np.arange(gr["nl"])
    keep = np.array([i for i in range(gr["nl"]) if i != l])
    out = dict(gr)
    for k in ("f", "t", "g", "b", "bsh", "tap", "shift"):
        out[k] = gr[k][keep]
    out["nl"] = gr["nl"] - 1
    return out, keep


def with_parallel(gr):
    """Add a branch parallel to branch 0 so that an outage of either keeps the entry."""
    out = dict(gr)
    for k in ("f", "t", "g", "b", "bsh", "tap", "shift"):
        v = gr[k][0] * (1.0 if k in ("f", "t", "tap", "shift") else 0.7)
        out[k] = np.concatenate([gr[k], [v]]).astype(gr[k].dtype)
    out["nl"] = gr["nl"] + 1
    return out


def _oracle_pq(gr, vm, va, outage, scenarios):
    """The oracle's P and Q of the listed scenarios, each on its grid without
    the outage branch (threads: the oracle's C calls release the GIL)."""
    from concurrent.futures import ThreadPoolExecutor

    def one(s):
        l = int(outage[s]) if outage is not None else -1
        skip = _skip(gr["nl"], l)
        return oracle.elementwise(gr, vm[s], va[s], oracle.ybus(gr, skip=skip), skip=skip, jac=False)[:2]

    with ThreadPoolExecutor(min(16, os.cpu_count() or 1)) as ex:
        return dict(zip(scenarios, ex.map(one, scenarios)))


def check_batch(pf, gr, vm, va, outage, scenarios=None, tol=TOL, cfg=None, pq_all=False):
    """Scenarios `scenarios` (all if None) in full: P, Q of all four batched
    calls, both Jacobians and the pattern against the oracle.  With pq_all,
    P and Q of every other scenario are compared as well."""
    import torch
    S, nb = vm.shape
    grid = pf.ybus_build(gr)
    if cfg:
        pf.grid_set_config(grid, **cfg)
    batch = pf.batch_create(grid, S, outage)
    joff = pf.batch_jac_offsets(batch).cpu().numpy()
    assert joff[0] == 0 and joff[-1] == batch.nnzJ_total
    P = torch.full((S * nb,), np.nan, dtype=torch.float64, device="cuda")
    Q = torch.full_like(P, np.nan)
    J = torch.full((batch.nnzJ_total,), np.nan, dtype=torch.float64, device="cuda")
    Pi = torch.full_like(P, np.nan)
    Qi = torch.full_like(P, np.nan)
    Py, Qy, Jy = torch.full_like(P, np.nan), torch.full_like(P, np.nan), torch.full_like(J, np.nan)
    Pyi, Qyi = torch.full_like(P, np.nan), torch.full_like(P, np.nan)
    pf.jac_elementwise_batched(batch, _d(vm), _d(va), P, Q, J)
    pf.inj_elementwise_batched(batch, _d(vm), _d(va), Pi, Qi)
    pf.jac_ybus_batched(batch, _d(vm), _d(va), Py, Qy, Jy)
    pf.inj_ybus_batched(batch, _d(vm), _d(va), Pyi, Qyi)
    torch.cuda.synchronize()
    pf.grid_check_error(grid)
    host = lambda x: x.cpu().numpy().reshape(S, nb)
    P, Q, J = host(P), host(Q), J.cpu().numpy()
    Pi, Qi = host(Pi), host(Qi)
    Py, Qy, Jy, Pyi, Qyi = host(Py), host(Qy), Jy.cpu().numpy(), host(Pyi), host(Qyi)
    for s in (range(S) if scenarios is None else scenarios):
        l = int(outage[s]) if outage is not None else -1
        skip = _skip(gr["nl"], l)
        Y = oracle.ybus(gr, skip=skip)
        jrp, jci = oracle.jac_pattern(Y)
        rp_s, ci_s = pf.batch_jac_pattern(batch, s)
        assert np.array_equal(rp_s, jrp) and np.array_equal(ci_s, jci), s
        assert joff[s + 1] - joff[s] == 4 * Y.nnz
        Pr, Qr, Jr = oracle.elementwise(gr, vm[s], va[s], Y, skip=skip)
        Js, Jys = J[joff[s]:joff[s + 1]], Jy[joff[s]:joff[s + 1]]
        errs = [relerr(x[s], r) for x, r in ((P, Pr), (Q, Qr), (Pi, Pr), (Qi, Qr), (Py, Pr), (Qy, Qr), (Pyi, Pr),
                                              (Qyi, Qr))]
        errs += [relerr(a, b) for a, b in zip(blocks(Js, jci, nb, Y.nnz), blocks(Jr, jci, nb, Y.nnz))]
        errs += [relerr(a, b) for a, b in zip(blocks(Jys, jci, nb, Y.nnz), blocks(Jr, jci, nb, Y.nnz))]
        assert max(errs) <= tol, (s, l, errs)
    if pq_all and scenarios is not None:
        rest = sorted(set(range(S)) - set(scenarios))
        for s, (Pr, Qr) in _oracle_pq(gr, vm, va, outage, rest).items():
            errs = [relerr(x[s], r) for x, r in ((P, Pr), (Q, Qr), (Pi, Pr), (Qi, Qr), (Py, Pr), (Qy, Qr), (Pyi, Pr),
                                                  (Qyi, Qr))]
            assert max(errs) <= tol, (s, errs)
    return batch


def test_small_batch_with_outages_and_parallels(pf):
    from paper_2302_10736_gb300 import synth
    gr = with_parallel(random_grid(400, 560, 21, shift_max=0.2))
    isb = synth.bridges(400, gr["f"], gr["t"])
    nonbridge = np.flatnonzero(~isb)
    outage = np.array([-1, int(nonbridge[3]), 0, gr["nl"] - 1, int(nonbridge[10]), int(np.flatnonzero(isb)[0]), -1,
                       int(nonbridge[20])], np.int32)   # none, plain, both of a parallel pair, a bridge
    vm, va = synth.voltages(400, len(outage), 21, 0, 0.93, 1.07, 0.25)
    check_batch(pf, gr, vm, va, outage)


@pytest.mark.parametrize("lanes", [1, 4, 32])
def test_ybus_batched_every_lane_count(pf, lanes):
    from paper_2302_10736_gb300 import synth
    gr = with_parallel(random_grid(300, 420, 23, shift_max=0.2))
    nonbridge = np.flatnonzero(~synth.bridges(300, gr["f"], gr["t"]))
    outage = np.array([int(nonbridge[5]), -1, 0, gr["nl"] - 1, int(nonbridge[40])], np.int32)
    vm, va = synth.voltages(300, len(outage), 23, 0, 0.93, 1.07, 0.25)
    check_batch(pf, gr, vm, va, outage, cfg=dict(ybus_lanes=lanes, ybus_block=128))


def test_launches_alternate_between_grids_of_different_shared_memory(pf):
    """The dynamic shared-memory limit is a per-kernel setting shared by every
    grid and batch: a grid whose windows need little of it, launched for the
    first time after one that needs more, must not lower it below what the
    larger one needs (its next launches would fail)."""
    import torch
    from paper_2302_10736_gb300 import synth
    grids = {"hub": hub_grid(400, 31), "small": random_grid(300, 400, 33, shift_max=0.2)}
    state = {}
    for key, gr in grids.items():
        nb = gr["nb"]
        vm, va = synth.voltages(nb, 2, 34, 0, 0.93, 1.07, 0.25)
        Y = oracle.ybus(gr)
        refs = [oracle.elementwise(gr, vm[s], va[s], Y) for s in range(2)]
        state[key] = (gr, vm, va, refs, Y)
    built = {}
    for rnd in range(3):
        for key in ("hub", "small"):
            gr, vm, va, refs, Y = state[key]
            nb = gr["nb"]
            if key not in built:
                grid = pf.ybus_build(gr)
                built[key] = (grid, pf.batch_create(grid, 2, None))
            grid, batch = built[key]
            P = torch.empty(nb, dtype=torch.float64, device="cuda")
            Q = torch.empty_like(P)
            J = torch.empty(grid.nnzJ, dtype=torch.float64, device="cuda")
            pf.jac_elementwise(grid, _d(vm[0]), _d(va[0]), P, Q, J)
            Pb = torch.empty(2 * nb, dtype=torch.float64, device="cuda")
            Qb = torch.empty_like(Pb)
            Jb = torch.empty(batch.nnzJ_total, dtype=torch.float64, device="cuda")
            pf.jac_elementwise_batched(batch, _d(vm), _d(va), Pb, Qb, Jb)
            torch.cuda.synchronize()
            pf.grid_check_error(grid)
            Pr, Qr, Jr = refs[0]
            assert relerr(P.cpu().numpy(), Pr) <= TOL and relerr(J.cpu().numpy(), Jr) <= TOL, (rnd, key)
            Jbh = Jb.cpu().numpy()
            for s in range(2):
                Pr, Qr, Jr = refs[s]
                assert relerr(Pb.cpu().numpy()[s * nb:(s + 1) * nb], Pr) <= TOL, (rnd, key, s)
                assert relerr(Jbh[s * grid.nnzJ:(s + 1) * grid.nnzJ], Jr) <= TOL, (rnd, key, s)


def test_batch_with_a_hub_bus(pf):
    """Windows whose single bus has more terminals than the CTA has threads,
    outages of a hub spoke, of one of a parallel pair of spokes and of a ring
    branch."""
    from paper_2302_10736_gb300 import synth
    gr = hub_grid(400, 32)
    S = 4
    hub = (gr["nb"] - 1) // 2
    spokes = [l for l in range(gr["nl"]) if hub in (gr["f"][l], gr["t"][l])]
    outage = np.array([spokes[3], -1, spokes[0], 5], np.int32)
    vm, va = synth.voltages(gr["nb"], S, 32, 0, 0.93, 1.07, 0.25)
    check_batch(pf, gr, vm, va, outage)


def test_batch_without_outages_equals_single_evaluation(pf):
    import torch
    gr = random_grid(2000, 2700, 22)
    vm, va = random_state(2000, 22, nscen=3)
    grid = pf.ybus_build(gr)
    batch = pf.batch_create(grid, 3, None)
    J = torch.empty(batch.nnzJ_total, dtype=torch.float64, device="cuda")
    P = torch.empty(3 * 2000, dtype=torch.float64, device="cuda")
    Q = torch.empty_like(P)
    pf.jac_elementwise_batched(batch, _d(vm), _d(va), P, Q, J)
    for s in range(3):
        P1 = torch.empty(2000, dtype=torch.float64, device="cuda")
        Q1 = torch.empty_like(P1)
        J1 = torch.empty(grid.nnzJ, dtype=torch.float64, device="cuda")
        pf.jac_elementwise(grid, _d(vm[s]), _d(va[s]), P1, Q1, J1)
        assert torch.equal(P[s * 2000:(s + 1) * 2000], P1) and torch.equal(Q[s * 2000:(s + 1) * 2000], Q1)
        assert torch.equal(J[s * grid.nnzJ:(s + 1) * grid.nnzJ], J1)
    # the Ybus method: the single evaluation's separate form runs the batch's
    # row kernel for one scenario, so with the same lanes it agrees bit for bit
    bc = pf.batch_get_config(batch)
    pf.grid_set_config(grid, ybus_lanes=bc["ybus_lanes"], ybus_block=bc["ybus_block"], ybus_fused=0)
    pf.jac_ybus_batched(batch, _d(vm), _d(va), P, Q, J)
    Pi, Qi = torch.empty_like(P), torch.empty_like(Q)
    pf.inj_ybus_batched(batch, _d(vm), _d(va), Pi, Qi)
    for s in range(3):
        P1 = torch.empty(2000, dtype=torch.float64, device="cuda")
        Q1 = torch.empty_like(P1)
        J1 = torch.empty(grid.nnzJ, dtype=torch.float64, device="cuda")
        pf.jac_ybus(grid, _d(vm[s]), _d(va[s]), P1, Q1, J1)
        assert torch.equal(P[s * 2000:(s + 1) * 2000], P1) and torch.equal(Q[s * 2000:(s + 1) * 2000], Q1)
        assert torch.equal(J[s * grid.nnzJ:(s + 1) * grid.nnzJ], J1)
        pf.inj_ybus(grid, _d(vm[s]), _d(va[s]), P1, Q1)
        assert torch.equal(Pi[s * 2000:(s + 1) * 2000], P1) and torch.equal(Qi[s * 2000:(s + 1) * 2000], Q1)


def test_workload3_n1_batch(pf):
    """10,000 buses x 1,024 scenarios with distinct non-bridge outages, against
    the oracle on each grid without its branch: P and Q of all 1,024
    scenarios (from all four batched calls), and the Jacobians (both methods)
    and patterns of 48 spread scenarios."""
    from paper_2302_10736_gb300 import synth
    w = synth.workload(3)
    sample = sorted(set(np.linspace(0, 1023, 48).astype(int).tolist()))
    batch = check_batch(pf, w, w["vm"], w["va"], w["outage"], scenarios=sample, pq_all=True)
    assert batch.nscen == 1024


def _adjoint_case(nb, nl, seed, S, outage=None):
    from paper_2302_10736_gb300 import synth
    gr = random_grid(nb, nl, seed, shift_max=0.2)
    vm, va = synth.voltages(nb, S, seed, 0, 0.95, 1.05, 0.2)
    vm2, va2 = synth.voltages(nb, 1, seed, 1, 0.95, 1.05, 0.2)
    Y = oracle.ybus(gr)
    Ps, Qs = oracle.inj_sparse(Y, vm2[0], va2[0])
    wP, wQ = synth.weights(nb, seed)
    return gr, vm, va, Ps, Qs, wP, wQ


def run_adjoint(pf, gr, vm, va, Ps, Qs, wP, wQ, outage=None):
    import torch
    S, nb = vm.shape
    grid = pf.ybus_build(gr)
    batch = pf.batch_create(grid, S, outage)
    L = torch.empty(S, dtype=torch.float64, device="cuda")
    gvm = torch.empty(S * nb, dtype=torch.float64, device="cuda")
    gva = torch.empty_like(gvm)
    gp = [torch.empty(gr["nl"], dtype=torch.float64, device="cuda") for _ in range(4)]
    pf.adjoint_elementwise(batch, _d(vm), _d(va), _d(Ps), _d(Qs), _d(wP), _d(wQ), L, gvm, gva, *gp)
    torch.cuda.synchronize()
    pf.grid_check_error(grid)
    return (L.cpu().numpy(), gvm.cpu().numpy().reshape(S, nb), gva.cpu().numpy().reshape(S, nb),
            [x.cpu().numpy() for x in gp])


def oracle_adjoint(gr, vm, va, Ps, Qs, wP, wQ, outage=None):
    S, nb = vm.shape
    Ls, gvm, gva = np.zeros(S), np.zeros((S, nb)), np.zeros((S, nb))
    gp = [np.zeros(gr["nl"]) for _ in range(4)]
    for s in range(S):
        l = int(outage[s]) if outage is not None else -1
        skip = _skip(gr["nl"], l)
        Y = oracle.ybus(gr, skip=skip)
        P, Q = oracle.inj_sparse(Y, vm[s], va[s])
        J = oracle.jac_ybus(Y, vm[s], va[s])
        Ls[s] = oracle.loss(P, Q, Ps, Qs, wP, wQ)
        gva[s], gvm[s] = oracle.adjoint_state(Y, J, P, Q, Ps, Qs, wP, wQ)
        gr_s, keep = _reduced(gr, l)
        Y_s = oracle.ybus(gr_s)
        for acc, part in zip(gp, oracle.adjoint_params_cstep(gr_s, Y_s, vm[s], va[s], Ps, Qs, wP, wQ)):
            acc[keep] += part
    return Ls, gvm, gva, gp


@pytest.mark.parametrize("S,with_outage", [(1, False), (1, True), (3, True)])
def test_adjoint_matches_oracle(pf, S, with_outage):
    gr, vm, va, Ps, Qs, wP, wQ = _adjoint_case(500, 700, 31 + S, S)
    outage = None
    if with_outage:
        from paper_2302_10736_gb300 import synth
        isb = synth.bridges(500, gr["f"], gr["t"])
        nb_ = np.flatnonzero(~isb)
        outage = np.array([int(nb_[0]), -1, int(nb_[5])][:S], np.int32)
    L, gvm, gva, gp = run_adjoint(pf, gr, vm, va, Ps, Qs, wP, wQ, outage)
    Lr, gvmr, gvar, gpr = oracle_adjoint(gr, vm, va, Ps, Qs, wP, wQ, outage)
    assert relerr(L, Lr) <= TOL
    for s in range(S):
        assert relerr(gvm[s], gvmr[s]) <= TOL and relerr(gva[s], gvar[s]) <= TOL, s
    for name, a, b in zip(("g", "b", "bsh", "tap"), gp, gpr):
        assert relerr(a, b) <= TOL, name


@pytest.mark.parametrize("S", [2, 170])
def test_adjoint_both_launch_forms_with_outages(pf, S):
    """Two scenarios on a 40-bus grid give fewer (scenario, window) items than
    SMs: one item per CTA with one grid barrier.  170 scenarios give more items
    than SMs: the throughput form with its phasor phase and two barriers.
    Every scenario but every fourth removes a non-bridge branch."""
    from paper_2302_10736_gb300 import synth
    gr, vm, va, Ps, Qs, wP, wQ = _adjoint_case(40, 55, 57, S)
    nbr = np.flatnonzero(~synth.bridges(40, gr["f"], gr["t"]))
    outage = np.array([-1 if s % 4 == 0 else int(nbr[s % len(nbr)]) for s in range(S)], np.int32)
    L, gvm, gva, gp = run_adjoint(pf, gr, vm, va, Ps, Qs, wP, wQ, outage)
    Lr, gvmr, gvar, gpr = oracle_adjoint(gr, vm, va, Ps, Qs, wP, wQ, outage)
    assert relerr(L, Lr) <= TOL
    assert relerr(gvm.ravel(), gvmr.ravel()) <= TOL and relerr(gva.ravel(), gvar.ravel()) <= TOL
    for s in (0, 1, S - 1):
        assert relerr(gvm[s], gvmr[s]) <= TOL and relerr(gva[s], gvar[s]) <= TOL, s
    for name, a, b in zip(("g", "b", "bsh", "tap"), gp, gpr):
        assert relerr(a, b) <= TOL, name


def test_adjoint_workload4_against_oracle_and_central_differences(pf):
    """25,000 buses: J^T r and complex-step parameter gradients to 1e-12, and
    central differences (h = 1e-7, long double) on 200 seeded coordinates."""
    from paper_2302_10736_gb300 import synth
    w = synth.workload(4)
    Y = oracle.ybus(w)
    Ps, Qs = oracle.inj_sparse(Y, w["vm2"], w["va2"])
    vm, va = w["vm"], w["va"]
    L, gvm, gva, gp = run_adjoint(pf, w, vm, va, Ps, Qs, w["wP"], w["wQ"])
    Lr, gvmr, gvar, gpr = oracle_adjoint(w, vm, va, Ps, Qs, w["wP"], w["wQ"])
    assert relerr(L, Lr) <= TOL
    assert relerr(gvm[0], gvmr[0]) <= TOL and relerr(gva[0], gvar[0]) <= TOL
    for a, b in zip(gp, gpr):
        assert relerr(a, b) <= TOL
    nb, nl = w["nb"], w["nl"]
    kinds = synth.randint(w["seed"], 7, 200, 6)
    idxs = np.array([synth.randint(w["seed"], 8 + i, 1, nb if k <= 1 else nl)[0] for i, k in enumerate(kinds)])
    fd = oracle.loss_central_diff(w, vm[0], va[0], Ps, Qs, w["wP"], w["wQ"], kinds, idxs, 1e-7)
    allg = [gva[0], gvm[0]] + gp
    ad = np.array([allg[k][i] for k, i in zip(kinds, idxs)])
    scale = np.array([np.max(np.abs(allg[k])) for k in kinds])
    err = np.abs(ad - fd) / np.maximum(np.abs(fd), 1e-3 * scale)
    assert err.max() <= 1e-6, err.max()


def test_adjoint_workload5_sixteen_scenarios(pf):
    """250,000 buses x 16 scenarios: losses and the scenario-summed parameter
    gradients against the oracle; state gradients of 4 scenarios."""
    from paper_2302_10736_gb300 import synth
    w = synth.workload(5)
    Y = oracle.ybus(w)
    Ps, Qs = oracle.inj_sparse(Y, w["vm2"], w["va2"])
    L, gvm, gva, gp = run_adjoint(pf, w, w["vm"], w["va"], Ps, Qs, w["wP"], w["wQ"])
    Lr = np.zeros(16)
    gpr = [np.zeros(w["nl"]) for _ in range(4)]
    for s in range(16):
        P, Q = oracle.inj_sparse(Y, w["vm"][s], w["va"][s])
        Lr[s] = oracle.loss(P, Q, Ps, Qs, w["wP"], w["wQ"])
        for acc, part in zip(gpr, oracle.adjoint_params_cstep(w, Y, w["vm"][s], w["va"][s], Ps, Qs, w["wP"],
                                                              w["wQ"])):
            acc += part
        if s % 5 == 0:
            P, Q = oracle.inj_sparse(Y, w["vm"][s], w["va"][s])
            J = oracle.jac_ybus(Y, w["vm"][s], w["va"][s])
            gar, gvr = oracle.adjoint_state(Y, J, P, Q, Ps, Qs, w["wP"], w["wQ"])
            assert relerr(gva[s], gar) <= TOL and relerr(gvm[s], gvr) <= TOL, s
    assert relerr(L, Lr) <= TOL
    for a, b in zip(gp, gpr):
        assert relerr(a, b) <= TOL


def test_mismatch_loss_autograd(pf):
    import torch
    gr, vm, va, Ps, Qs, wP, wQ = _adjoint_case(300, 420, 41, 2)
    grid = pf.ybus_build(gr)
    batch = pf.batch_create(grid, 2, None)
    t = lambda x, rg=False: torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda",
                                         requires_grad=rg)
    vm_t, va_t = t(vm, True), t(va, True)
    g_t, b_t, bsh_t, tap_t = t(gr["g"], True), t(gr["b"], True), t(gr["bsh"], True), t(gr["tap"], True)
    loss = pf.MismatchLoss.apply(batch, vm_t, va_t, g_t, b_t, bsh_t, tap_t, t(gr["shift"]), t(gr["gs"]),
                                 t(gr["bs"]), t(Ps), t(Qs), t(wP), t(wQ))
    (2.0 * loss).backward()
    Lr, gvmr, gvar, gpr = oracle_adjoint(gr, vm, va, Ps, Qs, wP, wQ)
    assert abs(loss.item() - Lr.sum()) <= TOL * abs(Lr.sum())
    assert relerr(vm_t.grad.cpu().numpy(), 2 * gvmr) <= TOL
    assert relerr(va_t.grad.cpu().numpy(), 2 * gvar) <= TOL
    for tt, ref in zip((g_t, b_t, bsh_t, tap_t), gpr):
        assert relerr(tt.grad.cpu().numpy(), 2 * ref) <= TOL


@pytest.mark.parametrize("nb,nl,S,form", [(2000, 2700, 3, "one item per CTA"), (10000, 13500, 8, "throughput")])
def test_loss_alone_total_and_upstream_scale(pf, nb, nl, S, form):
    """loss_elementwise: L_s and L_total against the oracle's loss of each
    scenario (outages honoured); L_total is bitwise the ascending sum of the
    L_s; adjoint_elementwise returns bitwise the same losses, and its
    gradients with an upstream scale Lbar are Lbar times the unscaled ones.
    Both kernel forms: a batch with fewer items than SMs (one per CTA) and a
    larger one."""
    import torch
    from paper_2302_10736_gb300 import synth
    gr, vm, va, Ps, Qs, wP, wQ = _adjoint_case(nb, nl, 61 + S, S)
    nonbridge = np.flatnonzero(~synth.bridges(nb, gr["f"], gr["t"]))
    outage = np.full(S, -1, np.int32)
    outage[1::2] = nonbridge[5:5 + len(outage[1::2])]
    grid = pf.ybus_build(gr)
    batch = pf.batch_create(grid, S, outage)
    args = [_d(x) for x in (vm.ravel(), va.ravel(), Ps, Qs, wP, wQ)]
    L = torch.full((S,), np.nan, dtype=torch.float64, device="cuda")
    Lt = torch.full((1,), np.nan, dtype=torch.float64, device="cuda")
    pf.loss_elementwise(batch, *args, L, Lt)
    Lt_only = torch.full((1,), np.nan, dtype=torch.float64, device="cuda")
    pf.loss_elementwise(batch, *args, None, Lt_only)
    torch.cuda.synchronize()
    pf.grid_check_error(grid)
    Lh = L.cpu().numpy()
    Lr = np.zeros(S)
    for s in range(S):
        skip = _skip(gr["nl"], int(outage[s]))
        Y = oracle.ybus(gr, skip=skip)
        P, Q = oracle.inj_sparse(Y, vm[s], va[s])
        Lr[s] = oracle.loss(P, Q, Ps, Qs, wP, wQ)
    assert relerr(Lh, Lr) <= TOL
    acc = 0.0
    for x in Lh:   # ascending s
        acc += x
    assert Lt.item() == acc and Lt_only.item() == acc
    # the adjoint: same losses bitwise; gradients scale with Lbar
    outs = {}
    for lbar in (None, 2.5):
        La = torch.full((S,), np.nan, dtype=torch.float64, device="cuda")
        Lta = torch.full((1,), np.nan, dtype=torch.float64, device="cuda")
        gvm = torch.empty(S * nb, dtype=torch.float64, device="cuda")
        gva = torch.empty_like(gvm)
        gp = [torch.empty(gr["nl"], dtype=torch.float64, device="cuda") for _ in range(4)]
        lb = None if lbar is None else torch.full((1,), lbar, dtype=torch.float64, device="cuda")
        pf.adjoint_elementwise(batch, *args, La, gvm, gva, *gp, Lbar=lb, Ltot=Lta)
        torch.cuda.synchronize()
        assert torch.equal(La, L) and torch.equal(Lta, Lt), form
        outs[lbar] = [x.cpu().numpy() for x in [gvm, gva] + gp]
    for a, b in zip(outs[2.5], outs[None]):
        assert relerr(a, 2.5 * b) <= 1e-14


def test_mismatch_loss_forward_runs_the_loss_alone(pf):
    """The autograd forward launches the loss kernel only; the backward the
    adjoint (library tracer)."""
    import torch
    gr, vm, va, Ps, Qs, wP, wQ = _adjoint_case(300, 420, 62, 2)
    grid = pf.ybus_build(gr)
    batch = pf.batch_create(grid, 2, None)
    t = lambda x: _d(x)
    vm_t = t(vm.ravel()).requires_grad_(True)
    va_t = t(va.ravel()).requires_grad_(True)
    g_t = t(gr["g"]).requires_grad_(True)
    pf.grid_trace_enable(grid, 64)
    loss = pf.MismatchLoss.apply(batch, vm_t, va_t, g_t, t(gr["b"]), t(gr["bsh"]), t(gr["tap"]), t(gr["shift"]),
                                 t(gr["gs"]), t(gr["bs"]), t(Ps), t(Qs), t(wP), t(wQ))
    torch.cuda.synchronize()
    fwd = [k for k, _ in pf.grid_trace_read(grid)]
    loss.backward()
    torch.cuda.synchronize()
    bwd = [k for k, _ in pf.grid_trace_read(grid)]
    pf.grid_trace_enable(grid, 0)
    assert "loss" in fwd and "adjoint" not in fwd, fwd
    assert "adjoint" in bwd and "loss" not in bwd, bwd
    assert vm_t.grad is not None and g_t.grad is not None


def test_every_batch_launch_shape_gives_the_same_results(pf):
    """Every launch configuration the autotuner may pick (window size x
    terminal cap x CTAs per SM, both adjoint forms, every batched-Ybus lane
    count): the batched Jacobians are bitwise those of the default shape (the
    sums per bus do not depend on the windows), the adjoint matches the oracle
    within 1e-12."""
    import torch
    from paper_2302_10736_gb300 import synth
    gr, vm, va, Ps, Qs, wP, wQ = _adjoint_case(2000, 2700, 67, 4)
    nonbridge = np.flatnonzero(~synth.bridges(2000, gr["f"], gr["t"]))
    outage = np.array([-1, nonbridge[3], nonbridge[70], -1], np.int32)
    grid = pf.ybus_build(gr)
    batch = pf.batch_create(grid, 4, outage)
    args = [_d(x) for x in (vm.ravel(), va.ravel())]
    spec = [_d(x) for x in (Ps, Qs, wP, wQ)]
    n = 4 * 2000

    def run():
        P, Q = torch.empty(n, dtype=torch.float64, device="cuda"), torch.empty(n, dtype=torch.float64, device="cuda")
        J = torch.empty(batch.nnzJ_total, dtype=torch.float64, device="cuda")
        Py, Qy = torch.empty_like(P), torch.empty_like(Q)
        Jy = torch.empty_like(J)
        pf.jac_elementwise_batched(batch, *args, P, Q, J)
        pf.jac_ybus_batched(batch, *args, Py, Qy, Jy)
        L = torch.empty(4, dtype=torch.float64, device="cuda")
        gvm, gva = torch.empty(n, dtype=torch.float64, device="cuda"), torch.empty(n, dtype=torch.float64, device="cuda")
        gp = [torch.empty(gr["nl"], dtype=torch.float64, device="cuda") for _ in range(4)]
        pf.adjoint_elementwise(batch, *args, *spec, L, gvm, gva, *gp)
        torch.cuda.synchronize()
        pf.grid_check_error(grid)
        return [x.cpu().numpy() for x in (P, Q, J, Py, Qy, Jy)], [x.cpu().numpy() for x in [L, gvm, gva] + gp]

    ref, _ = run()
    Lr, gvmr, gvar, gpr = oracle_adjoint(gr, vm, va, Ps, Qs, wP, wQ, outage)
    shapes = 0
    for window in (128, 256):
        for tpt in (1, 2, 3):
            for cps in (0, 1, 3):
                for form in (0, 1):
                    lanes = (1, 2, 4, 8, 16, 32)[shapes % 6]
                    try:
                        pf.batch_set_config(batch, window=window, terminals_per_thread=tpt, ctas_per_sm=cps,
                                            adjoint_form=form, ybus_lanes=lanes, ybus_block=128 * (1 + shapes % 3))
                    except pf.PfError as e:   # a window shape that does not fit in shared memory
                        assert e.status == pf.PF_EUNSUPPORTED
                        continue
                    got, adj = run()
                    cfg = pf.batch_get_config(batch)
                    for a, b in zip(got[:3], ref[:3]):
                        assert np.array_equal(a, b), cfg
                    for a, b in zip(got[3:], ref[3:]):
                        assert relerr(a, b) <= TOL, cfg
                    L, gvm, gva = adj[:3]
                    assert relerr(L, Lr) <= TOL and relerr(gvm.reshape(4, 2000), gvmr) <= TOL, cfg
                    assert relerr(gva.reshape(4, 2000), gvar) <= TOL, cfg
                    for a, b in zip(adj[3:], gpr):
                        assert relerr(a, b) <= TOL, cfg
                    shapes += 1
    assert shapes >= 12


def test_batch_autotune_and_its_cache(pf, tmp_path, monkeypatch):
    """batch_autotune picks a valid configuration, stores it under the
    batch's key in the PFGRID_TUNE_CACHE file, and a new batch of the same
    size class starts with it; results stay bitwise those of the default."""
    import torch
    from paper_2302_10736_gb300 import synth
    path = str(tmp_path / "tune.json")
    monkeypatch.setenv("PFGRID_TUNE_CACHE", path)
    gr = random_grid(3000, 4100, 68)
    nonbridge = np.flatnonzero(~synth.bridges(3000, gr["f"], gr["t"]))
    outage = np.array(nonbridge[:16], np.int32)
    vm, va = synth.voltages(3000, 16, 68, 0, 0.93, 1.07, 0.25)
    grid = pf.ybus_build(gr)
    batch = pf.batch_create(grid, 16, outage)
    J0 = torch.empty(batch.nnzJ_total, dtype=torch.float64, device="cuda")
    pf.jac_elementwise_batched(batch, _d(vm.ravel()), _d(va.ravel()), None, None, J0)
    best = pf.batch_autotune(batch, _d(vm.ravel()), _d(va.ravel()), reps=2)
    assert best == pf.batch_get_config(batch)
    assert pf.tune_cache_lookup(path, pf.batch_tune_key(batch)) == best
    J1 = torch.empty_like(J0)
    pf.jac_elementwise_batched(batch, _d(vm.ravel()), _d(va.ravel()), None, None, J1)
    batch2 = pf.batch_create(grid, 16, outage[::-1].copy())
    assert pf.batch_get_config(batch2) == best
    torch.cuda.synchronize()
    assert torch.equal(J0, J1)


def test_cuda_graph_capture_and_replay(pf):
    """The batched evaluation, the adjoint and the single evaluation can be
    captured in a CUDA graph (after one eager call) and replayed; replays give
    the eager bits."""
    import torch
    from paper_2302_10736_gb300 import synth
    gr = random_grid(3000, 4100, 71)
    grid = pf.ybus_build(gr)
    nonbridge = np.flatnonzero(~synth.bridges(3000, gr["f"], gr["t"]))
    outage = np.array([-1, int(nonbridge[3]), int(nonbridge[9])], np.int32)
    S = len(outage)
    batch = pf.batch_create(grid, S, outage)
    vm, va = synth.voltages(3000, S, 71, 0, 0.93, 1.07, 0.25)
    vmd, vad = _d(vm.ravel()), _d(va.ravel())
    P = torch.empty(S * 3000, dtype=torch.float64, device="cuda")
    Q = torch.empty_like(P)
    J = torch.empty(batch.nnzJ_total, dtype=torch.float64, device="cuda")
    P1 = torch.empty(3000, dtype=torch.float64, device="cuda")
    Q1 = torch.empty_like(P1)
    J1 = torch.empty(grid.nnzJ, dtype=torch.float64, device="cuda")
    Ps, Qs, wP, wQ = (_d(x) for x in (np.zeros(3000), np.zeros(3000), np.ones(3000), np.ones(3000)))
    L = torch.empty(S, dtype=torch.float64, device="cuda")
    gvm, gva = torch.empty_like(P), torch.empty_like(P)

    def work():
        pf.jac_elementwise_batched(batch, vmd, vad, P, Q, J)
        pf.adjoint_elementwise(batch, vmd, vad, Ps, Qs, wP, wQ, L, gvm, gva)
        pf.jac_elementwise(grid, vmd[:3000], vad[:3000], P1, Q1, J1)

    work()
    torch.cuda.synchronize()
    ref = [x.clone() for x in (P, Q, J, L, gvm, gva, P1, Q1, J1)]
    for x in (P, Q, J, L, gvm, gva, P1, Q1, J1):
        x.fill_(np.nan)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        work()
    for _ in range(2):
        g.replay()
    torch.cuda.synchronize()
    pf.grid_check_error(grid)
    for a, b in zip((P, Q, J, L, gvm, gva, P1, Q1, J1), ref):
        assert torch.equal(a, b)


def test_barrier_state_across_interleaved_kernels(pf):
    """The batched kernels of one grid share its grid-barrier state (a launch
    parity and two counters): alternate a small-batch adjoint (one item per
    CTA, one barrier), a throughput adjoint (two barriers) and a batched
    Jacobian (one barrier) with different grid sizes, 40 rounds; every launch
    must give bitwise the results of the first and no wait may time out."""
    import torch
    gr, vm, va, Ps, Qs, wP, wQ = _adjoint_case(200, 280, 61, 170)
    grid = pf.ybus_build(gr)
    big = pf.batch_create(grid, 170, None)          # more items than SMs: k_adj, k_ewb
    small = pf.batch_create(grid, 1, None)          # fewer: k_adj1
    d = _d
    vmb, vab = d(vm.ravel()), d(va.ravel())
    vm1, va1 = d(vm[0]), d(va[0])
    out = lambda n: torch.empty(n, dtype=torch.float64, device="cuda")
    first = None
    for r in range(40):
        L1, g1m, g1a = out(1), out(200), out(200)
        pf.adjoint_elementwise(small, vm1, va1, d(Ps), d(Qs), d(wP), d(wQ), L1, g1m, g1a)
        L2, g2m, g2a = out(170), out(170 * 200), out(170 * 200)
        pf.adjoint_elementwise(big, vmb, vab, d(Ps), d(Qs), d(wP), d(wQ), L2, g2m, g2a)
        P, Q, J = out(170 * 200), out(170 * 200), out(big.nnzJ_total)
        pf.jac_elementwise_batched(big, vmb, vab, P, Q, J)
        torch.cuda.synchronize()
        pf.grid_check_error(grid)
        now = [x.cpu().numpy() for x in (L1, g1m, g1a, L2, g2m, g2a, P, Q, J)]
        if first is None:
            first = now
        else:
            assert all(np.array_equal(a, b) for a, b in zip(first, now)), r
    # the single-state adjoint agrees with the first scenario of the big batch's
    np.testing.assert_allclose(first[0], first[3][:1], rtol=1e-12)
