"""Pins of the CPU oracle against facts other than itself (CPU only).

Each pin_* function returns the error it measures, so test_oracle_mutations
can show that a planted mistake in the oracle breaks at least one of them.
Sources of truth, none of which re-types an oracle formula:
  - hand-derived closed form of a lossless two-bus line (derived from Eq. 1);
  - Kirchhoff's current law on the physical branch model (ideal transformer
    m e^{j phi} : 1 plus a pi section), independent of the admittance stamps;
  - exact invariants: zero Ybus row sums without charging/taps, symmetry
    without phase shift, rotation invariance and degree-2 homogeneity of S;
  - complex-step derivatives of the real-form injections (every J entry);
  - series-branch loss identity (P_hk + P_kh = r |I_s|^2, ...);
  - long-double central differences of the loss (adjoint);
  - the paper's printed element count (16 values per line, Sec. V-A.2);
  - reduced Jacobian: the two-bus closed form, and Newton's method on it
    converging quadratically to a known solution (a wrong, transposed or
    misordered reduced Jacobian converges linearly at best).
"""
import math
import os

import numpy as np
import pytest

import oracle
from gridcases import (blocks, circuit_currents, make_grid, random_grid, random_state, relerr, series, superset_pattern,
                       three_bus_plus, two_bus_lossless)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
TOL = 1e-13


# ---------------------------------------------------------------- pins ----

def pin_two_bus():
    """Closed form of the lossless line x = 0.1 (y_s = -j10), V1 = 1, V2 = 1 at -0.1 rad.
    With d = th1 - th2:  P1 = 10 v1 v2 sin d,  Q1 = 10 v1^2 - 10 v1 v2 cos d,
                         P2 = -10 v1 v2 sin d, Q2 = 10 v2^2 - 10 v1 v2 cos d."""
    gr = two_bus_lossless()
    vm, va = np.array([1.0, 1.0]), np.array([0.0, -0.1])
    s, c = math.sin(0.1), math.cos(0.1)
    P_ref = np.array([10 * s, -10 * s])
    Q_ref = np.array([10 * (1 - c), 10 * (1 - c)])
    # rows (P1, P2, Q1, Q2) x columns (th1, th2, v1, v2)
    Jd = np.array([
        [10 * c, -10 * c, 10 * s, 10 * s],
        [-10 * c, 10 * c, -10 * s, -10 * s],
        [10 * s, -10 * s, 20 - 10 * c, -10 * c],
        [10 * s, -10 * s, -10 * c, 20 - 10 * c],
    ])
    Y = oracle.ybus(gr)
    jrp, jci = oracle.jac_pattern(Y)
    errs = []
    P, Q = oracle.inj_sparse(Y, vm, va)
    errs += [np.max(np.abs(P - P_ref)), np.max(np.abs(Q - Q_ref))]
    Pe, Qe, Je = oracle.elementwise(gr, vm, va, Y)
    errs += [np.max(np.abs(Pe - P_ref)), np.max(np.abs(Qe - Q_ref))]
    for J in (oracle.jac_ybus(Y, vm, va), oracle.jac_cstep(Y, vm, va), Je):
        for r in range(4):
            for e in range(jrp[r], jrp[r + 1]):
                errs.append(abs(J[e] - Jd[r, jci[e]]))
    Ydense = Y.dense()
    errs.append(np.max(np.abs(Ydense - np.array([[-10j, 10j], [10j, -10j]]))))
    return max(errs) / 10.0


def pin_circuit_law(gr, seed=1):
    """Ybus V equals the KCL bus currents of the physical model, and every
    injection path equals V conj(I_KCL)."""
    vm, va = random_state(gr["nb"], seed)
    V, Ikcl = circuit_currents(gr, vm, va)
    Y = oracle.ybus(gr)
    Ivec = Y.dense() @ V if gr["nb"] <= 400 else None
    S_ref = V * np.conj(Ikcl)
    errs = []
    if Ivec is not None:
        errs.append(relerr(Ivec, Ikcl))
    P, Q = oracle.inj_sparse(Y, vm, va)
    errs += [relerr(P, S_ref.real), relerr(Q, S_ref.imag)]
    Pe, Qe, _ = oracle.elementwise(gr, vm, va, Y, jac=False)
    errs += [relerr(Pe, S_ref.real), relerr(Qe, S_ref.imag)]
    if gr["nb"] <= 400:
        Yre, Yim = oracle.ybus_dense(gr)
        Pd, Qd = oracle.inj_dense(Yre, Yim, vm, va)
        errs += [relerr(Pd, S_ref.real), relerr(Qd, S_ref.imag)]
    return max(errs)


def pin_jacobian_cstep(gr, seed=2):
    vm, va = random_state(gr["nb"], seed)
    Y = oracle.ybus(gr)
    _, jci = oracle.jac_pattern(Y)
    Ja, Jc = oracle.jac_ybus(Y, vm, va), oracle.jac_cstep(Y, vm, va)
    return max(relerr(a, c) for a, c in zip(blocks(Ja, jci, gr["nb"], Y.nnz), blocks(Jc, jci, gr["nb"], Y.nnz)))


def pin_invariants(gr, seed=3):
    """Rotation invariance (theta columns of every row sum to 0) and degree-2
    homogeneity (sum_j dS_i/dv_j v_j = 2 S_i), for both Jacobian paths."""
    vm, va = random_state(gr["nb"], seed)
    Y = oracle.ybus(gr)
    nb, nnz = gr["nb"], Y.nnz
    jrp, jci = oracle.jac_pattern(Y)
    P, Q = oracle.inj_sparse(Y, vm, va)
    errs = []
    for J in (oracle.jac_ybus(Y, vm, va), oracle.elementwise(gr, vm, va, Y)[2]):
        rot = np.zeros(2 * nb)
        hom = np.zeros(2 * nb)
        scale = 0.0
        for r in range(2 * nb):
            for e in range(jrp[r], jrp[r + 1]):
                c = jci[e]
                if c < nb:
                    rot[r] += J[e]
                else:
                    hom[r] += J[e] * vm[c - nb]
                scale = max(scale, abs(J[e]))
        errs.append(np.max(np.abs(rot)) / scale)
        S2 = 2 * np.concatenate([P, Q])
        errs.append(relerr(hom, S2))
    return max(errs)


def pin_elementwise_equals_ybus(gr, seed=4, skip=None):
    vm, va = random_state(gr["nb"], seed)
    Y = oracle.ybus(gr, skip=skip)
    _, jci = oracle.jac_pattern(Y)
    P, Q = oracle.inj_sparse(Y, vm, va)
    J = oracle.jac_ybus(Y, vm, va)
    Pe, Qe, Je = oracle.elementwise(gr, vm, va, Y, skip=skip)
    errs = [relerr(Pe, P), relerr(Qe, Q)]
    errs += [relerr(a, b) for a, b in zip(blocks(Je, jci, gr["nb"], Y.nnz), blocks(J, jci, gr["nb"], Y.nnz))]
    return max(errs)


def pin_branch_loss(seed=5):
    """One branch, m = 1, phi = 0: P_hk + P_kh = r |I_s|^2 and
    Q_hk + Q_kh = x |I_s|^2 - (b_sh/2)(v_h^2 + v_k^2), I_s = y_s (V_h - V_k)."""
    rng = np.random.default_rng(seed)
    errs = []
    for _ in range(20):
        r, x, bsh = rng.uniform(0.001, 0.05), rng.uniform(0.01, 0.3), rng.uniform(0, 0.1)
        g, b = series(r, x)
        gr = make_grid(2, [(0, 1, g, b, bsh, 1.0, 0.0)])
        vm, va = rng.uniform(0.9, 1.1, 2), rng.normal(0, 0.2, 2)
        Y = oracle.ybus(gr)
        V = vm * np.exp(1j * va)
        Is = complex(g, b) * (V[0] - V[1])
        for P, Q in (oracle.inj_sparse(Y, vm, va), oracle.elementwise(gr, vm, va, Y, jac=False)[:2]):
            lossP = r * abs(Is) ** 2
            lossQ = x * abs(Is) ** 2 - bsh / 2 * (vm[0] ** 2 + vm[1] ** 2)
            errs.append(abs(P.sum() - lossP) / max(abs(P).max(), 1e-300))
            errs.append(abs(Q.sum() - lossQ) / max(abs(Q).max(), 1e-300))
    return max(errs)


def _loss_case(nb=150, nl=210, seed=7):
    gr = random_grid(nb, nl, seed, shift_max=0.2)
    vm, va = random_state(nb, seed)
    vm2, va2 = random_state(nb, seed, stream=1)
    Y = oracle.ybus(gr)
    Ps, Qs = oracle.inj_sparse(Y, vm2, va2)
    rng = np.random.default_rng(seed)
    wP, wQ = rng.uniform(0.5, 2, nb), rng.uniform(0.5, 2, nb)
    return gr, Y, vm, va, Ps, Qs, wP, wQ


def pin_loss_closed_form():
    """The mismatch loss L = sum_i wP_i (P_i - Ps_i)^2 + wQ_i (Q_i - Qs_i)^2 on the
    lossless two-bus line of pin_two_bus, from its closed-form injections
    (P1 = -P2 = 10 sin 0.1, Q1 = Q2 = 10 (1 - cos 0.1)) with targets and weights
    chosen so that every term differs (wP != wQ on each bus): a swapped weight,
    a dropped square or a sign error changes the value."""
    s, c = math.sin(0.1), math.cos(0.1)
    P = (10 * s, -10 * s)
    Q = (10 * (1 - c), 10 * (1 - c))
    Ps, Qs = (0.3, -0.7), (0.1, 0.2)
    wP, wQ = (1.5, 0.25), (0.75, 3.0)
    ref = sum(wP[i] * (P[i] - Ps[i]) ** 2 + wQ[i] * (Q[i] - Qs[i]) ** 2 for i in range(2))
    gr = two_bus_lossless()
    Y = oracle.ybus(gr)
    Po, Qo = oracle.inj_sparse(Y, np.array([1.0, 1.0]), np.array([0.0, -0.1]))
    L = oracle.loss(Po, Qo, np.array(Ps), np.array(Qs), np.array(wP), np.array(wQ))
    return abs(L - ref) / ref


def pin_loss_central_difference(nb=150, nl=210, seed=7, ncoord=24):
    """Central differences of oracle.loss over perturbed states (h = 1e-6, the
    injections from oracle.inj_sparse) against the long-double central
    differences of or_loss_central_diff, which evaluates the loss from the
    branch list without any oracle routine: a loss with a wrong weight, a
    dropped square or a missing bus has the wrong slope."""
    gr, Y, vm, va, Ps, Qs, wP, wQ = _loss_case(nb, nl, seed)
    rng = np.random.default_rng(seed + 1)
    kinds = rng.integers(0, 2, ncoord)
    idxs = rng.integers(0, nb, ncoord)
    h = 1e-6
    fd = oracle.loss_central_diff(gr, vm, va, Ps, Qs, wP, wQ, kinds, idxs, h)
    errs = []
    for c in range(ncoord):
        vals = []
        for sgn in (1.0, -1.0):
            vm2, va2 = vm.copy(), va.copy()
            (va2 if kinds[c] == 0 else vm2)[idxs[c]] += sgn * h
            P, Q = oracle.inj_sparse(Y, vm2, va2)
            vals.append(oracle.loss(P, Q, Ps, Qs, wP, wQ))
        d = (vals[0] - vals[1]) / (2 * h)
        errs.append(abs(d - fd[c]) / max(abs(fd).max(), 1e-300))
    return max(errs)


def pin_adjoint(nb=150, nl=210, seed=7):
    """J^T r and the complex-step parameter gradients against long-double
    central differences (h = 1e-7) of the loss."""
    gr, Y, vm, va, Ps, Qs, wP, wQ = _loss_case(nb, nl, seed)
    P, Q = oracle.inj_sparse(Y, vm, va)
    J = oracle.jac_ybus(Y, vm, va)
    gva, gvm = oracle.adjoint_state(Y, J, P, Q, Ps, Qs, wP, wQ)
    gg, gb, gbsh, gtap = oracle.adjoint_params_cstep(gr, Y, vm, va, Ps, Qs, wP, wQ)
    kinds = np.concatenate([np.zeros(nb, int), np.ones(nb, int)] + [np.full(nl, k) for k in (2, 3, 4, 5)])
    idxs = np.concatenate([np.arange(nb), np.arange(nb)] + [np.arange(nl)] * 4)
    fd = oracle.loss_central_diff(gr, vm, va, Ps, Qs, wP, wQ, kinds, idxs, 1e-7)
    ad = np.concatenate([gva, gvm, gg, gb, gbsh, gtap])
    errs = []
    off = 0
    for n in (nb, nb, nl, nl, nl, nl):
        errs.append(relerr(ad[off:off + n], fd[off:off + n]))
        off += n
    return max(errs)


# --------------------------------------------------------------- tests ----

def test_two_bus_closed_form():
    assert pin_two_bus() < 1e-14


@pytest.mark.parametrize("case", ["three_bus_plus", "random_shift", "random_plain"])
def test_circuit_law(case):
    gr = {"three_bus_plus": lambda: three_bus_plus(),
          "random_shift": lambda: random_grid(300, 420, 11, shift_max=0.3),
          "random_plain": lambda: random_grid(2000, 2700, 12)}[case]()
    assert pin_circuit_law(gr) < TOL


def test_row_sums_equal_shunts_without_charging_or_taps():
    gr = random_grid(500, 700, 21)
    gr["bsh"][:] = 0.0
    gr["tap"][:] = 1.0
    gr["shift"][:] = 0.0
    Y = oracle.ybus(gr)
    rows = np.add.reduceat(Y.yre + 1j * Y.yim, Y.rp[:-1])
    ysh = gr["gs"] + 1j * gr["bs"]
    scale = np.max(np.abs(Y.yre + 1j * Y.yim))
    assert np.max(np.abs(rows - ysh)) / scale < 1e-14


def test_symmetric_without_phase_shift():
    gr = random_grid(500, 700, 22)
    Yd = oracle.ybus(gr).dense()
    assert np.array_equal(Yd, Yd.T)
    gr2 = random_grid(300, 420, 23, shift_max=0.3)
    Yd2 = oracle.ybus(gr2).dense()
    assert not np.allclose(Yd2, Yd2.T)


@pytest.mark.parametrize("case", ["three_bus_plus", "random_shift", "c1_like"])
def test_jacobian_complex_step(case):
    gr = {"three_bus_plus": lambda: three_bus_plus(),
          "random_shift": lambda: random_grid(300, 420, 31, shift_max=0.3),
          "c1_like": lambda: random_grid(2000, 2700, 32)}[case]()
    assert pin_jacobian_cstep(gr) < TOL


@pytest.mark.parametrize("case", ["three_bus_plus", "random_shift"])
def test_jacobian_invariants(case):
    gr = three_bus_plus() if case == "three_bus_plus" else random_grid(400, 560, 41, shift_max=0.3)
    assert pin_invariants(gr) < TOL


@pytest.mark.parametrize("case", ["two_bus", "three_bus_plus", "random_shift", "c1_like", "outage"])
def test_elementwise_equals_ybus(case):
    skip = None
    if case == "two_bus":
        gr = two_bus_lossless()
    elif case == "three_bus_plus":
        gr = three_bus_plus()
    elif case == "random_shift":
        gr = random_grid(300, 420, 51, shift_max=0.3)
    elif case == "c1_like":
        gr = random_grid(2000, 2700, 52)
    else:
        gr = three_bus_plus()
        skip = np.array([0, 0, 0, 1], np.uint8)  # drop one of the parallel pair
    assert pin_elementwise_equals_ybus(gr, skip=skip) < TOL


def test_dense_equals_sparse():
    gr = random_grid(300, 420, 61, shift_max=0.2)
    vm, va = random_state(300, 61)
    Y = oracle.ybus(gr)
    P, Q = oracle.inj_sparse(Y, vm, va)
    Yre, Yim = oracle.ybus_dense(gr)
    Pd, Qd = oracle.inj_dense(Yre, Yim, vm, va)
    assert relerr(P, Pd) < TOL and relerr(Q, Qd) < TOL
    Yd = Y.dense()
    assert np.max(np.abs(Yd - (Yre + 1j * Yim))) == 0.0


def test_branch_loss_identity():
    assert pin_branch_loss() < 1e-12


def test_loss_closed_form():
    assert pin_loss_closed_form() < 1e-14


def test_loss_slope_against_central_differences():
    assert pin_loss_central_difference() < 1e-6


def test_adjoint_against_central_differences():
    assert pin_adjoint() < 1e-8


def test_jacobian_pattern_layout():
    gr = three_bus_plus()
    Y = oracle.ybus(gr)
    nb, nnz = gr["nb"], Y.nnz
    assert nnz == nb + 2 * 3  # the parallel pair merges into one off-diagonal pair
    jrp, jci = oracle.jac_pattern(Y)
    assert jrp[-1] == 4 * nnz
    for r in range(2 * nb):
        cols = jci[jrp[r]:jrp[r + 1]]
        assert np.all(np.diff(cols) > 0)
        i = r % nb
        ycols = Y.ci[Y.rp[i]:Y.rp[i + 1]]
        assert np.array_equal(cols, np.concatenate([ycols, nb + ycols]))
    assert Y.rp[4] - Y.rp[3] == 1  # isolated bus keeps its diagonal


def test_contingency_pattern():
    gr = random_grid(500, 700, 71)
    from paper_2302_10736_gb300 import synth
    isb = synth.bridges(500, gr["f"], gr["t"])
    l = int(np.flatnonzero(~isb)[0])
    skip = np.zeros(700, np.uint8)
    skip[l] = 1
    Y0, Y1 = oracle.ybus(gr), oracle.ybus(gr, skip=skip)
    assert Y1.nnz == Y0.nnz - 2
    # with a parallel pair, dropping one keeps the entries
    g3 = three_bus_plus()
    s3 = np.array([0, 0, 0, 1], np.uint8)
    assert oracle.ybus(g3, skip=s3).nnz == oracle.ybus(g3).nnz


def test_bridges_by_brute_force():
    """The generator's bridge list (used to draw N-1 outages) equals removal + BFS."""
    from paper_2302_10736_gb300 import synth
    gr = random_grid(60, 75, 81)
    isb = synth.bridges(60, gr["f"], gr["t"])

    def connected(skip):
        adj = [[] for _ in range(60)]
        for l in range(75):
            if l != skip:
                adj[gr["f"][l]].append(gr["t"][l])
                adj[gr["t"][l]].append(gr["f"][l])
        seen, st = {0}, [0]
        while st:
            u = st.pop()
            for w in adj[u]:
                if w not in seen:
                    seen.add(w)
                    st.append(w)
        return len(seen) == 60

    assert connected(-1)
    for l in range(75):
        assert isb[l] == (not connected(l))


def _read_golden(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for ln in fh:
            ln = ln.strip()
            if ln and not ln.startswith("#"):
                k, v = ln.split()
                vals[k] = int(v)
    return vals


def test_paper_element_count():
    """Sec. V-A.2: the element-wise evaluation of SyntheticUSA computes
    1,665,936 Jacobian element values, 16 per line; a generated grid with the
    same number of lines must yield exactly that many."""
    gv = _read_golden("paper_counts.txt")
    nl = gv["synthetic_usa_jacobian_elements"] // gv["partials_per_line"]
    assert nl * gv["partials_per_line"] == gv["synthetic_usa_jacobian_elements"]
    nb = 82000
    gr = random_grid(nb, nl, 91)
    vm, va = random_state(nb, 91)
    Y = oracle.ybus(gr)
    oracle.elementwise(gr, vm, va, Y, jac=False)
    assert oracle.elementwise.last_count == gv["synthetic_usa_jacobian_elements"]


# ------------------------------------------------------ reduced Jacobian ----

def pin_reduced_two_bus():
    """Bus types of the two-bus line (slack/PQ, slack/PV, PV/slack): the
    reduced Jacobian is the matching block of the hand-derived closed form,
    rows (P2, Q2) x columns (th2, v2) for a PQ bus 2, and F = S - S_spec."""
    gr = two_bus_lossless()
    vm, va = np.array([1.0, 1.0]), np.array([0.0, -0.1])
    s, c = math.sin(0.1), math.cos(0.1)
    Y = oracle.ybus(gr)
    P, Q, J = oracle.elementwise(gr, vm, va, Y)
    errs = []
    cases = [([3, 1], [0, 2, 4], [0, 1, 0, 1], [10 * c, -10 * s, -10 * s, 20 - 10 * c]),
             ([3, 2], [0, 1], [0], [10 * c]),
             ([2, 3], [0, 1], [0], [10 * c]),
             ([3, 4], [0], [], [])]
    for bt, cp, ri, vals in cases:
        colptr, rowidx, v = oracle.jac_reduced(Y, J, bt)
        if list(colptr) != cp or list(rowidx) != ri:
            return math.inf
        errs.append(np.max(np.abs(v - np.array(vals))) if vals else 0.0)
    F = oracle.mismatch(P, Q, [0.5, -0.25], [0.125, 0.0625], [3, 1])
    errs.append(np.max(np.abs(F - np.array([-10 * s + 0.25, 10 * (1 - c) - 0.0625]))))
    return max(errs)


def newton_errors(gr, bustype, vm_true, va_true, vm0, va0, iters=6, transpose=False):
    """Max-norm mismatch of each Newton iterate, solving the reduced system
    (dense solve of the CSC matrix) from (vm0, va0) towards the state whose
    injections define S_spec."""
    Y = oracle.ybus(gr)
    Ps, Qs = oracle.inj_sparse(Y, vm_true, va_true)
    red, npvpq, npq = oracle.reduced_index(bustype)
    n = npvpq + npq
    bt = np.asarray(bustype)
    pvpq, pq = np.flatnonzero((bt == 1) | (bt == 2)), np.flatnonzero(bt == 1)
    vm, va = vm0.copy(), va0.copy()
    out = []
    for _ in range(iters):
        P, Q = oracle.inj_sparse(Y, vm, va)
        F = oracle.mismatch(P, Q, Ps, Qs, bustype)
        out.append(float(np.max(np.abs(F))))
        colptr, rowidx, v = oracle.jac_reduced(Y, oracle.jac_ybus(Y, vm, va), bustype)
        A = np.zeros((n, n))
        for col in range(n):
            for e in range(colptr[col], colptr[col + 1]):
                A[rowidx[e], col] = v[e]
        dx = np.linalg.solve(A.T if transpose else A, -F)
        va[pvpq] += dx[:npvpq]
        vm[pq] += dx[npvpq:]
    return out


def pin_newton_quadratic():
    """A 30-bus meshed grid with phase shifters and a parallel pair, heavily
    loaded (angle differences up to ~0.5 rad): from a start within 2e-3 of
    the solution, Newton's mismatch falls quadratically to round-off."""
    gr = random_grid(30, 45, 41, shift_max=0.2)
    for k in ("f", "t", "g", "b", "bsh", "tap", "shift"):   # a parallel branch
        gr[k] = np.concatenate([gr[k], gr[k][:1] * (1.0 if k in ("f", "t", "tap", "shift") else 0.6)]).astype(gr[k].dtype)
    gr["nl"] += 1
    bt = np.ones(30, np.int32)
    bt[0], bt[[4, 9, 17]] = 3, 2
    vm_t, va_t = random_state(30, 41)
    va_t = va_t - va_t[0]
    rng = np.random.default_rng(41)
    vm0, va0 = vm_t.copy(), va_t.copy()
    vm0[bt == 1] += rng.uniform(-2e-3, 2e-3, int((bt == 1).sum()))
    va0[bt != 3] += rng.uniform(-2e-3, 2e-3, int((bt != 3).sum()))
    e = newton_errors(gr, bt, vm_t, va_t, vm0, va0)
    # quadratic: e_{k+1} <= C e_k^2 while above round-off, round-off reached by iteration 5
    worst = 0.0
    for a, b in zip(e, e[1:]):
        if a > 1e-6:
            worst = max(worst, b / (a * a))
    return max(e[4] * 1e12, worst / 1e3)


def test_reduced_two_bus_closed_form():
    assert pin_reduced_two_bus() < 1e-14


def test_newton_converges_quadratically():
    assert pin_newton_quadratic() < 1.0


def test_newton_pin_rejects_a_transposed_jacobian():
    """The pin has teeth: the same Newton run with the transpose of the
    (non-symmetric) reduced Jacobian does not reach round-off."""
    gr = random_grid(30, 45, 41, shift_max=0.2)
    bt = np.ones(30, np.int32)
    bt[0], bt[[4, 9, 17]] = 3, 2
    vm_t, va_t = random_state(30, 41)
    va_t = va_t - va_t[0]
    rng = np.random.default_rng(41)
    vm0, va0 = vm_t.copy(), va_t.copy()
    vm0[bt == 1] += rng.uniform(-2e-3, 2e-3, int((bt == 1).sum()))
    va0[bt != 3] += rng.uniform(-2e-3, 2e-3, int((bt != 3).sum()))
    good = newton_errors(gr, bt, vm_t, va_t, vm0, va0)
    bad = newton_errors(gr, bt, vm_t, va_t, vm0, va0, transpose=True)
    assert good[4] < 1e-12 and not bad[4] < 1e-9


def test_reduced_pattern_is_a_csc_of_the_kept_entries():
    gr = random_grid(200, 280, 42)
    vm, va = random_state(200, 42)
    Y = oracle.ybus(gr)
    J = oracle.jac_ybus(Y, vm, va)
    bt = np.ones(200, np.int32)
    bt[0], bt[7], bt[11::9] = 3, 4, 2
    colptr, rowidx, v = oracle.jac_reduced(Y, J, bt)
    red, npvpq, npq = oracle.reduced_index(bt)
    n = npvpq + npq
    assert colptr[0] == 0 and colptr[-1] == len(rowidx) and len(colptr) == n + 1
    for col in range(n):
        seg = rowidx[colptr[col]:colptr[col + 1]]
        assert np.all(np.diff(seg) > 0) and np.all((seg >= 0) & (seg < n))
    # dense comparison: the reduced matrix is the full one with rows/columns deleted
    jrp, jci = oracle.jac_pattern(Y)
    full = np.zeros((400, 400))
    for r in range(400):
        full[r, jci[jrp[r]:jrp[r + 1]]] = J[jrp[r]:jrp[r + 1]]
    keep = np.flatnonzero(red >= 0)
    keep = keep[np.argsort(red[keep])]
    A = np.zeros((n, n))
    for col in range(n):
        A[rowidx[colptr[col]:colptr[col + 1]], col] = v[colptr[col]:colptr[col + 1]]
    assert np.array_equal(A, full[np.ix_(keep, keep)])


def test_newton_oracle_finds_the_known_solution():
    """From a start within 1e-3, the oracle's Newton iteration reaches the
    state whose injections define the specification (the solution is unique
    nearby), and its final mismatch is at round-off."""
    pytest.importorskip("scipy")
    from paper_2302_10736_gb300 import synth
    w = synth.workload(1)
    bt = w["bustype"]
    vm_t, va_t = w["vm"][0].copy(), 0.1 * w["va"][0]
    Ps, Qs = oracle.inj_sparse(oracle.ybus(w), vm_t, va_t)
    rng = np.random.default_rng(54)
    vm0, va0 = vm_t.copy(), va_t.copy()
    pq, pvpq = bt == 1, (bt == 1) | (bt == 2)
    vm0[pq] += rng.uniform(-1e-3, 1e-3, int(pq.sum()))
    va0[pvpq] += rng.uniform(-1e-3, 1e-3, int(pvpq.sum()))
    vm, va, it, norms, ok = oracle.newton(w, bt, vm0, va0, Ps, Qs, tol=1e-11)
    assert ok and it <= 6, norms
    assert np.max(np.abs(vm - vm_t)) < 1e-10 and np.max(np.abs(va - va_t)) < 1e-10
    assert np.array_equal(vm[~pq], vm_t[~pq]) and va[0] == va_t[0]   # fixed quantities untouched


def _dense_jacobian_cstep(gr, vm, va, h=1e-30):
    """The dense 2nb x 2nb Jacobian of Eq. (2) by complex step of the real-form
    injections P_i = v_i sum_j v_j (G cos + B sin)(theta_i - theta_j),
    Q_i = v_i sum_j v_j (G sin - B cos)(theta_i - theta_j): columns theta then v."""
    Yd = oracle.ybus(gr).dense()
    G, B = Yd.real, Yd.imag
    nb = gr["nb"]

    def pq(th, v):
        d = th[:, None] - th[None, :]
        vv = v[:, None] * v[None, :]
        return np.concatenate([(vv * (G * np.cos(d) + B * np.sin(d))).sum(1),
                               (vv * (G * np.sin(d) - B * np.cos(d))).sum(1)])

    J = np.zeros((2 * nb, 2 * nb))
    for c in range(2 * nb):
        th, v = va.astype(complex), vm.astype(complex)
        if c < nb:
            th[c] += 1j * h
        else:
            v[c - nb] += 1j * h
        J[:, c] = pq(th, v).imag / h
    return J


def test_target_pattern_assembly_equals_the_dense_jacobian():
    """Alg. 2's placement into a larger pattern, against the dense Jacobian by
    complex step (independent of the sparse code): with a zeroed target every
    position holds the dense J's entry at its (row, column), the added
    positions zero; a pattern without one of Eq. (2)'s entries is rejected."""
    rng = np.random.default_rng(21)
    gr = random_grid(9, 14, 21, shift_max=0.3)
    vm, va = random_state(9, 21)
    Y = oracle.ybus(gr)
    Jd = _dense_jacobian_cstep(gr, vm, va)
    colptr, rowidx = superset_pattern(Y, rng, extra=25)
    out = oracle.jac_target(Y, oracle.jac_ybus(Y, vm, va), colptr, rowidx, np.zeros(len(rowidx)))
    cols = np.repeat(np.arange(2 * Y.nb), np.diff(colptr))
    ref = Jd[rowidx, cols]
    assert np.max(np.abs(out - ref)) <= 1e-12 * np.max(np.abs(Jd))
    assert np.count_nonzero(ref) > 0 and np.count_nonzero(out == 0.0) >= 25
    # a missing entry of the Ybus-block pattern
    jrp, jci = oracle.jac_pattern(Y)
    R, C = 1, int(jci[jrp[1]])
    k = next(k for k in range(colptr[C], colptr[C + 1]) if rowidx[k] == R)
    rowidx2 = np.delete(rowidx, k)
    colptr2 = colptr.copy()
    colptr2[C + 1:] -= 1
    with pytest.raises(ValueError):
        oracle.jac_target(Y, oracle.jac_ybus(Y, vm, va), colptr2, rowidx2, np.zeros(len(rowidx2)))
