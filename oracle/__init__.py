"""CPU FP64 oracle (test infrastructure).

Plain C (oracle.c, compiled with -ffp-contract=off) behind numpy wrappers.
Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may use
it; the product path (paper_2302_10736_gb300) never imports it, and this
module imports nothing from the product package.

Every function follows a passage of arXiv 2302.10736 (cited in oracle.c):
  ybus / ybus_dense        pi-model stamps consistent with Eqs. (5)-(6)
  inj_dense / inj_sparse   Eq. (1), steps of Sec. IV-B.1
  jac_pattern              Eq. (2) block layout on the Ybus pattern (Alg. 2 closed form)
  jac_ybus                 Eqs. (3)-(4), entry by entry
  jac_cstep                complex-step derivative of the real-form injections
  elementwise              Eqs. (5)-(7) + 16 partials, evaluation then reduction
  loss / adjoint_state     L = sum w (S - S_spec)^2 and J^T r
  adjoint_params_cstep     dL/d(g, b, b_sh, tap) by complex step
  loss_central_diff        long-double central differences of L
  reduced_index / jac_reduced / mismatch
                           the Newton step's Jacobian without the slack and PV
                           rows and columns, in CSC order, and its mismatch
                           vector (selection and reordering of Eq. (2)'s entries)
  newton                   Newton-Raphson on the reduced system (the textbook
                           iteration; a sparse LU is its linear-solve step)
  jac_target               Alg. 2: the Jacobian's values placed into a caller's
                           CSC pattern that contains the Ybus-block pattern, by
                           matching row and column coordinates
"""
import ctypes
import os
import shutil
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB = os.path.join(HERE, "liboracle.so")
SRC = os.path.join(HERE, "oracle.c")
_lib = None
_lock = threading.Lock()


def build(force=False):
    """Compile oracle.c in place (gcc, no FMA contraction)."""
    with _lock:
        if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
            return LIB
        cc = os.environ.get("CC") or shutil.which("gcc") or "cc"
        tmp = LIB + ".tmp"
        cmd = [cc, "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-o", tmp,
               SRC, "-lm"]
        r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
        if r.returncode != 0:
            raise RuntimeError("oracle build failed:\n" + r.stdout)
        os.replace(tmp, LIB)
        return LIB


def _load():
    global _lib
    if _lib is None:
        _lib = bind(build())
    return _lib


def bind(path):
    """Load an oracle build at `path` and declare its C signatures."""
    lib = ctypes.CDLL(path)
    i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
    f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
    ci, cd = ctypes.c_int, ctypes.c_double
    vp = ctypes.c_void_p
    lib.or_ybus.argtypes = [ci, ci, i32p, i32p, f64p, f64p, f64p, f64p, f64p, vp, vp, vp, i32p, i32p,
                            f64p, f64p]
    lib.or_ybus.restype = ci
    lib.or_ybus_dense.argtypes = [ci, ci, i32p, i32p, f64p, f64p, f64p, f64p, f64p, vp, vp, f64p, f64p]
    lib.or_inj_dense.argtypes = [ci, f64p, f64p, f64p, f64p, f64p, f64p]
    lib.or_inj_sparse.argtypes = [ci, i32p, i32p, f64p, f64p, f64p, f64p, f64p, f64p]
    lib.or_jac_pattern.argtypes = [ci, i32p, i32p, i32p, i32p]
    lib.or_jac_ybus.argtypes = [ci, i32p, i32p, f64p, f64p, f64p, f64p, f64p]
    lib.or_jac_cstep.argtypes = [ci, i32p, i32p, f64p, f64p, f64p, f64p, f64p]
    lib.or_elementwise.argtypes = [ci, ci, i32p, i32p, f64p, f64p, f64p, f64p, f64p, vp, vp, vp, f64p,
                                   f64p, i32p, i32p, f64p, f64p, vp]
    lib.or_loss.argtypes = [ci, f64p, f64p, f64p, f64p, f64p, f64p]
    lib.or_loss.restype = cd
    lib.or_adjoint_state.argtypes = [ci, i32p, i32p, f64p, f64p, f64p, f64p, f64p, f64p, f64p, f64p,
                                     f64p]
    lib.or_adjoint_params_cstep.argtypes = [ci, ci, i32p, i32p, f64p, f64p, f64p, f64p, f64p, i32p, i32p,
                                            f64p, f64p, f64p, f64p, f64p, f64p, f64p, f64p, f64p, f64p,
                                            f64p, f64p]
    lib.or_loss_central_diff.argtypes = [ci, ci, i32p, i32p, f64p, f64p, f64p, f64p, f64p, vp, vp, f64p,
                                         f64p, f64p, f64p, f64p, f64p, ci, i32p, i32p, cd, f64p]
    lib.or_loss_central_diff.restype = ci
    lib.or_elementwise.restype = ctypes.c_long
    return lib


def _f64(x):
    return np.ascontiguousarray(x, dtype=np.float64)


def _i32(x):
    return np.ascontiguousarray(x, dtype=np.int32)


def _opt(x, dtype):
    """(keep-alive array, pointer) for an optional array argument."""
    if x is None:
        return None, None
    a = np.ascontiguousarray(x, dtype=dtype)
    return a, a.ctypes.data_as(ctypes.c_void_p)


def _branches(gr):
    return (_i32(gr["f"]), _i32(gr["t"]), _f64(gr["g"]), _f64(gr["b"]), _f64(gr["bsh"]), _f64(gr["tap"]),
            _f64(gr["shift"]))


class Ybus:
    """CSR bus admittance matrix produced by the oracle."""

    def __init__(self, nb, rp, ci, yre, yim):
        self.nb, self.rp, self.ci, self.yre, self.yim = nb, rp, ci, yre, yim

    @property
    def nnz(self):
        return int(self.rp[-1])

    def dense(self):
        Y = np.zeros((self.nb, self.nb), complex)
        for i in range(self.nb):
            for e in range(self.rp[i], self.rp[i + 1]):
                Y[i, self.ci[e]] += self.yre[e] + 1j * self.yim[e]
        return Y


def ybus(gr, skip=None):
    lib = _load()
    nb, nl = int(gr["nb"]), int(gr["nl"])
    f, t, g, b, bsh, tap, sh = _branches(gr)
    gs, pgs = _opt(gr.get("gs"), np.float64)
    bs, pbs = _opt(gr.get("bs"), np.float64)
    sk, psk = _opt(None if skip is None else np.asarray(skip, np.uint8), np.uint8)
    cap = max(nb + 2 * nl, 1)
    rp = np.zeros(nb + 1, np.int32)
    ci, yre, yim = np.zeros(cap, np.int32), np.zeros(cap), np.zeros(cap)
    nnz = lib.or_ybus(nb, nl, f, t, g, b, bsh, tap, sh, pgs, pbs, psk, rp, ci, yre, yim)
    if nnz < 0:
        raise MemoryError("or_ybus")
    return Ybus(nb, rp, ci[:nnz].copy(), yre[:nnz].copy(), yim[:nnz].copy())


def ybus_dense(gr):
    lib = _load()
    nb, nl = int(gr["nb"]), int(gr["nl"])
    f, t, g, b, bsh, tap, sh = _branches(gr)
    gs, pgs = _opt(gr.get("gs"), np.float64)
    bs, pbs = _opt(gr.get("bs"), np.float64)
    Yre, Yim = np.zeros(nb * nb), np.zeros(nb * nb)
    lib.or_ybus_dense(nb, nl, f, t, g, b, bsh, tap, sh, pgs, pbs, Yre, Yim)
    return Yre.reshape(nb, nb), Yim.reshape(nb, nb)


def inj_dense(Yre, Yim, vm, va):
    lib = _load()
    nb = len(vm)
    P, Q = np.zeros(nb), np.zeros(nb)
    lib.or_inj_dense(nb, _f64(Yre).ravel(), _f64(Yim).ravel(), _f64(vm), _f64(va), P, Q)
    return P, Q


def inj_sparse(Y, vm, va):
    lib = _load()
    P, Q = np.zeros(Y.nb), np.zeros(Y.nb)
    lib.or_inj_sparse(Y.nb, Y.rp, Y.ci, Y.yre, Y.yim, _f64(vm), _f64(va), P, Q)
    return P, Q


def jac_pattern(Y):
    lib = _load()
    jrp = np.zeros(2 * Y.nb + 1, np.int32)
    jci = np.zeros(max(4 * Y.nnz, 1), np.int32)
    lib.or_jac_pattern(Y.nb, Y.rp, Y.ci, jrp, jci)
    return jrp, jci[:4 * Y.nnz]


def jac_ybus(Y, vm, va):
    lib = _load()
    J = np.zeros(max(4 * Y.nnz, 1))
    lib.or_jac_ybus(Y.nb, Y.rp, Y.ci, Y.yre, Y.yim, _f64(vm), _f64(va), J)
    return J[:4 * Y.nnz]


def jac_cstep(Y, vm, va):
    lib = _load()
    J = np.zeros(max(4 * Y.nnz, 1))
    lib.or_jac_cstep(Y.nb, Y.rp, Y.ci, Y.yre, Y.yim, _f64(vm), _f64(va), J)
    return J[:4 * Y.nnz]


def elementwise(gr, vm, va, Y, skip=None, jac=True):
    """Element-wise method: (P, Q, J or None).  Y gives the pattern of the
    same branch set (build it with the same skip mask)."""
    lib = _load()
    nb, nl = int(gr["nb"]), int(gr["nl"])
    f, t, g, b, bsh, tap, sh = _branches(gr)
    gs, pgs = _opt(gr.get("gs"), np.float64)
    bs, pbs = _opt(gr.get("bs"), np.float64)
    sk, psk = _opt(None if skip is None else np.asarray(skip, np.uint8), np.uint8)
    P, Q = np.zeros(nb), np.zeros(nb)
    J = np.zeros(max(4 * Y.nnz, 1)) if jac else None
    pJ = J.ctypes.data_as(ctypes.c_void_p) if jac else None
    nvalues = lib.or_elementwise(nb, nl, f, t, g, b, bsh, tap, sh, pgs, pbs, psk, _f64(vm), _f64(va), Y.rp, Y.ci,
                                 P, Q, pJ)
    elementwise.last_count = int(nvalues)
    return P, Q, (J[:4 * Y.nnz] if jac else None)


def loss(P, Q, Ps, Qs, wP, wQ):
    lib = _load()
    return float(lib.or_loss(len(P), _f64(P), _f64(Q), _f64(Ps), _f64(Qs), _f64(wP), _f64(wQ)))


def adjoint_state(Y, J, P, Q, Ps, Qs, wP, wQ):
    """(dL/dtheta, dL/dv) = (J11^T r_P + J21^T r_Q, J12^T r_P + J22^T r_Q)."""
    lib = _load()
    gva, gvm = np.zeros(Y.nb), np.zeros(Y.nb)
    lib.or_adjoint_state(Y.nb, Y.rp, Y.ci, _f64(J), _f64(P), _f64(Q), _f64(Ps), _f64(Qs), _f64(wP), _f64(wQ),
                         gva, gvm)
    return gva, gvm


def adjoint_params_cstep(gr, Y, vm, va, Ps, Qs, wP, wQ):
    lib = _load()
    nb, nl = int(gr["nb"]), int(gr["nl"])
    f, t, g, b, bsh, tap, sh = _branches(gr)
    out = [np.zeros(max(nl, 1)) for _ in range(4)]
    lib.or_adjoint_params_cstep(nb, nl, f, t, g, b, bsh, tap, sh, Y.rp, Y.ci, Y.yre, Y.yim, _f64(vm), _f64(va),
                                _f64(Ps), _f64(Qs), _f64(wP), _f64(wQ), *out)
    return tuple(o[:nl] for o in out)


def loss_central_diff(gr, vm, va, Ps, Qs, wP, wQ, kinds, idxs, step=1e-7):
    """Central differences of L; kinds 0 theta, 1 v, 2 g, 3 b, 4 b_sh, 5 tap."""
    lib = _load()
    nb, nl = int(gr["nb"]), int(gr["nl"])
    f, t, g, b, bsh, tap, sh = _branches(gr)
    gs, pgs = _opt(gr.get("gs"), np.float64)
    bs, pbs = _opt(gr.get("bs"), np.float64)
    kinds, idxs = _i32(kinds), _i32(idxs)
    out = np.zeros(max(len(kinds), 1))
    rc = lib.or_loss_central_diff(nb, nl, f, t, g, b, bsh, tap, sh, pgs, pbs, _f64(vm), _f64(va), _f64(Ps),
                                  _f64(Qs), _f64(wP), _f64(wQ), len(kinds), kinds, idxs, step, out)
    if rc != 0:
        raise MemoryError("or_loss_central_diff")
    return out[:len(kinds)]


# ----------------------------------------------------- reduced Jacobian ----
# Bus types as in MATPOWER: 1 PQ, 2 PV, 3 reference (slack), 4 isolated.
# A Newton step on the power-flow equations solves for theta of the PV and PQ
# buses and v of the PQ buses, from the P equations of the PV and PQ buses and
# the Q equations of the PQ buses: the blocks of Eq. (2) restricted to those
# rows and columns.  Ordering (this library's convention): theta / P part
# first, then v / Q, each in ascending bus order.

def reduced_index(bustype):
    """(red, n_pvpq, n_pq): red[R] is the reduced index of full row/column R
    of Eq. (2) (R < nb: theta_R / P_R, R >= nb: v_{R-nb} / Q_{R-nb}), or -1."""
    bt = np.asarray(bustype)
    nb = len(bt)
    pvpq = [i for i in range(nb) if bt[i] in (1, 2)]
    pq = [i for i in range(nb) if bt[i] == 1]
    red = -np.ones(2 * nb, np.int64)
    for k, i in enumerate(pvpq):
        red[i] = k
    for k, i in enumerate(pq):
        red[nb + i] = len(pvpq) + k
    return red, len(pvpq), len(pq)


def jac_reduced(Y, J, bustype):
    """The reduced Jacobian in CSC form (colptr [n+1], rowidx, values): every
    structural entry of the full Jacobian (canonical CSR of jac_pattern,
    values J) whose row and column are both kept, ordered by (column, row).
    Structural zeros are kept."""
    jrp, jci = jac_pattern(Y)
    red, npvpq, npq = reduced_index(bustype)
    n = npvpq + npq
    rows = np.repeat(np.arange(2 * Y.nb), np.diff(jrp))
    r, c = red[rows], red[np.asarray(jci, np.int64)]
    keep = (r >= 0) & (c >= 0)
    r, c, v = r[keep], c[keep], np.asarray(J)[keep]
    order = np.lexsort((r, c))
    colptr = np.zeros(n + 1, np.int64)
    colptr[1:] = np.cumsum(np.bincount(c, minlength=n))
    return colptr, r[order], v[order]


def mismatch(P, Q, Pspec, Qspec, bustype):
    """F = [P - Pspec on the PV and PQ buses; Q - Qspec on the PQ buses]."""
    bt = np.asarray(bustype)
    pvpq = (bt == 1) | (bt == 2)
    pq = bt == 1
    P, Q, Pspec, Qspec = (np.asarray(x, float) for x in (P, Q, Pspec, Qspec))
    return np.concatenate([(P - Pspec)[pvpq], (Q - Qspec)[pq]])


def newton(gr, bustype, vm, va, Pspec, Qspec, tol=1e-10, max_iter=20):
    """Newton-Raphson power flow: x <- x + dx with J_r(x) dx = -F(x), x = (theta
    of PV and PQ buses, v of PQ buses), until max |F| <= tol.  Returns
    (vm, va, iterations, max |F| per iterate, converged)."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    Y = ybus(gr)
    bt = np.asarray(bustype)
    red, npvpq, npq = reduced_index(bt)
    n = npvpq + npq
    pvpq = np.flatnonzero((bt == 1) | (bt == 2))
    pq = np.flatnonzero(bt == 1)
    vm, va = np.array(vm, float), np.array(va, float)
    norms = []
    for it in range(max_iter + 1):
        P, Q = inj_sparse(Y, vm, va)
        F = mismatch(P, Q, Pspec, Qspec, bt)
        norms.append(float(np.max(np.abs(F))) if n else 0.0)
        if norms[-1] <= tol:
            return vm, va, it, norms, True
        if it == max_iter:
            break
        colptr, rowidx, vals = jac_reduced(Y, jac_ybus(Y, vm, va), bt)
        dx = spla.splu(sp.csc_matrix((vals, rowidx, colptr), shape=(n, n))).solve(-F)
        va[pvpq] += dx[:npvpq]
        vm[pq] += dx[npvpq:]
    return vm, va, max_iter, norms, False


# ------------------------------------------------- caller's pattern (Alg. 2) --
def jac_target(Y, J, colptr, rowidx, out):
    """Sec. IV-B.3, Alg. 2: the Jacobian values J (the block layout of
    jac_pattern, rows 0 .. 2nb-1 = P then Q, columns = theta then v) placed
    into a CSC pattern (colptr [2nb+1], rowidx) that contains every entry of
    that layout: an entry at (row R, column C) goes to the position in column
    C whose row is R (the first such position).  `out` keeps its other
    entries.  ValueError if an entry has no position."""
    jrp, jci = jac_pattern(Y)
    colptr = np.asarray(colptr)
    rowidx = np.asarray(rowidx)
    for R in range(2 * Y.nb):
        for p in range(jrp[R], jrp[R + 1]):
            C = int(jci[p])
            hit = -1
            for k in range(int(colptr[C]), int(colptr[C + 1])):
                if rowidx[k] == R:
                    hit = k
                    break
            if hit < 0:
                raise ValueError("pattern lacks entry (%d, %d)" % (R, C))
            out[hit] = J[p]
    return out

