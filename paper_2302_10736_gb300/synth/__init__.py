"""Seeded synthetic inputs: grids shaped like the paper's MATPOWER cases,
voltage states, N-1 outage lists and loss weights.

This module holds no injection or Jacobian arithmetic; it only draws inputs
(via libsynth.so, plain C) that both the CPU oracle and the CUDA path use.

Workloads (seed = 20230221 + workload number; sub-streams per quantity):
  1  2,000 buses /   2,700 branches, 20% PV, one voltage state
  2  70,000 buses /  88,000 branches, 15% PV, one voltage state
  3  10,000 buses /  13,500 branches, 1,024 states (|V|~U[0.93,1.07],
     theta~N(0,0.25)) each paired with a distinct non-bridge outage
  4  25,000 buses /  33,000 branches, one state + a second state for the
     loss targets, weights ~U[0.5,2]
  5  250,000 buses / 330,000 branches, 16 states + loss data as in 4
  6  410,000 buses / 541,000 branches, one state (the size of the paper's
     largest replicated grid)
Replicated grids (replicated_workload): an 82,000-bus / 104,121-branch grid
(the bus and line counts of the paper's SyntheticUSA case) repeated 2 to 5
times as disjoint copies, 164,000 to 410,000 buses (the paper's ultra-large
cases, Sec. V-C).
"""
import ctypes
import os

import numpy as np

from .. import _build

_lib = None

WORKLOADS = {
    1: dict(nb=2000, nl=2700, pv=0.20, nscen=1),
    2: dict(nb=70000, nl=88000, pv=0.15, nscen=1),
    3: dict(nb=10000, nl=13500, pv=0.20, nscen=1024, vlo=0.93, vhi=1.07, sigma=0.25, outages=True),
    4: dict(nb=25000, nl=33000, pv=0.20, nscen=1, loss=True),
    5: dict(nb=250000, nl=330000, pv=0.20, nscen=16, loss=True),
    6: dict(nb=410000, nl=541000, pv=0.20, nscen=1),
}
BASE_SEED = 20230221
# the 82k-bus base of the replicated grids: bus and line counts of SyntheticUSA
REPLICA_BASE = dict(nb=82000, nl=104121, pv=0.20)


def _load():
    global _lib
    if _lib is None:
        path = _build.build_synth()
        lib = ctypes.CDLL(path)
        i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
        f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
        u8p = np.ctypeslib.ndpointer(np.uint8, flags="C_CONTIGUOUS")
        ci, cu64, cd = ctypes.c_int, ctypes.c_uint64, ctypes.c_double
        lib.sy_grid.argtypes = [ci, ci, cu64, cd, cd, cd, cd, i32p, i32p, f64p, f64p, f64p, f64p, f64p,
                                f64p, f64p, i32p, f64p, f64p]
        lib.sy_voltages.argtypes = [ci, ci, cu64, ci, cd, cd, cd, ci, f64p, f64p]
        lib.sy_bridges.argtypes = [ci, ci, i32p, i32p, u8p]
        lib.sy_outages.argtypes = [ci, u8p, ci, cu64, i32p]
        lib.sy_weights.argtypes = [ci, cu64, cd, cd, f64p, f64p]
        lib.sy_randint.argtypes = [cu64, ci, ci, ci, i32p]
        _lib = lib
    return _lib


def grid(nb, nl, seed, tx_frac=0.2, shift_max=0.0, shunt_frac=0.05, pv_frac=0.2):
    """One seeded grid as a dict of numpy arrays (branch arrays [nl], bus [nb])."""
    lib = _load()
    out = dict(
        nb=int(nb), nl=int(nl),
        f=np.zeros(nl, np.int32), t=np.zeros(nl, np.int32),
        g=np.zeros(nl), b=np.zeros(nl), bsh=np.zeros(nl), tap=np.zeros(nl), shift=np.zeros(nl),
        gs=np.zeros(nb), bs=np.zeros(nb), bustype=np.zeros(nb, np.int32),
        x=np.zeros(nb), y=np.zeros(nb),
    )
    rc = lib.sy_grid(nb, nl, seed, tx_frac, shift_max, shunt_frac, pv_frac, out["f"], out["t"], out["g"],
                     out["b"], out["bsh"], out["tap"], out["shift"], out["gs"], out["bs"], out["bustype"],
                     out["x"], out["y"])
    if rc != 0:
        raise ValueError("sy_grid failed (rc=%d) for nb=%d nl=%d" % (rc, nb, nl))
    return out


def voltages(nb, nscen, seed, stream=0, vlo=0.95, vhi=1.05, sigma=0.2, slack=0):
    """(vm, va) arrays of shape [nscen, nb]."""
    lib = _load()
    vm = np.zeros(nb * nscen)
    va = np.zeros(nb * nscen)
    lib.sy_voltages(nb, nscen, seed, stream, vlo, vhi, sigma, slack, vm, va)
    return vm.reshape(nscen, nb), va.reshape(nscen, nb)


def bridges(nb, f, t):
    lib = _load()
    nl = len(f)
    out = np.zeros(max(nl, 1), np.uint8)
    rc = lib.sy_bridges(nb, nl, np.ascontiguousarray(f, np.int32), np.ascontiguousarray(t, np.int32), out)
    if rc != 0:
        raise ValueError("sy_bridges failed")
    return out[:nl].astype(bool)


def outages(is_bridge, nscen, seed):
    lib = _load()
    isb = np.ascontiguousarray(np.asarray(is_bridge, np.uint8))
    out = np.zeros(max(nscen, 1), np.int32)
    rc = lib.sy_outages(len(isb), isb, nscen, seed, out)
    if rc != 0:
        raise ValueError("not enough non-bridge branches for %d outages" % nscen)
    return out[:nscen]


def weights(n, seed, lo=0.5, hi=2.0):
    lib = _load()
    wP, wQ = np.zeros(n), np.zeros(n)
    lib.sy_weights(n, seed, lo, hi, wP, wQ)
    return wP, wQ


def randint(seed, stream, count, n):
    lib = _load()
    out = np.zeros(max(count, 1), np.int32)
    lib.sy_randint(seed, stream, count, n, out)
    return out[:count]


def renumber_buses(gr, seed, stream=7):
    """The same grid (and voltage states) with its buses renumbered by a
    seeded random permutation: old bus i becomes bus perm[i].  Destroys the
    spatial locality of the numbering (a sensitivity case)."""
    nb = gr["nb"]
    keys = randint(seed, stream, nb, 2**31 - 1)
    perm = np.empty(nb, np.int64)
    perm[np.argsort(keys, kind="stable")] = np.arange(nb)
    out = dict(gr)
    out["f"] = perm[gr["f"]].astype(np.int32)
    out["t"] = perm[gr["t"]].astype(np.int32)
    for key in ("gs", "bs", "bustype", "x", "y", "vm2", "va2", "wP", "wQ"):
        if key in gr:
            v = np.empty_like(gr[key])
            v[perm] = gr[key]
            out[key] = v
    for key in ("vm", "va"):
        if key in gr:
            v = np.empty_like(gr[key])
            v[:, perm] = gr[key]
            out[key] = v
    out["perm"] = perm
    return out


def workload(k, nscen=None):
    """Full seeded input set of workload k (see the module docstring).

    nscen overrides the number of voltage states (outages are then the first
    nscen of the same draw order only if the override is not larger)."""
    w = WORKLOADS[k]
    seed = BASE_SEED + k
    ns = w["nscen"] if nscen is None else int(nscen)
    gr = grid(w["nb"], w["nl"], seed, pv_frac=w["pv"])
    vm, va = voltages(w["nb"], ns, seed, 0, w.get("vlo", 0.95), w.get("vhi", 1.05), w.get("sigma", 0.2))
    gr.update(workload=k, seed=seed, nscen=ns, vm=vm, va=va)
    if w.get("outages"):
        isb = bridges(w["nb"], gr["f"], gr["t"])
        gr["outage"] = outages(isb, ns, seed)
    if w.get("loss"):
        vm2, va2 = voltages(w["nb"], 1, seed, 1)
        gr["vm2"], gr["va2"] = vm2[0], va2[0]
        gr["wP"], gr["wQ"] = weights(w["nb"], seed)
    return gr


def replicated(base, copies):
    """`copies` disjoint copies of a grid: copy c's buses are c * nb + the
    base bus, its branches the base branches between them (every bus and line
    duplicated, no tie between copies)."""
    nb, nl = int(base["nb"]), int(base["nl"])
    off_b = np.repeat(np.arange(copies, dtype=np.int64) * nb, nl)
    out = dict(nb=nb * copies, nl=nl * copies)
    out["f"] = (np.tile(base["f"].astype(np.int64), copies) + off_b).astype(np.int32)
    out["t"] = (np.tile(base["t"].astype(np.int64), copies) + off_b).astype(np.int32)
    for key in ("g", "b", "bsh", "tap", "shift"):
        out[key] = np.tile(base[key], copies)
    for key in ("gs", "bs", "bustype", "x", "y"):
        if key in base:
            out[key] = np.tile(base[key], copies)
    return out


def replicated_workload(copies, same_state=False):
    """The 82k-bus base grid repeated `copies` times (2 .. 5 in the paper) with
    one voltage state: drawn for the whole grid, or (same_state) the base
    grid's state repeated in every copy."""
    seed = BASE_SEED + 7
    base = grid(REPLICA_BASE["nb"], REPLICA_BASE["nl"], seed, pv_frac=REPLICA_BASE["pv"])
    out = replicated(base, copies)
    if same_state:
        vm, va = voltages(base["nb"], 1, seed)
        vm, va = np.tile(vm, (1, copies)), np.tile(va, (1, copies))
    else:
        vm, va = voltages(out["nb"], 1, seed)
    out.update(workload="replicated_82k_x%d" % copies, seed=seed, nscen=1, vm=vm, va=va, copies=copies,
               base_nb=base["nb"], base_nl=base["nl"])
    return out
