"""C ABI checks that need no GPU: the library builds for sm_103a, loads,
exports every function include/pfgrid.h declares, and rejects invalid grids
on the host before touching the device."""
import ctypes
import subprocess

import numpy as np
import pytest

from paper_2302_10736_gb300 import _build
from gridcases import three_bus_plus


@pytest.fixture(scope="module")
def pf():
    _build.build_pfgrid()
    from paper_2302_10736_gb300 import pfgrid
    return pfgrid


def test_every_declared_symbol_is_exported(pf):
    names = pf.header_functions()
    assert {"ybus_build", "inj_ybus", "inj_elementwise", "jac_ybus", "jac_elementwise"} <= set(names)
    lib = ctypes.CDLL(_build.LIB_PFGRID)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", _build.LIB_PFGRID], stdout=subprocess.PIPE, text=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    assert set(names) <= exported


def test_status_names(pf):
    names = ["PF_OK", "PF_EINVAL", "PF_ENOMEM", "PF_ECUDA", "PF_ETOPO", "PF_EDEVICE", "PF_ETIMEOUT",
             "PF_EUNSUPPORTED", "PF_ENOCONV"]
    for code, name in enumerate(names):
        assert pf._status_name(code) == name and getattr(pf, name) == code
    assert pf._status_name(99) == "PF_UNKNOWN"


@pytest.mark.parametrize("mutate,code", [
    (lambda g: g["t"].__setitem__(0, g["f"][0]), 4),          # self loop
    (lambda g: g["t"].__setitem__(1, 17), 4),                 # bus out of range
    (lambda g: g["f"].__setitem__(2, -1), 4),                 # negative bus
    (lambda g: g["tap"].__setitem__(1, 0.0), 1),              # non-positive tap
    (lambda g: g["tap"].__setitem__(1, -1.05), 1),
    (lambda g: g["g"].__setitem__(0, np.nan), 1),             # non-finite parameter
    (lambda g: g["bsh"].__setitem__(3, np.inf), 1),
    (lambda g: g["gs"].__setitem__(2, np.nan), 1),            # non-finite shunt
])
def test_invalid_grids_rejected_on_host(pf, mutate, code):
    gr = three_bus_plus()
    mutate(gr)
    with pytest.raises(pf.PfError) as ei:
        pf.ybus_build(gr)
    assert ei.value.status == code
    assert pf.last_error()


def test_negative_sizes_rejected(pf):
    gr = three_bus_plus()
    gr["nl"] = -1
    with pytest.raises(pf.PfError) as ei:
        pf.ybus_build(gr)
    assert ei.value.status == 1


def test_oversized_grid_rejected(pf):
    # nb + 2 nl beyond the int32 Jacobian index range: refused before any allocation
    d = pf.pf_grid_desc(400_000_000, 200_000_000, None, None, None, None, None, None, None, None, None)
    out = ctypes.c_void_p()
    st = pf._lib.ybus_build(ctypes.byref(d), None, ctypes.byref(out))
    assert st == 7


@pytest.mark.parametrize("target", [0, 760, 3040])
@pytest.mark.parametrize("window", [128, 256])
@pytest.mark.parametrize("case", ["three_bus_plus", "parallel_star", "single_bus", "empty", "c1", "c2", "c3", "c4",
                                  "c5", "c6"])
def test_layout_selfcheck(pf, case, window, target):
    """Every index the kernels read or write stays inside its buffer (host check)."""
    from gridcases import make_grid
    from paper_2302_10736_gb300 import synth
    if case == "three_bus_plus":
        gr = three_bus_plus()
    elif case == "parallel_star":
        br = [(0, 1 + (i % 5), 1.0, -10.0, 0.0, 1.0, 0.0) for i in range(40)]
        gr = make_grid(7, br)
    elif case == "single_bus":
        gr = make_grid(1, [])
    elif case == "empty":
        gr = make_grid(0, [])
    else:
        w = synth.WORKLOADS[int(case[1])]
        gr = synth.grid(w["nb"], w["nl"], synth.BASE_SEED + int(case[1]), pv_frac=w["pv"])
    pf.grid_selfcheck(gr, window, target)


def test_selfcheck_rejects_bad_window(pf):
    with pytest.raises(pf.PfError):
        pf.grid_selfcheck(three_bus_plus(), 100)


@pytest.mark.parametrize("target", [0, 1520])
@pytest.mark.parametrize("window", [128, 256])
def test_layout_selfcheck_random_numbering(window, target):
    """The ghost-bus layout of a grid numbered without locality."""
    from paper_2302_10736_gb300 import pfgrid, synth
    w = synth.renumber_buses(synth.workload(1), 99)
    pfgrid.grid_selfcheck(w, window, target)


def test_replicated_grid_structure():
    """Host-only: the replicated 82k construction duplicates every bus and line
    with offset bus numbers and joins no copy to another."""
    from paper_2302_10736_gb300 import synth
    base = synth.grid(500, 660, 5)
    rep = synth.replicated(base, 3)
    assert rep["nb"] == 1500 and rep["nl"] == 1980
    for c in range(3):
        sl = slice(c * 660, (c + 1) * 660)
        assert np.array_equal(rep["f"][sl], base["f"] + 500 * c) and np.array_equal(rep["t"][sl], base["t"] + 500 * c)
        assert np.array_equal(rep["g"][sl], base["g"]) and np.array_equal(rep["gs"][c * 500:(c + 1) * 500], base["gs"])
    assert np.all(rep["f"] // 500 == rep["t"] // 500)   # no branch between copies
    w = synth.replicated_workload(2)
    assert w["nb"] == 164000 and w["nl"] == 2 * 104121
