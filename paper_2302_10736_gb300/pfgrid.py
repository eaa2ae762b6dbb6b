"""Thin ctypes binding of libpfgrid.so (the C ABI declared in include/pfgrid.h).

Argument marshalling only: every evaluation step runs in the library's CUDA
kernels.  Device arrays are torch CUDA tensors (float64, contiguous); the
stream defaults to torch's current stream.  There is no CPU fallback: if the
library is missing or fails to load, importing this module raises.
"""
import ctypes
import os
import re

import numpy as np

from . import _build

# PFGRID_LIB may name another build of the same library (the phase-probe build)
LIB_PATH = os.environ.get("PFGRID_LIB") or _build.LIB_PFGRID
HEADER = os.path.join(_build.INCLUDE, "pfgrid.h")

PF_OK, PF_EINVAL, PF_ENOMEM, PF_ECUDA, PF_ETOPO, PF_EDEVICE, PF_ETIMEOUT, PF_EUNSUPPORTED, PF_ENOCONV = range(9)


class PfError(RuntimeError):
    def __init__(self, status, name, msg):
        super().__init__("%s failed: %s (%s)" % (name, _status_name(status), msg))
        self.status = status


class pf_grid_desc(ctypes.Structure):
    _fields_ = [("nb", ctypes.c_int32), ("nl", ctypes.c_int32),
                ("from_", ctypes.c_void_p), ("to", ctypes.c_void_p),
                ("g", ctypes.c_void_p), ("b", ctypes.c_void_p), ("bsh", ctypes.c_void_p),
                ("tap", ctypes.c_void_p), ("shift", ctypes.c_void_p),
                ("gs", ctypes.c_void_p), ("bs", ctypes.c_void_p)]


class pf_config(ctypes.Structure):
    _fields_ = [("ybus_lanes", ctypes.c_int32), ("ybus_block", ctypes.c_int32), ("ew_window", ctypes.c_int32),
                ("ybus_fused", ctypes.c_int32)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class pf_batch_config(ctypes.Structure):
    _fields_ = [("window", ctypes.c_int32), ("terminals_per_thread", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("adjoint_form", ctypes.c_int32), ("ybus_lanes", ctypes.c_int32), ("ybus_block", ctypes.c_int32)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class pf_trace_rec(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_int32), ("ms", ctypes.c_float)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libpfgrid.so is not built (%s); run __graft_entry__.build() first" % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    vp, i32, pi32 = ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)
    st = ctypes.c_int32
    sig = {
        "pf_status_str": (ctypes.c_char_p, [st]),
        "pf_last_error": (ctypes.c_char_p, []),
        "ybus_build": (st, [ctypes.POINTER(pf_grid_desc), vp, ctypes.POINTER(vp)]),
        "grid_destroy": (None, [vp]),
        "grid_info": (st, [vp, pi32, pi32, pi32]),
        "grid_set_params": (st, [vp, vp, vp, vp, vp, vp, vp, vp, vp]),
        "ybus_get": (st, [vp, pi32, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp)]),
        "jac_pattern": (st, [vp, pi32, ctypes.POINTER(vp), ctypes.POINTER(vp)]),
        "inj_ybus": (st, [vp, vp, vp, vp, vp, vp]),
        "inj_elementwise": (st, [vp, vp, vp, vp, vp, vp]),
        "jac_ybus": (st, [vp, vp, vp, vp, vp, vp, vp]),
        "jac_elementwise": (st, [vp, vp, vp, vp, vp, vp, vp]),
        "eval_host": (st, [vp, i32, vp, vp, vp, vp, vp, vp]),
        "eval_host_async": (st, [vp, i32, vp, vp, vp, vp, vp, vp]),
        "grid_get_config": (st, [vp, ctypes.POINTER(pf_config)]),
        "grid_set_config": (st, [vp, ctypes.POINTER(pf_config), vp]),
        "grid_autotune": (st, [vp, vp, vp, i32, vp, ctypes.POINTER(pf_config)]),
        "grid_check_error": (st, [vp, vp]),
        "pf_kernel_name": (ctypes.c_char_p, [i32]),
        "grid_trace_enable": (st, [vp, i32]),
        "grid_trace_read": (st, [vp, ctypes.POINTER(pf_trace_rec), i32, pi32]),
        "grid_selfcheck": (st, [ctypes.POINTER(pf_grid_desc), i32, i32]),
        "phasor": (st, [i32, vp, vp, vp, vp, vp]),
        "grid_inject_barrier_fault": (st, [vp, vp]),
        "inj_ybus_noalloc": (st, [i32, vp, vp, vp, vp, vp, vp, vp, vp]),
        "grid_set_bus_types": (st, [vp, vp, vp]),
        "pf_debug_fail_allocations": (st, [i32]),
        "jac_elementwise_study": (st, [vp, i32, vp, vp, vp, vp, vp, vp]),
        "inj_ybus_study": (st, [vp, i32, vp, vp, vp, vp, vp]),
        "jac_reduced_info": (st, [vp, pi32, pi32, ctypes.POINTER(ctypes.c_int64)]),
        "jac_reduced_pattern": (st, [vp, ctypes.POINTER(vp), ctypes.POINTER(vp)]),
        "jac_reduced": (st, [vp, i32, vp, vp, vp, vp, vp, vp, vp]),
        "powerflow_newton": (st, [vp, i32, vp, vp, vp, vp, ctypes.c_double, i32, pi32, ctypes.POINTER(ctypes.c_double),
                                  vp]),
        "jac_set_target_pattern": (st, [vp, vp, vp, ctypes.c_int64, vp]),
        "jac_target": (st, [vp, i32, vp, vp, vp, vp, vp, vp]),
        "jac_reduced_solve": (st, [vp, vp, vp, vp, vp]),
        "pf_phase_probe_read": (st, [vp, i32, pi32]),
        "fp64_peak_probe": (st, [i32, i32, vp, ctypes.POINTER(ctypes.c_int64), vp]),
        "grid_ew_windows": (st, [vp, vp, i32, pi32]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = _load()


def _status_name(s):
    return _lib.pf_status_str(s).decode()


def last_error():
    return _lib.pf_last_error().decode()


def _check(status, name):
    if status != PF_OK:
        raise PfError(status, name, last_error())


def header_functions():
    """Names of the functions declared in include/pfgrid.h."""
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"^[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(", txt, flags=re.M)))


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _dptr(x, name, n=None):
    """Device pointer of a float64 contiguous CUDA tensor (None -> NULL)."""
    if x is None:
        return None
    import torch
    if not (isinstance(x, torch.Tensor) and x.is_cuda and x.dtype == torch.float64 and x.is_contiguous()):
        raise TypeError("%s must be a contiguous float64 CUDA tensor" % name)
    if n is not None and x.numel() < n:
        raise ValueError("%s has %d elements, needs %d" % (name, x.numel(), n))
    return ctypes.c_void_p(x.data_ptr())


def _hptr(a, dtype):
    if a is None:
        return None, None
    arr = np.ascontiguousarray(a, dtype=dtype)
    return arr, arr.ctypes.data_as(ctypes.c_void_p)


class Grid:
    """Owner of a pf_grid handle."""

    def __init__(self, handle):
        self.handle = ctypes.c_void_p(handle)
        nb, nl, nnz = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check(_lib.grid_info(self.handle, ctypes.byref(nb), ctypes.byref(nl), ctypes.byref(nnz)), "grid_info")
        self.nb, self.nl, self.nnz = nb.value, nl.value, nnz.value

    @property
    def nnzJ(self):
        return 4 * self.nnz

    def close(self):
        if self.handle:
            _lib.grid_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _desc(gr, keep):
    nb, nl = int(gr["nb"]), int(gr["nl"])

    def h(key, dtype):
        arr, p = _hptr(gr.get(key), dtype)
        keep.append(arr)
        return p

    return pf_grid_desc(nb, nl, h("f", np.int32), h("t", np.int32), h("g", np.float64), h("b", np.float64),
                        h("bsh", np.float64), h("tap", np.float64), h("shift", np.float64), h("gs", np.float64),
                        h("bs", np.float64))


def grid_selfcheck(gr, window, nwin_target=0):
    """Host-only check of every index invariant of the kernels (no GPU)."""
    keep = []
    d = _desc(gr, keep)
    _check(_lib.grid_selfcheck(ctypes.byref(d), int(window), int(nwin_target)), "grid_selfcheck")


def ybus_build(gr, stream=None):
    """Build a grid from a dict with nb, nl, f, t, g, b, bsh, tap, shift and
    optional gs, bs (host arrays)."""
    keep = []
    d = _desc(gr, keep)
    out = ctypes.c_void_p()
    s = ctypes.c_void_p(0) if stream is None and not _cuda_ready() else _stream(stream)
    _check(_lib.ybus_build(ctypes.byref(d), s, ctypes.byref(out)), "ybus_build")
    return Grid(out.value)


def _cuda_ready():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def grid_set_params(grid, g, b, bsh, tap, shift, gs=None, bs=None, stream=None):
    n, nb = grid.nl, grid.nb
    _check(_lib.grid_set_params(grid.handle, _dptr(g, "g", n), _dptr(b, "b", n), _dptr(bsh, "bsh", n),
                                _dptr(tap, "tap", n), _dptr(shift, "shift", n), _dptr(gs, "gs", nb),
                                _dptr(bs, "bs", nb), _stream(stream)), "grid_set_params")


def _device_copy(src_ptr, n, dtype):
    import torch
    out = torch.empty(n, dtype=dtype, device="cuda")
    if n:
        cudart = _cudart()
        nbytes = n * out.element_size()
        rc = cudart.cudaMemcpy(ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(src_ptr), ctypes.c_size_t(nbytes), 3)
        if rc != 0:
            raise RuntimeError("cudaMemcpy failed (%d)" % rc)
    return out


_cudart_lib = None


def _cudart():
    global _cudart_lib
    if _cudart_lib is None:
        for name in ("libcudart.so.13", "libcudart.so"):
            try:
                _cudart_lib = ctypes.CDLL(name)
                break
            except OSError:
                continue
        _cudart_lib.cudaMemcpy.restype = ctypes.c_int
        _cudart_lib.cudaMemcpy.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int]
    return _cudart_lib


def ybus_get(grid):
    """(rowptr, colidx, values[nnz, 2]) as new torch CUDA tensors (copies)."""
    import torch
    nnz = ctypes.c_int32()
    rp, ci, yv = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
    _check(_lib.ybus_get(grid.handle, ctypes.byref(nnz), ctypes.byref(rp), ctypes.byref(ci), ctypes.byref(yv)),
           "ybus_get")
    n = nnz.value
    return (_device_copy(rp.value, grid.nb + 1, torch.int32), _device_copy(ci.value, n, torch.int32),
            _device_copy(yv.value, 2 * n, torch.float64).view(n, 2))


def jac_pattern(grid):
    """(rowptr, colidx) of the canonical J as new torch CUDA tensors."""
    import torch
    nnzJ = ctypes.c_int32()
    rp, ci = ctypes.c_void_p(), ctypes.c_void_p()
    _check(_lib.jac_pattern(grid.handle, ctypes.byref(nnzJ), ctypes.byref(rp), ctypes.byref(ci)), "jac_pattern")
    return _device_copy(rp.value, 2 * grid.nb + 1, torch.int32), _device_copy(ci.value, nnzJ.value, torch.int32)


def inj_ybus(grid, vm, va, P, Q, stream=None):
    n = grid.nb
    _check(_lib.inj_ybus(grid.handle, _dptr(vm, "vm", n), _dptr(va, "va", n), _dptr(P, "P", n), _dptr(Q, "Q", n),
                         _stream(stream)), "inj_ybus")


def inj_elementwise(grid, vm, va, P, Q, stream=None):
    n = grid.nb
    _check(_lib.inj_elementwise(grid.handle, _dptr(vm, "vm", n), _dptr(va, "va", n), _dptr(P, "P", n),
                                _dptr(Q, "Q", n), _stream(stream)), "inj_elementwise")


def jac_ybus(grid, vm, va, P, Q, J, stream=None):
    n = grid.nb
    _check(_lib.jac_ybus(grid.handle, _dptr(vm, "vm", n), _dptr(va, "va", n), _dptr(P, "P", n), _dptr(Q, "Q", n),
                         _dptr(J, "J", grid.nnzJ), _stream(stream)), "jac_ybus")


def jac_elementwise(grid, vm, va, P, Q, J, stream=None):
    n = grid.nb
    _check(_lib.jac_elementwise(grid.handle, _dptr(vm, "vm", n), _dptr(va, "va", n), _dptr(P, "P", n),
                                _dptr(Q, "Q", n), _dptr(J, "J", grid.nnzJ), _stream(stream)), "jac_elementwise")


def _eval_host_call(fn, name, grid, method, vm, va, P, Q, J, stream):
    for nm, a, n in (("vm", vm, grid.nb), ("va", va, grid.nb), ("P", P, grid.nb), ("Q", Q, grid.nb),
                     ("J", J, grid.nnzJ)):
        if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous and a.size >= n):
            raise TypeError("%s must be a contiguous float64 numpy array with >= %d elements" % (nm, n))
    m = {"ybus": 0, "elementwise": 1}.get(method, method)
    vp = lambda a: ctypes.c_void_p(a.ctypes.data)
    _check(fn(grid.handle, int(m), vp(vm), vp(va), vp(P), vp(Q), vp(J), _stream(stream)), name)


def eval_host(grid, method, vm, va, P, Q, J, stream=None):
    """Host numpy buffers in and out (vm, va, P, Q [nb]; J [4 nnzY]).  With
    page-locked buffers the element-wise kernel reads and writes them directly.
    Returns once the results are in P, Q, J.  `stream` as an integer handle
    skips the per-call look-up of torch's current stream."""
    _eval_host_call(_lib.eval_host, "eval_host", grid, method, vm, va, P, Q, J, stream)


def eval_host_async(grid, method, vm, va, P, Q, J, stream=None):
    """eval_host that returns once the work is enqueued: all five buffers must
    be page-locked, and P, Q, J hold the results after `stream` is
    synchronized."""
    _eval_host_call(_lib.eval_host_async, "eval_host_async", grid, method, vm, va, P, Q, J, stream)


def phasor(vm, va, U, V, stream=None):
    """Phasor step alone: U [n, 4] = (cos, sin, vm, 1/vm), V [n, 2] = vm (cos, sin)."""
    n = vm.numel()
    _check(_lib.phasor(n, _dptr(vm, "vm", n), _dptr(va, "va", n), _dptr(U, "U", 4 * n), _dptr(V, "V", 2 * n),
                       _stream(stream)), "phasor")


def inj_ybus_noalloc(rowptr, colidx, yval, vm, va, P, Q, stream=None):
    """Ybus-method injections from a caller-owned CSR Ybus (int32 rowptr/colidx,
    float64 yval [nnz, 2]); the library allocates nothing for this call.  The
    lengths of colidx and yval are checked against rowptr[-1] (one read of
    that entry); column indices must lie in [0, nb)."""
    import torch
    nb = rowptr.numel() - 1
    for name, x in (("rowptr", rowptr), ("colidx", colidx)):
        if not (isinstance(x, torch.Tensor) and x.is_cuda and x.dtype == torch.int32 and x.is_contiguous()):
            raise TypeError("%s must be a contiguous int32 CUDA tensor" % name)
    cur = torch.cuda.current_device()
    for name, x in (("rowptr", rowptr), ("colidx", colidx), ("yval", yval), ("vm", vm), ("va", va), ("P", P),
                    ("Q", Q)):
        if isinstance(x, torch.Tensor) and x.is_cuda and x.device.index != cur:
            raise ValueError("%s is on cuda:%d, the current device is cuda:%d" % (name, x.device.index, cur))
    # the C call cannot read rowptr on the host: check the array lengths here
    nnz = int(rowptr[-1].item()) if nb >= 0 and rowptr.numel() else 0
    if colidx.numel() < nnz:
        raise ValueError("colidx has %d entries, rowptr[-1] = %d" % (colidx.numel(), nnz))
    _check(_lib.inj_ybus_noalloc(nb, ctypes.c_void_p(rowptr.data_ptr()), ctypes.c_void_p(colidx.data_ptr()),
                                 _dptr(yval, "yval", 2 * nnz), _dptr(vm, "vm", nb), _dptr(va, "va", nb),
                                 _dptr(P, "P", nb), _dptr(Q, "Q", nb), _stream(stream)), "inj_ybus_noalloc")


def grid_inject_barrier_fault(grid, stream=None):
    _check(_lib.grid_inject_barrier_fault(grid.handle, _stream(stream)), "grid_inject_barrier_fault")


def grid_get_config(grid):
    c = pf_config()
    _check(_lib.grid_get_config(grid.handle, ctypes.byref(c)), "grid_get_config")
    return c.as_dict()


def grid_set_config(grid, stream=None, **kw):
    c = pf_config(**{**grid_get_config(grid), **kw})
    _check(_lib.grid_set_config(grid.handle, ctypes.byref(c), _stream(stream)), "grid_set_config")


def grid_autotune(grid, vm, va, reps=20, stream=None):
    c = pf_config()
    _check(_lib.grid_autotune(grid.handle, _dptr(vm, "vm", grid.nb), _dptr(va, "va", grid.nb), int(reps),
                              _stream(stream), ctypes.byref(c)), "grid_autotune")
    return c.as_dict()


def grid_check_error(grid, stream=None):
    _check(_lib.grid_check_error(grid.handle, _stream(stream)), "grid_check_error")


def kernel_name(k):
    return _lib.pf_kernel_name(int(k)).decode()


def grid_trace_enable(grid, capacity):
    _check(_lib.grid_trace_enable(grid.handle, int(capacity)), "grid_trace_enable")


def grid_ew_windows(grid):
    """The element-wise windows: int32 array [nwin, 5] of {first bus, buses,
    first terminal, terminals, phasor slots}."""
    n = ctypes.c_int32()
    _check(_lib.grid_ew_windows(grid.handle, None, 0, ctypes.byref(n)), "grid_ew_windows")
    out = np.zeros((max(n.value, 0), 5), dtype=np.int32)
    if n.value:
        _check(_lib.grid_ew_windows(grid.handle, out.ctypes.data, n.value, ctypes.byref(n)), "grid_ew_windows")
    return out


def grid_trace_read(grid, cap=1 << 16):
    """List of (kernel name, ms) for the launches traced since the last read."""
    buf = (pf_trace_rec * cap)()
    n = ctypes.c_int32()
    _check(_lib.grid_trace_read(grid.handle, buf, cap, ctypes.byref(n)), "grid_trace_read")
    return [(kernel_name(buf[i].kernel), float(buf[i].ms)) for i in range(n.value)]


def jac_elementwise_study(grid, strategy, vm, va, P, Q, J, stream=None):
    """The paper's two-step element-wise structure (strategy 0 gather, 1 copy-add)."""
    nb = grid.nb
    _check(_lib.jac_elementwise_study(grid.handle, int(strategy), _dptr(vm, "vm", nb), _dptr(va, "va", nb),
                                      _dptr(P, "P", nb), _dptr(Q, "Q", nb), _dptr(J, "J", grid.nnzJ), _stream(stream)),
           "jac_elementwise_study")


def inj_ybus_study(grid, separate, vm, va, P, Q, stream=None):
    """Ybus injections with interleaved (0) or separate (1) voltage storage."""
    nb = grid.nb
    _check(_lib.inj_ybus_study(grid.handle, int(separate), _dptr(vm, "vm", nb), _dptr(va, "va", nb),
                               _dptr(P, "P", nb), _dptr(Q, "Q", nb), _stream(stream)), "inj_ybus_study")


def fp64_peak_probe(ctas, iters, sink, stream=None):
    """Launch the FP64 FMA throughput kernel; returns the FMAs it executes."""
    n = ctypes.c_int64()
    _check(_lib.fp64_peak_probe(int(ctas), int(iters), _dptr(sink, "sink", 1), ctypes.byref(n), _stream(stream)),
           "fp64_peak_probe")
    return n.value


def phase_probe_read(max_windows=8192):
    """Per-window phase records of the last single element-wise evaluation
    (probe builds only): uint64 array [n, 9], see pf_phase_probe_read."""
    out = np.zeros((max_windows, 9), np.uint64)
    n = ctypes.c_int32()
    _check(_lib.pf_phase_probe_read(out.ctypes.data_as(ctypes.c_void_p), int(max_windows), ctypes.byref(n)),
           "pf_phase_probe_read")
    return out[:n.value]


def debug_fail_allocations(after):
    """Test hook: the next `after` device allocations succeed, later ones fail
    (PF_ENOMEM); -1 turns it off."""
    _check(_lib.pf_debug_fail_allocations(int(after)), "pf_debug_fail_allocations")


# --------------------------------------------------- reduced Jacobian --

def grid_set_bus_types(grid, bus_type, stream=None):
    """Bus types (1 PQ, 2 PV, 3 reference, 4 isolated) for jac_reduced."""
    bt = np.ascontiguousarray(bus_type, dtype=np.int32)
    if bt.size != grid.nb:
        raise ValueError("bus_type must have nb = %d entries" % grid.nb)
    _check(_lib.grid_set_bus_types(grid.handle, bt.ctypes.data_as(ctypes.c_void_p), _stream(stream)),
           "grid_set_bus_types")


def jac_reduced_info(grid):
    """(n, n_pvpq, nnz) of the reduced system."""
    n, npvpq, nnz = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
    _check(_lib.jac_reduced_info(grid.handle, ctypes.byref(n), ctypes.byref(npvpq), ctypes.byref(nnz)),
           "jac_reduced_info")
    return n.value, npvpq.value, nnz.value


def jac_reduced_pattern(grid):
    """Host copies (colptr [n+1], rowidx [nnz]) of the reduced CSC pattern."""
    n, _, nnz = jac_reduced_info(grid)
    cp, ri = ctypes.c_void_p(), ctypes.c_void_p()
    _check(_lib.jac_reduced_pattern(grid.handle, ctypes.byref(cp), ctypes.byref(ri)), "jac_reduced_pattern")
    import torch
    return (_device_copy(cp.value, n + 1, torch.int32).cpu().numpy(),
            _device_copy(ri.value, nnz, torch.int32).cpu().numpy())


def jac_reduced(grid, method, vm, va, Pspec, Qspec, F, Jr, stream=None):
    """Mismatch F [n] and reduced Jacobian values Jr [nnz] (CSC order)."""
    n, _, nnz = jac_reduced_info(grid)
    nb = grid.nb
    m = {"ybus": 0, "elementwise": 1}.get(method, method)
    _check(_lib.jac_reduced(grid.handle, int(m), _dptr(vm, "vm", nb), _dptr(va, "va", nb),
                            _dptr(Pspec, "Pspec", nb), _dptr(Qspec, "Qspec", nb), _dptr(F, "F", n),
                            _dptr(Jr, "Jr", nnz), _stream(stream)), "jac_reduced")


def jac_set_target_pattern(grid, colptr, rowidx, stream=None):
    """A caller's Jacobian pattern (CSC, 2nb x 2nb, host int32 arrays) that
    contains the Ybus-block pattern (Alg. 2); later jac_target calls write
    into it."""
    cp, cpp = _hptr(colptr, np.int32)
    ri, rip = _hptr(rowidx, np.int32)
    if cp.size != 2 * grid.nb + 1:
        raise ValueError("colptr needs 2 nb + 1 = %d entries" % (2 * grid.nb + 1))
    grid._target_nnz = int(ri.size)
    _check(_lib.jac_set_target_pattern(grid.handle, cpp, rip, int(ri.size), _stream(stream)), "jac_set_target_pattern")


def jac_target(grid, method, vm, va, P, Q, Jt, stream=None):
    """Jacobian values into the caller's pattern: Jt [nnz] (only the Ybus-block
    positions are written), and P, Q [nb] unless None."""
    nb = grid.nb
    m = {"ybus": 0, "elementwise": 1}.get(method, method)
    nnz = getattr(grid, "_target_nnz", 0)
    _check(_lib.jac_target(grid.handle, int(m), _dptr(vm, "vm", nb), _dptr(va, "va", nb), _dptr(P, "P", nb),
                           _dptr(Q, "Q", nb), _dptr(Jt, "Jt", nnz), _stream(stream)), "jac_target")


def jac_reduced_solve(grid, Jr, F, dx, stream=None):
    """dx [n] with J_r dx = F, J_r given by its values Jr [nnz] in jac_reduced's
    CSC order (the library's sparse LU)."""
    n, _, nnz = jac_reduced_info(grid)
    _check(_lib.jac_reduced_solve(grid.handle, _dptr(Jr, "Jr", nnz), _dptr(F, "F", n), _dptr(dx, "dx", n),
                                  _stream(stream)), "jac_reduced_solve")


def powerflow_newton(grid, method, vm, va, Pspec, Qspec, tol=1e-10, max_iter=20, stream=None):
    """Newton-Raphson power flow from (vm, va) (device tensors, updated in
    place).  Returns (converged, iterations, final max |F|)."""
    nb = grid.nb
    m = {"ybus": 0, "elementwise": 1}.get(method, method)
    it, fmax = ctypes.c_int32(), ctypes.c_double()
    st = _lib.powerflow_newton(grid.handle, int(m), _dptr(vm, "vm", nb), _dptr(va, "va", nb),
                               _dptr(Pspec, "Pspec", nb), _dptr(Qspec, "Qspec", nb), float(tol), int(max_iter),
                               ctypes.byref(it), ctypes.byref(fmax), _stream(stream))
    if st not in (PF_OK, PF_ENOCONV):
        _check(st, "powerflow_newton")
    return st == PF_OK, it.value, fmax.value


# ------------------------------------------------------------------ batches --

def _bind_batches():
    vp, i32 = ctypes.c_void_p, ctypes.c_int32
    st = ctypes.c_int32
    sig = {
        "batch_create": (st, [vp, i32, vp, vp, ctypes.POINTER(vp)]),
        "batch_destroy": (None, [vp]),
        "batch_info": (st, [vp, ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_int64)]),
        "batch_jac_offsets": (st, [vp, ctypes.POINTER(vp)]),
        "batch_jac_pattern": (st, [vp, i32, vp, vp, ctypes.POINTER(i32)]),
        "inj_elementwise_batched": (st, [vp, vp, vp, vp, vp, vp]),
        "jac_elementwise_batched": (st, [vp, vp, vp, vp, vp, vp, vp]),
        "inj_ybus_batched": (st, [vp, vp, vp, vp, vp, vp]),
        "jac_ybus_batched": (st, [vp, vp, vp, vp, vp, vp, vp]),
        "adjoint_elementwise": (st, [vp] * 17),
        "batch_get_config": (st, [vp, ctypes.POINTER(pf_batch_config)]),
        "batch_set_config": (st, [vp, ctypes.POINTER(pf_batch_config), vp]),
        "batch_autotune": (st, [vp, vp, vp, i32, i32, vp, ctypes.POINTER(pf_batch_config)]),
        "batch_tune_key": (st, [vp, ctypes.c_char_p, i32]),
        "pf_tune_cache_lookup": (st, [ctypes.c_char_p, ctypes.c_char_p, ctypes.POINTER(pf_batch_config),
                                      ctypes.POINTER(i32)]),
        "pf_tune_cache_store": (st, [ctypes.c_char_p, ctypes.c_char_p, ctypes.POINTER(pf_batch_config)]),
        "loss_elementwise": (st, [vp] * 10),
    }
    for name, (res, args) in sig.items():
        fn = getattr(_lib, name)
        fn.restype = res
        fn.argtypes = args


_bind_batches()


class Batch:
    """Owner of a pf_batch handle (keeps its grid alive)."""

    def __init__(self, handle, grid):
        self.handle = ctypes.c_void_p(handle)
        self.grid = grid
        n, tot = ctypes.c_int32(), ctypes.c_int64()
        _check(_lib.batch_info(self.handle, ctypes.byref(n), ctypes.byref(tot)), "batch_info")
        self.nscen, self.nnzJ_total = n.value, tot.value

    def close(self):
        if self.handle:
            _lib.batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def batch_create(grid, nscen, outage=None, stream=None):
    """Batch of nscen scenarios; outage: host int array [nscen] (-1 = none) or None."""
    arr, p = _hptr(outage, np.int32) if outage is not None else (None, None)
    out = ctypes.c_void_p()
    _check(_lib.batch_create(grid.handle, int(nscen), p, _stream(stream), ctypes.byref(out)), "batch_create")
    return Batch(out.value, grid)


def batch_get_config(batch):
    c = pf_batch_config()
    _check(_lib.batch_get_config(batch.handle, ctypes.byref(c)), "batch_get_config")
    return c.as_dict()


def batch_set_config(batch, stream=None, **kw):
    c = pf_batch_config(**{**batch_get_config(batch), **kw})
    _check(_lib.batch_set_config(batch.handle, ctypes.byref(c), _stream(stream)), "batch_set_config")


PF_TUNE_JAC, PF_TUNE_YBUS, PF_TUNE_ADJOINT = 1, 2, 4


def batch_autotune(batch, vm, va, reps=5, kernels=0, stream=None):
    """Tune the batch's launch shapes on the states vm, va for the kernels in
    `kernels` (PF_TUNE_* bits, 0 = Jacobians of both methods); returns the
    chosen configuration (stored in the PFGRID_TUNE_CACHE file when set)."""
    n = batch.nscen * batch.grid.nb
    c = pf_batch_config()
    _check(_lib.batch_autotune(batch.handle, _dptr(vm, "vm", n), _dptr(va, "va", n), int(kernels), int(reps),
                               _stream(stream), ctypes.byref(c)), "batch_autotune")
    return c.as_dict()


def batch_tune_key(batch):
    buf = ctypes.create_string_buffer(512)
    _check(_lib.batch_tune_key(batch.handle, buf, 512), "batch_tune_key")
    return buf.value.decode()


def tune_cache_lookup(path, key):
    """The configuration stored under key in the tuning cache file, or None."""
    c, found = pf_batch_config(), ctypes.c_int32()
    _check(_lib.pf_tune_cache_lookup(os.fsencode(path), key.encode(), ctypes.byref(c), ctypes.byref(found)),
           "pf_tune_cache_lookup")
    return c.as_dict() if found.value else None


def tune_cache_store(path, key, cfg):
    c = pf_batch_config(**cfg)
    _check(_lib.pf_tune_cache_store(os.fsencode(path), key.encode(), ctypes.byref(c)), "pf_tune_cache_store")


def batch_jac_offsets(batch):
    """Offsets joff [nscen+1] of each scenario's Jacobian values (new torch CUDA tensor)."""
    import torch
    ptr = ctypes.c_void_p()
    _check(_lib.batch_jac_offsets(batch.handle, ctypes.byref(ptr)), "batch_jac_offsets")
    return _device_copy(ptr.value, batch.nscen + 1, torch.int64)


def batch_jac_pattern(batch, s):
    """(rowptr, colidx) numpy arrays of scenario s's Jacobian pattern."""
    n = ctypes.c_int32()
    _check(_lib.batch_jac_pattern(batch.handle, int(s), None, None, ctypes.byref(n)), "batch_jac_pattern")
    nb = batch.grid.nb
    rp = np.zeros(2 * nb + 1, np.int32)
    ci = np.zeros(max(n.value, 1), np.int32)
    _check(_lib.batch_jac_pattern(batch.handle, int(s), rp.ctypes.data_as(ctypes.c_void_p),
                                  ci.ctypes.data_as(ctypes.c_void_p), ctypes.byref(n)), "batch_jac_pattern")
    return rp, ci[:n.value]


def inj_elementwise_batched(batch, vm, va, P, Q, stream=None):
    n = batch.nscen * batch.grid.nb
    _check(_lib.inj_elementwise_batched(batch.handle, _dptr(vm, "vm", n), _dptr(va, "va", n), _dptr(P, "P", n),
                                        _dptr(Q, "Q", n), _stream(stream)), "inj_elementwise_batched")


def jac_elementwise_batched(batch, vm, va, P, Q, J, stream=None):
    n = batch.nscen * batch.grid.nb
    _check(_lib.jac_elementwise_batched(batch.handle, _dptr(vm, "vm", n), _dptr(va, "va", n), _dptr(P, "P", n),
                                        _dptr(Q, "Q", n), _dptr(J, "J", batch.nnzJ_total), _stream(stream)),
           "jac_elementwise_batched")


def inj_ybus_batched(batch, vm, va, P, Q, stream=None):
    n = batch.nscen * batch.grid.nb
    _check(_lib.inj_ybus_batched(batch.handle, _dptr(vm, "vm", n), _dptr(va, "va", n), _dptr(P, "P", n),
                                 _dptr(Q, "Q", n), _stream(stream)), "inj_ybus_batched")


def jac_ybus_batched(batch, vm, va, P, Q, J, stream=None):
    n = batch.nscen * batch.grid.nb
    _check(_lib.jac_ybus_batched(batch.handle, _dptr(vm, "vm", n), _dptr(va, "va", n), _dptr(P, "P", n),
                                 _dptr(Q, "Q", n), _dptr(J, "J", batch.nnzJ_total), _stream(stream)),
           "jac_ybus_batched")


def adjoint_elementwise(batch, vm, va, Pspec, Qspec, wP, wQ, L, gvm, gva, gg=None, gb=None, gbsh=None, gtap=None,
                        stream=None, Lbar=None, Ltot=None):
    """Loss per scenario L [S] (may be None), its total Ltot [1] (may be None),
    and the gradients scaled by the device scalar Lbar (None = 1)."""
    nb, nl, S = batch.grid.nb, batch.grid.nl, batch.nscen
    _check(_lib.adjoint_elementwise(batch.handle, _dptr(vm, "vm", S * nb), _dptr(va, "va", S * nb),
                                    _dptr(Pspec, "Pspec", nb), _dptr(Qspec, "Qspec", nb), _dptr(wP, "wP", nb),
                                    _dptr(wQ, "wQ", nb), _dptr(Lbar, "Lbar", 1), _dptr(L, "L", S),
                                    _dptr(Ltot, "Ltot", 1), _dptr(gvm, "gvm", S * nb), _dptr(gva, "gva", S * nb),
                                    _dptr(gg, "gg", nl), _dptr(gb, "gb", nl), _dptr(gbsh, "gbsh", nl),
                                    _dptr(gtap, "gtap", nl), _stream(stream)), "adjoint_elementwise")


def loss_elementwise(batch, vm, va, Pspec, Qspec, wP, wQ, L=None, Ltot=None, stream=None):
    """The mismatch loss alone: L [S] per scenario and/or their total Ltot [1]."""
    nb, S = batch.grid.nb, batch.nscen
    _check(_lib.loss_elementwise(batch.handle, _dptr(vm, "vm", S * nb), _dptr(va, "va", S * nb),
                                 _dptr(Pspec, "Pspec", nb), _dptr(Qspec, "Qspec", nb), _dptr(wP, "wP", nb),
                                 _dptr(wQ, "wQ", nb), _dptr(L, "L", S), _dptr(Ltot, "Ltot", 1), _stream(stream)),
           "loss_elementwise")


def _mismatch_loss_function():
    import torch

    class MismatchLoss(torch.autograd.Function):
        """Total mismatch loss sum_s L_s of a batch (see adjoint_elementwise) as a
        differentiable function of the voltage states and the branch parameters.

        forward(batch, vm, va, g, b, bsh, tap, shift, gs, bs, Pspec, Qspec, wP, wQ)
        sets the grid's parameters and runs the loss alone (loss_elementwise: no
        gradient work); backward sets them again and runs the adjoint kernel
        with the upstream gradient as its scale, so every operation on method
        values runs in the library."""

        @staticmethod
        def forward(ctx, batch, vm, va, g, b, bsh, tap, shift, gs, bs, Pspec, Qspec, wP, wQ):
            c = lambda x: None if x is None else x.detach().contiguous()
            params = tuple(c(x) for x in (g, b, bsh, tap, shift, gs, bs))
            grid_set_params(batch.grid, *params)
            state = tuple(c(x) for x in (vm, va, Pspec, Qspec, wP, wQ))
            Ltot = torch.empty(1, dtype=torch.float64, device=vm.device)
            loss_elementwise(batch, *state, None, Ltot)
            ctx.batch, ctx.params, ctx.state, ctx.shapes = batch, params, state, (vm.shape, va.shape)
            return Ltot.view(())

        @staticmethod
        def backward(ctx, grad):
            batch, (vm, va, Ps, Qs, wP, wQ) = ctx.batch, ctx.state
            grid = batch.grid
            grid_set_params(grid, *ctx.params)   # the parameters of the forward pass
            S, nb, nl, dev = batch.nscen, grid.nb, grid.nl, vm.device
            gvm = torch.empty(S * nb, dtype=torch.float64, device=dev)
            gva = torch.empty_like(gvm)
            gp = [torch.empty(nl, dtype=torch.float64, device=dev) for _ in range(4)]
            lbar = grad.detach().to(device=dev, dtype=torch.float64).reshape(1).contiguous()
            adjoint_elementwise(batch, vm, va, Ps, Qs, wP, wQ, None, gvm, gva, *gp, Lbar=lbar)
            return (None, gvm.view(ctx.shapes[0]), gva.view(ctx.shapes[1]), *gp,
                    None, None, None, None, None, None, None)

    return MismatchLoss


try:
    MismatchLoss = _mismatch_loss_function()
except ImportError:   # torch absent: the C ABI binding still works on numpy inputs
    MismatchLoss = None
