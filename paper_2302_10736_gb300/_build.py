"""In-tree compilation of the native parts (no cmake, no site-packages install).

libpfgrid.so  - the CUDA library (nvcc, sm_103a only) behind include/pfgrid.h
libsynth.so   - the seeded input generator (plain C99)
Both are rebuilt only when a source is newer than the library.
"""
import os
import shutil
import subprocess
import threading

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB_PFGRID = os.path.join(PKG, "libpfgrid.so")
# the same library with the element-wise kernel's phase probe compiled in
# (-DPF_PHASE_PROBE); never loaded unless PFGRID_LIB names it
LIB_PFGRID_PROBE = os.path.join(PKG, "libpfgrid_probe.so")
LIB_SYNTH = os.path.join(PKG, "synth", "libsynth.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
_lock = threading.Lock()


def _nvcc():
    cand = os.environ.get("NVCC") or shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return cand


def _cuda_home():
    nv = os.path.realpath(_nvcc())
    return os.path.dirname(os.path.dirname(nv))


def _stale(target, sources):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(s) > t for s in sources)


def _run(cmd):
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError("build failed: %s\n%s" % (" ".join(cmd), r.stdout))
    return r.stdout


def pfgrid_sources():
    srcs = sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cpp")))
    hdrs = sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh")))
    hdrs.append(os.path.join(INCLUDE, "pfgrid.h"))
    return srcs, hdrs


def build_pfgrid(force=False, verbose=False, extra_flags=(), phase_probe=False):
    """Compile every .cu/.cpp under csrc/ for sm_103a and link libpfgrid.so
    (libpfgrid_probe.so with the phase probe compiled in)."""
    srcs, hdrs = pfgrid_sources()
    lib = LIB_PFGRID_PROBE if phase_probe else LIB_PFGRID
    if phase_probe:
        extra_flags = tuple(extra_flags) + ("-DPF_PHASE_PROBE",)
    with _lock:
        if not force and not _stale(lib, srcs + hdrs):
            return lib
        objdir = os.path.join(PKG, "_build_probe" if phase_probe else "_build")
        os.makedirs(objdir, exist_ok=True)
        nvcc = _nvcc()
        common = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-O2,-fvisibility=hidden",
                  "-I", INCLUDE, "-I", CSRC] + ARCH + list(extra_flags)
        objs, procs = [], []
        for s in srcs:
            o = os.path.join(objdir, os.path.basename(s) + ".o")
            objs.append(o)
            cmd = [nvcc, "-c", s, "-o", o] + common
            if s.endswith(".cpp"):
                cmd = [nvcc, "-x", "cu", "-c", s, "-o", o] + common
            procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)))
        errs = []
        for cmd, p in procs:
            out, _ = p.communicate()
            if verbose and out:
                print(out)
            if p.returncode != 0:
                errs.append(" ".join(cmd) + "\n" + out)
        if errs:
            raise RuntimeError("nvcc failed:\n" + "\n".join(errs))
        lib64 = os.path.join(_cuda_home(), "lib64")
        tmp = lib + ".tmp"
        _run([nvcc, "-shared", "-o", tmp] + objs + ARCH +
             ["-cudart", "shared", "-Xlinker", "-rpath," + lib64])
        os.replace(tmp, lib)
        return lib


def build_synth(force=False):
    src = os.path.join(PKG, "synth", "synth.c")
    with _lock:
        if not force and not _stale(LIB_SYNTH, [src]):
            return LIB_SYNTH
        cc = os.environ.get("CC") or shutil.which("gcc") or "cc"
        tmp = LIB_SYNTH + ".tmp"
        _run([cc, "-O2", "-std=c99", "-fPIC", "-shared", "-o", tmp, src, "-lm"])
        os.replace(tmp, LIB_SYNTH)
        return LIB_SYNTH
