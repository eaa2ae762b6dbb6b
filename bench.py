"""Benchmark: injection + Jacobian evaluations/s on one GB300, element-wise vs
Ybus method, FP64, on the 70,000-bus / 88,000-branch synthetic grid.

One step = one full evaluation by the element-wise method (phasor step +
fused terminal evaluation and reduction) producing P, Q [nb] and all Jacobian
values J [4 nnzY] from (vm, va) already resident in HBM.  The Ybus method is
timed the same way and reported beside it.  L2 (129 MB) is flushed between
timed steps, outside the timed events, by writing a 512 MB buffer and then
reading a 256 MB one: the step's data is evicted, and the lines left in L2 are
clean, so the step does not pay for writing back the flush's own dirty lines.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun (N > 1) every rank evaluates its own replica of the workload
(the single-scenario path has no exchange step); rank 0 prints one JSON line.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = 2
METRIC = "injection+Jacobian evals/s (element-wise method, FP64)"
MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
# FP64 pipe peak derived from the nominal FP64 rate: 152 SMs x 2 FP64 ops/clk x 2.07 GHz
# (= 1.26 TFLOP/s counting an FMA as 2 flops, the nominal 1.25 TFLOP/s)
FP64_OPS_PEAK_G = 152 * 2 * 2.070
# the measured FP64 FMA rate of this run (measure_fp64_peak), once known
_FP64_MEASURED = {"g": None}


def fp64_peak_g():
    """The FP64 roof the fractions below are taken against: the rate measured
    in this run if there is one, else the nominal one."""
    return _FP64_MEASURED["g"] or FP64_OPS_PEAK_G
HBM_FALLBACK_GBS = 6800.0
# FP64 arithmetic instructions per unit of the element-wise Jacobian kernel
WORKLOAD_NAME = "synthetic grid, 70,000 buses / 88,000 branches, one voltage state"
# (the method's operations in its plain FP64 form: the roofline's algorithmic count)
EW_OPS_PER_TERMINAL = 12   # E = V_o conj(U_q) 4, G = conj(Yc) E 4, K = v_q G 2, sum K 2
EW_OPS_PER_BUS = 16        # phasor (1/v 4, V 2, v^2 1, 2v 1; sin/cos on the integer pipe) + diagonal entries and S (8)
# of which the kernel runs E, G, V and 2v in fixed point on the integer pipes: what is left on the FP64 pipe
EW_FP64_PIPE_PER_TERMINAL = 4   # K = v_q G 2, sum K 2
EW_FP64_PIPE_PER_BUS = 13       # 1/v 4, v^2 1, diagonal entries and S 8
YB_OPS_PER_NNZ = 16
YB_OPS_PER_ROW = 16
# DRAM bytes of one k_ew<1> launch on the 70k-bus grid (dram__bytes_read.sum + dram__bytes_write.sum
# of an ncu capture of that launch); None whenever the kernel changes, until it is captured again
EW_TRAFFIC_BYTES = 9941504


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default launch configuration")
    ap.add_argument("--no-extra", action="store_true", help="skip the batched and adjoint workloads")
    ap.add_argument("--phase-probe", action="store_true",
                    help="time the phases of the headline kernel with the phase-probe build of the library and exit")
    ap.add_argument("--phase-probe-child", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--profile-workload",
                    choices=["n1", "adjoint4", "batched5", "permuted", "reduced", "ultra", "newton", "sweep",
                             "study", "target", "replicated"],
                    help="run only this batched/adjoint workload (few launches, for profilers) and exit")
    ap.add_argument("--scenarios", type=int, default=None,
                    help="with --profile-workload n1: the first N scenarios of the 1,024 (a smaller case for profilers)")
    return ap.parse_args(argv)


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def hbm_peak():
    try:
        with open(MEASURED_PEAKS) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples while the GPU is busy."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.path = tempfile.mktemp(suffix=".csv")
        self.proc = None
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(index), "--query-gpu=" + self.QUERY,
                                          "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        for ln in open(self.path):
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append((float(f[1]), float(f[2]), f[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i in range(4) if r[i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "samples": len(rows), "reasons": reasons}


def host_cpu():
    """(CPU model, logical CPUs) of the host running this process."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.split(":")[0].strip() in ("Model name", "Model"):
                model = ln.split(":", 1)[1].strip()
                if ln.startswith("Model name"):
                    break
    except Exception:
        pass
    if not model:
        try:
            for ln in open("/proc/cpuinfo"):
                if ln.lower().startswith(("model name", "cpu part")):
                    model = ln.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    import platform
    return model or platform.processor() or platform.machine(), os.cpu_count() or 1


def oracle_batch_baseline(w, kind, seconds):
    """The oracle over the scenarios of a batched workload on all host cores
    (one thread per core; the oracle's C calls release the GIL), scenarios in
    order until `seconds` have passed (at least one round of one per core).
    kind "n1": injections + Jacobian of scenario s on its grid without its
    outage branch; "adjoint": injections, Jacobian, J^T r and the complex-step
    branch-parameter gradients of scenario s (the loss of the 250k workload)."""
    from concurrent.futures import ThreadPoolExecutor

    import oracle
    model, ncpu = host_cpu()
    S = w["nscen"]
    Y0 = oracle.ybus(w) if kind == "adjoint" else None

    def one(s):
        if kind == "n1":
            skip = np.zeros(w["nl"], np.uint8)
            skip[int(w["outage"][s])] = 1
            Y = oracle.ybus(w, skip=skip)
            oracle.elementwise(w, w["vm"][s], w["va"][s], Y, skip=skip)
        else:
            P, Q, J = oracle.elementwise(w, w["vm"][s], w["va"][s], Y0)
            oracle.adjoint_state(Y0, J, P, Q, w["Ps"], w["Qs"], w["wP"], w["wQ"])
            oracle.adjoint_params_cstep(w, Y0, w["vm"][s], w["va"][s], w["Ps"], w["Qs"], w["wP"], w["wQ"])
        return s

    nthr = min(ncpu, S)
    t0 = time.perf_counter()
    done = 0
    with ThreadPoolExecutor(nthr) as ex:
        # scenarios in order (again from the first once all are done) until the
        # time is up, a whole round of nthr at a time
        while True:
            list(ex.map(one, [(done + i) % S for i in range(nthr)]))
            done += nthr
            if time.perf_counter() - t0 >= seconds:
                break
    el = time.perf_counter() - t0
    return {"value": done / el, "unit": "scenarios/s", "cores": nthr, "nproc": ncpu, "cpu_model": model,
            "kind": "oracle", "sample": "%d scenario evaluations (%d distinct), %d threads, %.1f s"
                                        % (done, min(done, S), nthr, el)}


def run_oracle_steps(w, nsteps, seconds=None):
    """Oracle element-wise injection + Jacobian on the workload; returns (evals, s)."""
    import oracle
    Y = oracle.ybus(w)
    vm, va = w["vm"][0], w["va"][0]
    t0 = time.perf_counter()
    n = 0
    while True:
        oracle.elementwise(w, vm, va, Y)
        n += 1
        el = time.perf_counter() - t0
        if (seconds is not None and el >= seconds) or (seconds is None and n >= nsteps):
            return n, el


def reference_arm(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from paper_2302_10736_gb300 import synth
    w = synth.workload(WORKLOAD)
    run_oracle_steps(w, max(args.warmup, 1))
    n, el = run_oracle_steps(w, args.steps)
    v = n / el
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "evals/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / n, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD_NAME, "global_batch": 1, "seq_len": 0, "parallelism": "none"},
            "cpu_baseline": {"value": v, "unit": "evals/s", "cores": 1, "nproc": host_cpu()[1],
                             "cpu_model": host_cpu()[0], "kind": "oracle",
                             "sample": "%d full element-wise evaluations of the 70k-bus grid" % n},
            "e2e": {"value": v, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def phase_probe(args):
    """Builds the library with the phase probe compiled in and runs the
    headline kernel with it in a child process (PFGRID_LIB names the probe
    build there; the default library is never instrumented)."""
    from paper_2302_10736_gb300 import _build
    lib = _build.build_pfgrid(phase_probe=True)
    env = dict(os.environ, PFGRID_LIB=lib)
    cmd = [sys.executable, os.path.abspath(__file__), "--phase-probe-child", "--steps", str(args.steps),
           "--warmup", str(args.warmup)]
    return subprocess.call(cmd, env=env)


def phase_probe_child(args):
    """Per-phase times of k_ew<1> on the 70k-bus grid (L2 flushed before every
    launch, as in the timed loop): medians over windows and launches of each
    phase, the spread of CTA start and end times, and the per-SM end spread."""
    import torch

    from paper_2302_10736_gb300 import pfgrid, synth
    w = synth.workload(WORKLOAD)
    grid = pfgrid.ybus_build(w)
    dev = lambda x: torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")
    vm, va = dev(w["vm"][0]), dev(w["va"][0])
    P = torch.empty(w["nb"], dtype=torch.float64, device="cuda")
    Q = torch.empty_like(P)
    J = torch.empty(grid.nnzJ, dtype=torch.float64, device="cuda")
    flush = L2Flush(torch)
    names = ["loads", "phasors", "evaluation", "reduction", "stores"]
    per = {n: [] for n in names}
    span, end_med, start_spread, sm_end_spread, ev_us = [], [], [], [], []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for k in range(max(args.warmup, 3) + args.steps):
        flush.fill_(float(k))
        e0.record()
        pfgrid.jac_elementwise(grid, vm, va, P, Q, J)
        e1.record()
        torch.cuda.synchronize()
        if k < max(args.warmup, 3):
            continue
        ev_us.append(1e3 * e0.elapsed_time(e1))
        r = pfgrid.phase_probe_read().astype(np.float64)
        r = r[r[:, 1] > 0]
        gt0, gt1, sm, cyc = r[:, 0], r[:, 1], r[:, 2].astype(int), r[:, 3:8]
        ns_per_cycle = np.median((gt1 - gt0) / np.maximum(cyc[:, 4], 1))
        d = np.diff(np.concatenate([np.zeros((len(r), 1)), cyc], axis=1), axis=1) * ns_per_cycle / 1e3
        for i, n in enumerate(names):
            per[n].append(float(np.median(d[:, i])))
        t0 = gt0.min()
        span.append((gt1.max() - t0) / 1e3)
        end_med.append(float(np.median(gt1 - t0)) / 1e3)
        start_spread.append((gt0.max() - t0) / 1e3)
        sm_end = np.array([gt1[sm == m].max() for m in np.unique(sm)])
        sm_end_spread.append((sm_end.max() - sm_end.min()) / 1e3)
    med = lambda x: float(np.median(x))
    # the same kernel as the last launch of a stream of 40 over 16 grid copies
    # (the headline's form): when its launch wait returned, and what follows
    copies = [(grid, vm, va, P, Q, J)]
    for _ in range(STREAM_COPIES - 1):
        g2 = pfgrid.ybus_build(w)
        copies.append((g2, dev(w["vm"][0]), dev(w["va"][0]), torch.empty_like(P), torch.empty_like(Q),
                       torch.empty_like(J)))
    for k in range(3 * STREAM_COPIES):
        pfgrid.jac_elementwise(*copies[k % STREAM_COPIES])
    sper = {n: [] for n in names}
    rel_spread, post_span, post_med, end_spread = [], [], [], []
    for _ in range(max(3, min(args.steps, 20))):
        torch.cuda.synchronize()
        torch.cuda._sleep(int(2.1e9 * 2e-3))
        for k in range(40):
            pfgrid.jac_elementwise(*copies[k % STREAM_COPIES])
        torch.cuda.synchronize()
        r = pfgrid.phase_probe_read().astype(np.float64)
        r = r[r[:, 1] > 0]
        gt0, gt1, cyc, gtw = r[:, 0], r[:, 1], r[:, 3:8], r[:, 8]
        ns_per_cycle = np.median((gt1 - gt0) / np.maximum(cyc[:, 4], 1))
        d = np.diff(np.concatenate([np.zeros((len(r), 1)), cyc], axis=1), axis=1) * ns_per_cycle / 1e3
        for i, n in enumerate(names):
            sper[n].append(float(np.median(d[:, i])))
        rel_spread.append((gtw.max() - gtw.min()) / 1e3)
        post_span.append((gt1.max() - gtw.min()) / 1e3)
        post_med.append(float(np.median(gt1 - gtw)) / 1e3)
        end_spread.append((gt1.max() - np.median(gt1)) / 1e3)
    print(json.dumps({"kernel": "k_ew<1>", "workload": WORKLOAD_NAME, "launches": args.steps,
                      "event_us": med(ev_us), "cta_span_us": med(span), "cta_end_median_us": med(end_med),
                      "cta_start_spread_us": med(start_spread), "sm_end_spread_us": med(sm_end_spread),
                      "phase_median_us": {n: med(v) for n, v in per.items()},
                      "stream": {"phase_median_us": {n: med(v) for n, v in sper.items()},
                                 "wait_release_spread_us": med(rel_spread),
                                 "first_release_to_last_end_us": med(post_span),
                                 "release_to_end_median_us": med(post_med),
                                 "last_end_after_median_end_us": med(end_spread)}}), flush=True)


def job_throughput(torch, ms_local, world, dist, device):
    """(step time, whole-job evals/s) of `world` replicas that each evaluate
    one grid per step: the job's step time is the slowest rank's."""
    ms = ms_local
    if dist is not None:
        t = torch.tensor([ms_local], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, world * 1e3 / ms


class L2Flush:
    """Evicts the step's data from L2 (129 MB): writes a 512 MB buffer, then
    reads a 256 MB one so the lines left behind are clean.  With the write
    alone, L2 ends full of dirty lines and the timed step that follows pays
    their write-back on its own misses (about 2 us of the 70k-bus step)."""

    def __init__(self, torch, read=True):
        self.torch = torch
        self.w = torch.empty(64 << 20, dtype=torch.float64, device="cuda")
        self.r = torch.ones(32 << 20, dtype=torch.float64, device="cuda") if read else None
        self.acc = torch.zeros((), dtype=torch.float64, device="cuda")

    def fill_(self, x):
        self.w.fill_(x)
        if self.r is not None:
            self.torch.sum(self.r, dim=0, out=self.acc)


def time_loop(torch, fn, steps, flush, name):
    """Per-step device time (ms) of fn(), L2 flushed before every step outside
    the events; the loop is an NVTX range so profilers can select it."""
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    torch.cuda.nvtx.range_push(name)
    for k in range(steps):
        flush.fill_(float(k))
        ev0[k].record()
        fn()
        ev1[k].record()
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in zip(ev0, ev1)]


# copies of the headline grid evaluated in turn in the timed stream (16 x 19 MB
# of grid structure, state and outputs: above the 129 MB L2)
STREAM_COPIES = 16


def grid_bytes(grid):
    """Device bytes a grid's evaluation reads besides the state: Ybus CSR,
    terminal constants and index records (an estimate for the config line)."""
    return 4 * (grid.nb + 1) + 20 * grid.nnz + 60 * grid.nl + 60 * grid.nb


STREAM_HOST_MARGIN_S = 40e-6   # host time allowed per queued launch of a stream
# CUDA streams the headline's stream of independent evaluations alternates over:
# the CTAs of two evaluations then share the SMs in different phases of their
# windows (the integer-pipe phasor and coupling phases of one beside the FP64
# reduction of the other), which one launch alone cannot do
HEADLINE_STREAMS = 2


def stream_loop(torch, fn_k, steps, name, info=None, nstreams=1):
    """fn_k(k, stream) for k = 0 .. steps-1 back to back between one pair of
    CUDA events, step k on CUDA stream k mod nstreams (nstreams = 1: the
    current stream; stream None); mean ms per step.  A device-side wait
    (torch's spin kernel, before the first event) holds the GPU while the
    host queues all the launches, so the device time is the GPU's own
    back-to-back rate and not the host's launch rate (the end-to-end number
    includes the host).  If the host took longer than the wait, the run is
    repeated with a longer one."""
    margin = STREAM_HOST_MARGIN_S
    streams = [torch.cuda.Stream() for _ in range(nstreams)] if nstreams > 1 else [None]
    for _ in range(4):
        wait_s = steps * margin + 1e-3
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        torch.cuda._sleep(int(wait_s * 2.1e9))
        t0 = time.perf_counter()
        torch.cuda.nvtx.range_push(name)
        e0.record()
        if nstreams > 1:   # every stream starts after the first event
            go = torch.cuda.Event()
            go.record()
            for st in streams:
                st.wait_event(go)
        for k in range(steps):
            st = streams[k % len(streams)]
            fn_k(k, st.cuda_stream if st is not None else None)
        if nstreams > 1:   # the second event after every stream's last step
            cur = torch.cuda.current_stream()
            for st in streams:
                done = torch.cuda.Event()
                done.record(st)
                cur.wait_event(done)
        e1.record()
        torch.cuda.nvtx.range_pop()
        host_s = time.perf_counter() - t0
        torch.cuda.synchronize()
        if host_s < 0.8 * wait_s:
            break
        margin *= 2.0
    if info is not None:
        info["host_enqueue_us_per_step"] = host_s / steps * 1e6
        info["device_wait_ms"] = wait_s * 1e3
    return e0.elapsed_time(e1) / steps


def measure_fp64_peak(torch, pfgrid, ctas_per_sm=8, iters=2048):
    """FP64 FMA rate of this GPU from the library's probe kernel (best of 5
    launches, CUDA events): 8 CTAs of 256 threads per SM, 8 independent chains
    per thread."""
    sink = torch.zeros(1, dtype=torch.float64, device="cuda")
    nsm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    ctas = ctas_per_sm * nsm
    pfgrid.fp64_peak_probe(ctas, 64, sink)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    best = None
    for _ in range(5):
        e0.record()
        n = pfgrid.fp64_peak_probe(ctas, iters, sink)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        best = ms if best is None else min(best, ms)
    g = n / (best * 1e-3) / 1e9
    return {"gdfma_per_s": g, "per_sm_per_clock_at_max": g * 1e9 / nsm / 2.07e9, "ms": best, "dfma": n,
            "ctas": ctas, "source": "fp64_peak_probe"}


def graph_of(torch, fn):
    """Capture fn (one library launch) into a CUDA graph after one eager warm-up."""
    fn()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        fn()
    return g


def timed_replays(torch, g, reps, name="replays"):
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(2):
        g.replay()
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push(name)
    e0.record()
    for _ in range(reps):
        g.replay()
    e1.record()
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def extra_workloads(torch, pfgrid, synth, reps, only=None, cpu_seconds=None, n1_scenarios=None):
    """The batched and adjoint workloads, each timed from a CUDA-graph replay
    (inputs larger than L2 for the batched ones, so no flush is needed).
    `only` restricts the run to one of "n1", "adjoint4", "batched5", "permuted", "reduced", "ultra",
    "newton", "sweep", "study", "target"."""
    out = {}
    if only in (None, "n1"):
        out.update(_n1_workload(torch, pfgrid, synth, reps, cpu_seconds, n1_scenarios))
    for k, key, tag in ((4, "adjoint_25k", "adjoint4"), (5, "batched_jac_and_adjoint_250k_x16", "batched5")):
        if only in (None, tag):
            out[key] = _adjoint_workload(torch, pfgrid, synth, reps, k, cpu_seconds)
    if only in (None, "permuted"):
        out["c2_random_bus_order"] = _permuted_workload(torch, pfgrid, synth, max(reps, 20))
    if only in (None, "reduced"):
        out["reduced_newton_csc_70k"] = _reduced_workload(torch, pfgrid, synth, max(reps, 20))
    if only in (None, "target"):
        out["target_pattern_70k"] = _target_workload(torch, pfgrid, synth, max(reps, 20))
    if only in (None, "ultra"):
        out["single_410k"] = _single_workload(torch, pfgrid, synth, 6, max(reps, 20))
    if only in (None, "replicated"):
        out["replicated_82k"] = _replicated_workload(torch, pfgrid, synth, max(reps, 20))
    if only in (None, "study"):
        out["two_step_study_70k"] = _study_workload(torch, pfgrid, synth, max(reps, 20))
    if only in (None, "sweep"):
        out["size_sweep"] = _size_sweep(torch, pfgrid, synth, max(reps, 20))
    if only in (None, "newton"):
        out["newton_powerflow"] = {"2k": _newton_workload(torch, pfgrid, synth, 1),
                                   "10k": _newton_workload(torch, pfgrid, synth, 3)}
    return out


def _study_workload(torch, pfgrid, synth, steps):
    """The paper's two-step structure of the element-wise method (phasors,
    evaluation into an intermediate, then a gather or an atomic copy-add
    assembly) against the fused kernel, and its interleaved-vs-separate
    voltage storage for the Ybus injections, on the 70k-bus grid, L2 flushed."""
    dev = lambda x: torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")
    flush = L2Flush(torch)
    w = synth.workload(WORKLOAD)
    grid = pfgrid.ybus_build(w)
    vm, va = dev(w["vm"][0]), dev(w["va"][0])
    P = torch.empty(w["nb"], dtype=torch.float64, device="cuda")
    Q = torch.empty_like(P)
    J = torch.empty(grid.nnzJ, dtype=torch.float64, device="cuda")
    res = {}
    for name, f in (("fused", lambda: pfgrid.jac_elementwise(grid, vm, va, P, Q, J)),
                    ("two_step_gather", lambda: pfgrid.jac_elementwise_study(grid, 0, vm, va, P, Q, J)),
                    ("two_step_copy_add", lambda: pfgrid.jac_elementwise_study(grid, 1, vm, va, P, Q, J))):
        for _ in range(3):
            f()
        t = time_loop(torch, f, steps, flush, "study_" + name)
        res["%s_us" % name] = 1e3 * sum(t) / len(t)
    for name, sep in (("ybus_inj_interleaved", 0), ("ybus_inj_separate", 1)):
        f = lambda: pfgrid.inj_ybus_study(grid, sep, vm, va, P, Q)
        for _ in range(3):
            f()
        t = time_loop(torch, f, steps, flush, "study_" + name)
        res["%s_us" % name] = 1e3 * sum(t) / len(t)
    pfgrid.grid_check_error(grid)
    return res


# bus counts of the paper's test cases (Table VII and the replicated grids of Sec. V-F)
SWEEP_SIZES = (14, 118, 300, 1354, 2736, 9241, 25000, 70000, 82000, 164000, 410000)


def _size_sweep(torch, pfgrid, synth, steps):
    """Single evaluations by both methods on synthetic grids with the bus
    counts of the paper's cases (branches = 1.32 x buses, as in the 250k /
    330k workload), L2 flushed between steps: injections + Jacobian,
    injections alone, and the Ybus method's phasor launch (the steps of the
    paper's per-case table that separate launches expose), with the time of
    each relative to the 118-bus grid (the paper's complexity study)."""
    dev = lambda x: torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")
    flush = L2Flush(torch)
    rows = []
    for nb in SWEEP_SIZES:
        nl = int(round(1.32 * nb))
        gr = synth.grid(nb, nl, synth.BASE_SEED + 100 + nb)
        vm, va = synth.voltages(nb, 1, synth.BASE_SEED + 100 + nb)
        grid = pfgrid.ybus_build(gr)
        vmd, vad = dev(vm[0]), dev(va[0])
        pfgrid.grid_autotune(grid, vmd, vad, reps=10)
        P = torch.empty(nb, dtype=torch.float64, device="cuda")
        Q = torch.empty_like(P)
        J = torch.empty(grid.nnzJ, dtype=torch.float64, device="cuda")
        row = {"nb": nb, "nl": nl}
        for name, fn, jac in (("elementwise", pfgrid.jac_elementwise, True), ("ybus", pfgrid.jac_ybus, True),
                              ("elementwise_inj", pfgrid.inj_elementwise, False), ("ybus_inj", pfgrid.inj_ybus, False)):
            f = (lambda: fn(grid, vmd, vad, P, Q, J)) if jac else (lambda: fn(grid, vmd, vad, P, Q))
            for _ in range(3):
                f()
            t = time_loop(torch, f, steps, flush, "sweep_%s" % name)
            row["%s_us" % name] = 1e3 * sum(t) / len(t)   # mean: one event pair resolves about 1 us
        # the Ybus method's phasor step alone (its own launch), from the tracer
        pfgrid.grid_trace_enable(grid, 4 * steps + 16)
        time_loop(torch, lambda: pfgrid.inj_ybus(grid, vmd, vad, P, Q), steps, flush, "sweep_traced")
        ph = [ms for k, ms in pfgrid.grid_trace_read(grid) if k == "phasor"]
        pfgrid.grid_trace_enable(grid, 0)
        row["ybus_phasor_us_traced"] = 1e3 * sum(ph) / max(len(ph), 1)
        pfgrid.grid_check_error(grid)
        rows.append(row)
    base = next(r for r in rows if r["nb"] == 118)
    for r in rows:
        for name in ("elementwise", "ybus", "elementwise_inj", "ybus_inj"):
            r["%s_ratio_to_118" % name] = r["%s_us" % name] / base["%s_us" % name]
    return rows


def _replicated_workload(torch, pfgrid, synth, steps):
    """The paper's ultra-large cases (Sec. V-C): the 82k-bus grid repeated 2 to
    5 times as disjoint copies (164k to 410k buses); single evaluations of
    injections + Jacobian by both methods, L2 flushed between steps."""
    dev = lambda x: torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")
    flush = L2Flush(torch)
    rows = []
    for copies in (2, 3, 4, 5):
        w = synth.replicated_workload(copies)
        grid = pfgrid.ybus_build(w)
        vm, va = dev(w["vm"][0]), dev(w["va"][0])
        pfgrid.grid_autotune(grid, vm, va, reps=10)
        P = torch.empty(w["nb"], dtype=torch.float64, device="cuda")
        Q = torch.empty_like(P)
        J = torch.empty(grid.nnzJ, dtype=torch.float64, device="cuda")
        row = {"copies": copies, "nb": w["nb"], "nl": w["nl"]}
        for name, fn in (("elementwise", pfgrid.jac_elementwise), ("ybus", pfgrid.jac_ybus)):
            f = lambda: fn(grid, vm, va, P, Q, J)
            for _ in range(3):
                f()
            t = time_loop(torch, f, steps, flush, "replicated_%s" % name)
            row["%s_us" % name] = 1e3 * sum(t) / len(t)
        row["ybus_over_elementwise"] = row["ybus_us"] / row["elementwise_us"]
        pfgrid.grid_check_error(grid)
        rows.append(row)
        del grid
    return rows


def _newton_workload(torch, pfgrid, synth, k, reps=5):
    """Newton-Raphson power flow on workload k's grid and bus types, from a start
    within 1e-3 of a known operating point (the workload's angles scaled by 0.1),
    to max |F| <= 1e-10: wall time of the whole solve (host-timed, it synchronizes
    every iteration) and its iteration count."""
    w = synth.workload(k, nscen=1)
    nb, bt = w["nb"], w["bustype"]
    dev = lambda x: torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")
    grid = pfgrid.ybus_build(w)
    pfgrid.grid_set_bus_types(grid, bt)
    vm_t, va_t = dev(w["vm"][0]), dev(0.1 * w["va"][0])
    Ps = torch.empty(nb, dtype=torch.float64, device="cuda")
    Qs = torch.empty_like(Ps)
    pfgrid.inj_elementwise(grid, vm_t, va_t, Ps, Qs)
    rng = np.random.default_rng(56)
    pq, pvpq = bt == 1, (bt == 1) | (bt == 2)
    vm0, va0 = w["vm"][0].copy(), 0.1 * w["va"][0]
    vm0[pq] += rng.uniform(-1e-3, 1e-3, int(pq.sum()))
    va0[pvpq] += rng.uniform(-1e-3, 1e-3, int(pvpq.sum()))
    res = {"nb": nb, "n": pfgrid.jac_reduced_info(grid)[0]}
    for name, m in (("elementwise", 1), ("ybus", 0)):
        ts = []
        for r in range(reps + 1):
            vm, va = dev(vm0), dev(va0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ok, it, fmax = pfgrid.powerflow_newton(grid, m, vm, va, Ps, Qs, tol=1e-10, max_iter=20)
            ts.append(time.perf_counter() - t0)
        res[name] = {"converged": ok, "iterations": it, "max_mismatch": fmax,
                     "ms_per_solve": 1e3 * statistics.median(ts[1:])}
    pfgrid.grid_check_error(grid)
    return res


def _single_workload(torch, pfgrid, synth, k, steps):
    """Single evaluations of workload k by both methods, L2 flushed between steps."""
    dev = lambda x: torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")
    flush = L2Flush(torch)
    w = synth.workload(k)
    grid = pfgrid.ybus_build(w)
    vm, va = dev(w["vm"][0]), dev(w["va"][0])
    pfgrid.grid_autotune(grid, vm, va, reps=10)
    P = torch.empty(w["nb"], dtype=torch.float64, device="cuda")
    Q = torch.empty_like(P)
    J = torch.empty(grid.nnzJ, dtype=torch.float64, device="cuda")
    res = {"nb": w["nb"], "nl": w["nl"], "launch_config": pfgrid.grid_get_config(grid)}
    for name, fn in (("elementwise", pfgrid.jac_elementwise), ("ybus", pfgrid.jac_ybus)):
        f = lambda: fn(grid, vm, va, P, Q, J)
        for _ in range(3):
            f()
        t = time_loop(torch, f, steps, flush, "single%d_%s" % (k, name))
        res["%s_evals_per_s" % name] = 1e3 / (sum(t) / len(t))
    T, nb = 2 * w["nl"], w["nb"]
    ms = 1e3 / res["elementwise_evals_per_s"]
    res["elementwise_fp64_frac"] = (EW_OPS_PER_TERMINAL * T + EW_OPS_PER_BUS * nb) / (ms * 1e-3) / 1e9 / fp64_peak_g()
    pfgrid.grid_check_error(grid)
    return res


def _reduced_workload(torch, pfgrid, synth, steps):
    """The Newton step's inputs on the 70k-bus grid (15 % PV buses): mismatch
    vector and reduced Jacobian in CSC order, by both methods, L2 flushed
    between steps.  The element-wise method writes the reduced system from its
    kernel (one launch); the Ybus method's gather launch is timed by the
    tracer."""
    dev = lambda x: torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")
    flush = L2Flush(torch)
    w = synth.workload(WORKLOAD)
    grid = pfgrid.ybus_build(w)
    vm, va = dev(w["vm"][0]), dev(w["va"][0])
    pfgrid.grid_autotune(grid, vm, va, reps=10)
    pfgrid.grid_set_bus_types(grid, w["bustype"])
    n, npvpq, nnz = pfgrid.jac_reduced_info(grid)
    Ps = torch.zeros(w["nb"], dtype=torch.float64, device="cuda")
    Qs = torch.zeros_like(Ps)
    F = torch.empty(n, dtype=torch.float64, device="cuda")
    Jr = torch.empty(nnz, dtype=torch.float64, device="cuda")
    res = {"n": n, "nnz": nnz}
    for name, m in (("elementwise", 1), ("ybus", 0)):
        f = lambda: pfgrid.jac_reduced(grid, m, vm, va, Ps, Qs, F, Jr)
        for _ in range(3):
            f()
        t = time_loop(torch, f, steps, flush, "reduced_" + name)
        res["%s_evals_per_s" % name] = 1e3 / (sum(t) / len(t))
    pfgrid.grid_trace_enable(grid, 4 * steps + 16)
    time_loop(torch, lambda: pfgrid.jac_reduced(grid, 0, vm, va, Ps, Qs, F, Jr), steps, flush, "reduced_traced")
    tr = pfgrid.grid_trace_read(grid)
    pfgrid.grid_trace_enable(grid, 0)
    ms = [x for k, x in tr if k == "reduce"]
    if ms:
        mean = sum(ms) / len(ms)
        byt = 20 * nnz + 28 * n   # map, full value and reduced value per entry; map, P or Q, spec, F per row
        hbm, kind = hbm_peak()
        res["gather"] = {"us_per_launch": 1e3 * mean, "algorithmic_bytes": byt,
                         "gbs": byt / (mean * 1e-3) / 1e9, "frac_of_hbm": byt / (mean * 1e-3) / 1e9 / hbm,
                         "hbm_peak_source": kind}
    pfgrid.grid_check_error(grid)
    return res


def _target_workload(torch, pfgrid, synth, steps):
    """Alg. 2 on the 70k-bus grid: the Jacobian into a caller's CSC pattern
    that holds the Ybus blocks plus 16 coupled bus pairs (TCSC-like devices,
    all four blocks), by both methods, L2 flushed between steps."""
    dev = lambda x: torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")
    flush = L2Flush(torch)
    w = synth.workload(WORKLOAD)
    grid = pfgrid.ybus_build(w)
    nb = w["nb"]
    vm, va = dev(w["vm"][0]), dev(w["va"][0])
    rp, ci = (x.cpu().numpy() for x in pfgrid.jac_pattern(grid))
    rows = np.repeat(np.arange(2 * nb, dtype=np.int64), np.diff(rp))
    cols = ci.astype(np.int64)
    rng = np.random.default_rng(20230221)
    pairs = rng.choice(nb, size=(16, 2), replace=False)
    extra = [(x, y) for a, c in pairs for x in (a, c, nb + a, nb + c) for y in (a, c, nb + a, nb + c)]
    key = np.unique(np.concatenate([cols * (2 * nb) + rows, [y * (2 * nb) + x for x, y in extra]]))
    tcols, trows = key // (2 * nb), key % (2 * nb)
    colptr = np.zeros(2 * nb + 1, np.int32)
    np.add.at(colptr, tcols + 1, 1)
    colptr = np.cumsum(colptr).astype(np.int32)
    pfgrid.jac_set_target_pattern(grid, colptr, trows.astype(np.int32))
    Jt = torch.zeros(len(trows), dtype=torch.float64, device="cuda")
    P = torch.empty(nb, dtype=torch.float64, device="cuda")
    Q = torch.empty_like(P)
    res = {"nnz_target": int(len(trows)), "nnz_ybus_blocks": int(len(ci))}
    for name, m in (("elementwise", 1), ("ybus", 0)):
        f = lambda: pfgrid.jac_target(grid, m, vm, va, P, Q, Jt)
        for _ in range(3):
            f()
        t = time_loop(torch, f, steps, flush, "target_" + name)
        res["%s_evals_per_s" % name] = 1e3 / (sum(t) / len(t))
    pfgrid.grid_check_error(grid)
    return res


def _permuted_workload(torch, pfgrid, synth, steps):
    """The 70k-bus grid with its buses renumbered at random (no locality in
    the numbering): single evaluations by both methods, L2 flushed between
    steps, against the same grid in its own numbering."""
    dev = lambda x: torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")
    flush = L2Flush(torch)
    res = {}
    base = synth.workload(WORKLOAD)
    for tag, w in (("own_numbering", base), ("random_numbering", synth.renumber_buses(base, synth.BASE_SEED))):
        grid = pfgrid.ybus_build(w)
        pfgrid.grid_autotune(grid, dev(w["vm"][0]), dev(w["va"][0]), reps=10)
        vm, va = dev(w["vm"][0]), dev(w["va"][0])
        P = torch.empty(w["nb"], dtype=torch.float64, device="cuda")
        Q = torch.empty_like(P)
        J = torch.empty(grid.nnzJ, dtype=torch.float64, device="cuda")
        for name, fn in (("elementwise", pfgrid.jac_elementwise), ("ybus", pfgrid.jac_ybus)):
            f = lambda: fn(grid, vm, va, P, Q, J)
            for _ in range(3):
                f()
            t = time_loop(torch, f, steps, flush, "perm_" + name)
            res["%s_%s_evals_per_s" % (name, tag)] = 1e3 / (sum(t) / len(t))
        pfgrid.grid_check_error(grid)
    return res


def _n1_workload(torch, pfgrid, synth, reps, cpu_seconds=None, nscen=None):
    out = {}
    dev = lambda x: torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")

    # N-1 batch: 10,000 buses x 1,024 scenarios, each without a distinct non-bridge branch
    # (nscen: the first nscen of them)
    w = synth.workload(3, nscen=nscen)
    grid = pfgrid.ybus_build(w)
    S, nb, T = w["nscen"], w["nb"], 2 * w["nl"]
    batch = pfgrid.batch_create(grid, S, w["outage"])
    vm, va = dev(w["vm"]), dev(w["va"])
    default_cfg = pfgrid.batch_get_config(batch)
    tuned_cfg = pfgrid.batch_autotune(batch, vm, va, reps=3)
    P = torch.empty(S * nb, dtype=torch.float64, device="cuda")
    Q = torch.empty_like(P)
    J = torch.empty(batch.nnzJ_total, dtype=torch.float64, device="cuda")
    g = graph_of(torch, lambda: pfgrid.jac_elementwise_batched(batch, vm, va, P, Q, J))
    ms = timed_replays(torch, g, reps, "n1_batch")
    ops = S * (EW_OPS_PER_TERMINAL * T + EW_OPS_PER_BUS * nb)
    byt = S * (16 * nb + 16 * nb) + 8 * batch.nnzJ_total + 40 * T + 84 * nb
    name = "n1_batch_10k_x%d" % S
    out[name] = {
        "evals_per_s": S / (ms * 1e-3), "ms_per_launch": ms, "launches": 1, "graph": True,
        "fp64_gops": ops / (ms * 1e-3) / 1e9, "fp64_frac": ops / (ms * 1e-3) / 1e9 / fp64_peak_g(),
        "hbm_gbs": byt / (ms * 1e-3) / 1e9, "jacobian_values": batch.nnzJ_total,
        "launch_config": tuned_cfg, "default_launch_config": default_cfg}
    # the same batch by the Ybus method (phasor launch + row launch)
    g2 = graph_of(torch, lambda: pfgrid.jac_ybus_batched(batch, vm, va, P, Q, J))
    ms2 = timed_replays(torch, g2, reps, "n1_batch_ybus")
    out[name].update({"ybus_evals_per_s": S / (ms2 * 1e-3), "ybus_ms_per_launch": ms2, "ybus_launches": 2})
    # the plain single-scenario paths on the base grid, one state per launch (L2 warm)
    P1 = torch.empty(nb, dtype=torch.float64, device="cuda")
    Q1 = torch.empty_like(P1)
    J1 = torch.empty(grid.nnzJ, dtype=torch.float64, device="cuda")
    for key, fn in (("single_elementwise_evals_per_s", pfgrid.jac_elementwise),
                    ("single_ybus_evals_per_s", pfgrid.jac_ybus)):
        g3 = graph_of(torch, lambda: fn(grid, vm[:nb], va[:nb], P1, Q1, J1))
        out[name][key] = 1e3 / timed_replays(torch, g3, reps, "n1_single")
    pfgrid.grid_check_error(grid)
    if cpu_seconds:
        out[name]["cpu_baseline"] = oracle_batch_baseline(w, "n1", cpu_seconds)
    return out


def _adjoint_workload(torch, pfgrid, synth, reps, k, cpu_seconds=None):
    """Adjoint of the mismatch loss on workload k (25k buses x 1, or 250k x 16
    with the batched Jacobian and the single-scenario Ybus Jacobian beside it)."""
    dev = lambda x: torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")
    w = synth.workload(k)
    grid = pfgrid.ybus_build(w)
    S, nb, nl, T = w["nscen"], w["nb"], w["nl"], 2 * w["nl"]
    batch = pfgrid.batch_create(grid, S, None)
    default_cfg = pfgrid.batch_get_config(batch)
    # the adjoint is this workload's main call: tune for it (and the Jacobian beside it)
    tuned_cfg = pfgrid.batch_autotune(batch, dev(w["vm"]), dev(w["va"]), reps=3,
                                      kernels=pfgrid.PF_TUNE_ADJOINT | pfgrid.PF_TUNE_JAC | pfgrid.PF_TUNE_YBUS)
    Ps = torch.empty(nb, dtype=torch.float64, device="cuda")
    Qs = torch.empty_like(Ps)
    pfgrid.inj_elementwise(grid, dev(w["vm2"]), dev(w["va2"]), Ps, Qs)
    vm, va, wP, wQ = dev(w["vm"]), dev(w["va"]), dev(w["wP"]), dev(w["wQ"])
    L = torch.empty(S, dtype=torch.float64, device="cuda")
    gvm = torch.empty(S * nb, dtype=torch.float64, device="cuda")
    gva = torch.empty_like(gvm)
    gp = [torch.empty(nl, dtype=torch.float64, device="cuda") for _ in range(4)]
    g = graph_of(torch, lambda: pfgrid.adjoint_elementwise(batch, vm, va, Ps, Qs, wP, wQ, L, gvm, gva, *gp))
    ms = timed_replays(torch, g, reps, "adjoint%d" % k)
    ops = S * ((6 + 8 + 8) * nb + (10 + 22) * T + 48 * nl)   # phasor 1/v and V (sin/cos on the integer pipe)
    res = {"loss_and_gradients_per_s": S / (ms * 1e-3), "ms_per_launch": ms, "launches": 1, "graph": True,
           "launch_config": tuned_cfg, "default_launch_config": default_cfg,
           "fp64_gops": ops / (ms * 1e-3) / 1e9, "fp64_frac": ops / (ms * 1e-3) / 1e9 / fp64_peak_g()}
    if k == 5:
        P = torch.empty(S * nb, dtype=torch.float64, device="cuda")
        Q = torch.empty_like(P)
        J = torch.empty(batch.nnzJ_total, dtype=torch.float64, device="cuda")
        g2 = graph_of(torch, lambda: pfgrid.jac_elementwise_batched(batch, vm, va, P, Q, J))
        ms2 = timed_replays(torch, g2, reps, "batched5")
        ops2 = S * (EW_OPS_PER_TERMINAL * T + EW_OPS_PER_BUS * nb)
        res.update({"jac_evals_per_s": S / (ms2 * 1e-3), "jac_ms_per_launch": ms2,
                    "jac_fp64_frac": ops2 / (ms2 * 1e-3) / 1e9 / fp64_peak_g()})
        g4 = graph_of(torch, lambda: pfgrid.jac_ybus_batched(batch, vm, va, P, Q, J))
        res["ybus_batched_jac_evals_per_s"] = S * 1e3 / timed_replays(torch, g4, reps, "ybus_batched5")
        # the plain single-scenario Ybus path on the same grid, for comparison
        J1 = torch.empty(grid.nnzJ, dtype=torch.float64, device="cuda")
        P1 = torch.empty(nb, dtype=torch.float64, device="cuda")
        Q1 = torch.empty_like(P1)
        g3 = graph_of(torch, lambda: pfgrid.jac_ybus(grid, vm[:nb], va[:nb], P1, Q1, J1))
        res["single_scenario_ybus_jac_evals_per_s"] = 1e3 / timed_replays(torch, g3, reps, "ybus5")
    pfgrid.grid_check_error(grid)
    if cpu_seconds:
        import oracle
        Y = oracle.ybus(w)
        Psh, Qsh = oracle.inj_sparse(Y, w["vm2"], w["va2"])
        res["cpu_baseline"] = oracle_batch_baseline(dict(w, Ps=Psh, Qs=Qsh), "adjoint", cpu_seconds)
    return res


def main():
    args = parse_args()
    if args.impl == "reference":
        return reference_arm(args)
    if args.phase_probe:
        sys.exit(phase_probe(args))
    if args.phase_probe_child:
        return phase_probe_child(args)
    import torch

    from paper_2302_10736_gb300 import pfgrid, synth
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if args.profile_workload:
        _FP64_MEASURED["g"] = measure_fp64_peak(torch, pfgrid)["gdfma_per_s"]
        print(json.dumps(extra_workloads(torch, pfgrid, synth, max(1, args.steps), args.profile_workload,
                                         n1_scenarios=args.scenarios)))
        return
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    w = synth.workload(WORKLOAD)
    nb, nl = w["nb"], w["nl"]
    grid = pfgrid.ybus_build(w)
    dev = lambda x: torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")
    vm, va = dev(w["vm"][0]), dev(w["va"][0])
    P = torch.empty(nb, dtype=torch.float64, device="cuda")
    Q = torch.empty_like(P)
    J = torch.empty(grid.nnzJ, dtype=torch.float64, device="cuda")
    cfg = pfgrid.grid_get_config(grid) if args.no_autotune else pfgrid.grid_autotune(grid, vm, va, reps=20)
    flush = L2Flush(torch)
    T = 2 * nl

    # the headline stream: COPIES copies of the grid, each with its own state and
    # outputs, evaluated in turn, so that every step's grid, state and outputs
    # were last touched COPIES - 1 steps earlier (working set above L2)
    copies = [(grid, vm, va, P, Q, J)]
    for _ in range(STREAM_COPIES - 1):
        g2 = pfgrid.ybus_build(w)
        pfgrid.grid_set_config(g2, **cfg)
        copies.append((g2, dev(w["vm"][0]), dev(w["va"][0]), torch.empty_like(P), torch.empty_like(Q),
                       torch.empty_like(J)))
    footprint = STREAM_COPIES * (grid_bytes(grid) + 8 * (4 * nb + grid.nnzJ))
    # (with two streams step k goes to stream k mod 2 and copy k mod 16: the
    # streams never share a copy's outputs)
    ew_k = lambda k, st=None: pfgrid.jac_elementwise(*copies[k % STREAM_COPIES], stream=st)
    yb_k = lambda k, st=None: pfgrid.jac_ybus(*copies[k % STREAM_COPIES], stream=st)

    ew = lambda: pfgrid.jac_elementwise(grid, vm, va, P, Q, J)
    yb = lambda: pfgrid.jac_ybus(grid, vm, va, P, Q, J)
    iew = lambda: pfgrid.inj_elementwise(grid, vm, va, P, Q)
    iyb = lambda: pfgrid.inj_ybus(grid, vm, va, P, Q)
    for k in range(max(args.warmup, 3)):
        for f in (ew, yb, iew, iyb):
            flush.fill_(0.0)
            f()
    for k in range(max(args.warmup, 3) * STREAM_COPIES):
        ew_k(k)
        yb_k(k)
        pfgrid.inj_elementwise(*copies[k % STREAM_COPIES][:5])
        pfgrid.inj_ybus(*copies[k % STREAM_COPIES][:5])
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    time.sleep(0.3)

    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    stream_info = {}
    # the timed region of the headline
    ms_stream = stream_loop(torch, ew_k, args.steps, "ew_stream", stream_info, nstreams=HEADLINE_STREAMS)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms_stream_yb = stream_loop(torch, yb_k, args.steps, "ybus_stream", nstreams=HEADLINE_STREAMS)
    # the same streams on one CUDA stream: back-to-back launches of one evaluation at a time
    ms_stream1 = stream_loop(torch, ew_k, args.steps, "ew_stream_one")
    ms_stream1_yb = stream_loop(torch, yb_k, args.steps, "ybus_stream_one")
    # the injections alone, in the same stream form
    ms_stream_iew = stream_loop(torch, lambda k, st: pfgrid.inj_elementwise(*copies[k % STREAM_COPIES][:5], stream=st),
                                args.steps, "inj_ew_stream", nstreams=HEADLINE_STREAMS)
    ms_stream_iyb = stream_loop(torch, lambda k, st: pfgrid.inj_ybus(*copies[k % STREAM_COPIES][:5], stream=st),
                                args.steps, "inj_ybus_stream", nstreams=HEADLINE_STREAMS)
    # one evaluation at a time: L2 flushed before every step outside the events,
    # so each step also pays its launch (the latency form)
    t_ew = time_loop(torch, ew, args.steps, flush, "ew")
    t_yb = time_loop(torch, yb, args.steps, flush, "ybus")
    t_iew = time_loop(torch, iew, args.steps, flush, "inj_ew")
    t_iyb = time_loop(torch, iyb, args.steps, flush, "inj_ybus")
    # the latency form again after a write-only flush (L2 left full of dirty lines)
    t_dirty = time_loop(torch, ew, args.steps, L2Flush(torch, read=False), "ew_dirty_l2")
    torch.cuda.synchronize()
    # per-kernel times: the same loops again with the library's launch tracer on
    pfgrid.grid_trace_enable(grid, 8 * args.steps + 64)
    time_loop(torch, ew, args.steps, flush, "traced_ew")
    tr_ew = pfgrid.grid_trace_read(grid)
    time_loop(torch, yb, args.steps, flush, "traced_ybus")
    tr_yb = pfgrid.grid_trace_read(grid)
    time_loop(torch, iew, args.steps, flush, "traced_inj_ew")
    time_loop(torch, iyb, args.steps, flush, "traced_inj_ybus")
    tr_inj = pfgrid.grid_trace_read(grid)
    pfgrid.grid_trace_enable(grid, 0)
    # the FP64 roof of this GPU, measured under the same clocks
    fp64_peak = measure_fp64_peak(torch, pfgrid)
    _FP64_MEASURED["g"] = fp64_peak["gdfma_per_s"]
    clocks = sampler.stop()
    for c in copies:
        pfgrid.grid_check_error(c[0])

    ms_step, value = job_throughput(torch, ms_stream, world, dist, "cuda")

    def kmean(tr, name):
        xs = [ms for k, ms in tr if k == name]
        return (sum(xs) / len(xs), len(xs)) if xs else (None, 0)

    ms_jew, n_jew = kmean(tr_ew, "jac_ew")
    ms_pu, n_pu = kmean(tr_yb, "phasor")   # the Ybus path's separate phasor step
    ms_jyb, _ = kmean(tr_yb, "jac_ybus")
    ops_ew = EW_OPS_PER_TERMINAL * T + EW_OPS_PER_BUS * nb
    # the device's aggregate rate over the timed region: the method's operations
    # per evaluation x evaluations per second (one launch per evaluation, two in
    # flight at a time on two CUDA streams; the one-stream rate is beside it)
    achieved = ops_ew / (ms_stream * 1e-3) / 1e9
    hbm, hbm_kind = hbm_peak()
    # algorithmic bytes of an element-wise injection + Jacobian evaluation: branch ends and 5 parameters
    # per branch (48 B), vm, va, shunt and P, Q per bus (48 B), one value per Jacobian slot (32 B per nnzY)
    bytes_ew = 48 * nl + 48 * nb + 32 * grid.nnz
    roof = {"bound": "alu", "kernel": "k_ew<1>", "achieved": achieved, "peak": fp64_peak["gdfma_per_s"],
            "unit": "GFP64op/s", "frac": achieved / fp64_peak["gdfma_per_s"], "traffic": EW_TRAFFIC_BYTES,
            "ops_per_launch": ops_ew,
            "ops_note": "the method's operations in plain FP64 form (12 per terminal, 16 per bus); the kernel runs "
                        "8 per terminal and 3 per bus of them in 64-bit fixed point on the integer pipes, %d on "
                        "the FP64 pipe" % (EW_FP64_PIPE_PER_TERMINAL * T + EW_FP64_PIPE_PER_BUS * nb),
            "rate_note": "achieved = operations per evaluation x evaluations per second over the timed region "
                         "(%d CUDA streams, two evaluations' CTAs sharing the SMs); on one stream, launches back "
                         "to back: %.2f us per launch, frac %.3f" % (HEADLINE_STREAMS, ms_stream1 * 1e3,
                                                                     ops_ew / (ms_stream1 * 1e-3) / 1e9
                                                                     / fp64_peak["gdfma_per_s"]),
            "fp64_pipe_frac": (EW_FP64_PIPE_PER_TERMINAL * T + EW_FP64_PIPE_PER_BUS * nb) / (ms_stream * 1e-3) / 1e9
                              / fp64_peak["gdfma_per_s"],
            "peak_source": "measured: fp64_peak_probe (DFMA chains on every SM) in this run",
            "frac_of_nominal": achieved / FP64_OPS_PEAK_G,
            "nominal_peak": FP64_OPS_PEAK_G,
            "nominal_source": "152 SMs x 2 FP64 ops/clk x 2.07 GHz",
            "hbm": {"achieved": bytes_ew / (ms_stream * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
                    "frac": bytes_ew / (ms_stream * 1e-3) / 1e9 / hbm, "algorithmic_bytes": bytes_ew,
                    "peak_source": hbm_kind}}

    # end to end through the C ABI with pinned host buffers
    e2e = None
    try:
        if args.no_e2e:
            raise RuntimeError("skipped (--no-e2e)")
        hb = lambda n: torch.empty(n, dtype=torch.float64, pin_memory=True).numpy()
        # two sets of page-locked buffers, used in turn (a stream of states)
        sets = []
        for _ in range(2):
            vm_h, va_h, P_h, Q_h, J_h = hb(nb), hb(nb), hb(nb), hb(nb), hb(grid.nnzJ)
            vm_h[:], va_h[:] = w["vm"][0], w["va"][0]
            sets.append((vm_h, va_h, P_h, Q_h, J_h))
        st = torch.cuda.current_stream().cuda_stream   # passed as a handle: no stream lookup per call
        for k in range(8):
            pfgrid.eval_host(grid, 1, *sets[k % 2], stream=st)
        ne = min(args.steps, 100)
        # the synchronous call: returns with the results in host memory
        # (median of three runs of ne calls, as below)
        runs = []
        for _ in range(3):
            t0 = time.perf_counter()
            for k in range(ne):
                pfgrid.eval_host(grid, 1, *sets[k % 2], stream=st)
            runs.append(time.perf_counter() - t0)
        el_sync = statistics.median(runs)
        # the asynchronous call: a stream of states, each set of buffers on its
        # own CUDA stream so that one evaluation's start overlaps the previous
        # one's results crossing the host link; every step reads its state from
        # and writes its results to host memory; one synchronization at the end
        streams = [torch.cuda.Stream() for _ in sets]
        for k in range(8):
            pfgrid.eval_host_async(grid, 1, *sets[k % 2], stream=streams[k % 2].cuda_stream)
        torch.cuda.synchronize()
        runs = []
        for _ in range(3):
            t0 = time.perf_counter()
            for k in range(ne):
                pfgrid.eval_host_async(grid, 1, *sets[k % 2], stream=streams[k % 2].cuda_stream)
            torch.cuda.synchronize()
            runs.append(time.perf_counter() - t0)
        el = statistics.median(runs)
        e2e = {"value": world * ne / el, "unit": "evals/s", "h2d_bytes_per_step": 16 * nb,
               "d2h_bytes_per_step": 16 * nb + 8 * grid.nnzJ,
               "api": "eval_host_async, two buffer sets on two CUDA streams, one synchronization per run of %d "
                      "evaluations, median of 3 runs" % ne,
               "eval_host_sync_evals_per_s": world * ne / el_sync}
    except Exception as ex:  # reported, never silently replaced
        e2e = {"error": str(ex)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        n, el = run_oracle_steps(w, None, seconds=args.cpu_seconds)
        model, ncpu = host_cpu()
        cpu = {"value": n / el, "unit": "evals/s", "cores": 1, "nproc": ncpu, "cpu_model": model, "kind": "oracle",
               "sample": "%d full element-wise evaluations (P, Q, J) of the 70k-bus grid, single thread "
                         "(one evaluation has no independent parts to spread over cores)" % n}

    extra = None
    if rank == 0 and not args.no_extra:
        try:
            extra = extra_workloads(torch, pfgrid, synth, max(3, min(args.steps, 20)),
                                    cpu_seconds=None if args.no_cpu_baseline else min(args.cpu_seconds, 5.0))
        except Exception as ex:  # reported, never silently replaced
            extra = {"error": str(ex)}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD_NAME, "nnzY": grid.nnz, "nnzJ": grid.nnzJ,
                       "global_batch": world, "seq_len": 0, "parallelism": "replicas" if world > 1 else "none",
                       "l2": "inputs larger than L2: %d copies of the grid with their own states and outputs "
                             "(%.0f MB) evaluated in turn, %d steps back to back between one pair of CUDA events"
                             % (STREAM_COPIES, footprint / 1e6, args.steps),
                       "streams": "step k on CUDA stream k mod %d (independent evaluations: each reads its own "
                                  "copy's state and writes all its outputs)" % HEADLINE_STREAMS,
                       "launch_queue": "all %d launches queued behind a device-side wait of %.1f ms before the "
                                       "first event (host: %.1f us per launch), so the device time is the GPU's "
                                       "back-to-back rate" % (args.steps, stream_info["device_wait_ms"],
                                                              stream_info["host_enqueue_us_per_step"]),
                       "launch_config": cfg},
            "e2e": e2e, "gpu_launches": args.steps, "roofline": roof, "cpu_baseline": cpu, "clocks": clocks,
            "fp64_peak": fp64_peak,
            "compare": {
                "elementwise_jac_evals_per_s": 1e3 / ms_stream,
                "ybus_jac_evals_per_s_stream": 1e3 / ms_stream_yb,
                "elementwise_jac_evals_per_s_one_stream": 1e3 / ms_stream1,
                "ybus_jac_evals_per_s_one_stream": 1e3 / ms_stream1_yb,
                "elementwise_inj_evals_per_s_stream": 1e3 / ms_stream_iew,
                "ybus_inj_evals_per_s_stream": 1e3 / ms_stream_iyb,
                "elementwise_jac_evals_per_s_flush_per_step": 1e3 / (sum(t_ew) / len(t_ew)),
                "ybus_jac_evals_per_s_flush_per_step": 1e3 / (sum(t_yb) / len(t_yb)),
                "elementwise_inj_evals_per_s_flush_per_step": 1e3 / (sum(t_iew) / len(t_iew)),
                "ybus_inj_evals_per_s_flush_per_step": 1e3 / (sum(t_iyb) / len(t_iyb)),
                "elementwise_jac_evals_per_s_after_write_only_flush": 1e3 / (sum(t_dirty) / len(t_dirty)),
                "kernel_ms": {"phasor": ms_pu, "jac_ew": ms_jew, "jac_ybus": ms_jyb,
                              "inj_ew": kmean(tr_inj, "inj_ew")[0], "inj_ybus": kmean(tr_inj, "inj_ybus")[0]},
                "ybus_fp64_ops_per_launch": YB_OPS_PER_NNZ * grid.nnz + YB_OPS_PER_ROW * nb,
            },
            "workloads": extra,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
