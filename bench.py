"""Benchmark: dSDC steps/s of the T255 rotating shallow-water workload on one GB300.

Workload (the configuration the headline metric names): truncation T255 on a
384 x 768 Gauss grid, M = 4 Radau-right nodes, K = 5 sweeps, dt = 150 s,
seeded synthetic initial state (random vorticity/divergence spectra ~ n^-1.5
scaled to 20 m/s rms wind, one 100 m Gaussian height bump of 500 km radius).
A step is one full dSDC step (Algorithm 2): 1 + (K-1) M = 17 explicit
tendency evaluations through the spherical-harmonic transform and K sweep
kernels.

Arms:
  default            the CUDA library (FP64 transforms; the FP32 mixed mode is
                     timed beside it and reported with its error)
  --impl reference   the FP64 CPU oracle as it stands, on the host cores
Under torchrun (N > 1) every rank runs an independent replica of the
workload (no data-path collective): weak scaling, value = sum over ranks.
"""
from __future__ import annotations

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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import swe_inputs as si  # noqa: E402

METRIC = "SDC steps/s at T255 M=4 K=5: FP64 vs mixed at fixed error; adjoint/fwd ratio"
WORKLOAD = "t255"
L2_FLUSH_BYTES = 512 << 20          # > 129 MB L2
FP64_NOMINAL_TFLOPS = 1.25          # GB300 dense FP64: 152 SMs x 4 flops/clock x 2.07 GHz (nominal)
# FP32 SIMT: 152 SMs x 128 FMA lanes x 2 flops x 2.07 GHz (maximum SM clock)
FP32_SIMT_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
# DRAM bytes (read + write) of one launch of the FP64 ring kernel with a batch
# of 4 states at the T255 workload, from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum), and the SHA-256 prefix of
# the kernel's source (its function in transforms.cu and the FFT header) at
# that capture.  The traffic is the batch's F1 input, so a launch of b states
# moves b/4 of it.  When the source differs the counters no longer describe
# the kernel and the bench reports null.
RING_FP64_TRAFFIC_B4 = 25289216.0 + 192768.0
RING_FP64_SOURCES_SHA = "22cf27af41541150"


def _ring_fp64_source_sha() -> str:
    """SHA-256 prefix of the FP64 ring kernel's source text: the k2_ring
    function of transforms.cu and all of fft.cuh."""
    import hashlib
    csrc = os.path.join(ROOT, "paper_2403_20135_gb300", "csrc")
    with open(os.path.join(csrc, "transforms.cu")) as f:
        text = f.read()
    start = text.index("__global__ void k2_ring(")
    end = text.index("// -----", start)
    h = hashlib.sha256(text[start:end].encode())
    with open(os.path.join(csrc, "fft.cuh"), "rb") as f:
        h.update(f.read())
    return h.hexdigest()[:16]


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# ---------------------------------------------------------------------------
# algorithmic work per launch: flops per node evaluation times the batch
# ---------------------------------------------------------------------------
def stage_flops(wl, stage: str, batch: int) -> float:
    T, J2, L = wl.T, wl.nlat // 2, wl.nlon
    next_ = (T + 1) * (T + 4) // 2
    if stage == "synthesis":          # 4 complex fields x 2 real FMA per (n', j)
        return 16.0 * next_ * J2 * batch
    if stage == "analysis":           # 5 complex fields x 2 real FMA per (n', j)
        return 20.0 * next_ * J2 * batch
    if stage == "ring":               # 9 complex FFTs (5 L log2 L) + products per ring pair
        return (9 * 5.0 * L * np.log2(L) + 60.0 * L) * J2 * batch
    raise ValueError(stage)


def sweep_flops(wl, ybatch: int, nupdated: int) -> float:
    """FP64-mode flops of one sweep kernel per mode: for each updated node the
    quadrature (6 real components x M terms x 2 flops), the right side and the
    2x2 solve (about 24 flops); forming L_g u_j + T_E(u_j) (8 flops per node);
    the vector epilogue of the ybatch projected states (about 36 flops each)."""
    nc = (wl.T + 1) * (wl.T + 2) // 2
    M = wl.nodes
    return nc * ((12.0 * M + 24.0) * nupdated + 8.0 * M + 36.0 * ybatch)


def sweep_bytes(wl, all_nodes: bool, ybatch: int, y_elem: int = 16) -> float:
    """Bytes one sweep kernel moves per launch: u_n, the M node states, the
    projections (10 complex values per mode and projected state) and the
    states it writes (M, or 1 in the last sweep)."""
    nc = (wl.T + 1) * (wl.T + 2) // 2
    M = wl.nodes
    states = 1 + M + (M if all_nodes else 1)
    return nc * (states * 3 * 16.0 + ybatch * 10 * y_elem)


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# the oracle on the host cores
# ---------------------------------------------------------------------------
def oracle_steps_per_s(wl, budget_s: float, max_steps: int):
    """Time full oracle steps of the workload until the budget is spent."""
    from oracle import sdc as osdc
    from oracle import sht, swe
    o = swe.SWE(sht.Grid(wl.T, wl.nlat, wl.nlon), swe.default_physics())
    u = swe.initial_state(wl, o)
    coll = osdc.Collocation(wl.nodes)
    n, t0 = 0, time.perf_counter()
    while n < max_steps:
        u = osdc.swe_step(o, u, coll, wl.sweeps, wl.dt)
        n += 1
        if time.perf_counter() - t0 > budget_s:
            break
    el = time.perf_counter() - t0
    return n / el, n, el


def oracle_steps_per_s_single_thread(key: str, budget_s: float, max_steps: int):
    """oracle_steps_per_s in a fresh interpreter with every BLAS/OpenMP pool
    pinned to one thread (the pools size themselves at import)."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = ("import json, sys; sys.path.insert(0, %r); import bench, swe_inputs as si; "
            "print(json.dumps(bench.oracle_steps_per_s(si.WORKLOADS[%r], %r, %r)))" % (ROOT, key, budget_s, max_steps))
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                       timeout=4 * budget_s + 300)
    if r.returncode != 0:
        raise RuntimeError(f"single-thread oracle run failed: {r.stderr[-2000:]}")
    v, n, el = json.loads(r.stdout.strip().splitlines()[-1])
    return v, n, el


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the platform string)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


def cpu_baseline_entry(key: str, budget_s: float, max_steps: int) -> dict:
    """The oracle timed on the host cores twice: every pool pinned to one
    thread, and with the default pools (all cores the process may use)."""
    wl = si.WORKLOADS[key]
    v1, n1, el1 = oracle_steps_per_s_single_thread(key, budget_s, max_steps)
    va, na, ela = oracle_steps_per_s(wl, budget_s=budget_s, max_steps=max_steps)
    cores = host_cores()
    return {"value": va, "unit": "steps/s", "cores": cores, "kind": "oracle", "cpu_model": cpu_model(),
            "sample": f"{na} full T{wl.T} dSDC steps of the seeded state ({ela:.1f} s, numpy FP64, default "
                      f"thread pools over {cores} cores)",
            "single_thread": {"value": v1, "unit": "steps/s", "threads": 1,
                              "sample": f"{n1} full steps ({el1:.1f} s), BLAS/OpenMP pinned to 1 thread"},
            "all_cores": {"value": va, "unit": "steps/s", "threads": cores,
                          "sample": f"{na} full steps ({ela:.1f} s)"}}


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def reference_arm(args, rank: int, world: int):
    if rank != 0:
        return
    wl = si.WORKLOADS[WORKLOAD]
    for _ in range(args.warmup):
        pass                                  # the oracle has no warm-up state worth timing
    cap = max(1, min(args.steps, 12))         # keeps the whole run within a few minutes
    v, n, el = oracle_steps_per_s(wl, budget_s=150.0, max_steps=cap)
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "steps/s", "n_gpus": 1,
        "steps": n, "warmup": args.warmup, "ms_per_step": 1e3 * el / n, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl.describe(), "parallelism": "host cores"},
        "cpu_baseline": {"value": v, "unit": "steps/s", "cores": host_cores(), "kind": "oracle",
                         "cpu_model": cpu_model(),
                         "sample": f"{n} full T255 dSDC steps (of {args.steps} requested), default thread pools"},
        "e2e": {"value": v, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# the CUDA arm
# ---------------------------------------------------------------------------
def job_rate(local_ms: float, steps: int, world: int, device: str = "cpu"):
    """Whole-job throughput of `world` replicas that each ran `steps` steps:
    the slowest rank's time (MAX over ranks) bounds the job, and every rank
    processed `steps` units.  Returns (max_ms, steps/s of the whole job)."""
    total_ms = local_ms
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([local_ms], device=device, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    return total_ms, world * steps / (total_ms * 1e-3)


def time_device(s, state, steps: int, flush):
    """Sum of CUDA-event times of `steps` single-step graph replays, L2 flushed before each."""
    import torch
    stream = torch.cuda.current_stream()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    for i in range(steps):
        flush.zero_()
        starts[i].record(stream)
        s.run(state, 1)
        ends[i].record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in zip(starts, ends)]


def profile_stages(s, u0, flush, nprof: int):
    """Per-kernel-class device time of nprof steps launched kernel by kernel."""
    st = u0.clone()
    acc = {k: [0.0, 0] for k in s.STAGES}
    for _ in range(nprof):
        flush.zero_()
        for k, (ms, n) in s.profile_step(st).items():
            acc[k][0] += ms
            acc[k][1] += n
    tot = max(1e-12, sum(x[0] for x in acc.values()))
    prof = {k: {"ms_per_launch": (v[0] / v[1]) if v[1] else 0.0, "launches_per_step": v[1] // nprof,
                "share": v[0] / tot} for k, v in acc.items()}
    return prof, acc


def time_adjoint(Solver, wl, nsteps: int, nsnap: int, reps: int, precision: int = 0):
    """Adjoint/forward cost: one reversed step (retape + adjoint) against one forward
    step, and a checkpointed gradient run against the forward run of nsteps, both
    in the given precision mode."""
    import torch
    s = Solver.for_workload(wl, precision=precision)
    u0 = s.initial_state(wl)
    x = u0.clone()
    ub = torch.ones_like(u0)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    s.run(x, 2)
    s.step_adjoint(u0, ub)
    torch.cuda.synchronize()
    ev[0].record()
    for _ in range(reps):
        s.run(x, 1)
    ev[1].record()
    for _ in range(reps):
        s.step_adjoint(u0, ub)
    ev[2].record()
    torch.cuda.synchronize()
    fwd_ms = ev[0].elapsed_time(ev[1]) / reps
    rev_ms = ev[1].elapsed_time(ev[2]) / reps
    target = si.MEAN_DEPTH + s.spec_to_grid(u0[0].contiguous()) / si.GRAVITY
    x = u0.clone()
    ev[0].record()
    s.run(x, nsteps)
    ev[1].record()
    loss, g = s.adjoint_run(u0, nsteps, target, nsnap)
    ev[2].record()
    torch.cuda.synchronize()
    run_ms = ev[0].elapsed_time(ev[1])
    adj_ms = ev[1].elapsed_time(ev[2])
    _, nfwd = s.run_adjoint(u0, nsteps, ub, nsnap)
    s.close()
    return {"workload": wl.describe(), "step_fwd_ms": fwd_ms, "step_reverse_ms": rev_ms,
            "step_ratio": rev_ms / fwd_ms, "run_steps": nsteps, "snapshots": nsnap, "run_fwd_ms": run_ms,
            "run_adjoint_ms": adj_ms, "run_ratio": adj_ms / run_ms, "recomputed_forward_steps": nfwd}


def time_e2e(s, host_state, dev_state, host_out, steps: int):
    """Host-buffer path: pinned H2D copy, one step through the C ABI, D2H copy."""
    import torch
    stream = torch.cuda.current_stream()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        dev_state.copy_(host_state, non_blocking=True)
        s.run(dev_state, 1)
        host_out.copy_(dev_state, non_blocking=True)
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b)


def cuda_arm(args, rank: int, world: int):
    import torch
    import torch.distributed as dist

    from paper_2403_20135_gb300 import SDC_FP64, SDC_MIXED_BF16X3, SDC_MIXED_BF16X6, SDC_MIXED_FP32, Solver
    from paper_2403_20135_gb300.solver import fp64_fma_rate

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    wl = si.WORKLOADS[WORKLOAD]
    peaks, peak_kind = _peaks()

    s = Solver.for_workload(wl, precision=SDC_FP64)
    u0 = s.initial_state(wl)
    state = u0.clone()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")

    for _ in range(args.warmup):
        s.run(state, 1)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev0, _, l0 = s.counters()
    with ClockSampler(dev) as clk:
        times = time_device(s, state, args.steps, flush)
    ev1, _, l1 = s.counters()
    total_ms, steps_per_s = job_rate(float(sum(times)), args.steps, world, "cuda")
    clocks = clk.summary()

    # kernel-by-kernel profile of the same step (CUDA events between launches)
    prof, acc = profile_stages(s, u0, flush, max(3, min(10, args.steps)))
    dom = max(("synthesis", "ring", "analysis"), key=lambda k: acc[k][0])
    # average work per launch of the dominant stage: launches come with batch 1 (E0) and batch M
    K, M = wl.sweeps, wl.nodes
    nodes_per_step = 1 + (K - 1) * M
    launches_per_step = prof[dom]["launches_per_step"]
    flops_per_launch = stage_flops(wl, dom, nodes_per_step) / launches_per_step
    achieved_tf = flops_per_launch / (prof[dom]["ms_per_launch"] * 1e-3) / 1e12
    traffic = None
    if dom == "ring" and RING_FP64_SOURCES_SHA == _ring_fp64_source_sha():
        traffic = RING_FP64_TRAFFIC_B4 * (nodes_per_step / launches_per_step) / 4.0
    fp64_peak = fp64_fma_rate()
    roofline = {"bound": "alu", "achieved": achieved_tf, "peak": fp64_peak, "unit": "TFLOP/s",
                "frac": achieved_tf / fp64_peak, "traffic": traffic, "kernel": dom,
                "peak_kind": "measured FP64 FMA rate of this GPU (sdc_fp64_fma_rate, same run)",
                "peak_nominal": FP64_NOMINAL_TFLOPS, "frac_of_nominal": achieved_tf / FP64_NOMINAL_TFLOPS}
    # the whole step: algorithmic flops of every stage over the step time
    step_flops = sum(stage_flops(wl, k, nodes_per_step) for k in ("synthesis", "ring", "analysis"))
    step_flops += (sweep_flops(wl, 1, M) + (K - 2) * sweep_flops(wl, M, M) + sweep_flops(wl, M, 1))
    step_tf = step_flops / (total_ms / args.steps * 1e-3) / 1e12
    roofline_step = {"bound": "alu", "achieved": step_tf, "peak": fp64_peak, "unit": "TFLOP/s",
                     "frac": step_tf / fp64_peak, "frac_of_nominal": step_tf / FP64_NOMINAL_TFLOPS,
                     "flops_per_step": step_flops}
    # the sweep kernel (FP64 in every mode): FP64 flops and the bytes it moves
    sw_ms = prof["sweep"]["ms_per_launch"]
    # K sweeps per step: the first reads the projections of one state, the
    # others of M; sweeps 1..K-1 update all M nodes, the last one node
    sw_bytes = (sweep_bytes(wl, True, 1) + (K - 2) * sweep_bytes(wl, True, M) + sweep_bytes(wl, False, M)) / K
    sw_flops = (sweep_flops(wl, 1, M) + (K - 2) * sweep_flops(wl, M, M) + sweep_flops(wl, M, 1)) / K
    roofline_sweep = {"bound": "alu", "achieved": sw_flops / (sw_ms * 1e-3) / 1e12, "peak": fp64_peak,
                      "unit": "TFLOP/s", "frac": sw_flops / (sw_ms * 1e-3) / 1e12 / fp64_peak,
                      "hbm_gbs": sw_bytes / (sw_ms * 1e-3) / 1e9, "hbm_peak_gbs": peaks["hbm_gbs"],
                      "hbm_frac": sw_bytes / (sw_ms * 1e-3) / 1e9 / peaks["hbm_gbs"], "kernel": "sweep"}

    # end to end through host buffers
    host_state = u0.cpu().pin_memory()
    host_out = torch.empty_like(host_state).pin_memory()
    dev_state = torch.empty_like(u0)
    ne2e = max(3, min(args.steps, 50))
    time_e2e(s, host_state, dev_state, host_out, 2)
    e2e_ms = time_e2e(s, host_state, dev_state, host_out, ne2e)
    sbytes = 3 * s.ncoef * 16
    e2e = {"value": world * ne2e / (e2e_ms * 1e-3), "unit": "steps/s", "h2d_bytes_per_step": sbytes,
           "d2h_bytes_per_step": sbytes}

    # mixed modes beside it: throughput and error against the FP64 path, and the
    # fixed-error test: the mixed-mode error must stay below the FP64
    # discretisation error (FP64 at dt against FP64 at dt/4 over the same horizon)
    mixed = None
    if not args.no_mixed:
        nh = args.horizon
        a64, a64q = u0.clone(), u0.clone()
        s.run(a64, nh)
        sq = Solver(wl.T, wl.nlat, wl.nlon, wl.nodes, wl.sweeps, wl.dt / 4, si.RADIUS, si.OMEGA, si.GRAVITY,
                    si.MEAN_DEPTH, precision=SDC_FP64)
        sq.run(a64q, 4 * nh)
        sq.close()

        def rel(x, y):
            return ((x - y).abs().pow(2).sum(1) / y.abs().pow(2).sum(1)).sqrt().cpu().numpy()

        edisc = rel(a64, a64q)
        fields = ("phi", "zeta", "div")
        mixed = {"horizon_steps": nh, "fp64_discretisation_rel_l2": dict(zip(fields, map(float, edisc)))}
        for name, prec in (("fp32", SDC_MIXED_FP32), ("bf16x3", SDC_MIXED_BF16X3), ("bf16x6", SDC_MIXED_BF16X6)):
            sm = Solver.for_workload(wl, precision=prec)
            xs = u0.clone()
            for _ in range(args.warmup):
                sm.run(xs, 1)
            tm = time_device(sm, xs, args.steps, flush)
            mprof, _ = profile_stages(sm, u0, flush, max(3, min(10, args.steps)))
            am = u0.clone()
            sm.run(am, nh)
            sm.sync()
            err = rel(am, a64)
            mdom = max(("synthesis", "ring", "analysis"), key=lambda k: mprof[k]["ms_per_launch"])
            mfl = stage_flops(wl, mdom, nodes_per_step) / mprof[mdom]["launches_per_step"]
            mach = mfl / (mprof[mdom]["ms_per_launch"] * 1e-3) / 1e12
            mixed[name] = {"value": world * args.steps / (sum(tm) * 1e-3), "unit": "steps/s",
                           "ms_per_step": sum(tm) / args.steps, "stages": mprof,
                           "rel_l2_vs_fp64": dict(zip(fields, map(float, err))),
                           "fixed_error": bool(np.all(err < edisc)),
                           "roofline": {"bound": "alu", "kernel": mdom, "achieved": mach,
                                        "peak": FP32_SIMT_TFLOPS, "unit": "TFLOP/s",
                                        "frac": mach / FP32_SIMT_TFLOPS,
                                        "peak_kind": "nominal FP32 SIMT (algorithmic flops; the tensor-core "
                                                     "modes count their contractions at this rate too)"}}
            sm.close()
        mixed["fp32_legendre"] = legendre_compare(wl, args.steps, flush)
        ok = [k for k in ("fp32", "bf16x3", "bf16x6") if mixed[k]["fixed_error"]]
        if ok:
            best = max(ok, key=lambda k: mixed[k]["value"])
            mixed["best_at_fixed_error"] = {"mode": best, "value": mixed[best]["value"], "unit": "steps/s",
                                            "speedup_vs_fp64": mixed[best]["value"] / steps_per_s}
        else:
            mixed["best_at_fixed_error"] = None

    adjoint = None
    if not args.no_adjoint:
        adjoint = {"t255": time_adjoint(Solver, wl, 20, 8, 5),
                   "t127_differentiation": time_adjoint(Solver, si.WORKLOADS["t127adj"], 96, 8, 10),
                   "t255_fp32": time_adjoint(Solver, wl, 20, 8, 5, precision=PRECISIONS["fp32"])}

    t511 = None
    if not args.no_t511:
        t511 = t511_leg(max(3, min(args.steps, 10)), args.t511_horizon, args.t511_adjoint_steps, flush)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_entry(WORKLOAD, args.cpu_budget, 50)

    if rank == 0:
        line = {
            "metric": METRIC, "value": steps_per_s, "unit": "steps/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl.describe(), "precision": "FP64 transforms, FP64 solves",
                       "l2": "flushed (512 MiB write) before every timed step",
                       "parallelism": f"replicas x{world}"},
            "e2e": e2e, "gpu_launches": int(l1 - l0), "clocks": clocks, "roofline": roofline,
            "roofline_sweep": roofline_sweep, "roofline_step": roofline_step,
            "stages": prof, "mixed": mixed,
            "adjoint_fwd_ratio": adjoint["t255"]["step_ratio"] if adjoint else None, "adjoint": adjoint,
            "t511": t511,
            "cpu_baseline": cpu,
            "peaks_source": peak_kind,
        }
        print(json.dumps(line), flush=True)
    s.close()


PRECISIONS = {"fp64": 0, "fp32": 1, "bf16x3": 2, "bf16x6": 3}


def legendre_compare(wl, steps: int, flush) -> dict:
    """FP32 mode with the Legendre table against the on-the-fly recurrence:
    steps/s (CUDA events, L2 flushed per step) and the synthesis kernel's time
    per launch (kernel-by-kernel profile of the same steps)."""
    from paper_2403_20135_gb300 import SDC_LEGENDRE_RECURRENCE, Solver
    out = {}
    for name in ("table", "recurrence"):
        s = Solver.for_workload(wl, precision=PRECISIONS["fp32"])
        if name == "recurrence":
            s.set_legendre(SDC_LEGENDRE_RECURRENCE)
        u0 = s.initial_state(wl)
        x = u0.clone()
        s.run(x, 2)
        tm = time_device(s, x, steps, flush)
        prof, _ = profile_stages(s, u0, flush, 3)
        out[name] = {"steps_per_s": steps / (sum(tm) * 1e-3),
                     "synthesis_us_per_launch": 1e3 * prof["synthesis"]["ms_per_launch"]}
        s.close()
    return out


def t511_leg(steps: int, horizon: int, adj_steps: int, flush):
    """The largest combined form: T511 on 768 x 1536, M = 4, K = 5, dt = 75 s.
    Forward steps/s in every precision (CUDA events, L2 flushed before each
    step), per-field error of each mixed mode against the FP64 GPU path after
    `horizon` steps, the reversed-step/forward-step cost in FP64 and FP32 mode,
    the checkpointed gradient run over `adj_steps` steps with 16 snapshots in
    FP32 mode (the mixed form), and device memory: the library's own
    allocations (free-memory drop from before create) and torch's peak."""
    import torch
    from paper_2403_20135_gb300 import Solver
    wl = si.WORKLOADS["t511"]
    torch.cuda.synchronize()
    torch.cuda.reset_peak_memory_stats()
    free0 = torch.cuda.mem_get_info()[0]
    fields = ("phi", "zeta", "div")
    out = {"workload": wl.describe().replace(f"{wl.nsteps} steps", f"{horizon}-step horizon")}
    s64 = Solver.for_workload(wl, precision=0)
    u0 = s64.initial_state(wl)
    ref = u0.clone()
    s64.run(ref, horizon)
    s64.sync()

    def rate(s):
        x = u0.clone()
        s.run(x, 2)
        tm = time_device(s, x, steps, flush)
        return steps / (sum(tm) * 1e-3), sum(tm) / steps

    v64, ms64 = rate(s64)
    out["fp64"] = {"value": v64, "unit": "steps/s", "ms_per_step": ms64}
    min_free = torch.cuda.mem_get_info()[0]
    for name in ("fp32", "bf16x3", "bf16x6"):
        sm = Solver.for_workload(wl, precision=PRECISIONS[name])
        v, ms = rate(sm)
        x = u0.clone()
        sm.run(x, horizon)
        sm.sync()
        err = ((x - ref).abs().pow(2).sum(1) / ref.abs().pow(2).sum(1)).sqrt().cpu().numpy()
        out[name] = {"value": v, "unit": "steps/s", "ms_per_step": ms, "speedup_vs_fp64": v / v64,
                     "rel_l2_vs_fp64_gpu": dict(zip(fields, map(float, err)))}
        min_free = min(min_free, torch.cuda.mem_get_info()[0])
        sm.close()
    # reversed step against forward step, FP64 and FP32 mode
    for name, prec in (("fp64", 0), ("fp32", 1)):
        s = s64 if prec == 0 else Solver.for_workload(wl, precision=prec)
        ub = torch.ones_like(u0)
        x = u0.clone()
        s.run(x, 1)
        s.step_adjoint(u0, ub)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        torch.cuda.synchronize()
        ev[0].record()
        for _ in range(3):
            s.run(x, 1)
        ev[1].record()
        for _ in range(3):
            s.step_adjoint(u0, ub)
        ev[2].record()
        torch.cuda.synchronize()
        out[name]["adjoint_step_ratio"] = ev[1].elapsed_time(ev[2]) / ev[0].elapsed_time(ev[1])
        min_free = min(min_free, torch.cuda.mem_get_info()[0])
        if prec != 0:
            # the checkpointed gradient run of the mixed form
            target = si.MEAN_DEPTH + s.spec_to_grid(u0[0].contiguous()) / si.GRAVITY
            x = u0.clone()
            ev[0].record()
            s.run(x, adj_steps)
            ev[1].record()
            loss, g = s.adjoint_run(u0, adj_steps, target, 16)
            ev[2].record()
            torch.cuda.synchronize()
            out["fp32"]["adjoint_run"] = {"steps": adj_steps, "snapshots": 16,
                                          "fwd_ms": ev[0].elapsed_time(ev[1]), "adjoint_ms": ev[1].elapsed_time(ev[2]),
                                          "ratio": ev[1].elapsed_time(ev[2]) / ev[0].elapsed_time(ev[1]),
                                          "finite": bool(torch.isfinite(g).all().item())}
            min_free = min(min_free, torch.cuda.mem_get_info()[0])
            s.close()
    s64.close()
    out["fp32_legendre"] = legendre_compare(wl, steps, flush)
    out["device_memory"] = {"library_and_torch_peak_bytes": int(free0 - min_free),
                            "torch_max_allocated_bytes": int(torch.cuda.max_memory_allocated()),
                            "note": "free-memory drop from before the first create to its minimum over the leg "
                                    "(sampled between calls); one FP64 and one mixed context alive at a time"}
    return out


def work_precision(hours: float):
    """Synthetic work-precision study on the bench workload's grid and initial
    state: error after a fixed simulated time against GPU time for dSDC (FP64,
    FP32), serial IMEX SDC (FP64) and IMEX-o2 (FP64) over a time-step sweep.
    Reference: dSDC FP64 at 1/8 of the smallest step.  One JSON line."""
    import torch

    from paper_2403_20135_gb300 import (SDC_FP64, SDC_METHOD_DSDC, SDC_METHOD_IMEX2, SDC_METHOD_SERIAL_SDC,
                                        SDC_MIXED_FP32, Solver)
    wl = si.WORKLOADS[WORKLOAD]
    horizon = hours * 3600.0
    cases = [("dsdc", SDC_METHOD_DSDC, SDC_FP64, (900.0, 600.0, 450.0, 300.0, 150.0, 75.0)),
             ("dsdc", SDC_METHOD_DSDC, SDC_MIXED_FP32, (900.0, 600.0, 450.0, 300.0, 150.0, 75.0)),
             ("serial_sdc", SDC_METHOD_SERIAL_SDC, SDC_FP64, (900.0, 600.0, 300.0, 150.0, 75.0)),
             ("imex2", SDC_METHOD_IMEX2, SDC_FP64, (300.0, 150.0, 75.0, 37.5, 18.75))]

    def make(dt, method, prec):
        return Solver(wl.T, wl.nlat, wl.nlon, wl.nodes, wl.sweeps, dt, si.RADIUS, si.OMEGA, si.GRAVITY,
                      si.MEAN_DEPTH, precision=prec, method=method)

    s0 = make(wl.dt, SDC_METHOD_DSDC, SDC_FP64)
    u0 = s0.initial_state(wl)
    s0.close()
    dt_ref = 75.0 / 8
    sr = make(dt_ref, SDC_METHOD_DSDC, SDC_FP64)
    ref = u0.clone()
    sr.run(ref, int(round(horizon / dt_ref)))
    sr.sync()
    sr.close()
    fields = ("phi", "zeta", "div")
    rows = []
    for name, method, prec, dts in cases:
        for dt in dts:
            n = int(round(horizon / dt))
            s = make(dt, method, prec)
            x = u0.clone()
            s.run(x, 1)                       # graph capture and warm-up outside the timing
            x = u0.clone()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            s.run(x, n)
            e1.record()
            torch.cuda.synchronize()
            err = ((x - ref).abs().pow(2).sum(1) / ref.abs().pow(2).sum(1)).sqrt().cpu().numpy()
            rows.append({"method": name, "precision": "fp64" if prec == SDC_FP64 else "fp32", "dt": dt,
                         "steps": n, "gpu_ms": e0.elapsed_time(e1),
                         "rel_l2": dict(zip(fields, map(float, err))),
                         "finite": bool(np.all(np.isfinite(err)))})
            s.close()
    print(json.dumps({"work_precision": rows, "workload": wl.describe(), "simulated_hours": hours,
                      "reference": f"dSDC FP64, dt = {dt_ref} s"}), flush=True)


def profile_run(name: str, steps: int, adjoint: bool = False, chains: int = 0):
    """A few untimed steps of one precision mode (the command profilers wrap);
    with `adjoint`, reversed steps (retape + step adjoint) instead; `chains`
    (1 or 2) overrides the library's default chain count."""
    import torch
    from paper_2403_20135_gb300 import Solver
    wl = si.WORKLOADS[WORKLOAD]
    s = Solver.for_workload(wl, precision=PRECISIONS[name])
    if chains:
        s.set_chains(chains)
    u = s.initial_state(wl)
    if adjoint:
        ub = torch.ones_like(u)
        for _ in range(steps):
            s.step_adjoint(u, ub)
    else:
        s.run(u, steps)
    s.sync()
    kind = "reversed steps" if adjoint else "steps"
    print(f"profile-run {name}: {steps} {kind} of {wl.describe()} ok")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--no-t511", action="store_true", help="skip the T511 leg")
    ap.add_argument("--t511-horizon", type=int, default=400, help="steps of the T511 error comparison")
    ap.add_argument("--t511-adjoint-steps", type=int, default=400, help="steps of the T511 gradient run")
    ap.add_argument("--horizon", type=int, default=500, help="steps of the fixed-error comparison")
    ap.add_argument("--profile-run", choices=sorted(PRECISIONS), default=None,
                    help="only run --steps untimed steps of this precision (for profilers)")
    ap.add_argument("--adjoint", action="store_true", help="with --profile-run: reversed steps")
    ap.add_argument("--chains", type=int, default=0, help="with --profile-run: concurrent state chains (1 or 2)")
    ap.add_argument("--work-precision", type=float, default=None, metavar="HOURS",
                    help="only run the work-precision study over this simulated time")
    args = ap.parse_args()
    if args.work_precision:
        work_precision(args.work_precision)
        return
    if args.profile_run:
        profile_run(args.profile_run, args.steps, args.adjoint, args.chains)
        return
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "gloo" if args.impl == "reference" else "nccl"
        if args.impl == "ours":
            import torch
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group(backend)
    try:
        if args.impl == "reference":
            reference_arm(args, rank, world)
        else:
            cuda_arm(args, rank, world)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
